"""The row-tile enumeration of the row passes, checked on the CPU for every
compiled FFT length: each thread of a CTA of 32 * warps_for(N) threads visits the
(row, element) pairs of a 32-row x N tile at steps k < ceil(32 N / NT), either
with one fixed element per thread (when NT divides 32 N and N divides NT) or
with the running index tid + k NT (csrc/mbs_passes.cuh, TileMap). Every pair
must be visited once and lie inside the tile. warps_for is taken from the
library's header through a host program compiled with nvcc."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2410_02395_gb300", "csrc")


def _sizes():
    txt = open(os.path.join(CSRC, "mbs_fft_sizes.h")).read()
    return sorted({int(v) for v in re.findall(r"X\((\d+)\)", txt)})


def _warps(sizes):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "w.cu")
        with open(src, "w") as f:
            f.write('#include <cstdio>\n#include "mbs_fft.cuh"\nint main(){const int n[]={%s};'
                    'for(int v: n) printf("%%d %%d\\n", v, mbs::warps_for(v)); return 0;}\n'
                    % ",".join(map(str, sizes)))
        exe = os.path.join(d, "w")
        subprocess.run([nvcc, "-std=c++17", "-I", CSRC, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {int(a): int(b) for a, b in (ln.split() for ln in out.splitlines())}


def _visit(N, NT):
    pert = (32 * N + NT - 1) // NT
    fixed = NT % N == 0 and (32 * N) % NT == 0
    seen = {}
    for tid in range(NT):
        for k in range(pert):
            if fixed:
                r, e = tid // N + k * (NT // N), tid % N
                ok = r < 32
            else:
                idx = tid + k * NT
                r, e, ok = idx // N, idx % N, idx < 32 * N
            if ok:
                assert 0 <= r < 32 and 0 <= e < N, (N, tid, k, r, e)
                seen[(r, e)] = seen.get((r, e), 0) + 1
    return seen


def test_every_compiled_length_visits_each_tile_element_once():
    sizes = _sizes()
    assert len(sizes) == 106
    warps = _warps(sizes)
    for N in sizes:
        W = warps[N]
        assert 1 <= W <= 32
        seen = _visit(N, 32 * W)
        assert len(seen) == 32 * N and set(seen.values()) == {1}, N
