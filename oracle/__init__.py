"""FP64 CPU oracle of the modified Born series (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA product path never does.
"""
from .mbs_oracle import (  # noqa: F401
    Problem,
    fft_axis,
    fftn3,
    ifftn3,
    dft_direct,
    sinc_d2,
    correction_block,
    block_norm,
    frequencies_squared,
    split_sizes,
    absorbing_index,
    axis_flags,
    relative_l2,
)
