"""The plan-time tuner: it chooses launch shapes only (feed and resident CTAs of
the axis-1 pass, shape of the edge-correction kernels), so a tuned plan gives
the untuned plan's iterates bit for bit; its choices are cached on disk and a
second plan of the same geometry reads them instead of timing again."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from synth import point_source, spheres_medium  # noqa: E402

SHAPE = (128, 128, 64)   # axis-1 edge 64 has a TMA-fed pass; axes 0 and 1 are corrected
KW = dict(boundary_widths=((8, 8),) * 3, split=(2, 2, 1), truncation=8)


def _plan(**kw):
    import paper_2410_02395_gb300 as pkg

    n = spheres_medium(SHAPE, count=6, r_range=(4, 10), n_range=(1.1, 1.4), seed=71, margin=8)
    return pkg.Plan(SHAPE, 0.25, 1.0, torch.from_numpy(n).cuda(), **KW, **kw)


def test_tuned_and_untuned_plans_give_identical_iterates(tmp_path, monkeypatch):
    monkeypatch.setenv("MBS_TUNE_CACHE", str(tmp_path / "tune.txt"))
    src = torch.from_numpy(point_source(SHAPE)).cuda()
    tuned = _plan()
    plain = _plan(no_tune=True)
    it_t, it_p = tuned.info(), plain.info()
    assert it_t["tune_source"] == 1 and it_p["tune_source"] == 0
    assert "axis1/64:" in it_t["tuning"] and "corr01:" in it_t["tuning"]
    xt, _, _ = tuned.solve(src, tol=0.0, max_iter=12)
    xp, _, _ = plain.solve(src, tol=0.0, max_iter=12)
    assert torch.equal(xt, xp)
    tuned.close()
    plain.close()


def test_choices_are_cached_on_disk(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.txt"
    monkeypatch.setenv("MBS_TUNE_CACHE", str(path))
    first = _plan()
    assert first.info()["tune_source"] == 1
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and all("\t" in ln for ln in lines)   # axis-1 pass and corrections
    second = _plan()
    assert second.info()["tune_source"] == 2
    assert second.info()["tuning"] == first.info()["tuning"]
    assert len(path.read_text().splitlines()) == 2
    first.close()
    second.close()
    monkeypatch.setenv("MBS_TUNE_CACHE", "")                      # empty: no cache
    third = _plan()
    assert third.info()["tune_source"] == 1
    third.close()
