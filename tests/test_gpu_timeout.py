"""The bounded waits of the TMA-fed axis-1 passes, provoked without a fault.

Each wait for a tensor-map copy gives up after PassArgs::tma_wait SM cycles;
the kernel then marks the solver state MBS_ETIMEOUT and done, waits with the
full bound for the copies it still has in flight and leaves. A plan made with a
bound of one cycle makes the very first wait give up while its copy (a valid,
in-bounds box) is still on its way, so the path runs and every copy completes.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import point_source, random_field, spheres_medium  # noqa: E402

SHAPE = (32, 128, 64)       # axis-1 subdomain edge 64: a TMA-fed pass; row pitch 512 B
KW = dict(boundary_widths=((2, 2),) * 3, split=(1, 2, 1), truncation=4)


def _plan(**kw):
    import paper_2410_02395_gb300 as pkg

    n = spheres_medium(SHAPE, count=3, r_range=(2, 5), n_range=(1.1, 1.4), seed=41)
    return pkg, n, pkg.Plan(SHAPE, 0.25, 1.0, torch.from_numpy(n).cuda(), force_tma=True, **KW, **kw)


def test_expired_tma_wait_ends_the_solve_with_etimeout():
    pkg, n, plan = _plan(tma_wait_cycles=1)
    assert plan.info()["tma_groups"] >= 1
    src = torch.from_numpy(point_source(SHAPE)).cuda()
    with pytest.raises(pkg.MBSError) as ei:
        plan.solve(src, tol=0.0, max_iter=3)
    assert ei.value.status == 7
    plan.close()


def test_expired_tma_wait_in_an_operator_is_reported_and_the_plan_recovers():
    pkg, n, plan = _plan(tma_wait_cycles=1)
    x = torch.from_numpy(random_field(SHAPE, seed=42)).cuda()
    with pytest.raises(pkg.MBSError) as ei:
        plan.apply("PROPAGATE", x)
    assert ei.value.status == 7
    # the operator state was re-armed: an operator without tensor-map copies is exact
    ref = Problem(n, 0.25, 1.0, widths=KW["boundary_widths"], split=KW["split"], t=KW["truncation"])
    got = plan.apply("E", x)
    torch.cuda.synchronize()
    assert relative_l2(got.cpu().numpy(), ref.apply_E(x.cpu().numpy().astype(np.complex128))) < 2e-6
    plan.close()


def test_full_bound_with_forced_tma_matches_the_oracle():
    """The same plan with the default bound: the TMA-fed passes give the oracle's iterates."""
    pkg, n, plan = _plan()
    assert plan.info()["tma_groups"] >= 1
    src = point_source(SHAPE)
    x, it, _ = plan.solve(torch.from_numpy(src).cuda(), tol=0.0, max_iter=10)
    ref = Problem(n, 0.25, 1.0, widths=KW["boundary_widths"], split=KW["split"], t=KW["truncation"])
    xr, itr, _ = ref.solve(src, tol=0.0, max_iter=10)
    assert it == itr == 10
    assert relative_l2(x.cpu().numpy(), xr) < 1e-4
    plan.close()
