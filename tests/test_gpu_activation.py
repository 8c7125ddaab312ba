"""Subdomain activation (Sec. 3.1, "Implementation"): only the subdomains that
hold a source term start; a neighbour is activated once the field transferred
into it exceeds a threshold. The early iterates differ from the unmasked ones,
but the iteration converges from any start, so the converged field is the same
(checked against the unmasked plan and the FP64 oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import point_source, spheres_medium  # noqa: E402

SHAPE = (64, 48, 40)
KW = dict(boundary_widths=((6, 6), (6, 6), (4, 4)), split=(2, 2, 2), truncation=6)
SRC = (12, 10, 9)  # inside subdomain (0, 0, 0), away from its faces


def _plan(**kw):
    import paper_2410_02395_gb300 as pkg

    n = spheres_medium(SHAPE, count=5, r_range=(3, 7), n_range=(1.1, 1.4), seed=61, margin=6)
    return pkg, n, pkg.Plan(SHAPE, 0.25, 1.0, torch.from_numpy(n).cuda(), graph_iters=5, **KW, **kw)


def test_only_the_source_subdomain_starts_and_the_others_follow():
    pkg, n, plan = _plan(activation=True)
    src = point_source(SHAPE, SRC)
    plan.set_source(torch.from_numpy(src).cuda())
    flags = plan.active_subdomains()
    assert flags.shape == (2, 2, 2) and flags.sum() == 1 and flags[0, 0, 0] == 1
    plan.iterate(5, 0.0)
    x = plan.field(like=torch.zeros(1, device="cuda")).cpu().numpy()
    # while a subdomain is inactive its field stays exactly zero
    for j in np.argwhere(plan.active_subdomains() == 0):
        sl = tuple(slice(int(j[d]) * SHAPE[d] // 2, (int(j[d]) + 1) * SHAPE[d] // 2) for d in range(3))
        assert not np.any(x[sl])
    seen = [int(plan.active_subdomains().sum())]
    for _ in range(40):
        plan.iterate(5, 0.0)
        seen.append(int(plan.active_subdomains().sum()))
    assert seen == sorted(seen) and seen[-1] == 8  # activation spreads and never reverts
    plan.close()


def test_activation_converges_to_the_unmasked_solution():
    pkg, n, masked = _plan(activation=True)
    _, _, plain = _plan()
    src = point_source(SHAPE, SRC)
    s = torch.from_numpy(src).cuda()
    xa, ita, ra = masked.solve(s, tol=1e-5, max_iter=20000)
    xp, itp, rp = plain.solve(s, tol=1e-5, max_iter=20000)
    assert ra < 1e-5 and rp < 1e-5
    assert abs(ita - itp) <= max(10, 0.05 * itp)  # the iteration count barely changes (Sec. 3.1)
    ref = Problem(n, 0.25, 1.0, widths=KW["boundary_widths"], split=KW["split"], t=KW["truncation"])
    xr, _, _ = ref.solve(src, tol=1e-8, max_iter=40000)
    ea = relative_l2(xa.cpu().numpy(), xr)
    ep = relative_l2(xp.cpu().numpy(), xr)
    assert ea < 1e-3 and ep < 1e-3, (ea, ep)
    assert masked.active_subdomains().sum() == 8
    masked.close()
    plain.close()


def test_activation_is_refused_where_it_does_not_apply():
    import paper_2410_02395_gb300 as pkg

    n = torch.ones(SHAPE, dtype=torch.complex64, device="cuda")
    for bad in (dict(residual_form=True), dict(plain_steps=True)):
        with pytest.raises(pkg.MBSError) as ei:
            pkg.Plan(SHAPE, 0.25, 1.0, n, activation=True, **KW, **bad)
        assert ei.value.status == 1
    kw0 = dict(KW, truncation=0)
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Plan(SHAPE, 0.25, 1.0, n, activation=True, **kw0)
    assert ei.value.status == 8
    plan = pkg.Plan(SHAPE, 0.25, 1.0, n, activation=True, **KW)
    with pytest.raises(pkg.MBSError) as ei:
        pkg.Batch([plan])
    assert ei.value.status == 1
    # a warm start activates every subdomain
    plan.set_source(torch.from_numpy(point_source(SHAPE, SRC)).cuda())
    assert plan.active_subdomains().sum() == 1
    plan.set_initial_field(torch.zeros(SHAPE, dtype=torch.complex64, device="cuda"))
    assert plan.active_subdomains().sum() == 8
    plan.close()
