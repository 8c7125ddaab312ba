"""Batches of independent solves: one graph over several plans gives exactly the
iterates and iteration counts of the plans run one by one, and each batched solve
matches the FP64 oracle on its own grid at equal iteration counts."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import Problem, relative_l2  # noqa: E402
from synth import frequency_batch  # noqa: E402


def _plans(problems, **kw):
    import paper_2410_02395_gb300 as pkg

    out = []
    for params, n, src in problems:
        p = pkg.Plan(params["shape"], params["pixel"], params["wavelength"], torch.from_numpy(n).cuda(),
                     boundary_widths=params["widths"], split=params["split"], truncation=params["t"],
                     periodic=params["periodic"], split_sizes=params["split_sizes"], **kw)
        p.set_source(torch.from_numpy(src).cuda())
        out.append(p)
    return out


@pytest.fixture(scope="module")
def problems():
    return frequency_batch(count=4, seed=7, box=7.0, spheres=5, r_range=(0.5, 1.5), t=4)


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("n_iter", [7, 25])
def test_batch_equals_individual_plans(problems, n_iter, fused):
    """Both forms of the batch: one launch per pass and edge over all plans, and a
    graph of every plan's own launches."""
    import paper_2410_02395_gb300 as pkg

    assert len({p["shape"] for p, _, _ in problems}) > 1  # uneven grids in one batch
    batched = _plans(problems)
    b = pkg.Batch(batched, graph_iters=10, fused=fused)
    assert b.launches_per_iteration()[1] == fused
    res = b.iterate(n_iter, 0.0, no_poll=True)
    assert [r[1] for r in res] == [n_iter] * len(problems)
    single = _plans(problems)
    for pb, ps in zip(batched, single):
        ps.iterate(n_iter, 0.0)
        xb = pb.field(like=torch.zeros(1, device="cuda"))
        xs = ps.field(like=torch.zeros(1, device="cuda"))
        assert torch.equal(xb, xs)
        np.testing.assert_array_equal(pb.history(n_iter), ps.history(n_iter))
    b.close()
    for p in batched + single:
        p.close()


def test_batch_solves_each_to_its_own_tolerance(problems):
    import paper_2410_02395_gb300 as pkg

    batched = _plans(problems)
    b = pkg.Batch(batched, graph_iters=10)
    res = b.iterate(5000, 1e-5)
    single = _plans(problems)
    for (st, it, eps), ps in zip(res, single):
        st1, it1, eps1 = ps.iterate(5000, 1e-5)
        assert st == st1 == "MBS_OK"
        assert it == it1 and eps == eps1 and eps < 1e-5
    # a new source on one plan is picked up by the batch (graphs are captured again)
    params, n, src = problems[0]
    batched[0].set_source(torch.from_numpy(2 * src).cuda())
    res2 = b.iterate(5000, 1e-5)
    assert res2[0][1] == res[0][1]  # linear problem: same iteration count for a scaled source
    x = batched[0].field(like=torch.zeros(1, device="cuda"))
    single[0].set_source(torch.from_numpy(src).cuda())
    single[0].iterate(5000, 1e-5)
    x1 = single[0].field(like=torch.zeros(1, device="cuda"))
    assert torch.allclose(x, 2 * x1, rtol=1e-5, atol=1e-9)
    b.close()
    for p in batched + single:
        p.close()


@pytest.mark.parametrize("form", ["x", "residual", "tf32"])
def test_batched_solves_match_the_oracle(problems, form):
    """Every solve of the batch (uneven grids, explicit uneven subdomain sizes)
    against the oracle at 30 iterations (3 replays of a graph of 10)."""
    import paper_2410_02395_gb300 as pkg

    kw = {"residual_form": form == "residual", "corr_tf32": form == "tf32"}
    batched = _plans(problems, **kw)
    b = pkg.Batch(batched, graph_iters=10)
    res = b.iterate(30, 0.0, no_poll=True)
    for (params, n, src), p, r in zip(problems, batched, res):
        assert r[1] == 30
        ref = Problem(n, params["pixel"], params["wavelength"], widths=params["widths"], split=params["split"],
                      periodic=params["periodic"], t=params["t"], split_sizes_=params["split_sizes"])
        xr, itr, histr = ref.solve(src, tol=0.0, max_iter=30)
        x = p.field(like=torch.zeros(1, device="cuda")).cpu().numpy()
        assert relative_l2(x, xr) < 1e-4, (params["shape"], relative_l2(x, xr))
        np.testing.assert_allclose(p.history(30), histr, rtol=1e-4, atol=1e-6)
    b.close()
    for p in batched:
        p.close()


def test_batch_of_x_form_plans_runs_fused(problems):
    """The x-form plans with mixed-radix edges run as one launch per pass and edge
    over all plans: far fewer launches per iteration than the plans' own."""
    import paper_2410_02395_gb300 as pkg

    plans = _plans(problems)
    b = pkg.Batch(plans, graph_iters=10)
    n, fused = b.launches_per_iteration()
    assert fused
    own = pkg.Batch(_plans(problems, corr_tf32=True), graph_iters=10)  # not fusable: each plan's launches
    n_own, fused_own = own.launches_per_iteration()
    assert not fused_own and n < n_own
    own.close()
    b.close()
    for p in plans:
        p.close()
