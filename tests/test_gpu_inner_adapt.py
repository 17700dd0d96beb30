"""The adaptive inner tolerance of the mixed solver (sem_pcg_opts.inner_adapt):
a refinement round that starts near the outer target stops once the target
is within reach.  Whatever the inner tolerance, the FP64 true residual
decides convergence, so every solution here is checked by the oracle's own
residual; from a guess whose residual is three times the target, the adapted
round needs fewer FP32 iterations than a full reduction by inner_tol."""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-8


def _t():
    import torch
    return torch


def _setup(case):
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    return om, gm


def _rel_res(om, b, x):
    r = b - om.apply(x)
    return float(np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)))


def _near_guess(om, case, b, factor, seed=5):
    """x0 = x* + s e: x* a tight oracle solution, e a continuous random
    field (zero on Dirichlet nodes), s chosen so that the relative residual
    of x0 is `factor` times TOL."""
    xo, _, _, so = om.pcg(b, tol=1e-13, max_iter=20000)
    assert so == 0
    g = np.random.default_rng(seed).standard_normal(case.rhs_global().shape)
    e = om.apply_mask(om.scatter(g))
    re = om.apply(e)
    s = factor * TOL * np.sqrt(om.glsc3(b, b) / om.glsc3(re, re))
    return xo + s * e


@pytest.mark.parametrize("schwarz", [False, True], ids=["jacobi", "schwarz"])
def test_near_guess_adapted_round_is_shorter(schwarz):
    torch = _t()
    case = inputs.channel(5, 7)
    om, gm = _setup(case)
    b = om.scatter(case.rhs_global())
    x0 = _near_guess(om, case, b, 3.0)
    assert 2.5 < _rel_res(om, b, x0) / TOL < 3.5
    kw = dict(tol=TOL, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2, check_every=8)
    if schwarz:
        gc = binding.Mesh(1, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
        kw.update(schwarz=binding.Schwarz(gm, gc), coarse_iters=3, coarse_tol=1e-2)
    bd = torch.from_numpy(b).cuda()
    res = {}
    for theta in (0.0, 0.5):
        x, st = gm.pcg(bd, torch.from_numpy(x0.copy()).cuda(), inner_adapt=theta, **kw)
        assert st["status"] == 0, st
        assert st["outer_iters"] == 1, st
        rel = _rel_res(om, b, x.cpu().numpy())
        assert rel <= 1.05 * TOL, (theta, rel)
        assert abs(st["rel_res"] - rel) <= 1e-3 * TOL
        res[theta] = st["iters"]
    assert res[0.5] < res[0.0], res


def test_far_start_keeps_inner_tol_until_the_last_round():
    """From x = 0 the first rounds reduce by inner_tol as before; only the
    last round, whose remaining reduction is smaller than inner_tol, is
    shortened."""
    torch = _t()
    case = inputs.deformed_cube(4, 5)
    om, gm = _setup(case)
    b = om.scatter(case.rhs_global())
    bd = torch.from_numpy(b).cuda()
    out = {}
    for theta in (0.0, 0.5):
        x, st = gm.pcg(bd, tol=TOL, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3,
                       check_every=4, inner_adapt=theta)
        assert st["status"] == 0, st
        assert _rel_res(om, b, x.cpu().numpy()) <= 1.05 * TOL
        out[theta] = st
    assert out[0.5]["iters"] <= out[0.0]["iters"], (out[0.5]["iters"], out[0.0]["iters"])


def test_batched_rounds_adapt_per_solve():
    torch = _t()
    cases = [inputs.BoxCase("a", 5, (3, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=1),
             inputs.BoxCase("b", 7, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=2),
             inputs.channel(3, 7)]
    meshes, oms, bs = [], [], []
    for c in cases:
        om, gm = _setup(c)
        meshes.append(gm)
        oms.append(om)
        bs.append(torch.from_numpy(om.scatter(c.rhs_global())).cuda())
    its = {}
    for theta in (0.0, 0.5):
        xs, stats = binding.pcg_solve_batched(meshes, bs, tol=TOL, max_iter=20000, inner_tol=1e-3, check_every=4,
                                              inner_adapt=theta)
        for i, (om, st) in enumerate(zip(oms, stats)):
            assert st["status"] == 0, (theta, i, st)
            assert _rel_res(om, bs[i].cpu().numpy(), xs[i].cpu().numpy()) <= 1.05 * TOL
        its[theta] = sum(st["iters"] for st in stats)
    assert its[0.5] <= its[0.0], its


@pytest.mark.parametrize("theta", [-0.1, 1.0, float("nan")])
def test_inner_adapt_out_of_range_rejected(theta):
    torch = _t()
    case = inputs.deformed_cube(2, 3)
    om, gm = _setup(case)
    b = torch.from_numpy(om.scatter(case.rhs_global())).cuda()
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, precision=binding.SEM_PCG_MIXED, inner_adapt=theta)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
