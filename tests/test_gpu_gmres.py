"""Flexible restarted GMRES as the inner solver of the mixed solve
(sem_pcg_opts.krylov = SEM_KRYLOV_FGMRES) against the FP64 oracle: with the
Jacobi diagonal, the two-level and the three-level hybrid Schwarz
preconditioner, the solution of the oracle's tight solve to 1e-10 and the
oracle's true residual within the tolerance; the iteration count of one long
cycle against the oracle's own flexible GMRES with the same preconditioner;
short cycles (many restarts) still converge; bad options are rejected."""
import numpy as np
import pytest

import oracle
from oracle import schwarz as sw
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import _dev, _host, _rel

pytestmark = pytest.mark.gpu

CASES = [inputs.channel(4, 7), inputs.deformed_cube(4, 5),
         inputs.BoxCase("n3_per", 3, (4, 3, 3), (1, 0, 1), inputs.Y_FACES, jitter=0.1, seed=3),
         # 27 x 125 = 3375 local points: not a multiple of 4 (the float4 passes' scalar tail)
         inputs.BoxCase("n4_odd", 4, (3, 3, 3), (0, 0, 0), inputs.ALL_FACES, jitter=0.1, seed=6)]
IDS = [c.name for c in CASES]


def _setup(case, mid=None):
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V, mid_order=mid, mid_weight=0.15)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    keep = [gc]
    kw = dict(schwarz=S, coarse_iters=3, coarse_tol=1e-2)
    if mid:
        gmid = binding.Mesh(mid, case.nel, case.periodic, case.faces, V, geom_f32=True)
        keep.append(gmid)
        kw.update(schwarz_mid=binding.Schwarz(gmid, gc), mid_weight=0.15)
    return H, gm, kw, keep


@pytest.mark.parametrize("prec", ["jacobi", "schwarz2", "schwarz3"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fgmres_matches_oracle(case, prec):
    H, gm, kw, keep = _setup(case, mid=3 if prec == "schwarz3" and case.N > 3 else None)
    if prec == "jacobi":
        kw = {}
    om = H.m
    b = om.scatter(case.rhs_global())
    xo, _, _, so = om.pcg(b, tol=1e-13, max_iter=20000)
    assert so == 0
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3,
                    krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=40, check_every=8, **kw)
    assert st["status"] == 0, st
    assert st["rel_res"] <= 1e-12
    assert _rel(_host(xg), xo) <= 1e-10
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-12
    if prec != "jacobi":
        # about as many iterations as flexible CG with the same preconditioner
        _, sc = gm.pcg(_dev(b), tol=1e-12, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3,
                       check_every=8, **kw)
        assert st["iters"] <= 1.3 * sc["iters"] + 2, (st["iters"], sc["iters"])


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_one_cycle_iterations_match_oracle_fgmres(case):
    """A single long cycle (inner tolerance equal to the outer one, within
    FP32 reach) is plain flexible GMRES: its iterations to 1e-5 match the
    oracle's FP64 flexible GMRES with the FP64 hybrid Schwarz preconditioner
    (coarse level solved to convergence on both sides) within the FP32
    differences (+-20 %, and at most 3)."""
    H, gm, kw, keep = _setup(case)
    kw.update(coarse_iters=150, coarse_tol=1e-7)
    om = H.m
    b = om.scatter(case.rhs_global())
    _, it_o, rel_o = sw.fgmres(om, b, H.apply, restart=100, tol=1e-5, max_iter=100)
    assert rel_o <= 1e-5
    _, st = gm.pcg(_dev(b), tol=1e-5, max_iter=100, precision=binding.SEM_PCG_MIXED, inner_tol=1e-5,
                   krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=100, check_every=4, **kw)
    assert st["status"] == 0, st
    assert st["outer_iters"] == 1, st
    assert abs(st["iters"] - it_o) <= max(3, 0.2 * it_o), (st["iters"], it_o)


def test_short_cycles_restart_and_converge():
    case = inputs.deformed_cube(4, 5)
    H, gm, kw, keep = _setup(case)
    om = H.m
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-10, max_iter=50000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3,
                    krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=3, check_every=2, **kw)
    assert st["status"] == 0, st
    assert st["outer_iters"] >= 4
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.05e-10


def test_zero_rhs_and_bad_options():
    import torch
    case = inputs.deformed_cube(3, 3)
    H, gm, kw, keep = _setup(case)
    b = torch.zeros(gm.nloc, dtype=torch.float64, device="cuda")
    x, st = gm.pcg(b, precision=binding.SEM_PCG_MIXED, krylov=binding.SEM_KRYLOV_FGMRES, **kw)
    assert st["status"] == 0 and float(x.abs().max()) == 0.0
    b = _dev(H.m.scatter(case.rhs_global()))
    for bad, code in ((dict(krylov=2), binding.SEM_ERR_INVALID_ARG),
                      (dict(krylov=1, gmres_restart=129), binding.SEM_ERR_INVALID_ARG),
                      (dict(krylov=1, gmres_restart=-1), binding.SEM_ERR_INVALID_ARG)):
        with pytest.raises(binding.SemError) as ei:
            gm.pcg(b, precision=binding.SEM_PCG_MIXED, **bad)
        assert ei.value.status == code, bad
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, precision=binding.SEM_PCG_F64, krylov=binding.SEM_KRYLOV_FGMRES)
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED
    with pytest.raises(binding.SemError) as ei:
        binding.pcg_solve_batched([gm], [b], krylov=binding.SEM_KRYLOV_FGMRES)
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED


@pytest.mark.slow
def test_full_size_fgmres_schwarz_true_residual():
    """The 32^3 channel (16.8 M local points), three-level Schwarz FGMRES:
    the oracle's true residual of the solution meets the tolerance."""
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gmid = binding.Mesh(3, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S, Smid = binding.Schwarz(gm, gc), binding.Schwarz(gmid, gc)
    b = gm.scatter(_dev(case.rhs_global()))
    x, st = gm.pcg(b, tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2, check_every=8,
                   schwarz=S, coarse_iters=3, coarse_tol=1e-2, schwarz_mid=Smid, mid_weight=0.15,
                   krylov=binding.SEM_KRYLOV_FGMRES, gmres_restart=30, inner_adapt=0.5)
    assert st["status"] == 0, st
    xh, bh = _host(x), _host(b)
    del x, b, S, Smid, gm, gc, gmid
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    r = bh - om.apply(xh)
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(bh, bh)) <= 1.05e-8


def test_nan_rhs_and_converged_guess():
    """A NaN in the right-hand side is reported as SEM_ERR_NAN; a guess that
    already meets the tolerance returns at once with no inner iteration."""
    import torch
    case = inputs.deformed_cube(3, 5)
    H, gm, kw, keep = _setup(case)
    om = H.m
    b = om.scatter(case.rhs_global())
    bn = b.copy()
    bn[len(bn) // 2] = np.nan
    _, st = gm.pcg(_dev(bn), precision=binding.SEM_PCG_MIXED, krylov=binding.SEM_KRYLOV_FGMRES,
                   raise_on_error=False, **kw)
    assert st["status"] == binding.SEM_ERR_NAN, st
    xo, _, _, so = om.pcg(b, tol=1e-13, max_iter=20000)
    assert so == 0
    x, st = gm.pcg(_dev(b), torch.from_numpy(xo.copy()).cuda(), tol=1e-8, precision=binding.SEM_PCG_MIXED,
                   krylov=binding.SEM_KRYLOV_FGMRES, **kw)
    assert st["status"] == 0 and st["iters"] == 0 and st["outer_iters"] == 0, st
