"""The hybrid Schwarz preconditioner (sem_schwarz_apply, FP32) against the
FP64 oracle (oracle/schwarz.py), and the solves that use it: FP64 refinement
around flexible FP32 CG preconditioned by it (solutions and true residuals
against the oracle, fewer iterations than Jacobi, error paths, the 32^3
channel), and the FP32-pair outer residual option of the mixed solver.

Bar: FP32 data and arithmetic through six 1-D contractions, a division by the
eigenvalue sums and the overlap sums: 1e-4 relative 2-norm (the local
operators of stretched cells have eigenvalue spreads of ~1e4, which the FP32
eigenvectors carry into the result); the coarse level with its CG iterated to
convergence.  Copies of a node are bit-identical (fixed summation order)."""
import numpy as np
import pytest

import oracle
from oracle import schwarz as sw
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import _dev, _host, _rel

pytestmark = pytest.mark.gpu

SW_TOL = 1e-4

SW_CASES = [
    inputs.BoxCase("stretch", 3, (3, 4, 3), (1, 0, 1), inputs.Y_FACES, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5),
                   tanh_beta=(0.0, 2.0, 0.0)),
    inputs.deformed_cube(3, 4),
    inputs.channel(4, 7),
    inputs.BoxCase("n2_jit", 2, (3, 3, 2), (0, 0, 1), 0b001111, jitter=0.1, seed=4),
    inputs.BoxCase("n4_x1", 4, (1, 3, 2), (1, 0, 1), inputs.Y_FACES),
]
IDS = [c.name for c in SW_CASES]


def _setup(case):
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    return H, gm, gc, S


def _rhs(H):
    m = H.m
    r = m.apply_mask(m.scatter(np.random.default_rng(9).standard_normal(m.nglob)))
    return r.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("case", SW_CASES, ids=IDS)
def test_schwarz_levels_match_oracle(case):
    import torch
    H, gm, gc, S = _setup(case)
    r = _rhs(H)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z0 = _host(S.apply(rt, coarse_iters=0)).astype(np.float64)
    ref0 = H.m.apply_mask(H.sw.apply(r))
    assert _rel(z0, ref0) <= SW_TOL
    z1 = _host(S.apply(rt, coarse_iters=400, coarse_tol=1e-9)).astype(np.float64)
    assert _rel(z1, H.apply(r)) <= SW_TOL
    # continuity: every copy of a node holds the same bits; Dirichlet nodes 0
    one = np.zeros(H.m.nglob)
    one[H.m.gid] = z1
    np.testing.assert_array_equal(z1, one[H.m.gid])
    assert np.all(z1[H.m.apply_mask(np.ones(H.m.nloc)) == 0] == 0)


def test_schwarz_rejects_wrong_coarse_mesh():
    case = SW_CASES[0]
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    wrong = binding.Mesh(2, case.nel, case.periodic, case.faces, V, geom_f32=True)
    with pytest.raises(binding.SemError) as ei:
        binding.Schwarz(gm, wrong)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


# ------------------------------------------------------------------ the preconditioned solve

SOLVE_CASES = [SW_CASES[0], SW_CASES[2], SW_CASES[3], SW_CASES[4], inputs.deformed_cube(5, 5)]
SOLVE_IDS = [c.name for c in SOLVE_CASES]


@pytest.mark.parametrize("coarse_iters", [0, 5], ids=["one_level", "two_level"])
@pytest.mark.parametrize("case", SOLVE_CASES, ids=SOLVE_IDS)
def test_pcg_schwarz_matches_oracle(case, coarse_iters):
    """FP64 refinement around flexible FP32 CG with the hybrid Schwarz
    preconditioner: the solution of the FP64 oracle's solve to 1e-10, the
    reported residual the true one, and fewer inner iterations than the
    Jacobi-preconditioned mixed solve."""
    H, gm, gc, S = _setup(case)
    om = H.m
    b = om.scatter(case.rhs_global())
    xo, _, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4,
                    schwarz=S, coarse_iters=coarse_iters, coarse_tol=1e-3)
    assert sto == 0 and st["status"] == 0, st
    assert st["rel_res"] <= 1e-12
    assert _rel(_host(xg), xo) <= 1e-10
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-12
    _, sj = gm.pcg(_dev(b), tol=1e-12, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4)
    assert st["iters"] < sj["iters"], (st["iters"], sj["iters"])


def test_pcg_schwarz_zero_rhs_and_wrong_mesh():
    case = SW_CASES[0]
    H, gm, gc, S = _setup(case)
    import torch
    b = torch.zeros(gm.nloc, dtype=torch.float64, device="cuda")
    x, st = gm.pcg(b, tol=1e-10, precision=binding.SEM_PCG_MIXED, schwarz=S, coarse_iters=5)
    assert st["status"] == 0 and st["iters"] == 0
    assert float(x.abs().max()) == 0.0
    other = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
    with pytest.raises(binding.SemError) as ei:
        other.pcg(b + 1.0, tol=1e-10, precision=binding.SEM_PCG_MIXED, schwarz=S)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b + 1.0, tol=1e-10, schwarz=S)  # FP64 solver: Jacobi only
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED


def test_full_size_pcg_schwarz_true_residual():
    """The 32^3 channel (N = 7) to 1e-8: oracle-computed true residual, and
    several times fewer inner iterations than with Jacobi."""
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                    schwarz=S, coarse_iters=5, coarse_tol=1e-2)
    assert st["status"] == 0
    r = b - om.apply(_host(xg))
    rel = np.sqrt(om.glsc3(r, r) / om.glsc3(b, b))
    assert rel <= 1.05e-8, rel
    assert st["iters"] < 200, st["iters"]


# ------------------------------------------------------------------ FP32-pair outer residual

@pytest.mark.parametrize("case", [inputs.channel(5, 7), inputs.deformed_cube(4, 5)], ids=["channel5", "deformed4"])
@pytest.mark.parametrize("use_schwarz", [False, True], ids=["jacobi", "schwarz"])
def test_pcg_mixed_outer_pair_true_residual(case, use_schwarz):
    """The mixed solver with its FP64 outer residual formed by the FP32-pair
    operator: the oracle-computed true residual meets the tolerance and the
    solution matches the FP64 oracle's."""
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_pair=True)
    kw = {}
    if use_schwarz:
        gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
        kw = dict(schwarz=binding.Schwarz(gm, gc), coarse_iters=3)
    b = om.scatter(case.rhs_global())
    xo, _, _, _ = om.pcg(b, tol=1e-12, max_iter=20000)
    xg, st = gm.pcg(_dev(b), tol=1e-10, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3,
                    outer_pair=True, **kw)
    assert st["status"] == 0, st
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.05e-10
    assert _rel(_host(xg), xo) <= 1e-8


def test_pcg_outer_pair_needs_pair_geometry():
    case = SW_CASES[0]
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
    import torch
    b = torch.ones(gm.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, tol=1e-8, precision=binding.SEM_PCG_MIXED, outer_pair=True)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


def test_full_size_pcg_schwarz_outer_pair_true_residual():
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_pair=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                    schwarz=S, coarse_iters=3, coarse_tol=1e-2, outer_pair=True)
    assert st["status"] == 0
    r = b - om.apply(_host(xg))
    rel = np.sqrt(om.glsc3(r, r) / om.glsc3(b, b))
    assert rel <= 1.05e-8, rel


# ------------------------------------------------------------------ the intermediate multigrid level

MID_CASES = [(inputs.channel(4, 7), 3), (inputs.deformed_cube(3, 5), 3), (SW_CASES[0], 2),
             (inputs.BoxCase("n9", 9, (2, 3, 2), (0, 1, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=5), 4)]
MID_IDS = [f"{c.name}_M{M}" for c, M in MID_CASES]


def _setup_mid(case, M):
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V, mid_order=M, mid_weight=0.15)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gmid = binding.Mesh(M, case.nel, case.periodic, case.faces, V, geom_f32=True)
    return H, gm, binding.Schwarz(gm, gc), binding.Schwarz(gmid, gc), gc, gmid


@pytest.mark.parametrize("case,M", MID_CASES, ids=MID_IDS)
def test_schwarz_three_levels_match_oracle(case, M):
    """z = S_N r + 0.15 P_M S_M P_M^T r + coarse (sem_schwarz_apply3) against
    the oracle's three-level preconditioner, at the two-level bar; copies
    bit-identical and Dirichlet nodes 0."""
    import torch
    H, gm, S, Smid, gc, gmid = _setup_mid(case, M)
    r = _rhs(H)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z = _host(S.apply3(Smid, rt, mid_weight=0.15, coarse_iters=400, coarse_tol=1e-9)).astype(np.float64)
    assert _rel(z, H.apply(r)) <= SW_TOL
    one = np.zeros(H.m.nglob)
    one[H.m.gid] = z
    np.testing.assert_array_equal(z, one[H.m.gid])
    assert np.all(z[H.m.apply_mask(np.ones(H.m.nloc)) == 0] == 0)


@pytest.mark.parametrize("case,M", MID_CASES[:2], ids=MID_IDS[:2])
def test_pcg_schwarz_three_levels_matches_oracle(case, M):
    """The mixed solver with the three-level preconditioner: the FP64
    oracle's solution to 1e-10 at tau = 1e-12, the true residual, and on the
    channel fewer inner iterations than with two levels."""
    H, gm, S, Smid, gc, gmid = _setup_mid(case, M)
    om = H.m
    b = om.scatter(case.rhs_global())
    xo, _, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    kw = dict(tol=1e-12, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4, schwarz=S,
              coarse_iters=5, coarse_tol=1e-3)
    xg, st = gm.pcg(_dev(b), schwarz_mid=Smid, mid_weight=0.15, **kw)
    assert sto == 0 and st["status"] == 0, st
    assert _rel(_host(xg), xo) <= 1e-10
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-12
    if case.name == "channel":
        _, s2 = gm.pcg(_dev(b), **kw)
        assert st["iters"] < s2["iters"], (st["iters"], s2["iters"])


def test_full_size_pcg_schwarz_three_levels_true_residual():
    """The 32^3 channel (N = 7) to 1e-8 with the three-level preconditioner
    (intermediate order 3, weight 0.15): oracle-computed true residual, and
    fewer inner iterations than with two levels."""
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gmid = binding.Mesh(3, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S, Smid = binding.Schwarz(gm, gc), binding.Schwarz(gmid, gc)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    kw = dict(tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2, schwarz=S,
              coarse_iters=3, coarse_tol=1e-2, check_every=8)
    xg, st = gm.pcg(_dev(b), schwarz_mid=Smid, mid_weight=0.15, **kw)
    assert st["status"] == 0
    r = b - om.apply(_host(xg))
    rel = np.sqrt(om.glsc3(r, r) / om.glsc3(b, b))
    assert rel <= 1.05e-8, rel
    _, s2 = gm.pcg(_dev(b), **kw)
    assert st["iters"] < s2["iters"], (st["iters"], s2["iters"])


def test_schwarz_three_levels_reject_mismatched_mid():
    case = inputs.channel(3, 5)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    other = inputs.channel(4, 3)
    go = binding.Mesh(3, other.nel, other.periodic, other.faces, other.vertices(), geom_f32=True)
    goc = binding.Mesh(1, other.nel, other.periodic, other.faces, other.vertices(), geom_f32=True)
    bad = binding.Schwarz(go, goc)
    b = _dev(np.zeros(gm.nloc))
    for mid in (bad, S):  # other elements; same order
        with pytest.raises(binding.SemError) as ei:
            gm.pcg(b + 1.0, precision=binding.SEM_PCG_MIXED, schwarz=S, schwarz_mid=mid)
        assert ei.value.status == binding.SEM_ERR_INVALID_ARG
