"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: integer/index work and the gather-scatter (pure additions in the same
ascending order) are bit-exact; the FP64 operator is within 1e-12 in the
relative 2-norm (pointwise relative error is meaningless where A u ~ 0); the
converged CG solution within 1e-10 relative when both sides converge to a
tight 1e-12 residual (two correct CG runs at residual tau differ by up to
~kappa tau, so the gate uses a tolerance where that bound is far below 1e-10).
"""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

AX_TOL = 1e-12
SOL_TOL = 1e-10


def _torch():
    import torch
    return torch


def _pair(case, geom_f32=False):
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=geom_f32)
    return om, gm


def _dev(a):
    return _torch().from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    _torch().cuda.synchronize()
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    inputs.BoxCase("n1_single", 1, (1, 1, 1), (0, 0, 0), 0),
    inputs.BoxCase("n2_jitter", 2, (3, 2, 2), (0, 0, 0), inputs.ALL_FACES, jitter=0.15, seed=1),
    inputs.BoxCase("n3_periodic1", 3, (1, 2, 3), (1, 0, 1), inputs.Y_FACES, jitter=0.1, seed=2),
    inputs.BoxCase("n4_even", 4, (2, 3, 2), (0, 1, 0), inputs.ALL_FACES, perturb_amp=0.2, seed=3),
    inputs.BoxCase("n5_deformed", 5, (5, 4, 3), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=4),
    inputs.channel(6, 7),
    inputs.BoxCase("n7_ragged", 7, (13, 11, 7), (0, 0, 1), 0b000011, perturb_amp=0.05, seed=5),
    inputs.BoxCase("n9_deformed", 9, (4, 3, 5), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=6),
    inputs.BoxCase("n11_deformed", 11, (3, 3, 2), (1, 1, 0), 0b110000, jitter=0.1, seed=7),
]
IDS = [c.name for c in CASES]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_geometry_and_mesh_arrays(case):
    om, gm = _pair(case)
    xyz = _host(gm.coords())
    np.testing.assert_allclose(xyz, om.xyz, rtol=0, atol=1e-14 * max(1.0, np.abs(om.xyz).max()))
    for c in range(6):
        g = _host(gm.field(3 + c)).reshape(om.E, -1)
        scale = np.abs(om.G[:, :3]).max()
        np.testing.assert_allclose(g, om.G[:, c], rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(_host(gm.field(binding.FIELD_MASS)), om.B.reshape(-1), rtol=1e-12)
    np.testing.assert_array_equal(_host(gm.field(binding.FIELD_MULT)), om.mult)
    np.testing.assert_allclose(_host(gm.field(binding.FIELD_DINV)), om.dinv, rtol=1e-12, atol=0)
    assert gm.nglob == om.nglob


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_ax_f64_matches_oracle(case):
    om, gm = _pair(case)
    rng = np.random.default_rng(11)
    for u in (rng.standard_normal(om.nloc), om.scatter(rng.standard_normal(om.nglob))):
        w = _host(gm.ax(_dev(u)))
        assert _rel(w, om.ax_local(u)) <= AX_TOL


@pytest.mark.parametrize("case", CASES[:7], ids=IDS[:7])
def test_helmholtz_matches_oracle(case):
    om, gm = _pair(case)
    u = np.random.default_rng(3).standard_normal(om.nloc)
    for h1, h2 in ((1.0, 0.0), (0.00625, 1500.0), (0.0, 1.0), (2.5, 0.0)):
        w = _host(gm.helmholtz(h1, h2, _dev(u)))
        ref = oracle.helmholtz_local(om.N, om.D, om.G, om.B, h1, h2, u.reshape(om.E, -1)).reshape(-1)
        assert _rel(w, ref) <= AX_TOL


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_dssum_bit_exact(case):
    om, gm = _pair(case)
    u = np.random.default_rng(5).standard_normal(om.nloc)
    for mask in (False, True):
        t = _dev(u)
        gm.dssum(t, mask=mask)
        ref = om.dssum(u)
        if mask:
            ref = om.apply_mask(ref)
        np.testing.assert_array_equal(_host(t), ref)


@pytest.mark.parametrize("case", CASES[:6], ids=IDS[:6])
def test_scatter_and_inner_product(case):
    om, gm = _pair(case)
    rng = np.random.default_rng(8)
    ug = rng.standard_normal(om.nglob)
    ul = _host(gm.scatter(_dev(ug)))
    np.testing.assert_array_equal(ul, om.scatter(ug))
    a, b = om.scatter(rng.standard_normal(om.nglob)), om.scatter(rng.standard_normal(om.nglob))
    ref = om.glsc3(a, b)
    assert abs(gm.glsc3(_dev(a), _dev(b)) - ref) <= 1e-13 * (np.abs(a * b / om.mult).sum())


def _manufactured_rhs(om):
    x, y, z = om.xyz
    f = inputs.manufactured_f(x, y, z).reshape(-1)
    return om.apply_mask(om.dssum(om.B.reshape(-1) * f))


def test_pcg_cube_manufactured_matches_oracle():
    case = inputs.cube_manufactured(4, 7)
    om, gm = _pair(case)
    b = _manufactured_rhs(om)
    # the GPU path builds its own right-hand side from its own mass and coordinates
    xyz = gm.coords()
    f = _dev(inputs.manufactured_f(*_host(xyz)).reshape(-1))
    bg = gm.helmholtz(0.0, 1.0, f)
    gm.dssum(bg, mask=True)
    assert _rel(_host(bg), b) <= 1e-13
    xo, ito, rro, sto = om.pcg(b, tol=1e-12, max_iter=5000)
    xg, st = gm.pcg(bg, tol=1e-12, max_iter=5000, check_every=8)
    assert sto == 0 and st["status"] == 0
    assert st["rel_res"] <= 1e-12
    assert _rel(_host(xg), xo) <= SOL_TOL
    assert abs(st["iters"] - ito) <= max(3, ito // 20)
    # the paper-independent check: the discrete solution approximates u*
    x, y, z = om.xyz
    assert np.abs(_host(xg) - inputs.manufactured_u(x, y, z).reshape(-1)).max() < 1e-5


@pytest.mark.parametrize("case", [inputs.channel(5, 7), inputs.deformed_cube(6, 5),
                                  inputs.BoxCase("n9", 9, (3, 4, 3), (0, 0, 0), inputs.ALL_FACES,
                                                 perturb_amp=0.05, seed=2)], ids=["channel5", "deformed6", "n9"])
def test_pcg_random_rhs_matches_oracle(case):
    om, gm = _pair(case)
    b = om.scatter(case.rhs_global())
    xo, ito, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=20000)
    assert sto == 0 and st["status"] == 0
    assert _rel(_host(xg), xo) <= SOL_TOL
    # x is continuous: every copy of a node holds the same value
    xh = _host(xg)
    one = np.zeros(om.nglob)
    one[om.gid] = xh
    np.testing.assert_array_equal(xh, one[om.gid])


# Topologies that stress the axis-by-axis gather-scatter of the CG loop: a
# single periodic element along x (its two x faces are one node layer), odd
# N + 1 (no vector loads), N = 2 .. 11, periodic axes mixed with Dirichlet
# faces on the others.
TOPO = [c for c in CASES if c.name in ("n2_jitter", "n3_periodic1", "n4_even", "n7_ragged", "n11_deformed")]


@pytest.mark.parametrize("mixed", [False, True], ids=["f64", "mixed"])
@pytest.mark.parametrize("case", TOPO, ids=[c.name for c in TOPO])
def test_pcg_topologies_match_oracle(case, mixed):
    om, gm = _pair(case, geom_f32=mixed)
    b = om.scatter(case.rhs_global())
    xo, _, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    kw = dict(precision=binding.SEM_PCG_MIXED, inner_tol=1e-4) if mixed else {}
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=20000, **kw)
    assert sto == 0 and st["status"] == 0, st
    xh = _host(xg)
    assert _rel(xh, xo) <= SOL_TOL
    one = np.zeros(om.nglob)
    one[om.gid] = xh
    np.testing.assert_array_equal(xh, one[om.gid])


def test_pcg_initial_guess_and_absolute_tolerance():
    case = inputs.deformed_cube(4, 5)
    om, gm = _pair(case)
    b = om.scatter(case.rhs_global())
    xo, *_ = om.pcg(b, tol=1e-13, max_iter=20000)
    x0 = _dev(xo * (1 + 1e-6))
    xg, st = gm.pcg(_dev(b), x=x0, tol=1e-12, max_iter=20000)
    _, st0 = gm.pcg(_dev(b), tol=1e-12, max_iter=20000)
    assert st["status"] == 0 and st["iters"] < 0.75 * st0["iters"]
    assert _rel(_host(xg), xo) <= SOL_TOL
    xg2, st2 = gm.pcg(_dev(b), tol=1e-9, relative=False, max_iter=20000)
    assert st2["abs_res"] <= 1e-9


def test_pcg_error_paths():
    case = inputs.deformed_cube(3, 3)
    om, gm = _pair(case)
    b = om.scatter(case.rhs_global())
    bad = b.copy()
    bad[17] = np.inf
    _, st = gm.pcg(_dev(bad), raise_on_error=False)
    assert st["status"] == binding.SEM_ERR_NAN
    x, st = gm.pcg(_dev(b), tol=1e-14, max_iter=3, raise_on_error=False)
    assert st["status"] == binding.SEM_ERR_NOT_CONVERGED and st["iters"] == 3
    # stats are still filled and consistent with a fresh residual
    assert st["rel_res"] > 1e-14
    assert gm.check_device_error() == 0


def test_bad_mesh_and_small_workspace_rejected():
    V = inputs.box_vertices((2, 1, 1))
    V[0, :, 0] *= -1.0
    with pytest.raises(binding.SemError) as ei:
        binding.Mesh(3, (2, 1, 1), (0, 0, 0), 0, V)
    assert ei.value.status == binding.SEM_ERR_MESH
    case = inputs.deformed_cube(3, 3)
    om, gm = _pair(case)
    opts = gm.pcg_opts()
    small = gm.pcg_scratch(opts)[:1024]
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(_dev(om.scatter(case.rhs_global())), scratch=small)
    assert ei.value.status == binding.SEM_ERR_WORKSPACE


# ------------------------------------------------------------------ full sizes
# The 32^3-element channel at N = 7 (16.8 M local points) in the launch
# configuration the benchmark times.  The oracle checks sampled elements (the
# operator is element-local) and sampled gather-scatter groups, and the
# converged solution through its own residual.


@pytest.fixture(scope="module")
def channel32():
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    return case, V, gm


@pytest.mark.slow
def test_full_size_ax_sampled_elements(channel32):
    case, V, gm = channel32
    rng = np.random.default_rng(21)
    u = rng.standard_normal(case.nloc)
    w = _host(gm.ax(_dev(u))).reshape(case.E, -1)
    sel = np.unique(np.concatenate([[0, case.E - 1], rng.integers(0, case.E, 300)]))
    _, G, _, st = oracle.geometry(case.N, V[sel])
    assert st == 0
    D = oracle.deriv(case.N)
    ref = oracle.ax_local(case.N, D, G, u.reshape(case.E, -1)[sel])
    assert _rel(w[sel], ref) <= AX_TOL


@pytest.mark.slow
def test_full_size_pcg_true_residual(channel32):
    case, V, gm = channel32
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-8, max_iter=20000)
    assert st["status"] == 0
    x = _host(xg)
    r = b - om.apply(x)
    rel = np.sqrt(om.glsc3(r, r) / om.glsc3(b, b))
    assert rel <= 1.05e-8, rel
    # dssum of the full-size field is still bit-exact against the oracle
    u = np.random.default_rng(4).standard_normal(case.nloc)
    t = _dev(u)
    gm.dssum(t, mask=True)
    np.testing.assert_array_equal(_host(t), om.apply_mask(om.dssum(u)))


# ------------------------------------------------------------------ FP32 operator and mixed precision
# FP32 storage and accumulation: the operator error is a few units of FP32
# rounding (2^-24 = 6e-8) times the ~3(N+1) terms of each contraction chain,
# so 5e-6 in the relative 2-norm bounds it for N <= 11.
F32_AX_TOL = 5e-6


@pytest.mark.parametrize("case", [c for c in CASES if c.N in (1, 3, 5, 7, 9, 11)],
                         ids=[c.name for c in CASES if c.N in (1, 3, 5, 7, 9, 11)])
def test_ax_f32_matches_oracle(case):
    torch = _torch()
    om, gm = _pair(case, geom_f32=True)
    u = np.random.default_rng(12).standard_normal(om.nloc).astype(np.float32)
    w = _host(gm.ax(torch.from_numpy(u).cuda())).astype(np.float64)
    assert _rel(w, om.ax_local(u.astype(np.float64))) <= F32_AX_TOL


@pytest.mark.parametrize("case", CASES[:7], ids=IDS[:7])
def test_dssum_f32(case):
    torch = _torch()
    om, gm = _pair(case, geom_f32=True)
    u = np.random.default_rng(6).standard_normal(om.nloc).astype(np.float32)
    t = torch.from_numpy(u).cuda()
    gm.dssum(t, mask=True)
    ref = om.apply_mask(om.dssum(u.astype(np.float64)))
    np.testing.assert_allclose(_host(t), ref, rtol=0, atol=4 * 2.0 ** -24 * 8 * np.abs(u).max())


@pytest.mark.parametrize("case", [inputs.channel(5, 7), inputs.deformed_cube(6, 5),
                                  inputs.BoxCase("n9", 9, (3, 4, 3), (0, 0, 0), inputs.ALL_FACES,
                                                 perturb_amp=0.05, seed=2)], ids=["channel5", "deformed6", "n9"])
def test_pcg_mixed_matches_oracle(case):
    om, gm = _pair(case, geom_f32=True)
    b = om.scatter(case.rhs_global())
    xo, ito, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4)
    assert sto == 0 and st["status"] == 0, st
    assert st["rel_res"] <= 1e-12 and st["outer_iters"] >= 2
    assert _rel(_host(xg), xo) <= SOL_TOL
    # the reported FP64 residual is the true one
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-12


def test_pcg_mixed_needs_f32_geometry_and_poisson():
    case = inputs.deformed_cube(3, 3)
    om, gm = _pair(case)
    b = _dev(om.scatter(case.rhs_global()))
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, precision=binding.SEM_PCG_MIXED)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    om, gm = _pair(case, geom_f32=True)
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, precision=binding.SEM_PCG_MIXED, h2=1.0)
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED


@pytest.mark.slow
def test_full_size_pcg_mixed_true_residual():
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4)
    assert st["status"] == 0
    r = b - om.apply(_host(xg))
    rel = np.sqrt(om.glsc3(r, r) / om.glsc3(b, b))
    assert rel <= 1.05e-8, rel


@pytest.mark.slow
def test_full_size_deformed64_mixed_true_residual():
    """The 64^3 deformed cube (134 M local points): the solutions of FP64
    refinement around FP32 Jacobi-PCG and around flexible FP32 CG with the
    hybrid Schwarz preconditioner (mean-edge-length local solves, approximate
    on deformed elements) have oracle-computed true residuals within the
    tolerance; the Schwarz solve needs fewer inner iterations."""
    case = inputs.deformed_cube(64, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    bg = case.rhs_global()
    b = _dev(bg)
    b = gm.scatter(b)
    x, st = gm.pcg(b, tol=1e-8, max_iter=100000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2, check_every=32)
    assert st["status"] == 0
    xs, sts = gm.pcg(b, tol=1e-8, max_iter=100000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                     check_every=8, schwarz=S, coarse_iters=3, coarse_tol=1e-2)
    assert sts["status"] == 0
    assert sts["iters"] < st["iters"], (sts["iters"], st["iters"])
    xh, xsh = _host(x), _host(xs)
    bh = _host(b)
    del x, xs, b, S, gc, gm
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    for sol in (xh, xsh):
        r = bh - om.apply(sol)
        rel = np.sqrt(om.glsc3(r, r) / om.glsc3(bh, bh))
        assert rel <= 1.05e-8, rel


def test_autotune_reports_and_keeps_the_fastest():
    """The autotuner times every launch shape of the operator -- FP32:
    pipeline depth x CTA cap x elements per CTA (N = 5: 36 of 64 threads of
    a one-element CTA have a line), FP64: CTA cap -- keeps the fastest in the
    launch table, and the operator stays correct under it."""
    torch = _torch()
    case = inputs.channel(6, 5)
    om, gm = _pair(case, geom_f32=True)
    try:
        for dt, cg, n in ((binding.SEM_F32, True, 36), (binding.SEM_F64, False, 4)):
            r = gm.autotune(dt, cg)
            assert len(r["table"]) == n
            best = min(r["table"], key=lambda t: t[3])
            assert (r["best_stages"], r["best_cap"], r["best_epc"]) == best[:3]
            assert r["best_ms"] == pytest.approx(best[3])
        u = np.random.default_rng(3).standard_normal(om.nloc)
        assert _rel(_host(gm.ax(_dev(u))), om.ax_local(u)) <= AX_TOL
    finally:
        binding.lib().sem_autotune_reset()


@pytest.mark.parametrize("epc", [2, 4])
@pytest.mark.parametrize("stages", [1, 2])
def test_fp32_operator_element_groups_match_oracle(epc, stages):
    """Block shapes of 2 and 4 elements per CTA (incl. a last group with
    fewer elements: E = 3 x 4 x 5 = 60 is not a multiple of 8 groups of 4 in
    a wave): the FP32 operator and the mixed solve against the oracle."""
    torch = _torch()
    for case in (inputs.BoxCase("g5", 5, (3, 4, 5), (0, 1, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=7),
                 inputs.BoxCase("g9", 9, (3, 1, 3), (1, 0, 0), inputs.Y_FACES, jitter=0.05, seed=8)):
        om, gm = _pair(case, geom_f32=True)
        try:
            gm.autotune_set(binding.SEM_F32, False, stages, 0, epc)
            gm.autotune_set(binding.SEM_F32, True, stages, 0, epc)
            u = np.random.default_rng(4).standard_normal(om.nloc)
            w = _host(gm.ax(_dev(u).float()).double())
            assert _rel(w, om.ax_local(u)) <= 5e-6
            b = om.scatter(case.rhs_global())
            xg, st = gm.pcg(_dev(b), tol=1e-10, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2)
            assert st["status"] == 0
            r = b - om.apply(_host(xg))
            assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.05e-10
        finally:
            binding.lib().sem_autotune_reset()
