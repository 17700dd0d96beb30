"""Pins of the hybrid Schwarz oracle (oracle/schwarz.py): the fast-
diagonalisation local solve against a dense solve of the SEM operator on the
extended subdomain (exact on axis-aligned tensor-product meshes), symmetry and
definiteness of the preconditioner, the coarse transfer pair, and the
flexible PCG against the plain oracle solve."""
import math

import numpy as np
import pytest

import oracle
from oracle import schwarz as sw
from paper_2405_05640_gb300 import inputs


def _dense(m):
    """Assembled operator on the unique (global) nodes, by columns."""
    n = m.nglob
    first = np.zeros(n, dtype=np.int64)
    first[m.gid[::-1]] = np.arange(m.nloc)[::-1]
    A = np.zeros((n, n))
    for c in range(n):
        eg = np.zeros(n)
        eg[c] = 1.0
        A[:, c] = m.apply(eg[m.gid])[first]
    return A


STRETCH = inputs.BoxCase("stretch", 3, (3, 4, 3), (1, 0, 1), inputs.Y_FACES, lo=(0.0, -1.0, 0.0),
                         hi=(2.0, 1.0, 1.5), tanh_beta=(0.0, 2.0, 0.0))


def test_fdm_local_solve_equals_dense_subdomain_solve():
    case = STRETCH
    V = case.vertices()
    S = sw.SchwarzFDM(case.N, case.nel, case.periodic, case.faces, V)
    A = _dense(S.m)
    rng = np.random.default_rng(3)
    rg = rng.standard_normal(S.m.nglob)
    for e in (0, 5, 17, S.m.E - 1):
        g = S.gid_ext[e]
        ok = g >= 0
        ge = g[ok]
        assert len(np.unique(ge)) == len(ge)
        u_dense = np.linalg.solve(A[np.ix_(ge, ge)], rg[ge])
        rext = np.where(ok, rg[np.where(ok, g, 0)], 0.0)
        u = S.local_solve(e, rext)[ok]
        assert np.abs(u - u_dense).max() <= 1e-11 * np.abs(u_dense).max()


def test_preconditioner_symmetric_positive_definite():
    case = inputs.deformed_cube(3, 4)
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    m = H.m
    rng = np.random.default_rng(5)
    x = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
    y = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
    a, b = m.glsc3(x, H.apply(y)), m.glsc3(y, H.apply(x))
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    assert m.glsc3(x, H.apply(x)) > 0 and m.glsc3(y, H.apply(y)) > 0


def test_coarse_transfer_pair():
    case = inputs.BoxCase("aff", 5, (2, 3, 2), (0, 0, 0), inputs.ALL_FACES, lo=(0.0, -1.0, 0.5), hi=(2.0, 1.0, 1.5))
    V = case.vertices()
    m = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    C = sw.CoarseLevel(case.N, case.nel, case.periodic, case.faces, V, m)
    # prolongation reproduces trilinear (here: linear) functions exactly
    xc_, yc_, zc_ = C.mc.xyz
    f = lambda x, y, z: 0.7 * x - 1.3 * y + 0.4 * z + 2.0
    pf = C.prolong(f(xc_, yc_, zc_).reshape(-1))
    x, y, z = m.xyz
    assert np.abs(pf - f(x, y, z).reshape(-1)).max() <= 1e-13
    # restriction is its adjoint in the unique-node products
    rng = np.random.default_rng(7)
    r = m.scatter(rng.standard_normal(m.nglob))
    xc = C.mc.scatter(rng.standard_normal(C.mc.nglob))
    lhs = float(np.sum(C.prolong(xc) * r / m.mult))
    rc = C.mc.dssum(np.einsum("ia,jb,kc,ekji->ecba", C.J1, C.J1, C.J1,
                              (r / m.mult).reshape(m.E, case.N + 1, case.N + 1, case.N + 1)).reshape(-1))
    rhs = float(np.sum(xc * rc / C.mc.mult))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("case", [inputs.channel(4, 5), inputs.deformed_cube(4, 5), STRETCH],
                         ids=["channel4", "deformed4", "stretch"])
def test_flexible_pcg_converges_faster_to_the_same_solution(case):
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    m = H.m
    b = m.scatter(case.rhs_global())
    xo, itj, _, st = m.pcg(b, tol=1e-12, max_iter=20000)
    x, its, rel = sw.fpcg(m, b, H.apply, tol=1e-12)
    assert st == 0 and rel <= 1e-12
    assert its <= 0.5 * itj, (its, itj)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)


def test_fgmres_equals_dense_solve_and_matches_fcg():
    """Restarted flexible GMRES: without preconditioner on a tiny mesh it
    reproduces the dense solve (also across restarts); with the hybrid
    Schwarz preconditioner it reaches the plain solution in about as many
    iterations as flexible CG (the preconditioner is symmetric positive
    definite, so CG's short recurrence loses nothing)."""
    case = inputs.BoxCase("tiny", 3, (2, 2, 1), (0, 0, 0), inputs.ALL_FACES, jitter=0.1, seed=5)
    V = case.vertices()
    m = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    A = _dense(m)
    free = m.apply_mask(np.ones(m.nloc))
    rng = np.random.default_rng(11)
    b = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
    first = np.zeros(m.nglob, dtype=np.int64)
    first[m.gid[::-1]] = np.arange(m.nloc)[::-1]
    keep = free[first] != 0
    bg = b[first]
    xd = np.zeros(m.nglob)
    xd[keep] = np.linalg.solve(A[np.ix_(keep, keep)], bg[keep])
    for restart in (200, 7):
        x, it, rel = sw.fgmres(m, b, lambda r: r, restart=restart, tol=1e-12)
        assert rel <= 1e-12
        assert np.abs(x[first] - xd).max() <= 1e-9 * np.abs(xd).max(), restart
    case = inputs.channel(4, 5)
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    m = H.m
    b = m.scatter(case.rhs_global())
    xo, itj, _, _ = m.pcg(b, tol=1e-10, max_iter=20000)
    xf, itf, relf = sw.fpcg(m, b, H.apply, tol=1e-10)
    xg, itg, relg = sw.fgmres(m, b, H.apply, restart=30, tol=1e-10)
    assert relg <= 1e-10
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert itg <= 1.5 * itf and itf <= 1.5 * itg, (itg, itf)
    assert itg <= 0.5 * itj, (itg, itj)


def test_multiplicative_levels_gain_nothing_over_additive():
    """The reading of 'hybrid' as additive between the two levels: applying
    the coarse correction first and the local solves to the updated residual
    costs an extra operator application per step and converges in the same
    number of flexible-CG iterations."""
    case = inputs.channel(4, 5)
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    m = H.m
    b = m.scatter(case.rhs_global())
    xa, ita, rela = sw.fpcg(m, b, H.apply, tol=1e-10)
    xm, itm, relm = sw.fpcg(m, b, H.apply_multiplicative, tol=1e-10)
    assert rela <= 1e-10 and relm <= 1e-10
    assert np.linalg.norm(xa - xm) <= 1e-8 * np.linalg.norm(xa)
    assert abs(ita - itm) <= max(2, ita // 10), (ita, itm)


# ------------------------------------------------------------------ intermediate (order-M) level

@pytest.mark.parametrize("M,N", [(1, 3), (2, 5), (3, 7), (4, 9)])
def test_lagrange_interp_exact_to_degree_M(M, N):
    xm, _ = oracle.gll(M)
    xn, _ = oracle.gll(N)
    J = sw.lagrange_interp(M, N)
    for k in range(M + 1):
        assert np.abs(J @ xm ** k - xn ** k).max() <= 1e-13
    # and not beyond: degree M + 1 is not reproduced
    assert np.abs(J @ xm ** (M + 1) - xn ** (M + 1)).max() > 1e-3
    # the end points map to end points exactly (faces to faces)
    assert np.array_equal(J[0], np.eye(M + 1)[0]) and np.array_equal(J[N], np.eye(M + 1)[M])
    assert np.abs(J.sum(axis=1) - 1.0).max() <= 1e-14


def test_mid_transfer_pair():
    case = inputs.BoxCase("aff", 5, (2, 3, 2), (0, 0, 0), inputs.ALL_FACES, lo=(0.0, -1.0, 0.5), hi=(2.0, 1.0, 1.5))
    V = case.vertices()
    m = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    L = sw.MidLevel(case.N, 3, case.nel, case.periodic, case.faces, V, m)
    # on affine elements the prolongation reproduces polynomials of degree <= M exactly
    f = lambda x, y, z: 0.3 * x ** 3 - 1.1 * x * y * z + 0.7 * y ** 2 + z - 0.5
    xm, ym, zm = L.mm.xyz
    pf = L.prolong(f(xm, ym, zm).reshape(-1))
    x, y, z = m.xyz
    assert np.abs(pf - f(x, y, z).reshape(-1)).max() <= 1e-12
    # the restriction is its adjoint in the unique-node products
    rng = np.random.default_rng(9)
    r = m.scatter(rng.standard_normal(m.nglob))
    xmid = L.mm.scatter(rng.standard_normal(L.mm.nglob))
    lhs = float(np.sum(L.prolong(xmid) * r / m.mult))
    rm = L.mm.dssum(np.einsum("ia,jb,kc,ekji->ecba", L.J, L.J, L.J,
                              (r / m.mult).reshape(m.E, case.N + 1, case.N + 1, case.N + 1)).reshape(-1))
    rhs = float(np.sum(xmid * rm / L.mm.mult))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_three_level_preconditioner_spd_and_solves():
    case = inputs.deformed_cube(3, 5)
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V, mid_order=3)
    m = H.m
    rng = np.random.default_rng(11)
    x = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
    y = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
    a, b = m.glsc3(x, H.apply(y)), m.glsc3(y, H.apply(x))
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    assert m.glsc3(x, H.apply(x)) > 0 and m.glsc3(y, H.apply(y)) > 0
    bb = m.scatter(case.rhs_global())
    xo, _, _, st = m.pcg(bb, tol=1e-12, max_iter=20000)
    x3, _, rel = sw.fpcg(m, bb, H.apply, tol=1e-12)
    assert st == 0 and rel <= 1e-12
    assert np.linalg.norm(x3 - xo) <= 1e-9 * np.linalg.norm(xo)


def test_three_level_fewer_iterations_on_the_channel():
    case = inputs.channel(4, 7)
    V = case.vertices()
    H2 = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    H3 = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V, mesh=H2.m, mid_order=3)
    m = H2.m
    b = m.scatter(case.rhs_global())
    _, i2, _ = sw.fpcg(m, b, H2.apply, tol=1e-10)
    _, i3, _ = sw.fpcg(m, b, H3.apply, tol=1e-10)
    assert i3 <= 0.9 * i2, (i3, i2)
