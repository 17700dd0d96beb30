"""Pins of the oracle's geometry, gather-scatter, stiffness operator, Jacobi
diagonal and PCG against closed forms, invariants and an independent
brute-force dense assembly (tests/_sem_dense.py)."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import inputs
from tests._sem_dense import assemble, coordinate_numbering, physical_points


def _mesh(N, nel, periodic=(0, 0, 0), faces=0, **kw):
    case = inputs.BoxCase("t", N, tuple(nel), tuple(periodic), faces, **kw)
    return oracle.Mesh(N, case.nel, case.periodic, faces, case.vertices()), case


# ---------------------------------------------------------------- geometry


def test_affine_geometry_closed_form():
    N = 5
    m, case = _mesh(N, (3, 2, 4), lo=(0.0, -1.0, 2.0), hi=(3.0, 1.0, 3.0))
    h = np.array([1.0, 1.0, 0.25])
    detJ = np.prod(h) / 8.0
    rho = m.rho
    w3 = np.einsum("k,j,i->kji", rho, rho, rho).reshape(-1)
    for e in range(m.E):
        np.testing.assert_allclose(m.B[e], w3 * detJ, rtol=1e-12)
        for c in range(3):
            np.testing.assert_allclose(m.G[e, c], w3 * detJ * (2.0 / h[c]) ** 2, rtol=1e-12)
        np.testing.assert_allclose(m.G[e, 3:], 0.0, atol=1e-14)
    # coordinates of the GLL points of element 0
    xi = m.xi
    X = m.xyz[0, 0].reshape(N + 1, N + 1, N + 1)
    np.testing.assert_allclose(X[0, 0, :], 0.0 + (xi + 1) / 2 * h[0], atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 7])
def test_mass_sums_to_volume_on_deformed_box(N):
    m, _ = _mesh(N, (3, 3, 2), perturb_amp=0.05 * 8, seed=3, hi=(1.0, 2.0, 0.5))
    assert abs(m.B.sum() - 1.0 * 2.0 * 0.5) < 1e-13


def test_geometry_rotation_invariant():
    N = 4
    case = inputs.BoxCase("t", N, (2, 1, 1), (0, 0, 0), 0, perturb_amp=0.4, seed=5)
    V = case.vertices()
    a, b = 0.3, -1.1
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    R = Rz @ Rx
    _, G0, B0, s0 = oracle.geometry(N, V)
    _, G1, B1, s1 = oracle.geometry(N, V @ R.T + np.array([1.0, -2.0, 0.5]))
    assert s0 == s1 == 0
    np.testing.assert_allclose(G1, G0, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(B1, B0, rtol=1e-13)


def test_inverted_element_is_rejected():
    V = inputs.box_vertices((1, 1, 1))
    V[:, :, 0] *= -1.0  # mirror: det J < 0
    assert oracle.geometry(3, V)[3] == oracle.EMESH


# ---------------------------------------------------------------- numbering / dssum


@pytest.mark.parametrize("nel,periodic", [((2, 3, 2), (0, 0, 0)), ((3, 2, 2), (1, 0, 1)),
                                          ((1, 2, 1), (1, 1, 1)), ((2, 2, 2), (1, 1, 1))])
def test_numbering_matches_coordinate_matching(nel, periodic):
    N = 3
    case = inputs.BoxCase("t", N, nel, periodic, 0, hi=(2.0, 1.0, 3.0))
    gid, ng = oracle.box_numbering(N, nel, periodic)
    P = physical_points(N, case.vertices())
    period = [(2.0, 1.0, 3.0)[a] if periodic[a] else 0 for a in range(3)]
    gid2, ng2 = coordinate_numbering(P, period)
    assert ng == ng2
    # same partition of local points into global nodes
    pairs = set(zip(gid.tolist(), gid2.tolist()))
    assert len(pairs) == ng


@pytest.mark.parametrize("nel,periodic", [((4, 4, 4), (0, 0, 0)), ((4, 3, 5), (1, 0, 1)),
                                          ((2, 2, 2), (1, 1, 1))])
def test_multiplicity_counts(nel, periodic):
    N = 7
    m, _ = _mesh(N, nel, periodic)
    assert set(np.unique(m.mult)) <= {1.0, 2.0, 4.0, 8.0}
    expect = np.prod([nel[a] * N + (0 if periodic[a] else 1) for a in range(3)])
    assert m.nglob == expect
    assert abs(np.sum(1.0 / m.mult) - expect) < 1e-8
    # interior (non-face) points of every element have multiplicity one
    n1 = N + 1
    mm = m.mult.reshape(m.E, n1, n1, n1)
    assert np.all(mm[:, 1:-1, 1:-1, 1:-1] == 1.0)


def test_unique_counts_of_the_named_configs():
    # cube 4^3 N=7: 29^3 nodes with boundary; channel 32^3 periodic x,z
    assert oracle.box_numbering(7, (4, 4, 4), (0, 0, 0))[1] == 29 ** 3 == 24389
    assert inputs.global_dims(7, (32, 32, 32), (1, 0, 1)) == (224, 225, 224)


def test_dssum_idempotent_up_to_multiplicity():
    m, _ = _mesh(3, (3, 2, 2), (1, 0, 0))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(m.nloc)
    s = m.dssum(u)
    np.testing.assert_allclose(m.dssum(s / m.mult), s, rtol=1e-13, atol=1e-13)
    # dssum of a continuous field is the field times its multiplicity
    c = m.scatter(rng.standard_normal(m.nglob))
    np.testing.assert_allclose(m.dssum(c), c * m.mult, rtol=1e-14)


def test_mask_marks_exactly_the_dirichlet_faces():
    N = 3
    m, _ = _mesh(N, (2, 2, 2), (1, 0, 1), inputs.Y_FACES, hi=(1.0, 1.0, 1.0))
    y = m.xyz[1].reshape(-1)
    np.testing.assert_array_equal(m.mask.astype(bool), np.isclose(y, 0) | np.isclose(y, 1))
    mg = inputs.global_masked(N, (2, 2, 2), (1, 0, 1), inputs.Y_FACES)
    np.testing.assert_array_equal(mg[m.gid], m.mask.astype(bool))


# ---------------------------------------------------------------- stiffness operator


TINY = [
    (1, (2, 1, 1), (0, 0, 0), dict()),
    (2, (2, 2, 1), (0, 0, 0), dict(perturb_amp=0.3, seed=1)),
    (3, (2, 1, 2), (0, 0, 0), dict(perturb_amp=0.3, seed=2, hi=(1.0, 0.5, 2.0))),
    (3, (2, 2, 1), (1, 0, 0), dict(hi=(1.0, 1.0, 1.0))),
    (2, (1, 1, 2), (1, 1, 0), dict()),
    (2, (2, 1, 2), (0, 0, 0), dict(jitter=0.15, seed=3)),
    (3, (1, 2, 2), (0, 0, 0), dict(jitter=0.15, seed=4, hi=(0.7, 1.0, 1.3))),
]


@pytest.mark.parametrize("N,nel,periodic,kw", TINY)
def test_assembled_operator_matches_dense_galerkin(N, nel, periodic, kw):
    m, case = _mesh(N, nel, periodic, **kw)
    period = [(case.hi[a] - case.lo[a]) if periodic[a] else 0 for a in range(3)]
    A, Bm, gid2, ng, _ = assemble(N, case.vertices(), period)
    assert ng == m.nglob
    # map oracle global ids -> coordinate ids (a bijection)
    perm = np.zeros(ng, dtype=np.int64)
    perm[m.gid] = gid2
    Aor = np.zeros((ng, ng))
    for g in range(ng):
        e = np.zeros(ng)
        e[g] = 1.0
        col = m.dssum(m.ax_local(m.scatter(e)))
        # any copy holds the assembled value; collect one per global node
        y = np.zeros(ng)
        y[m.gid] = col
        Aor[np.ix_(perm, [perm[g]])] = y[:, None]
    np.testing.assert_allclose(Aor, A, atol=1e-12 * np.abs(A).max())
    # mass and the Jacobi diagonal
    bor = np.zeros(ng)
    bor[perm[m.gid]] = m.dssum(m.B.reshape(-1))
    np.testing.assert_allclose(bor, Bm, rtol=1e-13)
    # The preconditioner's diagonal is Q Q^T diag(A_L).  It equals diag(A)
    # unless one element holds two copies of a node (a periodic axis of a
    # single element), where A also gets the element's cross couplings.
    if not any(periodic[a] and nel[a] == 1 for a in range(3)):
        dor = np.zeros(ng)
        dor[perm[m.gid]] = m.diag
        np.testing.assert_allclose(dor, np.diag(A), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 0, 1)])
def test_operator_symmetric_and_annihilates_constants(periodic):
    N = 5
    m, _ = _mesh(N, (3, 2, 2), periodic, perturb_amp=0.05 * 6, seed=7)
    rng = np.random.default_rng(1)
    u = m.scatter(rng.standard_normal(m.nglob))
    v = m.scatter(rng.standard_normal(m.nglob))
    Au, Av = m.apply(u), m.apply(v)
    a, b = m.glsc3(v, Au), m.glsc3(u, Av)
    assert abs(a - b) <= 1e-13 * (abs(a) + abs(b))
    Ac = m.dssum(m.ax_local(np.ones(m.nloc)))
    assert np.max(np.abs(Ac)) <= 1e-13 * np.max(np.abs(Au))
    assert m.glsc3(u, Au) > 0


def test_operator_positive_definite_with_mask():
    m, _ = _mesh(4, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.2, seed=4)
    rng = np.random.default_rng(2)
    for _ in range(5):
        u = m.apply_mask(m.scatter(rng.standard_normal(m.nglob)))
        assert m.glsc3(u, m.apply(u)) > 0


@pytest.mark.parametrize("case", [inputs.cube_manufactured(3, 5), inputs.channel(3, 4)])
def test_linear_functions_in_kernel_on_affine_meshes(case):
    m = oracle.Mesh(case.N, case.nel, (0, 0, 0), 0, case.vertices())
    x, y, z = m.xyz
    u = (2.0 * x - 0.5 * y + 3.0 * z + 1.0).reshape(-1)
    Au = m.dssum(m.ax_local(u))
    # zero at nodes not on the domain boundary (affine: A u = -lap u = 0 weakly)
    interior = np.ones(m.nloc, dtype=bool)
    xyz = m.xyz.reshape(3, -1)
    for a in range(3):
        interior &= ~np.isclose(xyz[a], case.lo[a]) & ~np.isclose(xyz[a], case.hi[a])
    assert interior.any()
    assert np.max(np.abs(Au[interior])) < 1e-11


# ---------------------------------------------------------------- PCG


def test_pcg_matches_dense_solve():
    N = 3
    m, case = _mesh(N, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.3, seed=9)
    bg = inputs.random_rhs_global(N, case.nel, case.periodic, inputs.ALL_FACES, seed=4)
    b = m.scatter(bg)
    x, it, rr, st = m.pcg(b, tol=1e-14, max_iter=500)
    assert st == 0 and rr <= 1e-14
    # dense solve on the free unknowns with the independent assembly
    A, _, gid2, ng, _ = assemble(N, case.vertices())
    perm = np.zeros(ng, dtype=np.int64)
    perm[m.gid] = gid2
    free_or = ~inputs.global_masked(N, case.nel, case.periodic, inputs.ALL_FACES)
    free = np.zeros(ng, dtype=bool)
    free[perm] = free_or
    rhs = np.zeros(ng)
    rhs[perm] = bg
    xd = np.zeros(ng)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], rhs[free])
    np.testing.assert_allclose(x, xd[perm[m.gid]], atol=1e-12 * np.abs(xd).max())


def test_pcg_reports_nan_and_non_convergence():
    m, case = _mesh(2, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES)
    b = m.scatter(case.rhs_global())
    bad = b.copy()
    bad[5] = np.nan
    assert m.pcg(bad)[3] == oracle.ENAN
    x, it, rr, st = m.pcg(b, tol=1e-14, max_iter=2)
    assert st == oracle.ENOTCONV and it == 2


def _manufactured_error(N, nel):
    case = inputs.cube_manufactured(nel, N)
    m = oracle.Mesh(N, case.nel, case.periodic, case.faces, case.vertices())
    x, y, z = m.xyz
    f = inputs.manufactured_f(x, y, z).reshape(-1)
    b = m.apply_mask(m.dssum(m.B.reshape(-1) * f))
    u, it, rr, st = m.pcg(b, tol=1e-13, max_iter=5000)
    assert st == 0
    return np.max(np.abs(u - inputs.manufactured_u(x, y, z).reshape(-1)))


def test_spectral_convergence_manufactured_solution():
    errs = [_manufactured_error(N, 2) for N in range(3, 11)]
    # exponential decay: every two orders gain well over a decade
    for a, b in zip(errs[:-2], errs[2:]):
        assert b < a / 8, errs
    assert errs[-1] < 1e-8
    # log-linear fit: slope of ln(err) vs N clearly negative
    slope = np.polyfit(np.arange(3, 11), np.log(errs), 1)[0]
    assert slope < -1.5, slope
