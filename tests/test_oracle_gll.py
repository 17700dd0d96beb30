"""Pins of the oracle's GLL nodes, weights and derivative matrix against
closed forms and exactness properties (Deville, Fischer & Mund 2002, the SEM
reference of the paper's section 3.1)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from tests._sem_dense import bary_deriv, gll_numpy


CLOSED = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("N", sorted(CLOSED))
def test_gll_closed_forms(N):
    xi, rho = oracle.gll(N)
    np.testing.assert_allclose(xi, CLOSED[N][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(rho, CLOSED[N][1], rtol=1e-14, atol=0)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_against_numpy_legendre(N):
    xi, rho = oracle.gll(N)
    x2, w2 = gll_numpy(N)
    np.testing.assert_allclose(xi, x2, atol=1e-14)
    np.testing.assert_allclose(rho, w2, rtol=1e-12)
    assert abs(rho.sum() - 2.0) < 1e-14
    # symmetry about 0
    np.testing.assert_array_equal(xi, -xi[::-1])


@pytest.mark.parametrize("N", range(1, 12))
def test_legendre_recurrence(N):
    c = np.zeros(N + 1)
    c[N] = 1
    for x in (-0.9, -0.31, 0.0, 0.42, 0.999):
        P, dP = oracle.legendre(N, x)
        assert abs(P - npleg.legval(x, c)) < 1e-14
        assert abs(dP - npleg.legval(x, npleg.legder(c))) < 1e-12 * max(1, N * N)


@pytest.mark.parametrize("N", range(1, 13))
def test_quadrature_exact_to_degree_2N_minus_1(N):
    xi, rho = oracle.gll(N)
    for m in range(0, 2 * N):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(rho, xi ** m) - exact) < 1e-13, m
    # ... and not for degree 2N (a negative test: GLL is not Gauss)
    m = 2 * N
    assert abs(np.dot(rho, xi ** m) - 2.0 / (m + 1)) > 1e-10


@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_exact_on_polynomials(N):
    xi, _ = oracle.gll(N)
    D = oracle.deriv(N, xi)
    np.testing.assert_allclose(D @ np.ones(N + 1), 0.0, atol=1e-12 * N * N)
    for m in range(1, N + 1):
        np.testing.assert_allclose(D @ xi ** m, m * xi ** (m - 1), atol=2e-12 * N * N)
    # degree N+1 is not reproduced (the interpolant has degree N)
    assert np.max(np.abs(D @ xi ** (N + 1) - (N + 1) * xi ** N)) > 1e-6


def test_derivative_N1_closed_form():
    np.testing.assert_array_equal(oracle.deriv(1), [[-0.5, 0.5], [-0.5, 0.5]])


@pytest.mark.parametrize("N", range(1, 14))
def test_derivative_matches_barycentric(N):
    xi, _ = oracle.gll(N)
    np.testing.assert_allclose(oracle.deriv(N, xi), bary_deriv(xi), atol=1e-12 * N * N)


@pytest.mark.parametrize("N", range(1, 12))
def test_derivative_centro_antisymmetric(N):
    D = oracle.deriv(N)
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-14 * N * N)
    assert D[0, 0] == -0.25 * N * (N + 1) and D[N, N] == 0.25 * N * (N + 1)
