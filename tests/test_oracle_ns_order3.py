"""Pins of the NS oracle's third-order stepping and dealiased advection
(the high-order splitting of Karniadakis, Israeli & Orszag 1991 that the
paper cites in section 3.1; over-integration on 3(N+1)/2 Gauss points)."""
import math

import numpy as np
import pytest

import oracle
from oracle import ns
from paper_2405_05640_gb300 import inputs


def test_lagrange_matrix_identity_and_exactness():
    xi = oracle.gll(5)[0]
    np.testing.assert_allclose(ns.lagrange_matrix(xi, xi), np.eye(6), atol=1e-14)
    z, _ = np.polynomial.legendre.leggauss(9)
    f = lambda x: 3 * x ** 5 - x ** 4 + 0.5 * x - 2.0
    np.testing.assert_allclose(ns.lagrange_matrix(xi, z) @ f(xi), f(z), rtol=0, atol=1e-13)
    assert ns.dealias_points(7) == 12 and ns.dealias_points(4) == 8


def _tgv_like(o):
    x, y, z = o.m.xyz
    return [(np.sin(x) * np.cos(y) * np.cos(z)).reshape(-1), (-np.cos(x) * np.sin(y) * np.cos(z)).reshape(-1),
            (0.3 * np.sin(z) * np.cos(x)).reshape(-1)]


def test_dealiased_weak_form_is_exact_on_trilinear_elements():
    # the integrand phi_i C(u) d_a u is a polynomial of degree <= 3N+2 per
    # direction on trilinear elements: M = 3(N+1)/2 Gauss points integrate it
    # exactly, so more points change nothing
    case = inputs.BoxCase("jit", 4, (3, 2, 2), (1, 1, 1), 0, lo=(0, 0, 0), hi=(2 * math.pi,) * 3,
                          jitter=0.12, seed=3)
    o = ns.NSOracle(case.N, case.nel, case.vertices(), 100.0, dealias=True)
    u = _tgv_like(o)
    W1 = o.advect_weak(u)
    W2 = o.advect_weak(u, M=o.M + 3)
    for a, b in zip(W1, W2):
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    # fewer points than the 3/2 rule is not exact
    W0 = o.advect_weak(u, M=case.N + 1)
    assert max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(W0, W2)) > 1e-6


def test_dealiased_equals_collocation_for_linear_fields():
    # (u . grad) u of a linear field is linear: both forms are exact and the
    # lumped GLL mass integrates phi_i times a linear function exactly
    case = inputs.BoxCase("aff", 4, (2, 3, 2), (0, 0, 0), 0, lo=(0.0, -1.0, 0.5), hi=(2.0, 1.0, 1.5))
    o = ns.NSOracle(case.N, case.nel, case.vertices(), 100.0, periodic=(0, 0, 0), dealias=True)
    x, y, z = [c.reshape(-1) for c in o.m.xyz]
    u = [0.3 * x - 1.1 * y + 0.2, 0.7 * z + 0.5 * x - 0.1, -0.4 * y + 0.9 * z + 1.3]
    nd, nc = o.advect_dealiased(u), o.advect(u)
    for a, b in zip(nd, nc):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def _tgv2d(o, t, nu):
    x, y, _ = [c.reshape(-1) for c in o.m.xyz]
    f = math.exp(-2.0 * nu * t)
    return [np.sin(x) * np.cos(y) * f, -np.cos(x) * np.sin(y) * f, np.zeros_like(x)]


def _run(order, dt, T, dealias=False, Re=2.0):
    # N = 9 on 3 x 3 x 1 elements: the interpolated start is then discretely
    # divergence-free to ~1e-10; at N = 5 the first projection of the history
    # leaves a dt-dependent jump near 1e-5 that hides the third-order error
    case = inputs.BoxCase("tgv2d", 9, (3, 3, 1), (1, 1, 1), 0, lo=(0, 0, 0), hi=(2 * math.pi, 2 * math.pi, 1.0))
    o = ns.NSOracle(case.N, case.nel, case.vertices(), Re, order=order, dealias=dealias)
    nu = 1.0 / Re
    # exact start: the history holds the exact solution at the previous times
    o.set_velocity(_tgv2d(o, 0.0, nu))
    hist = [_tgv2d(o, -j * dt, nu) for j in range(1, order)]
    adv = o.advect_dealiased if dealias else o.advect
    o.u_hist = hist
    o.nl_hist = [adv(h) for h in hist]
    o.steps = order - 1
    n = int(round(T / dt))
    for _ in range(n):
        o.step(dt, p_tol=1e-13, v_tol=1e-13)
    return o.u


@pytest.mark.slow
@pytest.mark.parametrize("order,dealias", [(3, False), (3, True), (2, False)])
def test_temporal_order(order, dealias):
    # self-convergence on the 2-D Taylor-Green vortex (an exact NS solution):
    # halving dt divides the error by 2^order
    T = 0.4
    ref = _run(order, T / 160, T, dealias)
    errs = []
    for n in (10, 20, 40):
        u = _run(order, T / n, T, dealias)
        errs.append(max(np.abs(a - b).max() for a, b in zip(u, ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    lo, hi = (6.0, 10.5) if order == 3 else (3.0, 5.2)
    assert lo <= r1 <= hi and lo <= r2 <= hi, (errs, r1, r2)
