"""Pins of the Navier-Stokes oracle (oracle/ns.py) against closed forms of
the Taylor-Green vortex and operator identities.  The TGV on [0, 2 pi]^3 with
u = (sin x cos y cos z, -cos x sin y cos z, 0) has kinetic energy 1/8, the
pressure p = (cos 2x + cos 2y)(cos 2z + 2)/16 + const (which solves
lap p = -div((u . grad) u) exactly) and dE/dt(0) = -3 nu / 4."""
import math

import numpy as np
import pytest

import oracle
from oracle.ns import NSOracle
from paper_2405_05640_gb300 import inputs


def _tgv(nel, N, Re=1600.0, jitter=0.0):
    case = inputs.tgv_box(nel, N)
    case.jitter = jitter
    ns = NSOracle(N, case.nel, case.vertices(), Re)
    x, y, z = ns.m.xyz
    ns.set_velocity([c.reshape(-1) for c in inputs.tgv_velocity(x, y, z)])
    return ns


def test_gradient_exact_on_linear_and_spectral_on_trig():
    case = inputs.BoxCase("t", 5, (2, 3, 2), (0, 0, 0), 0, hi=(1.0, 2.0, 0.5), jitter=0.1, seed=3)
    ns = NSOracle(5, case.nel, case.vertices(), 1.0, periodic=(0, 0, 0))
    x, y, z = (a.reshape(-1) for a in ns.m.xyz)
    g = ns.grad(3 * x - 2 * y + 0.5 * z + 1)
    for gm, c in zip(g, (3.0, -2.0, 0.5)):
        np.testing.assert_allclose(gm, c, atol=1e-11)
    g = ns.grad(np.sin(x) * np.cos(y))
    np.testing.assert_allclose(g[0], np.cos(x) * np.cos(y), atol=1e-4)
    np.testing.assert_allclose(g[1], -np.sin(x) * np.sin(y), atol=1e-4)


def test_weak_divergence_of_gradient_is_the_stiffness_operator():
    # wdiv(grad q) = sum_ab D_a^T G_ab D_b q = A_L q, computed through an
    # independent path (inverse Jacobian + mass vs the C operator with G)
    case = inputs.BoxCase("t", 4, (2, 2, 2), (0, 0, 0), 0, jitter=0.12, seed=5)
    ns = NSOracle(4, case.nel, case.vertices(), 1.0, periodic=(0, 0, 0))
    q = np.random.default_rng(0).standard_normal(ns.m.nloc)
    a = ns.wdiv(ns.grad(q))
    b = ns.m.ax_local(q)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_advection_of_linear_field():
    case = inputs.BoxCase("t", 3, (2, 2, 1), (0, 0, 0), 0, jitter=0.1, seed=1)
    ns = NSOracle(3, case.nel, case.vertices(), 1.0, periodic=(0, 0, 0))
    x, y, z = (a.reshape(-1) for a in ns.m.xyz)
    nl = ns.advect([x, 2 * y, np.zeros_like(x)])
    np.testing.assert_allclose(nl[0], -x, atol=1e-12)
    np.testing.assert_allclose(nl[1], -4 * y, atol=1e-12)
    np.testing.assert_allclose(nl[2], 0.0, atol=1e-12)


def test_tgv_kinetic_energy_and_divergence_free_start():
    ns = _tgv(4, 7)
    assert abs(ns.kinetic_energy() - 0.125) < 1e-12
    # the interpolant is divergence-free up to the spectral truncation error
    div = sum(ns.grad(ns.u[m])[m] for m in range(3))
    assert np.max(np.abs(div)) < 5e-6


@pytest.mark.parametrize("N", [5, 7, 9])
def test_tgv_pressure_spectrally_accurate(N):
    ns = _tgv(4, N)
    b = ns.pressure_rhs(ns.advect(ns.u))
    p, it, st = ns.solve_pressure(b, 1e-13)
    assert st == 0
    x, y, z = ns.m.xyz
    pe = inputs.tgv_pressure(x, y, z).reshape(-1)
    pe = pe - ns.unique_mean(pe)
    err = np.max(np.abs(p - pe))
    assert err < {5: 5e-3, 7: 2e-4, 9: 5e-6}[N], err


def test_tgv_pressure_converges_exponentially():
    errs = []
    for N in (4, 6, 8, 10):
        ns = _tgv(3, N)
        p, _, _ = ns.solve_pressure(ns.pressure_rhs(ns.advect(ns.u)), 1e-13)
        x, y, z = ns.m.xyz
        pe = inputs.tgv_pressure(x, y, z).reshape(-1)
        errs.append(np.max(np.abs(p - (pe - ns.unique_mean(pe)))))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 4, errs


def test_tgv_energy_decay_rate_and_monotone():
    Re = 100.0
    ns = _tgv(4, 7, Re)
    dt = 1e-3
    E = [ns.kinetic_energy()]
    for _ in range(4):
        ns.step(dt, p_tol=1e-12, v_tol=1e-12)
        E.append(ns.kinetic_energy())
    assert all(b < a for a, b in zip(E, E[1:]))
    rate = (E[-1] - E[0]) / (4 * dt)
    assert abs(rate - (-3.0 / (4.0 * Re))) < 0.02 * 3.0 / (4.0 * Re), rate
    div = sum(ns.grad(ns.u[m])[m] for m in range(3))
    assert np.max(np.abs(div)) < 1e-3
