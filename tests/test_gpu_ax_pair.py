"""The FP64-in/out operator evaluated in double-float arithmetic (sem_ax,
SEM_F64_PAIR) against the FP64 oracle.  It is not FP64 arithmetic and its
bars are those of its format, not FP64's:

Rough fields: the 1e-12 relative 2-norm of the FP64 operator.  The pair
format carries 48 significant bits and every product and line sum keeps its
exact rounding error, but the anchored sums and the FP32 low parts leave
about 2^-42 of the line-wise magnitudes |D^T||G||D||u|; on smooth fields,
where A u cancels strongly, that measure is the bar (2^-41, pointwise) with
1e-11 in the relative 2-norm.  The element-wise power-of-two scaling makes
the result exactly homogeneous: w(2^k u) = 2^k w(u) bit for bit.

Solves with FP64 vectors around this operator (SEM_PCG_F64_PAIR) are gated
like the other non-FP64 paths: the oracle's own true residual of the
returned solution, the iteration count of the FP64 solver (same Krylov
process) and continuity.
"""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import AX_TOL, CASES, IDS, _dev, _host, _rel

pytestmark = pytest.mark.gpu


def _meshes(case):
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_pair=True)
    return om, gm


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_ax_pair_matches_oracle(case):
    om, gm = _meshes(case)
    rng = np.random.default_rng(12)
    for u in (rng.standard_normal(om.nloc), om.scatter(rng.standard_normal(om.nglob)),
              rng.uniform(0.0, 1.0, om.nloc)):
        w = _host(gm.ax(_dev(u), pair=True))
        assert _rel(w, om.ax_local(u)) <= AX_TOL


@pytest.mark.parametrize("case", [CASES[4], CASES[6]], ids=[IDS[4], IDS[6]])
def test_ax_pair_smooth_field(case):
    # A smooth continuous field: A u cancels strongly, so the error is bounded
    # against the line-wise magnitudes |D^T| |G| |D| |u| (pointwise, 2^-41).
    om, gm = _meshes(case)
    x, y, z = om.xyz
    u = (np.sin(np.pi * x) * np.cos(2 * y) * np.sin(np.pi * z + 0.3) + 0.5 * x * y).reshape(-1)
    ref = om.ax_local(u)
    mag = oracle.ax_local(om.N, np.abs(om.D), np.abs(om.G), np.abs(u).reshape(om.E, -1)).reshape(-1)
    wp = _host(gm.ax(_dev(u), pair=True))
    assert np.all(np.abs(wp - ref) <= 2.0 ** -41 * mag)
    assert _rel(wp, ref) <= 1e-11


def test_ax_pair_exactly_homogeneous_and_scale_free():
    om, gm = _meshes(CASES[5])
    u = np.random.default_rng(13).standard_normal(om.nloc)
    w = _host(gm.ax(_dev(u), pair=True))
    for k in (-700, -200, 200, 700):
        wk = _host(gm.ax(_dev(np.ldexp(u, k)), pair=True))
        np.testing.assert_array_equal(wk, np.ldexp(w, k))


def test_ax_pair_mixed_magnitudes_zero_and_nan_elements():
    om, gm = _meshes(CASES[4])
    rng = np.random.default_rng(14)
    u = rng.standard_normal((om.E, om.npt))
    u[1] *= 1e-30           # a tiny element next to O(1) ones: element-wise accuracy holds
    u[2] = 0.0              # exact zeros
    u[3, 5] = np.nan        # a NaN poisons its own element only
    w = _host(gm.ax(_dev(u.reshape(-1)), pair=True)).reshape(om.E, -1)
    assert np.isnan(w[3]).all()
    assert np.array_equal(w[2], np.zeros(om.npt))
    ok = np.ones(om.E, bool)
    ok[3] = False
    ref = oracle.ax_local(om.N, om.D, om.G[ok], u[ok])
    got = w[ok]
    assert np.isfinite(got).all()
    for e in range(got.shape[0]):
        if np.linalg.norm(ref[e]) > 0:
            assert _rel(got[e], ref[e]) <= AX_TOL


def test_ax_pair_needs_pair_geometry():
    case = CASES[2]
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    with pytest.raises(binding.SemError) as ei:
        gm.ax(_dev(np.zeros(gm.nloc)), pair=True)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


@pytest.mark.slow
def test_full_size_ax_pair_sampled_elements():
    # the 32^3 channel at N = 7 in the benchmark's launch configuration
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_pair=True)
    rng = np.random.default_rng(22)
    u = rng.standard_normal(case.nloc)
    w = _host(gm.ax(_dev(u), pair=True)).reshape(case.E, -1)
    sel = np.unique(np.concatenate([[0, case.E - 1], rng.integers(0, case.E, 300)]))
    _, G, _, st = oracle.geometry(case.N, V[sel])
    assert st == 0
    ref = oracle.ax_local(case.N, oracle.deriv(case.N), G, u.reshape(case.E, -1)[sel])
    assert _rel(w[sel], ref) <= AX_TOL


# ------------------------------------------------------------------ FP64 vectors around the double-float operator
# Gate as for the other non-FP64 paths: the oracle's own residual of the
# returned solution, the iteration count of the FP64 solver (same Krylov
# process), and continuity (every copy of a node holds the same value).
PCG_CASES = [inputs.channel(5, 7), inputs.deformed_cube(6, 5),
             inputs.BoxCase("n9", 9, (3, 4, 3), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=2)] + \
            [c for c in CASES if c.name in ("n2_jitter", "n3_periodic1", "n11_deformed")]


@pytest.mark.parametrize("case", PCG_CASES, ids=[c.name for c in PCG_CASES])
def test_pcg_f64_pair_matches_oracle(case):
    om, gm = _meshes(case)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-10, max_iter=20000, precision=binding.SEM_PCG_F64_PAIR)
    _, s64 = gm.pcg(_dev(b), tol=1e-10, max_iter=20000)
    assert st["status"] == 0, st
    assert abs(st["iters"] - s64["iters"]) <= max(3, 0.02 * s64["iters"])
    xh = _host(xg)
    r = b - om.apply(xh)
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 2e-10
    xo, _, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    assert sto == 0 and _rel(xh, xo) <= 1e-6
    one = np.zeros(om.nglob)
    one[om.gid] = xh
    np.testing.assert_array_equal(xh, one[om.gid])


def test_pcg_f64_pair_needs_pair_geometry_and_poisson():
    case = CASES[4]
    om, gm = _meshes(case)
    b = _dev(om.scatter(case.rhs_global()))
    with pytest.raises(binding.SemError) as ei:
        gm.pcg(b, precision=binding.SEM_PCG_F64_PAIR, h2=1.0)
    assert ei.value.status == binding.SEM_ERR_UNSUPPORTED
    g2 = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices())
    with pytest.raises(binding.SemError) as ei:
        g2.pcg(b, precision=binding.SEM_PCG_F64_PAIR)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


@pytest.mark.slow
def test_full_size_pcg_f64_pair_true_residual():
    case = inputs.channel(32, 7)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_pair=True)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-8, max_iter=20000, precision=binding.SEM_PCG_F64_PAIR)
    assert st["status"] == 0
    x = _host(xg)
    r = b - om.apply(x)
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.05e-8
