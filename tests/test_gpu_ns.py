"""Parity of the Navier-Stokes building blocks and time stepper (CUDA path,
through the C ABI) with the FP64 oracle (oracle/ns.py)."""
import numpy as np
import pytest

from oracle.ns import NSOracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _t():
    import torch
    return torch


def _dev(a):
    return _t().from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    _t().cuda.synchronize()
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = [
    inputs.BoxCase("n3_jit", 3, (3, 2, 2), (0, 0, 0), 0, jitter=0.12, seed=1),
    inputs.BoxCase("n5_per", 5, (2, 3, 2), (1, 1, 1), 0, hi=(6.283185307179586,) * 3),
    inputs.BoxCase("n7_jit", 7, (3, 2, 3), (1, 0, 1), 0, jitter=0.08, seed=2),
    inputs.BoxCase("n9", 9, (2, 2, 2), (0, 0, 0), 0, jitter=0.05, seed=3),
]


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_gradient_advect_wdiv_match_oracle(case):
    V = case.vertices()
    on = NSOracle(case.N, case.nel, V, 1.0, periodic=case.periodic)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_rx=True)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(on.m.nloc)
    g = _host(gm.gradient(_dev(f)))
    for m, ref in enumerate(on.grad(f)):
        assert _rel(g[m], ref) <= TOL
    u = [rng.standard_normal(on.m.nloc) for _ in range(3)]
    nl = _host(gm.advect(_dev(np.stack(u))))
    for c, ref in enumerate(on.advect(u)):
        assert _rel(nl[c], ref) <= TOL
    F = [rng.standard_normal(on.m.nloc) for _ in range(3)]
    w = _host(gm.weak_div(_dev(np.stack(F))))
    assert _rel(w, on.wdiv(F)) <= TOL


def _tgv_pair(nel, N, Re, geom_f32=False):
    case = inputs.tgv_box(nel, N)
    V = case.vertices()
    on = NSOracle(N, case.nel, V, Re)
    x, y, z = on.m.xyz
    u0 = [c.reshape(-1) for c in inputs.tgv_velocity(x, y, z)]
    on.set_velocity(u0)
    gm = binding.Mesh(N, case.nel, case.periodic, case.faces, V, geom_rx=True, geom_f32=geom_f32)
    st = binding.NSState(gm, Re)
    st.set_velocity(_dev(np.stack(u0)))
    return on, gm, st


def test_ns_steps_match_oracle():
    on, gm, st = _tgv_pair(3, 5, 400.0)
    assert abs(st.kinetic_energy() - on.kinetic_energy()) < 1e-14
    po = gm.pcg_opts(tol=1e-13, max_iter=20000, use_initial_guess=True)
    vo = gm.pcg_opts(tol=1e-13, max_iter=20000)
    p_prev = None
    for n in range(4):
        ref = on.step(2e-3, p_tol=1e-13, v_tol=1e-13)
        ps, vs = st.step(2e-3, po, vo)
        if p_prev is not None:  # the pressure history ring: slot 4 holds p^{n-1}
            assert _rel(_host(st.get(4)), p_prev) <= 1e-9
        p_prev = on.p.copy()
        assert ps["status"] == 0 and all(v["status"] == 0 for v in vs)
        assert _rel(_host(st.get(6)), ref["p_rhs"]) <= 1e-11
        for c in range(3):
            assert _rel(_host(st.get(c)), on.u[c]) <= 1e-10, (n, c)
        assert _rel(_host(st.get(3)), on.p) <= 1e-9, n
        assert abs(st.kinetic_energy() - on.kinetic_energy()) < 1e-13


def test_ns_mixed_pressure_and_guess():
    on, gm, st = _tgv_pair(3, 5, 400.0, geom_f32=True)
    po = gm.pcg_opts(tol=1e-11, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3)
    vo = gm.pcg_opts(tol=1e-12, max_iter=20000)
    for n in range(3):
        on.step(2e-3, p_tol=1e-12, v_tol=1e-12)
        guess = st.get(3)
        ps, vs = st.step(2e-3, po, vo, p_guess=guess)
        assert ps["status"] == 0 and ps["outer_iters"] >= 1
        assert _rel(_host(st.get(3)), on.p) <= 1e-8
        for c in range(3):
            assert _rel(_host(st.get(c)), on.u[c]) <= 1e-9


def test_ns_stop_at_k_and_resume_is_bitwise():
    """Checkpoint / resume: stop after step k, keep every state field on the
    host (as a checkpoint file would), restore it into a new stepper on the
    same mesh and step on; the result equals the uninterrupted run bit for
    bit (BDF3 / EXT3 with dealiased advection, so the whole history is in
    the state)."""
    on, gm, st = _tgv_pair(3, 5, 400.0)
    st.set_scheme(3, dealias=True)
    po = gm.pcg_opts(tol=1e-12, max_iter=20000, use_initial_guess=True)
    vo = gm.pcg_opts(tol=1e-12, max_iter=20000)
    for _ in range(3):
        st.step(2e-3, po, vo)
    fields, steps = st.checkpoint()
    saved = [_host(f).copy() for f in fields]
    for _ in range(3):
        st.step(2e-3, po, vo)
    ref = [_host(f).copy() for f in st.checkpoint()[0]]
    st2 = binding.NSState(gm, 400.0)
    st2.set_scheme(3, dealias=True)
    st2.restore(([_dev(a) for a in saved], steps))
    for _ in range(3):
        st2.step(2e-3, po, vo)
    got = [_host(f) for f in st2.checkpoint()[0]]
    assert len(got) == len(ref)
    for w, (a, b) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(a, b, err_msg=f"slot {w}")


def test_ns_schwarz_pressure_matches_oracle():
    """The pressure solved by the mixed solver with the hybrid Schwarz
    preconditioner on the fully periodic TGV box (singular pressure system,
    coarse level on the periodic vertex grid)."""
    on, gm, st = _tgv_pair(3, 5, 400.0, geom_f32=True)
    case = inputs.tgv_box(3, 5)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, case.vertices(), geom_f32=True)
    S = binding.Schwarz(gm, gc)
    po = gm.pcg_opts(tol=1e-11, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-3, schwarz=S,
                     use_initial_guess=True)
    vo = gm.pcg_opts(tol=1e-12, max_iter=20000)
    for n in range(3):
        on.step(2e-3, p_tol=1e-12, v_tol=1e-12)
        ps, vs = st.step(2e-3, po, vo)
        assert ps["status"] == 0 and ps["outer_iters"] >= 1
        assert _rel(_host(st.get(3)), on.p) <= 1e-8
        for c in range(3):
            assert _rel(_host(st.get(c)), on.u[c]) <= 1e-9
