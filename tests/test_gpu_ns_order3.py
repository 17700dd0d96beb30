"""Third-order stepping (BDF3 / EXT3) and dealiased advection of the NS
stepper (CUDA path, through the C ABI) against the FP64 oracle."""
import math

import numpy as np
import pytest

from oracle.ns import NSOracle
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_ns import _dev, _host, _rel

pytestmark = pytest.mark.gpu

DA_CASES = [
    inputs.BoxCase("n2_per_jit", 2, (3, 2, 3), (1, 1, 1), 0, hi=(2 * math.pi,) * 3, jitter=0.1, seed=5),
    inputs.BoxCase("n5_per_jit", 5, (3, 2, 2), (1, 1, 1), 0, hi=(2 * math.pi,) * 3, jitter=0.12, seed=3),
    inputs.BoxCase("n6_per", 6, (2, 2, 2), (1, 1, 1), 0, hi=(2 * math.pi,) * 3),
    inputs.BoxCase("n7_per_jit", 7, (2, 3, 2), (1, 1, 1), 0, hi=(2 * math.pi,) * 3, jitter=0.08, seed=4),
    inputs.BoxCase("n9_per", 9, (2, 2, 1), (1, 1, 1), 0, hi=(2 * math.pi,) * 3),
]


@pytest.mark.parametrize("case", DA_CASES, ids=[c.name for c in DA_CASES])
def test_dealiased_advection_matches_oracle(case):
    V = case.vertices()
    on = NSOracle(case.N, case.nel, V, 100.0, dealias=True)
    x, y, z = on.m.xyz
    u = [(np.sin(x) * np.cos(y) * np.cos(z)).reshape(-1), (-np.cos(x) * np.sin(y) * np.cos(z)).reshape(-1),
         (0.3 * np.sin(z + x) * np.cos(y)).reshape(-1)]
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_rx=True)
    st = binding.NSState(gm, 100.0)
    st.set_scheme(3, dealias=True)
    nl = _host(st.advect(_dev(np.stack(u))))
    for c, ref in enumerate(on.advect_dealiased(u)):
        assert _rel(nl[c], ref) <= 1e-12, c
    # collocation form through the same entry point
    st.set_scheme(2, dealias=False)
    nl = _host(st.advect(_dev(np.stack(u))))
    for c, ref in enumerate(on.advect(u)):
        assert _rel(nl[c], ref) <= 1e-12, c


@pytest.mark.parametrize("dealias", [False, True], ids=["colloc", "dealias"])
def test_ns_order3_steps_match_oracle(dealias):
    case = inputs.tgv_box(3, 5)
    V = case.vertices()
    Re = 400.0
    on = NSOracle(case.N, case.nel, V, Re, order=3, dealias=dealias)
    x, y, z = on.m.xyz
    u0 = [c.reshape(-1) for c in inputs.tgv_velocity(x, y, z)]
    on.set_velocity(u0)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_rx=True)
    st = binding.NSState(gm, Re)
    st.set_scheme(3, dealias=dealias)
    st.set_velocity(_dev(np.stack(u0)))
    po = gm.pcg_opts(tol=1e-13, max_iter=20000, use_initial_guess=True)
    vo = gm.pcg_opts(tol=1e-13, max_iter=20000)
    for n in range(5):
        on.step(2e-3, p_tol=1e-13, v_tol=1e-13)
        ps, vs = st.step(2e-3, po, vo)
        assert ps["status"] == 0 and all(v["status"] == 0 for v in vs)
        for c in range(3):
            assert _rel(_host(st.get(c)), on.u[c]) <= 1e-10, (n, c)
        assert _rel(_host(st.get(3)), on.p) <= 1e-9, n
    # the checkpoint slots of the third level hold u^{n-2} and NL^{n-2}
    assert _rel(_host(st.get(13)), on.u_hist[1][0]) <= 1e-10
    assert _rel(_host(st.get(16)), on.nl_hist[1][0]) <= 1e-9


def test_scheme_arguments_rejected():
    case = inputs.tgv_box(2, 3)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, case.vertices(), geom_rx=True)
    st = binding.NSState(gm, 100.0)
    with pytest.raises(binding.SemError) as ei:
        st.set_scheme(4)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    h = binding.lib().sem_ns_set_scheme(st.handle, 3, 1, None, 0, None)
    assert h == binding.SEM_ERR_WORKSPACE
