"""Failure detection without a GPU fault: every device wait of the library is
bounded; a wait that runs out records a code in the mesh's error word, the
kernel returns and the context stays usable.  The self-test entry point makes
the library's own two wait forms (an mbarrier of the bulk-copy pipelines, the
grid barrier of the cooperative coarse solve) wait on something nothing
completes, with a short limit."""
import time

import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _mesh(geom_f32=False):
    case = inputs.deformed_cube(3, 5)
    V = case.vertices()
    return case, binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=geom_f32), \
        oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)


@pytest.mark.parametrize("kind,code", [(0, 1), (1, 2)], ids=["mbarrier", "grid_barrier"])
def test_wait_runs_out_reports_and_clears(kind, code):
    import torch
    case, gm, om = _mesh()
    assert gm.check_device_error() == 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    scr = gm.wait_selftest(kind, 0.02)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert 0.02 <= waited < 2.0, waited  # it waited its limit, then gave up
    assert gm.check_device_error() == code
    assert gm.check_device_error() == 0  # read and cleared
    del scr
    # the context is still usable: the operator matches the oracle
    u = np.random.default_rng(5).standard_normal(om.nloc)
    w = gm.ax(torch.from_numpy(u).cuda()).cpu().numpy()
    ref = om.ax_local(u)
    assert np.linalg.norm(w - ref) <= 1e-12 * np.linalg.norm(ref)


def test_solve_after_a_timeout_reports_only_its_own():
    import torch
    case, gm, om = _mesh(geom_f32=True)
    b = torch.from_numpy(om.scatter(case.rhs_global())).cuda()
    for kind in (0, 1):
        gm.wait_selftest(kind, 0.01)
        torch.cuda.synchronize()
        # the solver clears the earlier give-up at entry: its own kernels did
        # not time out, so it converges and reports OK
        _, st = gm.pcg(b, tol=1e-10, max_iter=5000)
        assert st["status"] == 0
        _, st = gm.pcg(b, tol=1e-10, max_iter=5000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2)
        assert st["status"] == 0
        assert gm.check_device_error() == 0


def test_selftest_rejects_bad_arguments():
    case, gm, om = _mesh()
    for kind, lim in ((2, 0.01), (0, 0.0), (0, 11.0)):
        with pytest.raises(binding.SemError) as ei:
            gm.wait_selftest(kind, lim)
        assert ei.value.status == binding.SEM_ERR_INVALID_ARG
    st = binding.lib().sem_wait_selftest(gm.handle, 1, 0.01, None, 0, None)
    assert st == binding.SEM_ERR_WORKSPACE
