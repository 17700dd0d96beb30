"""The FP32 operator reading BF16 geometric factors (SEM_GEOM_BF16), the
"BF16" option of the inner operator of the mixed solver.

Bar: every factor is rounded to BF16 (relative error <= 2^-9), so the operator
error is bounded pointwise by 2^-9 of the line-wise magnitudes |D^T||G||D||u|
plus FP32 rounding; tested at 2^-8.  The mixed solver still converges to the
FP64 tolerance (its FP64 refinement corrects the inner operator), only with
more inner iterations (measured: 1.85x on the 32^3 channel).
"""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import CASES, IDS, _dev, _host

pytestmark = pytest.mark.gpu


def _meshes(case):
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_bf16=True)
    return om, gm


@pytest.mark.parametrize("case", CASES[1:], ids=IDS[1:])
def test_ax_f32_bf16_factors_bounded_by_rounding(case):
    import torch
    om, gm = _meshes(case)
    u = np.random.default_rng(41).standard_normal(om.nloc).astype(np.float32).astype(np.float64)
    w = _host(gm.ax(torch.from_numpy(u.astype(np.float32)).cuda())).astype(np.float64)
    ref = om.ax_local(u)
    mag = oracle.ax_local(om.N, np.abs(om.D), np.abs(om.G), np.abs(u).reshape(om.E, -1)).reshape(-1)
    assert np.all(np.abs(w - ref) <= 2.0 ** -8 * mag)


@pytest.mark.parametrize("case", [inputs.channel(5, 7), inputs.deformed_cube(6, 5)], ids=["channel5", "deformed6"])
def test_pcg_mixed_bf16_converges_to_fp64_tolerance(case):
    om, gm = _meshes(case)
    b = om.scatter(case.rhs_global())
    xg, st = gm.pcg(_dev(b), tol=1e-10, max_iter=40000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2)
    assert st["status"] == 0, st
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-10
