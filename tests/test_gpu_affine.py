"""The affine-element form of the FP32 operator (SEM_GEOM_AFFINE): on axis-
aligned box elements G is diagonal and factorises, G_rr = rho_i rho_j rho_k
hy hz / (2 hx) etc., so the operator reads 3 scalars per element instead of 6
factors per point.  Same operator, same FP32 bar as the general FP32 path
(5e-6 relative 2-norm against the FP64 oracle); the mixed solver on such a
mesh converges to the oracle's solution like the general one.
"""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import SOL_TOL, _dev, _host, _rel

pytestmark = pytest.mark.gpu

F32_AX_TOL = 5e-6

AFFINE = [inputs.channel(6, 7), inputs.cube_manufactured(4, 5),
          inputs.BoxCase("n3_periodic_x1", 3, (1, 3, 2), (1, 0, 1), inputs.Y_FACES),
          inputs.BoxCase("n9_box", 9, (3, 2, 4), (0, 0, 0), inputs.ALL_FACES, lo=(-1.0, 0.0, 2.0), hi=(3.0, 0.5, 2.5))]
IDS = [c.name for c in AFFINE]


def _meshes(case, affine=True):
    V = case.vertices()
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_affine=affine)
    return om, gm


@pytest.mark.parametrize("case", AFFINE, ids=IDS)
def test_ax_f32_affine_matches_oracle(case):
    import torch
    om, gm = _meshes(case)
    _, gg = _meshes(case, affine=False)
    u = np.random.default_rng(31).standard_normal(om.nloc)
    ut = torch.from_numpy(u.astype(np.float32)).cuda()
    w = _host(gm.ax(ut)).astype(np.float64)
    ref = om.ax_local(u.astype(np.float32).astype(np.float64))
    assert _rel(w, ref) <= F32_AX_TOL
    wg = _host(gg.ax(ut)).astype(np.float64)   # the general FP32 path on the same mesh
    assert _rel(w, wg) <= F32_AX_TOL


@pytest.mark.parametrize("case", AFFINE, ids=IDS)
def test_pcg_mixed_affine_matches_oracle(case):
    om, gm = _meshes(case)
    b = om.scatter(case.rhs_global())
    xo, _, _, sto = om.pcg(b, tol=1e-12, max_iter=20000)
    xg, st = gm.pcg(_dev(b), tol=1e-12, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-4)
    assert sto == 0 and st["status"] == 0, st
    assert _rel(_host(xg), xo) <= SOL_TOL
    r = b - om.apply(_host(xg))
    assert np.sqrt(om.glsc3(r, r) / om.glsc3(b, b)) <= 1.5e-12


def test_affine_flag_rejects_deformed_and_needs_f32():
    case = inputs.deformed_cube(3, 3)
    V = case.vertices()
    with pytest.raises(binding.SemError) as ei:
        binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True, geom_affine=True)
    assert ei.value.status == binding.SEM_ERR_MESH
    c2 = inputs.channel(3, 3)
    with pytest.raises(binding.SemError) as ei:
        binding.Mesh(c2.N, c2.nel, c2.periodic, c2.faces, c2.vertices(), geom_affine=True)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
