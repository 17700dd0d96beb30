"""The hybrid Schwarz preconditioner (sem_schwarz_apply, FP32) against the
FP64 oracle (oracle/schwarz.py).

Bar: FP32 data and arithmetic through six 1-D contractions, a division by the
eigenvalue sums and the overlap sums: 1e-4 relative 2-norm (the local
operators of stretched cells have eigenvalue spreads of ~1e4, which the FP32
eigenvectors carry into the result); the coarse level with its CG iterated to
convergence.  Copies of a node are bit-identical (fixed summation order)."""
import numpy as np
import pytest

import oracle
from oracle import schwarz as sw
from paper_2405_05640_gb300 import binding, inputs

from test_gpu_parity import _dev, _host, _rel

pytestmark = pytest.mark.gpu

SW_TOL = 1e-4

SW_CASES = [
    inputs.BoxCase("stretch", 3, (3, 4, 3), (1, 0, 1), inputs.Y_FACES, lo=(0.0, -1.0, 0.0), hi=(2.0, 1.0, 1.5),
                   tanh_beta=(0.0, 2.0, 0.0)),
    inputs.deformed_cube(3, 4),
    inputs.channel(4, 7),
    inputs.BoxCase("n2_jit", 2, (3, 3, 2), (0, 0, 1), 0b001111, jitter=0.1, seed=4),
    inputs.BoxCase("n4_x1", 4, (1, 3, 2), (1, 0, 1), inputs.Y_FACES),
]
IDS = [c.name for c in SW_CASES]


def _setup(case):
    V = case.vertices()
    H = sw.HybridSchwarz(case.N, case.nel, case.periodic, case.faces, V)
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    gc = binding.Mesh(1, case.nel, case.periodic, case.faces, V, geom_f32=True)
    S = binding.Schwarz(gm, gc)
    return H, gm, gc, S


def _rhs(H):
    m = H.m
    r = m.apply_mask(m.scatter(np.random.default_rng(9).standard_normal(m.nglob)))
    return r.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("case", SW_CASES, ids=IDS)
def test_schwarz_levels_match_oracle(case):
    import torch
    H, gm, gc, S = _setup(case)
    r = _rhs(H)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z0 = _host(S.apply(rt, coarse_iters=0)).astype(np.float64)
    ref0 = H.m.apply_mask(H.sw.apply(r))
    assert _rel(z0, ref0) <= SW_TOL
    z1 = _host(S.apply(rt, coarse_iters=400, coarse_tol=1e-9)).astype(np.float64)
    assert _rel(z1, H.apply(r)) <= SW_TOL
    # continuity: every copy of a node holds the same bits; Dirichlet nodes 0
    one = np.zeros(H.m.nglob)
    one[H.m.gid] = z1
    np.testing.assert_array_equal(z1, one[H.m.gid])
    assert np.all(z1[H.m.apply_mask(np.ones(H.m.nloc)) == 0] == 0)


def test_schwarz_rejects_wrong_coarse_mesh():
    case = SW_CASES[0]
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    wrong = binding.Mesh(2, case.nel, case.periodic, case.faces, V, geom_f32=True)
    with pytest.raises(binding.SemError) as ei:
        binding.Schwarz(gm, wrong)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
