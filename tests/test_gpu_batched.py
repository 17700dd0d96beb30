"""Batched mixed-precision solves (one CUDA graph launch per batch: a
device-side WHILE loop of rounds per solve) against the FP64 oracle, solve by
solve."""
import numpy as np
import pytest

import oracle
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


def _t():
    import torch
    return torch


def test_batched_solves_match_oracle_and_single_solves():
    torch = _t()
    cases = [inputs.BoxCase("a", 5, (3, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=1),
             inputs.BoxCase("b", 7, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=2),
             inputs.BoxCase("c", 3, (4, 3, 2), (1, 0, 0), inputs.Y_FACES, jitter=0.1, seed=3),
             inputs.BoxCase("d", 9, (2, 1, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=4),
             inputs.channel(3, 7)]
    meshes, oms, bs = [], [], []
    for c in cases:
        V = c.vertices()
        meshes.append(binding.Mesh(c.N, c.nel, c.periodic, c.faces, V, geom_f32=True))
        om = oracle.Mesh(c.N, c.nel, c.periodic, c.faces, V)
        oms.append(om)
        bs.append(torch.from_numpy(om.scatter(c.rhs_global())).cuda())
    xs, stats = binding.pcg_solve_batched(meshes, bs, tol=1e-11, max_iter=20000, inner_tol=1e-2, check_every=8)
    for i, (om, st) in enumerate(zip(oms, stats)):
        assert st["status"] == 0, (i, st)
        assert st["rel_res"] <= 1e-11
        x = xs[i].cpu().numpy()
        xo, _, _, so = om.pcg(bs[i].cpu().numpy(), tol=1e-13, max_iter=20000)
        assert so == 0
        assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo), i
        # the same solve alone takes the same number of inner iterations
        _, s1 = meshes[i].pcg(bs[i], tol=1e-11, max_iter=20000, precision=binding.SEM_PCG_MIXED, inner_tol=1e-2,
                              check_every=8)
        assert abs(s1["iters"] - st["iters"]) <= 2, (i, s1["iters"], st["iters"])
        assert st["wall_ms"] > 0
        # the rounds of each solve ran in the device-side loop of the one
        # graph launch (8 FP32 iterations per round)
        assert st["ax_launches"] >= st["iters"] / 8, st
    # the solves finish at their own pace: the one with the fewest rounds
    # before the one with the most
    few = min(range(len(cases)), key=lambda i: stats[i]["ax_launches"])
    many = max(range(len(cases)), key=lambda i: stats[i]["ax_launches"])
    assert stats[few]["wall_ms"] <= stats[many]["wall_ms"]


def test_batched_reports_non_convergence_per_solve():
    torch = _t()
    c = inputs.deformed_cube(3, 5)
    V = c.vertices()
    m = binding.Mesh(c.N, c.nel, c.periodic, c.faces, V, geom_f32=True)
    om = oracle.Mesh(c.N, c.nel, c.periodic, c.faces, V)
    b = torch.from_numpy(om.scatter(c.rhs_global())).cuda()
    xs, stats = binding.pcg_solve_batched([m, m], [b, b.clone()], tol=1e-12, max_iter=5, check_every=4,
                                          raise_on_error=False)
    assert all(s["status"] == binding.SEM_ERR_NOT_CONVERGED for s in stats)
