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


def test_batched_schwarz_matches_oracle_and_single_solves():
    """The batched solve with a hybrid Schwarz preconditioner per solve
    (flexible CG restarted at every refinement, coarse CG as separate
    launches inside the one graph): each solution against the oracle, the
    iterations of the same solve alone, and far fewer iterations than the
    Jacobi batch."""
    torch = _t()
    cases = [inputs.BoxCase("a", 5, (3, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=1),
             inputs.BoxCase("b", 7, (2, 2, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=2),
             inputs.BoxCase("c", 3, (4, 3, 2), (1, 0, 0), inputs.Y_FACES, jitter=0.1, seed=3),
             inputs.BoxCase("d", 9, (2, 1, 2), (0, 0, 0), inputs.ALL_FACES, perturb_amp=0.05, seed=4),
             inputs.channel(4, 7)]
    meshes, coarse, sws, oms, bs = [], [], [], [], []
    for c in cases:
        V = c.vertices()
        m = binding.Mesh(c.N, c.nel, c.periodic, c.faces, V, geom_f32=True)
        gc = binding.Mesh(1, c.nel, c.periodic, c.faces, V, geom_f32=True)
        meshes.append(m)
        coarse.append(gc)
        sws.append(binding.Schwarz(m, gc))
        om = oracle.Mesh(c.N, c.nel, c.periodic, c.faces, V)
        oms.append(om)
        bs.append(torch.from_numpy(om.scatter(c.rhs_global())).cuda())
    kw = dict(tol=1e-11, max_iter=20000, inner_tol=1e-2, check_every=8, coarse_iters=3, coarse_tol=1e-2)
    xs, stats = binding.pcg_solve_batched(meshes, bs, schwarz=sws, **kw)
    _, jstats = binding.pcg_solve_batched(meshes, bs, tol=1e-11, max_iter=20000, inner_tol=1e-2, check_every=8)
    for i, (om, st) in enumerate(zip(oms, stats)):
        assert st["status"] == 0, (i, st)
        assert st["rel_res"] <= 1e-11
        x = xs[i].cpu().numpy()
        xo, _, _, so = om.pcg(bs[i].cpu().numpy(), tol=1e-13, max_iter=20000)
        assert so == 0
        assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo), i
        _, s1 = meshes[i].pcg(bs[i], precision=binding.SEM_PCG_MIXED, schwarz=sws[i], **kw)
        assert abs(s1["iters"] - st["iters"]) <= max(3, 0.1 * s1["iters"]), (i, s1["iters"], st["iters"])
        assert st["iters"] < jstats[i]["iters"], (i, st["iters"], jstats[i]["iters"])


def test_batched_schwarz_rejects_a_foreign_schwarz_object():
    torch = _t()
    c1, c2 = inputs.deformed_cube(2, 4), inputs.deformed_cube(3, 4)
    m1 = binding.Mesh(c1.N, c1.nel, c1.periodic, c1.faces, c1.vertices(), geom_f32=True)
    m2 = binding.Mesh(c2.N, c2.nel, c2.periodic, c2.faces, c2.vertices(), geom_f32=True)
    g2 = binding.Mesh(1, c2.nel, c2.periodic, c2.faces, c2.vertices(), geom_f32=True)
    s2 = binding.Schwarz(m2, g2)
    b = torch.ones(m1.nloc, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.SemError) as ei:
        binding.pcg_solve_batched([m1], [b], schwarz=[s2], tol=1e-8)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
