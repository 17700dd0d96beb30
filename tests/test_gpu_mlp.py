"""The element-local guess network on the tensor cores against the FP64
oracle (oracle/mlp.py) on the same BF16-rounded weights and inputs.

Two comparisons.  (1) Against the oracle with the GPU's rounding points
mirrored (BF16 hidden activations and back-propagated gradients): the ReLU
decisions are then taken on the same values and the remaining difference is
FP32 accumulation and rare re-roundings: 5e-3 in the relative 2-norm.
(2) Against the plain FP64 oracle: five BF16 roundings (2^-9 each) along the
chain plus ReLU decisions flipped by them bound the gradients at 5e-2."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2405_05640_gb300 import binding, inputs

pytestmark = pytest.mark.gpu
MIRROR_TOL = 5e-3
BF16_TOL = 5e-2


def _t():
    import torch
    return torch


def _bf16_round(a):
    torch = _t()
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("I,H,O,R,real", [(256, 128, 128, 256, 200), (2048, 256, 512, 512, 512)])
def test_forward_and_gradients_match_oracle(I, H, O, R, real):
    torch = _t()
    p = inputs.mlp_init(I, H, O, seed=5)
    net = binding.MLP(I, H, O, R)
    net.set_params(p)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((R, I)).astype(np.float32)
    T = rng.standard_normal((R, O)).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Y = net.forward(Xb).cpu().numpy()
    pr = {k: (_bf16_round(v) if k.startswith("W") else v.astype(np.float64)) for k, v in p.items()}
    Xr = _bf16_round(X)
    Yo, _ = omlp.forward(pr, Xr)
    assert _rel(Y, Yo) <= BF16_TOL
    loss = net.grad(Xb, torch.from_numpy(T).cuda(), rows_real=real, outs_real=O - 8)
    Lo, go = omlp.loss_and_grads(pr, Xr, T.astype(np.float64), rows=real, outs=O - 8)
    assert abs(loss - Lo) <= BF16_TOL * Lo
    g = net.get_grads()
    for k in omlp.NAMES:
        assert _rel(g[k], go[k]) <= BF16_TOL, (k, _rel(g[k], go[k]))
    Lq, gq = omlp.loss_and_grads(pr, Xr, T.astype(np.float64), rows=real, outs=O - 8, q=_bf16_round)
    Yq, _ = omlp.forward(pr, Xr, q=_bf16_round)
    assert _rel(Y, Yq) <= MIRROR_TOL
    assert abs(loss - Lq) <= MIRROR_TOL * Lq
    for k in omlp.NAMES:
        assert _rel(g[k], gq[k]) <= MIRROR_TOL, (k, _rel(g[k], gq[k]))


def test_training_reduces_loss():
    torch = _t()
    I, H, O, R = 256, 128, 128, 512
    net = binding.MLP(I, H, O, R)
    net.set_params(inputs.mlp_init(I, H, O, seed=2))
    rng = np.random.default_rng(3)
    X = rng.standard_normal((R, I)).astype(np.float32)
    M = rng.standard_normal((I, O)).astype(np.float32) / np.sqrt(I)
    T = np.tanh(X @ M)
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    first = net.grad(Xb, Td)
    for _ in range(150):
        net.adam(2e-3)
        last = net.grad(Xb, Td)
    assert last < 0.2 * first, (first, last)


def test_guess_kernels_match_definitions():
    torch = _t()
    import oracle
    case = inputs.tgv_box(3, 5)
    gm = binding.Mesh(5, case.nel, case.periodic, case.faces, case.vertices())
    om = oracle.Mesh(5, case.nel, case.periodic, case.faces, case.vertices())
    E, npt = gm.E, gm.npt
    rng = np.random.default_rng(9)
    f = [om.scatter(rng.standard_normal(om.nglob)) for _ in range(5)]  # continuous fields
    d = [torch.from_numpy(a).cuda() for a in f]
    ext = 3 * f[0] - 3 * f[1] + f[2]
    # residual of the extrapolation: b - A p_ext
    r = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
    work = torch.empty_like(r)
    binding.guess_residual(gm, d[3], d[0], d[1], d[2], r, work)
    ref_r = f[3] - om.apply(ext)
    assert np.linalg.norm(r.cpu().numpy() - ref_r) <= 1e-12 * np.linalg.norm(ref_r)
    ldx = 4 * npt + 40
    X = torch.zeros((E, ldx), dtype=torch.bfloat16, device="cuda")
    binding.guess_features(gm, d[0], d[1], d[2], d[4], r, 2.0, 4.0, 8.0, X)
    rr = r.cpu().numpy()
    d3 = f[0] - 3 * f[1] + 3 * f[2] - f[4]
    Xr = np.concatenate([((f[0] - f[1]) / 2).reshape(E, npt), ((f[1] - f[2]) / 2).reshape(E, npt),
                         (rr / 4).reshape(E, npt), (d3 / 8).reshape(E, npt)], axis=1)
    np.testing.assert_array_equal(X[:, :4 * npt].float().cpu().numpy(), _bf16_round(Xr))
    assert float(X[:, 4 * npt:].abs().max()) == 0.0
    binding.guess_features(gm, d[0], d[1], d[2], None, r, 2.0, 4.0, 8.0, X)  # fourth field p1
    Xr[:, 3 * npt:] = (f[0] / 8).reshape(E, npt)
    np.testing.assert_array_equal(X[:, :4 * npt].float().cpu().numpy(), _bf16_round(Xr))
    T = torch.zeros((E, npt + 8), dtype=torch.float32, device="cuda")
    binding.guess_target(gm, d[4], d[0], d[1], d[2], 2.0, T)
    np.testing.assert_allclose(T[:, :npt].cpu().numpy(), ((f[4] - ext) / 2).reshape(E, npt), rtol=1e-6, atol=1e-6)
    Y = torch.from_numpy(rng.standard_normal((E, npt + 8)).astype(np.float32)).cuda()
    g = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
    binding.guess_apply(gm, Y, d[0], d[1], d[2], 2.0, g)
    loc = ext + 2.0 * Y[:, :npt].double().cpu().numpy().reshape(-1)
    np.testing.assert_allclose(g.cpu().numpy(), om.dssum(loc) / om.mult, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("lam,assembled", [(0.0, False), (2.5, False), (1.0, True)])
def test_energy_norm_gradients_match_oracle(lam, assembled):
    """sem_mlp_grad_energy (element stiffness in FP32 on the FP32 geometric
    factors, plus lambda times the mass) against the oracle's K-norm loss in
    FP64 with K = A_e + lambda B_e, or for the averaged correction
    K = S M^-1 (A_L + lambda B) M^-1 S (S: sum of the copies): the same two
    bars as the mean square."""
    torch = _t()
    import oracle
    case = inputs.BoxCase("energy", 3, (8, 4, 4), (0, 0, 0), 0, perturb_amp=0.05, seed=3)
    V = case.vertices()
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    om = oracle.Mesh(case.N, case.nel, case.periodic, case.faces, V)
    E, npt = om.E, om.npt
    I, H, O, R = 4 * npt, 128, 128, 128
    assert E == R and npt < O
    p = inputs.mlp_init(I, H, O, seed=6)
    net = binding.MLP(I, H, O, R)
    net.set_params(p)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((R, I)).astype(np.float32)
    T = rng.standard_normal((R, O)).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    loss = net.grad_energy(Xb, torch.from_numpy(T).cuda(), gm, lam, assembled=assembled)
    g = net.get_grads()
    pr = {k: (_bf16_round(v) if k.startswith("W") else v.astype(np.float64)) for k, v in p.items()}
    Xr = _bf16_round(X)

    def K(d):
        d = d.reshape(-1)
        if assembled:
            d = om.dssum(d) * om.minv
        k = om.ax_local(d) + lam * om.B.reshape(-1) * d
        if assembled:
            k = om.dssum(k * om.minv)
        return k.reshape(E, npt)

    Lo, go = omlp.loss_and_grads(pr, Xr, T.astype(np.float64), rows=E, outs=npt, K=K)
    assert abs(loss - Lo) <= BF16_TOL * Lo
    for k in omlp.NAMES:
        assert _rel(g[k], go[k]) <= BF16_TOL, (k, _rel(g[k], go[k]))
    Lq, gq = omlp.loss_and_grads(pr, Xr, T.astype(np.float64), rows=E, outs=npt, q=_bf16_round, K=K)
    assert abs(loss - Lq) <= MIRROR_TOL * Lq
    for k in omlp.NAMES:
        assert _rel(g[k], gq[k]) <= MIRROR_TOL, (k, _rel(g[k], gq[k]))


def test_energy_norm_argument_checks():
    torch = _t()
    case = inputs.BoxCase("energy", 3, (8, 4, 4), (0, 0, 0), 0, seed=3)
    V = case.vertices()
    net = binding.MLP(256, 128, 128, 128)
    X = torch.zeros((128, 256), dtype=torch.bfloat16, device="cuda")
    T = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    g64 = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V)  # no FP32 geometry
    for mesh, lam, st in ((g64, 1.0, binding.SEM_ERR_INVALID_ARG),
                          (binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True), -1.0,
                           binding.SEM_ERR_INVALID_ARG)):
        with pytest.raises(binding.SemError) as ei:
            net.grad_energy(X, T, mesh, lam)
        assert ei.value.status == st
    gm = binding.Mesh(case.N, case.nel, case.periodic, case.faces, V, geom_f32=True)
    with pytest.raises(binding.SemError) as ei:
        net.grad_energy(X, T, gm, 1.0, work=torch.empty(gm.nloc, dtype=torch.float32, device="cuda"))
    assert ei.value.status == binding.SEM_ERR_WORKSPACE


def test_guess_residual_pair_matches_oracle():
    """The residual feature with the FP32-pair operator: b - A p_ext within
    the double-float error (~2^-42 of the line-wise magnitudes) of the FP64
    oracle; a mesh without the pair factors is rejected."""
    torch = _t()
    import oracle
    case = inputs.tgv_box(3, 7)
    V = case.vertices()
    gm = binding.Mesh(7, case.nel, case.periodic, case.faces, V, geom_pair=True)
    om = oracle.Mesh(7, case.nel, case.periodic, case.faces, V)
    rng = np.random.default_rng(4)
    f = [om.scatter(rng.standard_normal(om.nglob)) for _ in range(4)]
    d = [torch.from_numpy(a).cuda() for a in f]
    r = torch.empty(gm.nloc, dtype=torch.float64, device="cuda")
    work = torch.empty_like(r)
    binding.guess_residual(gm, d[3], d[0], d[1], d[2], r, work, pair=True)
    ref = f[3] - om.apply(3 * f[0] - 3 * f[1] + f[2])
    assert np.linalg.norm(r.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    g64 = binding.Mesh(7, case.nel, case.periodic, case.faces, V)
    with pytest.raises(binding.SemError) as ei:
        binding.guess_residual(g64, d[3], d[0], d[1], d[2], r, work, pair=True)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG
