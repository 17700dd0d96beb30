"""The tcgen05 BF16 GEMM against an FP64 product of the same BF16-rounded
operands.  FP32 accumulation of K products of BF16 values: the error is
bounded by ~K * 2^-24 * sum|a||b|, checked per element against that bound."""
import numpy as np
import pytest

from paper_2405_05640_gb300 import binding

pytestmark = pytest.mark.gpu


def _case(M, N, K, seed, bias, act, splitk=False):
    import torch
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bb = torch.randn(N, generator=g).float() if bias else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    work = binding.gemm_splitk_work(M, N, K) if splitk else None
    c32, c16 = binding.gemm_bf16(A.cuda(), B.cuda(), bb.cuda() if bias else None, act, True, True, err, work=work)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a = A.double().numpy()
    b = B.double().numpy()
    ref = a @ b.T
    if bias:
        ref = ref + bb.double().numpy()[None, :]
    if act == 1:
        ref = np.maximum(ref, 0.0)
    bound = 4 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    got = c32.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= bound + 1e-6 * np.abs(ref)), np.max(np.abs(got - ref) / bound)
    # the BF16 output is the FP32 result rounded to BF16
    np.testing.assert_array_equal(c16.cpu().float().numpy(), c32.cpu().to(torch.bfloat16).float().numpy())
    return c32


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 256, 128), (256, 256, 2048), (384, 512, 256),
                                   (512, 128, 640)])
def test_gemm_matches_fp64(M, N, K):
    _case(M, N, K, seed=M + N + K, bias=False, act=0)


def test_gemm_bias_relu():
    _case(256, 256, 256, seed=7, bias=True, act=1)


def test_gemm_rejects_ragged_shapes():
    import torch
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(binding.SemError) as ei:
        binding.gemm_bf16(A, B)
    assert ei.value.status == binding.SEM_ERR_INVALID_ARG


@pytest.mark.parametrize("M,N,K", [(256, 2048, 8192), (512, 256, 16384), (256, 256, 8192), (128, 128, 1088)])
def test_gemm_splitk_matches_fp64_and_is_deterministic(M, N, K):
    """Split-K for small outputs with a long K (the network's weight
    gradients; K = 1088 = 17 K-blocks: the slice count is reduced so that no
    slice is empty): the same bound against FP64, the bias and activation
    after the slices are summed, and the same bits on a second call."""
    c1 = _case(M, N, K, seed=M + N + K, bias=True, act=1, splitk=True)
    c2 = _case(M, N, K, seed=M + N + K, bias=True, act=1, splitk=True)
    np.testing.assert_array_equal(c1.cpu().numpy(), c2.cpu().numpy())
