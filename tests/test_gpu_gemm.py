"""The proposal's tcgen05 BF16 GEMM (C = A B^T, FP32 accumulation) against
numpy's FP64 matmul of the same BF16 values: products of BF16 numbers are
exact in FP32, so the only error is FP32 accumulation (relative ~K * 2^-24)."""
import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc.Context()


def bf16(shape, seed):
    x = sg.Rng(seed).normal(int(np.prod(shape))).reshape(shape).astype(np.float32)
    t = torch.tensor(x).to(torch.bfloat16)
    return t, t.float().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K,split", [(128, 16, 64, 1), (1, 32, 64, 1), (100, 48, 128, 1), (300, 64, 320, 1),
                                         (257, 128, 1152, 1), (64, 200, 256, 1), (130, 1024, 1536, 1),
                                         (32, 64, 8448 * 64, 128), (96, 320, 4096, 4), (1000, 250, 192, 1),
                                         (256, 256, 512, 1), (129, 17, 64, 1), (385, 144, 640, 2)])
def test_gemm_matches_fp64(ctx, M, N, K, split):
    A, a = bf16((M, K), 1 + M)
    B, b = bf16((N, K), 2 + N)
    ref = a @ b.T
    C = torch.full((M, N), float("nan"), device="cuda:0")
    ctx.gemm_bf16(A.cuda(), B.cuda(), C, split_k=split)
    got = C.cpu().numpy().astype(np.float64)
    scale = np.sqrt(np.abs(a) ** 2 @ (np.abs(b) ** 2).T)      # |row| |col| bound of the sum
    err = np.abs(got - ref) / np.maximum(scale, 1e-30)
    assert np.isfinite(got).all()
    # FP32 accumulation: error grows like sqrt(K) * 2^-24 for random signs
    assert err.max() < 4 * np.sqrt(K) * 2.0 ** -24 + 1e-6, err.max()


def test_gemm_bias_relu(ctx):
    A, a = bf16((200, 128), 11)
    B, b = bf16((64, 128), 12)
    bias = np.linspace(-3, 3, 64).astype(np.float32)
    ref = np.maximum(a @ b.T + bias, 0)
    C = torch.empty((200, 64), device="cuda:0")
    ctx.gemm_bf16(A.cuda(), B.cuda(), C, bias=torch.tensor(bias, device="cuda:0"), relu=True)
    assert np.abs(C.cpu().numpy() - ref).max() < 1e-3
