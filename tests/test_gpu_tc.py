"""Tensor-core building blocks of the BF16 verify kernel in isolation:
swizzled K-major shared-memory tiles, tcgen05.mma accumulation in tensor
memory over two passes, tcgen05.ld read-back.  D = 2 A B^T is compared with
an FP64 product of the same bf16 values; products of bf16 are exact in FP32,
so only the accumulation rounds.  The bound used by the pruning margin is
n_mma * 2^-20 * sum |a b| per output (n_mma = MMA instructions accumulated)."""
import numpy as np
import pytest
import torch

import paper_2510_00566_gb300 as pano

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_00566_gb300 import _build
    _build.build()
    pano.lib()


@pytest.mark.parametrize("N,K", [(16, 16), (64, 32), (64, 64), (32, 128),
                                 (256, 64), (48, 192)])
def test_tc_gemm_matches_fp64(N, K):
    g = torch.Generator().manual_seed(N * 1000 + K)
    A = (torch.randn(128, K, generator=g) * torch.exp(-0.02 * torch.arange(K))).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    D = pano.panorama_debug_tc_gemm(A.cuda(), B.cuda()).cpu().double()
    a, b = A.double(), B.double()
    ref = 2.0 * (a @ b.T)
    mag = 2.0 * (a.abs() @ b.abs().T)
    n_mma = 2 * K // 16
    err = (D - ref).abs()
    assert torch.all(err <= n_mma * 2.0 ** -20 * mag + 1e-30), float((err / mag).max())
    # in practice far tighter than the bound
    assert float((err / mag).max()) < 1e-5


def test_tc_gemm_cancellation():
    """Large terms that cancel: the error stays relative to sum |a b|."""
    K, N = 64, 32
    a = torch.zeros(128, K)
    a[:, 0::2] = 1000.0
    a[:, 1::2] = -1000.0
    b = torch.ones(N, K)
    b[:, 1::2] = 1.0 + 2.0 ** -7
    A, B = a.to(torch.bfloat16), b.to(torch.bfloat16)
    D = pano.panorama_debug_tc_gemm(A.cuda(), B.cuda()).cpu().double()
    ref = 2.0 * (A.double() @ B.double().T)
    mag = 2.0 * (A.double().abs() @ B.double().abs().T)
    assert torch.all((D - ref).abs() <= (2 * K // 16) * 2.0 ** -20 * mag)
