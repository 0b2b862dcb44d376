"""Tensor-core building blocks of the BF16 and FP8 verify kernels in
isolation: swizzled K-major shared-memory tiles, tcgen05.mma accumulation in
tensor memory over two passes, tcgen05.ld read-back.  D = 2 A B^T is compared
with an FP64 product of the same bf16 (or E4M3) values; their products are
exact in FP32, so only the accumulation rounds.  The bound used by the
pruning margin is n_mma * 2^-20 * sum |a b| per output (n_mma = MMA
instructions accumulated: 16 K elements each for bf16, 32 for E4M3)."""
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


E4M3 = torch.float8_e4m3fn


def _fp8_check(A, B):
    D = pano.panorama_debug_tc_gemm_fp8(A.view(torch.uint8).cuda(),
                                        B.view(torch.uint8).cuda()).cpu().double()
    a, b = A.double(), B.double()
    ref = 2.0 * (a @ b.T)
    mag = 2.0 * (a.abs() @ b.abs().T)
    n_mma = 2 * A.shape[1] // 32
    err = (D - ref).abs()
    assert torch.all(err <= n_mma * 2.0 ** -20 * mag + 1e-30), float((err / mag).max())
    return float((err / mag.clamp_min(1e-300)).max())


@pytest.mark.parametrize("N,K", [(16, 32), (64, 64), (32, 128), (256, 128), (48, 384),
                                 (64, 512)])
def test_tc_gemm_fp8_matches_fp64(N, K):
    g = torch.Generator().manual_seed(N * 1000 + K)
    A = (torch.randn(128, K, generator=g) * torch.exp(-0.01 * torch.arange(K))).to(E4M3)
    B = torch.randn(N, K, generator=g).to(E4M3)
    assert _fp8_check(A, B) < 1e-6


def test_tc_gemm_fp8_wide_range_and_cancellation():
    """Products over 2^40 of dynamic range (subnormal E4M3 included), and
    large terms that cancel: the error stays within the per-MMA model."""
    g = torch.Generator().manual_seed(7)
    scale_a = torch.pow(2.0, torch.randint(-12, 8, (128, 256), generator=g).float())
    scale_b = torch.pow(2.0, torch.randint(-12, 8, (64, 256), generator=g).float())
    A = (torch.randn(128, 256, generator=g) * scale_a).clamp(-448, 448).to(E4M3)
    B = (torch.randn(64, 256, generator=g) * scale_b).clamp(-448, 448).to(E4M3)
    _fp8_check(A, B)
    a = torch.zeros(128, 128)
    a[:, 0::2] = 448.0
    a[:, 1::2] = -448.0
    b = torch.ones(32, 128)
    b[:, 1::2] = 1.125
    assert _fp8_check(a.to(E4M3), b.to(E4M3)) == 0.0


def test_sqrt_up_bounds_the_root_from_above():
    """The last level's upper bounds take square roots with the approximate
    square root times 1 + 2^-18, rounded up: on every binade of FP32 (zero,
    subnormals, normals up to 2^127) and many mantissas it must be at least
    the exact root, within 2^-17 of it for normal inputs, and at most 2^-62
    below 2^-126 (where the input is raised to 2^-126)."""
    g = torch.Generator().manual_seed(11)
    exps = torch.arange(-149, 128, dtype=torch.float64)
    mant = 1.0 + torch.rand(exps.numel(), 64, generator=g, dtype=torch.float64)
    x = (mant * torch.pow(2.0, exps)[:, None]).reshape(-1)
    x = torch.cat([x, torch.tensor([0.0, 2.0 ** -149, 2.0 ** -126, 1.0, 4.0,
                                    float(torch.finfo(torch.float32).max)],
                                   dtype=torch.float64)])
    x32 = x.to(torch.float32)
    x32 = x32[torch.isfinite(x32)]
    r = pano.panorama_debug_sqrt_up(x32.to("cuda:0")).cpu().double()
    exact = x32.double().sqrt()
    assert torch.all(r >= exact)
    normal = x32.double() >= 2.0 ** -126
    assert torch.all(r[normal] <= exact[normal] * (1 + 2.0 ** -17)), \
        float((r[normal] / exact[normal]).max())
    assert torch.all(r[~normal] <= 2.0 ** -62)
