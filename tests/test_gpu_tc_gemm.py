"""The tcgen05 3xTF32 contraction (dr_tf32x3_gemm) against an FP64 matrix product.

FP32-accurate means: |C - C64| <= 2^-18 * (|A| |B|) elementwise (a single TF32 pass is off by ~2^-11).
Shapes cover every tile width (N = 12..512), ragged M, N and K, and K not a multiple of 32; the
four tall shapes have at least two 128 x 128 tiles per SM, which the persistent kernel takes."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 256, 512), (300, 200, 100), (1000, 12, 256), (4096, 512, 512), (5, 16, 40),
                                   (129, 129, 33), (257, 64, 64), (640, 32, 1000),
                                   (19000, 130, 64), (40000, 257, 96), (38000, 512, 512), (20000, 256, 160)])
def test_tf32x3_gemm_matches_fp64(M, N, K):
    from paper_2605_25346_b300 import _lib
    lib = _lib.load()
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g, dtype=torch.float32)
    BT = torch.randn(N, K, device="cuda", generator=g, dtype=torch.float32) / np.sqrt(K)
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    torch.cuda.synchronize()
    rc = lib.dr_tf32x3_gemm(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(BT.data_ptr()),
                            ctypes.c_void_p(C.data_ptr()), None)
    assert rc == 0, lib.dr_last_error(None)
    ref = A.double() @ BT.double().T
    mag = A.double().abs() @ BT.double().abs().T
    err = ((C.double() - ref).abs() / mag.clamp_min(1e-30)).max().item()
    assert torch.isfinite(C).all()
    assert err <= 2.0 ** -18, f"max elementwise error {err:.3e} of |A||B|"
