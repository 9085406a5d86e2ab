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


# The persistent GEMM's launch shapes on the staged path: clusters of two CTAs sharing the right
# operand's tiles (1), one CTA per tile row (5), and the pair form, one cta_group::2 MMA of M = 256
# over two CTAs with B's columns split between them (6).  They run the same products in the same
# order, so the bounds agree bit for bit, and they match the FP64 oracle on a few domains.  Widths
# include columns that are no multiple of 128 (partial tiles and B halves) and an odd number of row
# tiles (the last pair's second CTA has no rows).
@pytest.mark.parametrize("widths,D", [([16, 512, 512, 512, 512, 8], 96), ([4, 200, 150, 130, 3], 37)])
def test_persistent_launch_shapes_agree(widths, D):
    import dataclasses
    from oracle import reach as orc
    from paper_2605_25346_b300 import api
    from paper_2605_25346_b300 import workloads as wl
    if widths[0] == 16:
        p = dataclasses.replace(wl.large16().subset(np.arange(D)), H=2)
    else:
        p = wl.random_problem(81, widths, D=D, H=2, eps=0.2)
    out = {}
    for tuning in (101, 105, 106):
        r = api.Reach(0).load(p, precision=2)
        r.set_options(precision=2, tuning=tuning)
        out[tuning] = r.bounds(on_device=False)
        r.close()
    for t in (101, 106):
        np.testing.assert_array_equal(out[t]["lo"], out[105]["lo"])
        np.testing.assert_array_equal(out[t]["hi"], out[105]["hi"])
    q = p.subset(np.arange(3))
    o = orc.reach(q)
    olo, ohi = o["lo"].numpy(), o["hi"].numpy()
    scale = np.maximum(np.maximum(np.abs(olo), np.abs(ohi)), ohi - olo)
    err = np.maximum(np.abs(out[106]["lo"][:3] - olo), np.abs(out[106]["hi"][:3] - ohi)) / scale
    assert err.max() <= 1e-5


# The GEMM autotuner's choices persist in the file DR_GEMM_TUNE_CACHE: the first process times the
# candidates and writes one "key variant" line per GEMM shape; a second process takes the file's
# choices without trials (its report says so) and computes the same bounds.
_CACHE_SCRIPT = """
import sys
import numpy as np
from paper_2605_25346_b300 import api
from paper_2605_25346_b300 import workloads as wl
p = wl.random_problem(79, [6, 256, 256, 200, 3], D=64, H=2, eps=0.15)
r = api.Reach(0).load(p, precision=2)
b = r.bounds(on_device=False)
np.save(sys.argv[1], np.concatenate([b["lo"].ravel(), b["hi"].ravel()]))
r.close()
print(api.gemm_tuning_report())
"""


def test_gemm_tuning_cache_file(tmp_path):
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, DR_GEMM_TUNE_CACHE=str(tmp_path / "gemm_cache.txt"))
    runs = []
    for k in range(2):
        out = subprocess.run([sys.executable, "-c", _CACHE_SCRIPT, str(tmp_path / f"b{k}.npy")], cwd=root, env=env,
                             capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        runs.append(out.stdout)
    lines = (tmp_path / "gemm_cache.txt").read_text().split("\n")
    entries = [ln.split() for ln in lines if ln.strip()]
    assert entries and all(len(e) == 2 and e[0].startswith("epi") and 1 <= int(e[1]) <= 6 for e in entries), lines
    assert "(ms:" in runs[0] and "from DR_GEMM_TUNE_CACHE" in runs[1], runs
    assert "(ms:" not in runs[1], runs[1]
    np.testing.assert_array_equal(np.load(tmp_path / "b0.npy"), np.load(tmp_path / "b1.npy"))
