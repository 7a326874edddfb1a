"""The network's BF16 GEMM on the 5th-generation tensor cores (tcgen05, FP32
accumulator in tensor memory) against FP64 numpy products of the same
BF16-rounded operands, on the shapes the learned guess uses (rows = atom
pairs, 96/256-wide layers, block-sized heads) including ragged edges and both
transpositions. Each case runs in a child process, so that a device error in
one cannot affect the others."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1601_02713_gb300 import native
M, N, K, ta, tb = map(int, sys.argv[2:7])
g = torch.Generator().manual_seed(M * 7 + N * 13 + K)
A = (torch.randn((K, M) if ta else (M, K), generator=g) * 0.5).to(torch.bfloat16).cuda()
B = (torch.randn((N, K) if tb else (K, N), generator=g) * 0.5).to(torch.bfloat16).cuda()
C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
rc = native.pimd_bf16_gemm_dev(A, B, C, bool(ta), bool(tb))
torch.cuda.synchronize()
a = A.double().cpu().numpy(); b = B.double().cpu().numpy()
ref = (a.T if ta else a) @ (b.T if tb else b)
got = C.double().cpu().numpy()
err = float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30))
print(json.dumps({"rc": rc, "rel": err, "nan": bool(np.isnan(got).any())}))
"""

CASES = [(256, 256, 96, 0, 0), (300, 256, 256, 0, 0), (300, 25, 256, 0, 0), (256, 70, 300, 1, 0),
         (96, 256, 300, 1, 0), (77, 256, 25, 0, 1), (1000, 196, 256, 0, 0), (13, 9, 5, 1, 1)]


@pytest.mark.parametrize("case", CASES)
def test_bf16_gemm(case):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT, *map(str, case)], capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["rc"] == 0 and not r["nan"], r
    # FP32 accumulation of at most 300 exact BF16 products
    assert r["rel"] < 1e-5, r
