"""Small case for an ncu capture of the ragged-batch split kernel (not a test):
the first 128 problems of the seed-0 ragged 2-D workload (N in
{32,64,128,256}^2, m in 2..6, mixed boundaries), dissipative, split precision,
two full steps on a non-default stream, with the item size and blocks per SM
the autotuner picks on the full workload (split: 256 nodes, 8 blocks per SM;
FP64: 256 nodes, 2 blocks per SM).  Usage: python tests/ncu_batch_case.py [fp64]"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import paper_1802_05246_b300 as hb  # noqa: E402

rng = np.random.default_rng(0)
probs = []
for _ in range(128):
    Np = int(rng.choice([32, 64, 128, 256]))
    m = int(rng.integers(2, 7))
    bc = int(rng.integers(0, 3))
    rng.integers(1, 5)  # pulse draws of the workload generator are not needed here
    probs.append((2, m, Np, 1.0, 1.0 / Np, 0.9 / Np, hb.DISSIPATIVE, bc))
fp64 = len(sys.argv) > 1 and sys.argv[1] == "fp64"
b = hb.HermiteBatch(probs, precision=hb.FP64 if fp64 else hb.SPLIT32)
b.set_stream(torch.cuda.Stream())
b.config(256, 2 if fp64 else 8)
b.step(2)
torch.cuda.synchronize()
print("ok", b.dof_per_step)
