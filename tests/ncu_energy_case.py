"""Small case for an ncu capture of the energy kernels (not a test): 3-D,
m = 3, 64^3 periodic, dissipative, random data; one energy call (both
forms).  Usage: python tests/ncu_energy_case.py [split|fp64] (default split)"""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_1802_05246_b300 as hb  # noqa: E402

N, m = 64, 3
h = 1.0 / N
prec = hb.FP64 if len(sys.argv) > 1 and sys.argv[1] == "fp64" else hb.SPLIT32
g = hb.Hermite(3, m, N, 1.0, h, 0.9 * h, hb.DISSIPATIVE, hb.PERIODIC, precision=prec)
u = torch.randn(N ** 3, (m + 1) ** 3, dtype=torch.float64, device="cuda")
v = torch.randn(N ** 3, m ** 3, dtype=torch.float64, device="cuda")
g.set_state_device(u, v)
print("ok", g.energy())
