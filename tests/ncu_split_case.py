"""Small case for an ncu capture of the split-precision half-step (not a
test): 3-D, m = 3, 64^3 periodic, c dt/h = 0.9, random data, three
half-steps.  Usage: python tests/ncu_split_case.py [variant] (default 0,
the full dissipative method)."""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_1802_05246_b300 as hb  # noqa: E402

N, m = 64, 3
h = 1.0 / N
variant = int(sys.argv[1]) if len(sys.argv) > 1 else 0
g = hb.Hermite(3, m, N, 1.0, h, 0.9 * h, variant, hb.PERIODIC, precision=hb.SPLIT32)
u = torch.randn(N ** 3, (m + 1) ** 3, dtype=torch.float64, device="cuda")
v = torch.randn(N ** 3, m ** 3, dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
g.set_state_device(u, v)
g.advance_half(3)
torch.cuda.synchronize()
print("ok")
