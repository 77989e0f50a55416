import sys, torch
sys.path.insert(0, '.')
import paper_1802_05246_b300 as hb
N, m = 64, 3; h = 1.0 / N
variant = int(sys.argv[1]) if len(sys.argv) > 1 else 0
g = hb.Hermite(3, m, N, 1.0, h, 0.9 * h, variant, 0, precision=hb.SPLIT32)
u = torch.randn(N**3, (m+1)**3, dtype=torch.float64, device='cuda')
v = torch.randn(N**3, m**3, dtype=torch.float64, device='cuda')
torch.cuda.synchronize()
g.set_state_device(u, v)
g.advance_half(3)
torch.cuda.synchronize()
print("ok")
