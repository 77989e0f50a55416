"""Small case for an ncu capture of the network kernels (not a test): 64
images of 128 x 128 with 64 channels (134 MB of BF16 activations, above the
126 MB L2), dilation 8; three forward launches, then three weight-gradient
launches.  Usage: python tests/ncu_conv_case.py"""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_1802_05246_b300 as hb  # noqa: E402

B, C, dil = 64, 64, 8
L = hb.lib()
s = torch.cuda.current_stream().cuda_stream
x = torch.randn((B, 128, 128, C), device="cuda").to(torch.bfloat16)
dy = torch.randn((B, 128, 128, C), device="cuda").to(torch.bfloat16)
w = (torch.randn((C, 9, C), device="cuda") * 0.05).to(torch.bfloat16)
y = torch.empty_like(x)
dw = torch.zeros((C, 9, C), device="cuda")
for _ in range(3):
    assert L.hnn_conv3x3_fwd(x.data_ptr(), w.data_ptr(), None, None, B, 128, 128, C, C, dil, 1, y.data_ptr(), None,
                             s) == 0
for _ in range(3):
    assert L.hnn_conv3x3_wgrad(x.data_ptr(), dy.data_ptr(), B, 128, 128, C, C, dil, dw.data_ptr(), s) == 0
torch.cuda.synchronize()
print("ok")
