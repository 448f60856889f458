"""The torch.autograd.Function wrapper: its gradient is the library's adjoint, and a
torch.optim.Adam loop on theta follows the library's own Adam update."""
import numpy as np
import pytest

import synth
from gpu_common import Case, rel_l2, torch

pytestmark = pytest.mark.gpu


def test_autograd_gradient_is_library_adjoint():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    c.gpu_zf()
    th = T.nn.Parameter(c.theta.clone())
    loss = fd.fddpd_loss(th, c.plan, c.s, c.H, c.W, c.alpha, c.pa)
    loss.backward()
    g_ref, met = c.gpu_backward()
    assert abs(loss.item() - met[0]) <= 1e-6 * met[0]
    assert rel_l2(th.grad.cpu().numpy(), g_ref) <= 1e-6


def test_torch_adam_loop_matches_library_adam():
    import paper_2205_05158_gb300 as fd
    T = torch()
    c = Case(synth.CONFIGS["m16_k2_n64"], fc_scale=0.3)
    c.gpu_zf()
    th0 = c.theta.clone()
    th = T.nn.Parameter(th0.clone())
    opt = T.optim.Adam([th], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    losses = []
    for _ in range(4):
        opt.zero_grad()
        loss = fd.fddpd_loss(th, c.plan, c.s, c.H, c.W, c.alpha, c.pa)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    lib = th0.clone()
    c.plan.reset_optimizer()
    c.plan.update(c.s, c.H, c.W, c.alpha, c.pa, lib, 1e-3, 4, fd.FDDPD_ADAM)
    T.cuda.synchronize()
    d_t = (th.detach() - th0).cpu().numpy()
    d_l = (lib - th0).cpu().numpy()
    mask = np.abs(d_l) > 1e-6
    assert mask.sum() > 100
    assert rel_l2(d_t[mask], d_l[mask]) <= 1e-3
    assert losses[-1] < losses[0]
