"""PyTorch autograd boundary of the neural deferred renderer (Sec. 3.3, training): the U-Net's
forward and backward passes and the L1 reconstruction loss as torch.autograd.Function objects
whose forward and backward call the library's kernels through the C ABI, and an optimiser that
runs the library's Adam kernel.  They marshal tensors only: every arithmetic step runs in the
library.

    net = NrvUNet(c_in=5, prec=nrv.PREC_BF16)
    opt = NrvAdam(net.parameters(), lr=1e-3)
    for x, target in batches:
        opt.zero_grad()
        loss = nrv_l1(net(x, height, width), target)
        loss.backward()
        opt.step()

One handle keeps the activations of its last training forward: run backward before the next
forward of the same module (a second forward first makes the earlier graph unusable, and its
backward raises).
"""
from __future__ import annotations

import torch

from . import nrv


class NrvUNetFunction(torch.autograd.Function):
    """rgb = U-Net(netin; params) through nrv_net_forward_train; the backward returns
    dL/dparams from nrv_net_backward (no gradient for the network input, which the method
    never needs: it comes from the rasterizer)."""

    @staticmethod
    def forward(ctx, netin, params, handle, prec, height, width):
        handle.load_params(params)
        n = netin.shape[0]
        rgb = torch.empty((n, height, width, 3), dtype=torch.float32, device=netin.device)
        handle.net.forward_train(netin.contiguous(), n, height, width, prec, rgb)
        handle.forwards += 1
        ctx.handle, ctx.token = handle, handle.forwards
        ctx.save_for_backward(netin, params)   # the backward reads the input of the first layer
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        h = ctx.handle
        if h.forwards != ctx.token:
            raise RuntimeError("NrvUNet: another forward ran after this one; its activations are "
                               "gone (run backward before the next forward)")
        netin, params = ctx.saved_tensors
        grad = torch.empty_like(params)
        h.net.backward(grad_rgb.contiguous(), grad)
        return None, grad, None, None, None, None


class NrvL1Function(torch.autograd.Function):
    """mean |y - t| and its gradient sign(y - t) / numel (sign(0) = 0) from nrv_l1_loss; the
    gradient is computed in the forward's kernel and scaled by the incoming gradient (1 for a
    loss that is the graph's output)."""

    @staticmethod
    def forward(ctx, y, t):
        y, t = y.contiguous(), t.contiguous()
        loss = torch.empty((), dtype=torch.float32, device=y.device)
        dy = torch.empty_like(y)
        nrv.l1_loss(y, t, loss.view(1), dy)
        ctx.save_for_backward(dy)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dy,) = ctx.saved_tensors
        return dy * g, None


def nrv_l1(y, t):
    return NrvL1Function.apply(y, t)


class NrvReconFunction(torch.autograd.Function):
    """Eq. 1 without its perceptual term -- l1 mean|y - t| + l2 mean (y - t)^2 + tv TV(y) --
    from nrv_recon_loss on RGB images [n][h][w][3]; gradient as for NrvL1Function."""

    @staticmethod
    def forward(ctx, y, t, weights):
        y, t = y.contiguous(), t.contiguous()
        loss = torch.empty((), dtype=torch.float32, device=y.device)
        dy = torch.empty_like(y)
        nrv.recon_loss(y, t, weights, loss.view(1), dy)
        ctx.save_for_backward(dy)
        return loss

    @staticmethod
    def backward(ctx, g):
        (dy,) = ctx.saved_tensors
        return dy * g, None, None


def nrv_recon(y, t, l1=0.0, l2=1.0, tv=0.0):
    return NrvReconFunction.apply(y, t, (l1, l2, tv))


# Parameter writes made by library kernels (NrvAdam), which torch's version counter does not
# see: data pointer -> number of writes.
_library_writes: dict[int, int] = {}


class _Handle:
    """A library network handle plus the parameter version it last loaded."""

    def __init__(self, c_in):
        self.net = nrv.Net(c_in)
        self.loaded = None
        self.forwards = 0

    def load_params(self, params):
        ptr = params.data_ptr()
        key = (ptr, params._version, _library_writes.get(ptr, 0))
        if key != self.loaded:
            self.net.set_params(params.detach())
            self.loaded = key


class NrvUNet(torch.nn.Module):
    """The U-Net of the neural deferred renderer with its flat FP32 parameter vector (the
    layout of include/nrv.h) as one nn.Parameter.  forward(netin, height, width): netin is the
    packed G-buffer [n][Hn][Wn][C] (float32 for PREC_F32, bfloat16 for PREC_BF16), the result
    RGB [n][height][width][3] float32.  Initialised with the library's seeded Xavier draw."""

    def __init__(self, c_in: int, prec: int = nrv.PREC_BF16, seed: int = 1, device=None):
        super().__init__()
        if prec not in (nrv.PREC_F32, nrv.PREC_BF16):
            raise ValueError("training runs in PREC_F32 or PREC_BF16")
        self.prec = prec
        self.h = _Handle(c_in)
        device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        p = torch.empty((nrv.param_count(c_in),), dtype=torch.float32, device=device)
        self.h.net.init_params(seed, p)
        self.params = torch.nn.Parameter(p)

    def forward(self, netin, height: int, width: int):
        return NrvUNetFunction.apply(netin, self.params, self.h, self.prec, height, width)


class NrvAdam(torch.optim.Optimizer):
    """Adam (Sec. 3.3 trains with Adam, lr 1e-3) through nrv_adam_step: FP32 moments, no
    weight decay, the library's kernel for every update."""

    def __init__(self, params, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        super().__init__(params, dict(lr=lr, betas=betas, eps=eps))

    @torch.no_grad()
    def step(self, closure=None):
        loss = closure() if closure is not None else None
        for group in self.param_groups:
            b1, b2 = group["betas"]
            for p in group["params"]:
                if p.grad is None:
                    continue
                st = self.state[p]
                if not st:
                    st["step"] = 0
                    st["m"] = torch.zeros_like(p)
                    st["v"] = torch.zeros_like(p)
                st["step"] += 1
                nrv.adam_step(p.data, p.grad.contiguous(), st["m"], st["v"], st["step"],
                              group["lr"], b1, b2, group["eps"])
                ptr = p.data_ptr()
                _library_writes[ptr] = _library_writes.get(ptr, 0) + 1
        return loss
