"""Differentiable butterfly apply: a torch.autograd.Function over the
bf_diff_* entry points of libbfly.so, and a module holding the factor blocks
as trainable parameters.

u = K_bf g with K_bf = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*
(Eq. Kfactors).  The backward pass gives the gradient with respect to g
(the adjoint apply K_bf^* ubar) and to every V/H/S/G/U block, in PyTorch's
convention for complex tensors.  The forward pass keeps the input of every
k-th factor (k chosen by the plan from a memory budget, or forced); the
backward pass recomputes the rest.  Every step runs in the library's CUDA
kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import capi


class ButterflyApplyFunction(torch.autograd.Function):
    """u = K_bf g for g of shape (nrhs, N) complex64 (one vector per row)."""

    @staticmethod
    def forward(ctx, plan, g, VL, S, UL, *HG):
        h = len(HG) // 2
        H, G = list(HG[:h]), list(HG[h:])
        g = g.contiguous()
        nrhs = g.shape[0]
        saved = torch.empty(capi.bf_diff_saved_bytes(plan, nrhs) // 8, dtype=torch.complex64, device=g.device)
        u = torch.empty_like(g)
        capi.bf_diff_forward(plan, (VL, H, S, G, UL), g, u, saved, nrhs=nrhs)
        ctx.plan = plan
        ctx.h = h
        ctx.save_for_backward(saved, VL, S, UL, *HG)
        return u

    @staticmethod
    def backward(ctx, ubar):
        saved, VL, S, UL, *HG = ctx.saved_tensors
        h = ctx.h
        H, G = list(HG[:h]), list(HG[h:])
        ubar = ubar.contiguous()
        gbar = torch.empty_like(ubar)
        gVL, gS, gUL = torch.empty_like(VL), torch.empty_like(S), torch.empty_like(UL)
        gH = [torch.empty_like(a) for a in H]
        gG = [torch.empty_like(a) for a in G]
        capi.bf_diff_backward(ctx.plan, (VL, H, S, G, UL), ubar, gbar, saved, (gVL, gH, gS, gG, gUL),
                              nrhs=ubar.shape[0])
        return (None, gbar, gVL, gS, gUL, *gH, *gG)


class ButterflyOperator(torch.nn.Module):
    """The factors of one butterfly factorization as parameters; forward(g)
    applies K_bf to g of shape (nrhs, N) complex64 on the parameters' device."""

    def __init__(self, factors, nrhs_max: int, device="cuda", stride: int = 0, saved_budget: int = 0):
        super().__init__()
        dev = torch.device(device)
        self.L, self.n0, self.r = int(factors.L), int(factors.n0), int(factors.r)
        self.h = self.L // 2
        self.N = self.n0 << self.L
        c64 = torch.complex64
        self.VL = torch.nn.Parameter(torch.as_tensor(factors.VL).to(dev, c64).contiguous())
        self.UL = torch.nn.Parameter(torch.as_tensor(factors.UL).to(dev, c64).contiguous())
        self.S = torch.nn.Parameter(torch.as_tensor(factors.S).to(dev, torch.float32).contiguous())
        self.H = torch.nn.ParameterList([torch.nn.Parameter(torch.as_tensor(a).to(dev, c64).contiguous())
                                         for a in factors.H])
        self.G = torch.nn.ParameterList([torch.nn.Parameter(torch.as_tensor(a).to(dev, c64).contiguous())
                                         for a in factors.G])
        self.plan = capi.bf_diff_create(self.L, self.n0, self.r, nrhs_max, stride=stride,
                                        saved_budget=saved_budget)

    @property
    def stride(self) -> int:
        return capi.bf_diff_stride(self.plan)

    def forward(self, g: torch.Tensor) -> torch.Tensor:
        return ButterflyApplyFunction.apply(self.plan, g, self.VL, self.S, self.UL, *self.H, *self.G)
