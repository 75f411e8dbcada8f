"""``torch.autograd.Function`` over T unrolled primal-form ADMM iterations (Algorithm 1).

``unrolled_admm(c_lower, b, handle, T, ckpt_every)`` returns X_T, the affine iterate of iteration T
on the lower pattern E_L (the handle's order), as a differentiable function of the lower-pattern
values of C and of b. The forward and the reverse pass are the library's kernels
(``sdp_unrolled_forward`` / ``sdp_unrolled_backward``); this module only moves tensors.

The handle holds the iteration state, so one handle serves one graph at a time: a second forward on
the same handle before the first backward invalidates the first (its backward then raises).
"""

from __future__ import annotations

import torch

from . import sdp_get_sizes, sdp_set_cost, sdp_set_rhs, sdp_unrolled_backward, sdp_unrolled_forward


class UnrolledADMM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c_lower, b, handle, T, ckpt_every):
        c_lower = c_lower.detach().contiguous()
        b = b.detach().contiguous()
        sdp_set_cost(handle, c_lower)
        sdp_set_rhs(handle, b)
        x = torch.empty(sdp_get_sizes(handle)["nE_lower"], dtype=torch.float64, device=c_lower.device)
        sdp_unrolled_forward(handle, int(T), int(ckpt_every), x_out=x)
        ctx.handle = handle
        return x

    @staticmethod
    def backward(ctx, gx):
        h = ctx.handle
        sz = sdp_get_sizes(h)
        gc = torch.empty(sz["nE_lower"], dtype=torch.float64, device=gx.device)
        gb = torch.empty(sz["m"], dtype=torch.float64, device=gx.device)
        sdp_unrolled_backward(h, gx.detach().contiguous().to(torch.float64), gc, gb)
        return gc, gb, None, None, None


def unrolled_admm(c_lower: torch.Tensor, b: torch.Tensor, handle, T: int = 200, ckpt_every: int = 20):
    """X_T on E_L as a differentiable function of (C on E_L, b)."""
    return UnrolledADMM.apply(c_lower, b, handle, T, ckpt_every)


def lower_weights(handle, device="cuda") -> torch.Tensor:
    """w_e = 1 on the diagonal and 2 off it, so sum_e w_e a_e b_e = <A, B> for symmetric A, B."""
    from . import sdp_get_maps
    mp = sdp_get_maps(handle)
    w = (mp["pat_row"] != mp["pat_col"]).astype("float64") + 1.0
    return torch.tensor(w, device=device)
