"""torch.autograd.Function wrappers around libhp's forward and adjoint kernels.

The backward passes are hand-written kernels behind the C ABI:
``hp_filterbank3d_adjoint`` (flipped-kernel correlation with the reflect
fold-back per axis; gradient magnitude through D_a / GM) and
``hp_morph3d_backward`` (subgradient routed to the extreme source, ties to
the smallest linear index). torch only supplies memory and streams.
"""
from __future__ import annotations

import torch

from . import api


def _as_list(filters):
    return [(int(k), float(s)) for k, s in filters]


class FilterBank(torch.autograd.Function):
    """outputs = bank(x) for filters [(kind, sigma), ...]; float32 outputs."""

    @staticmethod
    def forward(ctx, x, filters):
        filters = _as_list(filters)
        outs = api.filterbank3d(x, filters, out_dtype=api.HP_F32)
        ctx.save_for_backward(x)
        ctx.filters = filters
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        (x,) = ctx.saved_tensors
        used = [(f, g.contiguous()) for f, g in zip(ctx.filters, grads) if g is not None]
        if not used:
            return None, None
        gin = api.filterbank3d_adjoint(x, [g for _, g in used], [f for f, _ in used])
        return gin, None


class Morph(torch.autograd.Function):
    """Grayscale erosion (dilate=False) or dilation with its subgradient."""

    @staticmethod
    def forward(ctx, x, dilate: bool, se: str, radius: int):
        out = (api.dilate3d if dilate else api.erode3d)(x, se, radius)
        ctx.save_for_backward(x)
        ctx.cfg = (bool(dilate), se, int(radius))
        return out

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        dilate, se, radius = ctx.cfg
        gin = api.morph3d_backward(x, g.contiguous(), dilate, se, radius)
        return gin, None, None, None


class BankAndErosion(torch.autograd.Function):
    """The differentiable feature stack: the filter bank plus one erosion of
    the same input; backward writes the bank adjoint and accumulates the
    erosion subgradient into the same buffer."""

    @staticmethod
    def forward(ctx, x, filters, se: str, radius: int):
        filters = _as_list(filters)
        outs = api.filterbank3d(x, filters, out_dtype=api.HP_F32)
        e = api.erode3d(x, se, radius)
        ctx.save_for_backward(x)
        ctx.cfg = (filters, se, int(radius))
        return (*outs, e)

    @staticmethod
    def backward(ctx, *grads):
        (x,) = ctx.saved_tensors
        filters, se, radius = ctx.cfg
        used = [(f, g.contiguous()) for f, g in zip(filters, grads[:-1]) if g is not None]
        if used:
            gin = api.filterbank3d_adjoint(x, [g for _, g in used], [f for f, _ in used])
            if grads[-1] is not None:
                api.morph3d_backward(x, grads[-1].contiguous(), False, se, radius, gin=gin,
                                     accumulate=True)
        elif grads[-1] is not None:
            gin = api.morph3d_backward(x, grads[-1].contiguous(), False, se, radius)
        else:
            gin = None
        return gin, None, None, None


def filterbank(x, filters):
    return FilterBank.apply(x, filters)


def morph(x, dilate=False, se="cube", radius=1):
    return Morph.apply(x, dilate, se, radius)


def bank_and_erosion(x, filters, se="cube", radius=2):
    return BankAndErosion.apply(x, filters, se, radius)
