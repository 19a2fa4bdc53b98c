"""Learned normalized/offset min-sum: autograd binding and training loop.

``NomsLoss`` wraps the library's forward and backward kernels
(``ldpc_noms_forward`` / ``ldpc_noms_backward``) in a ``torch.autograd.Function``
over the T unrolled iterations; the activations stay inside the library (with
checkpoints every ``ckpt_every`` iterations).  ``train_noms`` draws training
frames with the device channel (``ldpc_channel``) at Eb/N0 uniform in a range,
and steps Adam on the [T][J*L][2] parameters (w, o).  Everything that touches a
message runs in the CUDA kernels; torch holds the parameters and the optimizer.
"""
from __future__ import annotations

import math

from . import (ALGO_NOMS, MSG_F16, MSG_F32, QCCode, default_opts, ldpc_channel, ldpc_ber_sim, ldpc_noms_backward,
               ldpc_noms_forward)


def _torch():
    import torch

    return torch


class NomsLoss:
    """loss = NomsLoss.apply(params, llr, code_handle, msg, ckpt_every, clip)."""

    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            torch = _torch()

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(ctx, params, llr, code, msg, ckpt_every, clip):
                    loss, _ = ldpc_noms_forward(code, llr.contiguous(), params.detach(), msg, ckpt_every, clip)
                    ctx.save_for_backward(params)
                    ctx.code = code
                    return loss[0]

                @staticmethod
                def backward(ctx, gout):
                    (params,) = ctx.saved_tensors
                    grad = torch.zeros_like(params)
                    ldpc_noms_backward(ctx.code, params.detach(), grad)
                    return grad * gout, None, None, None, None, None

            cls._fn = _Fn
        return cls._fn.apply(*args)


def init_params(T: int, ncirc: int, device="cuda", w0: float = 1.0, o0: float = 0.0):
    """[T][ncirc][2] with w = w0, o = o0 (w = 1, o = 0 is plain min-sum)."""
    torch = _torch()
    p = torch.empty((T, ncirc, 2), dtype=torch.float32, device=device)
    p[..., 0] = w0
    p[..., 1] = o0
    return p


def draw_frames(code: QCCode, batch: int, seed: int, first_frame: int, ebn0_lo: float, ebn0_hi: float,
                groups: int = 8, stream=None):
    """Training frames from the device channel, Eb/N0 drawn uniformly per group of frames."""
    torch = _torch()
    llr = torch.empty((batch, code.N), dtype=torch.float32, device="cuda")
    g = torch.Generator().manual_seed(seed * 7919 + first_frame)
    per = math.ceil(batch / groups)
    for i in range(groups):
        lo, hi = i * per, min(batch, (i + 1) * per)
        if lo >= hi:
            break
        e = ebn0_lo + (ebn0_hi - ebn0_lo) * float(torch.rand(1, generator=g))
        ldpc_channel(code.handle, e, seed, first_frame + lo, llr[lo:hi], stream)
    return llr


def train_noms(code: QCCode, T: int = 10, steps: int = 200, batch: int = 1024, ebn0=(2.5, 4.5), lr: float = 0.02,
               seed: int = 1, msg: int = MSG_F16, ckpt_every: int = 2, clip: float = 30.0, params=None, log=None):
    """Adam on the NOMS parameters; returns (params, list of losses)."""
    torch = _torch()
    ncirc = _ncirc(code)
    p = (params if params is not None else init_params(T, ncirc)).clone().requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr)
    losses = []
    frame = 0
    for it in range(steps):
        llr = draw_frames(code, batch, seed, frame, *ebn0)
        frame += batch
        opt.zero_grad()
        loss = NomsLoss.apply(p, llr, code.handle, msg, ckpt_every, clip)
        loss.backward()
        opt.step()
        with torch.no_grad():
            p[..., 1].clamp_(min=0.0)
        losses.append(float(loss.detach()))
        if log and (it % max(1, steps // 10) == 0 or it == steps - 1):
            log(f"step {it}: loss {losses[-1]:.5f}")
    return p.detach(), losses


def _ncirc(code: QCCode) -> int:
    import numpy as np

    J, L = np.asarray(code.shifts).shape
    return J * L


def ber(code: QCCode, params, ebn0_db: float, frames: int, seed: int = 99, gamma: int = 4096, max_iter=None,
        msg: int = MSG_F16, early_stop: bool = True, target_frame_errors: int = 1 << 40):
    """BER/FER of the NOMS decoder (params [T][J*L][2]) through ldpc_ber_sim."""
    T = params.shape[0] if max_iter is None else max_iter
    o = default_opts(max_iter=T, early_stop=int(early_stop), algo=ALGO_NOMS, msg=msg)
    o.noms_params = params.contiguous().data_ptr()
    r = ldpc_ber_sim(code.handle, ebn0_db, seed, 0, frames, target_frame_errors, gamma, o)
    r["ber"] = r["bit_errors"] / (r["frames"] * code.N)
    r["fer"] = r["frame_errors"] / r["frames"]
    return r
