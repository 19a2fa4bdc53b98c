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
               seed: int = 1, msg: int = MSG_F16, ckpt_every: int = 2, clip: float = 30.0, params=None, log=None,
               unroll: int = 0, dist=None):
    """Adam on the NOMS parameters; returns (params, list of losses).

    unroll > T trains the decoder as it runs for `unroll` iterations: iterations beyond T use the
    last trained row (the parameters are tied, their gradients summed by autograd).
    dist: a torch.distributed process group of several ranks -- data-parallel training, each rank on
    its own frames (frame ids offset by rank), gradients averaged over all frames every step."""
    from .shard import average_gradient

    torch = _torch()
    ncirc = _ncirc(code)
    p = (params if params is not None else init_params(T, ncirc)).clone().requires_grad_(True)
    opt = torch.optim.Adam([p], lr=lr)
    losses = []
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    frame = rank << 40
    for it in range(steps):
        llr = draw_frames(code, batch, seed, frame, *ebn0)
        frame += batch
        opt.zero_grad()
        P = extend_params(p, unroll) if unroll > T else p
        loss = NomsLoss.apply(P, llr, code.handle, msg, ckpt_every, clip)
        loss.backward()
        p.grad = average_gradient(p.grad, batch, dist)
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


def clopper_pearson(k: int, n: int, conf: float = 0.95):
    """Exact binomial confidence interval of a rate k/n."""
    from scipy.stats import beta

    a = 1.0 - conf
    lo = 0.0 if k == 0 else float(beta.ppf(a / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - a / 2, k + 1, n - k))
    return lo, hi


def ber_interval(r: dict, N: int, conf: float = 0.95):
    """Confidence interval of the BER from ldpc_ber_sim's counts.  Frames are independent, the bits
    of one frame are not (a failed frame carries many wrong bits), so the interval is the normal
    one of the mean of the per-frame error counts e_f (variance from sum e_f and sum e_f^2), divided
    by N.  With no frame error the BER is 0 and bounded by the FER's Clopper-Pearson upper limit
    (BER <= FER, since a frame has at most N wrong bits)."""
    from scipy.stats import norm

    n = int(r["frames"])
    if r["frame_errors"] == 0 or n < 2:
        return 0.0, clopper_pearson(int(r["frame_errors"]), n, conf)[1]
    m = r["bit_errors"] / n
    var = max(0.0, (r["bit_errors_sq"] - n * m * m) / (n - 1))
    h = float(norm.ppf(0.5 + conf / 2)) * math.sqrt(var / n)
    return max(0.0, (m - h) / N), (m + h) / N


def _timed_ber(code, opts, ebn0, frames, gamma, target_fe, seed=4242):
    torch = _torch()
    torch.cuda.synchronize()
    r = ldpc_ber_sim(code.handle, ebn0, seed, 0, frames, target_fe, gamma, opts)
    r["mbit_s"] = r["frames"] * code.K / r["seconds"] / 1e6
    nb = r["frames"] * code.N
    r["ber"] = r["bit_errors"] / nb
    r["ber_ci95"] = ber_interval(r, code.N)
    r["fer"] = r["frame_errors"] / r["frames"]
    r["fer_ci95"] = clopper_pearson(r["frame_errors"], r["frames"])
    return r


def extend_params(params, iters: int):
    """[iters][ncirc][2]: the trained rows, then the last trained row repeated for the later iterations."""
    torch = _torch()
    T = params.shape[0]
    if iters <= T:
        return params[:iters].contiguous()
    return torch.cat([params, params[-1:].expand(iters - T, -1, -1)], dim=0).contiguous()


def _overlap(a, b) -> bool:
    return a[0] <= b[1] and b[0] <= a[1]


def evaluate(code, params, ebn0_points, frames=1 << 20, gamma=8192, target_fe=100, sp_iters=30, long_iters=50,
             frame_caps=None):
    """At each Eb/N0: sum-product (sp_iters iterations, FP32 messages) and the trained NOMS run for
    long_iters iterations (FP16 messages; iterations past the trained rows reuse the last row), both
    with early stop on the same frames, each until target_fe frame errors or its frame cap
    (frame_caps[e] if given, else `frames`); plus untrained min-sum (w = 1, o = 0) as the method
    without the learned parameters.  Every arm reports BER and FER with 95% intervals (exact for the
    FER, frame-clustered for the BER) and decoded Mbit/s; `match` records whether NOMS's intervals
    overlap sum-product's, and `faster` whether NOMS decodes more Mbit/s."""
    T = params.shape[0]
    ncirc = params.shape[1]
    out = {}
    for e in ebn0_points:
        cap = (frame_caps or {}).get(e, frames)
        row = {}
        o = default_opts(max_iter=sp_iters, early_stop=1, msg=MSG_F32)
        sp = _timed_ber(code, o, e, cap, gamma, target_fe)
        row[f"sp{sp_iters}_f32"] = sp
        o = default_opts(max_iter=long_iters, early_stop=1, algo=ALGO_NOMS, msg=MSG_F16)
        prm = extend_params(params, long_iters)
        o.noms_params = prm.data_ptr()
        nm = _timed_ber(code, o, e, cap, gamma, target_fe)
        row[f"noms_trained_{long_iters}it_f16"] = nm
        o = default_opts(max_iter=long_iters, early_stop=1, algo=ALGO_NOMS, msg=MSG_F16)
        plain = init_params(long_iters, ncirc)
        o.noms_params = plain.data_ptr()
        row[f"minsum_untrained_{long_iters}it_f16"] = _timed_ber(code, o, e, min(cap, 1 << 18), gamma, target_fe)
        row["match"] = {"fer_intervals_overlap": _overlap(sp["fer_ci95"], nm["fer_ci95"]),
                        "ber_intervals_overlap": _overlap(sp["ber_ci95"], nm["ber_ci95"]),
                        "both_reached_target": sp["frame_errors"] >= target_fe and nm["frame_errors"] >= target_fe,
                        "faster": nm["mbit_s"] > sp["mbit_s"]}
        out[str(e)] = row
    return out


def main(argv=None):
    import argparse
    import json
    import time

    import numpy as np

    torch = _torch()
    ap = argparse.ArgumentParser(description="train the learned normalized/offset min-sum and compare it with "
                                             "sum-product on a seeded QC code")
    ap.add_argument("--J", type=int, default=4)
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--p", type=int, default=765)
    ap.add_argument("--shift-seed", type=int, default=2)
    ap.add_argument("--T", type=int, default=10, help="trained parameter rows (iterations)")
    ap.add_argument("--unroll", type=int, default=20, help="iterations unrolled in training (rows past T tied)")
    ap.add_argument("--steps", type=int, default=768)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=0.01)
    ap.add_argument("--train-ebn0", type=float, nargs=2, default=[2.9, 3.6])
    ap.add_argument("--ebn0", type=float, nargs="*", default=[3.0, 3.25, 3.375, 3.5])
    ap.add_argument("--eval-frames", type=int, default=1 << 24, help="frame cap per arm")
    ap.add_argument("--frames-3p5", type=int, default=1 << 27, help="frame cap per arm at 3.5 dB")
    ap.add_argument("--long-iters", type=int, default=50, help="iterations of the trained decoder")
    ap.add_argument("--target-errors", type=int, default=100)
    ap.add_argument("--params", default=None, help="evaluate these trained parameters (torch.save of [T][J*L][2]) "
                                                   "instead of training")
    ap.add_argument("--frames-at", type=float, nargs=2, action="append", default=[], metavar=("EBN0", "FRAMES"),
                    help="frame cap per arm at one Eb/N0 (repeatable)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    import sys
    import os

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth

    code = QCCode(synth.qc_shifts(a.J, a.L, a.p, seed=a.shift_seed), a.p)
    caps = {3.5: a.frames_3p5}
    caps.update({float(e): int(f) for e, f in a.frames_at})
    res = {"code": f"QC {a.J}x{a.L} p={a.p} n={code.N}", "T": a.T, "unroll": a.unroll}
    if a.params:
        params = torch.load(a.params).cuda()
        res["params_from"] = a.params
    else:
        t0 = time.time()
        params, losses = train_noms(code, T=a.T, steps=a.steps, batch=a.batch, lr=a.lr, ebn0=tuple(a.train_ebn0),
                                    unroll=a.unroll, log=print)
        torch.cuda.synchronize()
        res["training"] = {"frames": a.steps * a.batch, "ebn0": a.train_ebn0, "seconds": time.time() - t0,
                           "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:]))}
    res.update({
           "eval": evaluate(code, params, a.ebn0, frames=a.eval_frames, target_fe=a.target_errors,
                            long_iters=a.long_iters, frame_caps=caps),
           "params_w_mean_per_iter": params[..., 0].mean(dim=1).tolist(),
           "params_o_mean_per_iter": params[..., 1].mean(dim=1).tolist()})
    print(json.dumps(res, indent=1))
    if a.out and not a.params:
        torch.save(params.cpu(), os.path.splitext(a.out)[0] + "_params.pt")
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
