"""BER/FER of the message precisions on one code: sum-product with FP32 and FP16 messages
and integer min-sum, each through ldpc_ber_sim (device channel, continuous simulation) on
the same frames, with 95% confidence intervals (exact for the FER; for the BER from the
frame-level variance of the error counts, since the bits of a frame do not fail independently).

    python -m paper_1204_0334_gb300.precision --ebn0 3.0 3.25 --target-errors 200
"""
from __future__ import annotations

import argparse
import json
import os
import sys

from . import ALGO_MS, ALGO_SP, MSG_F16, MSG_F32, MSG_I8, QCCode, default_opts, ldpc_ber_sim
from .noms import ber_interval, clopper_pearson

CASES = [("sp_f32", dict(algo=ALGO_SP, msg=MSG_F32)), ("sp_f16", dict(algo=ALGO_SP, msg=MSG_F16)),
         ("minsum_i8", dict(algo=ALGO_MS, msg=MSG_I8))]


def run(code: QCCode, ebn0_points, max_frames: int, target_errors: int, iters: int, gamma: int, seed: int):
    out = {}
    for e in ebn0_points:
        row = {}
        for name, kw in CASES:
            o = default_opts(max_iter=iters, early_stop=1, **kw)
            r = ldpc_ber_sim(code.handle, e, seed, 0, max_frames, target_errors, gamma, o)
            nb = r["frames"] * code.N
            r["ber"] = r["bit_errors"] / nb
            r["ber_ci95"] = ber_interval(r, code.N)
            r["fer"] = r["frame_errors"] / r["frames"]
            r["fer_ci95"] = clopper_pearson(r["frame_errors"], r["frames"])
            r["mean_iters"] = r["iters_sum"] / r["frames"]
            r["mbit_s"] = r["frames"] * code.K / r["seconds"] / 1e6
            row[name] = r
        out[str(e)] = row
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--J", type=int, default=4)
    ap.add_argument("--L", type=int, default=24)
    ap.add_argument("--p", type=int, default=765)
    ap.add_argument("--shift-seed", type=int, default=2)
    ap.add_argument("--ebn0", type=float, nargs="*", default=[3.0, 3.25])
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--gamma", type=int, default=4096)
    ap.add_argument("--max-frames", type=int, default=1 << 20)
    ap.add_argument("--target-errors", type=int, default=200)
    ap.add_argument("--seed", type=int, default=777)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth

    code = QCCode(synth.qc_shifts(a.J, a.L, a.p, seed=a.shift_seed), a.p)
    res = {"code": f"QC {a.J}x{a.L} p={a.p} n={code.N}", "iters": a.iters,
           "eval": run(code, a.ebn0, a.max_frames, a.target_errors, a.iters, a.gamma, a.seed)}
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
