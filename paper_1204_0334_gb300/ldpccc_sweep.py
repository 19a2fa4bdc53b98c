"""BER of the pipelined LDPCCC decoder (Algorithm 2) over an Eb/N0 sweep, for the code derived
by the Sec. II-D unwrapping and for the time-invariant code with delays D^{a_jl}, both from the
same QC base: all-zero frames from the device channel (ldpccc_channel), decoded window by window
(ldpccc_decode_window); bit errors of the decided frames with exact 95% confidence intervals.

    python -m paper_1204_0334_gb300.ldpccc_sweep --ebn0 1.5 1.75 2.0 2.25 2.5 2.75 3.0
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

from . import LDPCCC, ldpccc_channel, ldpccc_decode_window
from .noms import clopper_pearson


def run_point(cc: LDPCCC, ebn0: float, seed: int, info_bits: int, window: int, stream=None) -> dict:
    """Decode until at least info_bits information bits have been decided past the pipeline's fill."""
    import torch

    g, c = cc.gamma, cc.c
    llr = torch.empty((g, window, c), dtype=torch.float32, device="cuda")
    hard = torch.empty((g, window, c), dtype=torch.uint8, device="cuda")
    from . import ldpccc_reset

    ldpccc_reset(cc.handle)
    first, errors, decided = 0, 0, 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while decided * g * cc.b < info_bits:
        ldpccc_channel(cc.handle, ebn0, seed, first, llr, stream)
        _, n = ldpccc_decode_window(cc.handle, llr, 30.0, hard, None, stream)
        first += window
        if n:
            errors += int(hard[:, :n].sum().item())
            decided += n
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    nb = decided * g * c
    return {"frames_decided_per_stream": decided, "streams": g, "bit_errors": errors, "ber": errors / nb,
            "ber_ci95": clopper_pearson(errors, nb), "mbit_s": decided * g * cc.b / secs / 1e6}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--J", type=int, default=3)
    ap.add_argument("--L", type=int, default=6)
    ap.add_argument("--p", type=int, default=128)
    ap.add_argument("--I", type=int, default=30)
    ap.add_argument("--streams", type=int, default=1024)
    ap.add_argument("--shift-seed", type=int, default=3)
    ap.add_argument("--ebn0", type=float, nargs="*", default=[1.5, 1.75, 2.0, 2.25, 2.5, 2.75, 3.0])
    ap.add_argument("--info-bits", type=float, default=2e8, help="information bits decided per point and code")
    ap.add_argument("--seed", type=int, default=515)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import synth

    shifts = synth.qc_shifts(a.J, a.L, a.p, seed=a.shift_seed)
    res = {"base": f"QC {a.J}x{a.L} p={a.p}", "I": a.I, "streams": a.streams}
    for name, tanner in (("sec2d_unwrapping", False), ("time_invariant_delays", True)):
        cc = LDPCCC(shifts, a.p, a.I, a.streams, tanner=tanner)
        window = max(16, (4096 * 256) // cc.c // 4)
        res[name] = {"c": cc.c, "b": cc.b, "ms": cc.ms,
                     "points": {str(e): run_point(cc, e, a.seed, int(a.info_bits), window) for e in a.ebn0}}
        cc.close()
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
