import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print the FP32 parity figures the GPU tests recorded (frames and elements that needed the
    conditioning arm, largest relative deviation from the FP64 oracle)."""
    try:
        from helpers import PARITY_RECORDS
    except ImportError:
        return
    if not PARITY_RECORDS:
        return
    tr = terminalreporter
    tr.section("FP32 parity against the FP64 oracle")
    arm_f = sum(r.get("arm_frames", 0) for r in PARITY_RECORDS)
    arm_e = sum(r.get("arm_elems", 0) for r in PARITY_RECORDS)
    tot_f = sum(r.get("frames", 0) for r in PARITY_RECORDS)
    tot_e = sum(r.get("elems", 0) for r in PARITY_RECORDS)
    tr.write_line(f"{len(PARITY_RECORDS)} comparisons, {tot_f} frames, {tot_e} posteriors; conditioning arm: "
                  f"{arm_f} frames, {arm_e} posteriors")
    for r in PARITY_RECORDS:
        extra = "".join(f" {k}={v:.3g}" if isinstance(v, float) else f" {k}={v}" for k, v in r.items()
                        if k not in ("label",))
        tr.write_line(f"  {r['label']}:{extra}")
