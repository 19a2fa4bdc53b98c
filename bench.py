#!/usr/bin/env python
"""Throughput benchmark of the GB300 LDPC decoder.

Workload (one step = one ldpc_ber_sim call through the whole block-code path):
  QC-LDPC 4 x 24, p = 765 (n = 18360, K = N - M = 15300 design information bits),
  seeded shifts, 131072 frames per step decoded in 4096 frame slots (a slot takes
  the next frame as soon as its frame stops), all-zero codeword over BPSK/AWGN at
  Eb/N0 = 3.5 dB generated on the device (Philox + Box-Muller), sum-product with
  FP32 messages, at most 30 iterations with syndrome early stop, device-side
  error counting.

Metric: decoded information Mbit/s = frames * 15300 / seconds (whole job over
all ranks).  Ranks decode disjoint frame ranges (weak scaling, no collective on
the data path; the only collectives are the timing barrier and max).

--impl reference runs the CPU oracle (FP64, OpenMP over frames) on the host
cores on a bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

J, L, P_CIRC, SHIFT_SEED = 4, 24, 765, 2
N_BITS = L * P_CIRC
K_INFO = N_BITS - J * P_CIRC  # 15300
E_EDGES = J * L * P_CIRC
METRIC = "decoded info Mbit/s (n=18360, 30 iters) at BER matching FP64 oracle"
# DRAM bytes (read + write) per check-pass launch, averaged over the launches of one
# default-size call, measured with ncu (dram__bytes_{read,write}.sum) on the default
# workload of this file (FP32 messages, early stop, 3.5 dB, 4096 slots, 131072 frames),
# with the hash of the kernel sources it was measured on: reported only while the
# sources hash the same (null as soon as a kernel changes, until re-measured).
CN_DRAM_BYTES_PER_LAUNCH = {"f32": (2277.8e6, "f63b990e626641ef")}
KERNEL_SOURCES = ("qc_pipe.cu", "qc_device.cuh", "ldpc_internal.cuh")


def kernel_source_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1204_0334_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ebn0", type=float, default=3.5)
    ap.add_argument("--gamma", type=int, default=4096, help="frame slots decoded together")
    ap.add_argument("--frames", type=int, default=131072, help="frames simulated per step")
    ap.add_argument("--iters", type=int, default=30)
    ap.add_argument("--msg", default="f32", choices=["f32", "f16", "i8"])
    ap.add_argument("--no-early-stop", action="store_true")
    ap.add_argument("--codewords", default="zero", choices=["zero", "random"],
                    help="transmitted codewords: all-zero (the paper's protocol) or random, encoded on the device")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ldpccc", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sparse", action="store_true")
    ap.add_argument("--no-noms", action="store_true")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's codes A-D and LDPCCCs A'-D'")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU seconds of the oracle baseline")
    ap.add_argument("--seed", type=int, default=20120403)
    return ap.parse_args()


def workload_name(a) -> str:
    es = "early-stop" if not a.no_early_stop else "fixed"
    cw = ", random codewords" if getattr(a, "codewords", "zero") == "random" else ""
    return (f"QC-LDPC 4x24 p=765 n=18360, {a.frames} frames/step in {a.gamma} slots, {a.iters} iters {es}, "
            f"Eb/N0 {a.ebn0} dB, {a.msg} msgs{cw}")


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                    power.append(float(f[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p >= 0.5 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(a, nframes: int, threads: int, first_frame: int, ebn0=None):
    """Channel + FP64 decode + error count of frames first_frame .. first_frame + nframes - 1 on the host
    cores; returns (seconds, counts) with the counts ldpc_ber_sim reports."""
    import numpy as np
    import oracle
    import synth

    shifts = synth.qc_shifts(J, L, P_CIRC, seed=SHIFT_SEED)
    if not hasattr(oracle_sample, "graph"):
        H = oracle.qc_parity_check(shifts, P_CIRC)
        oracle_sample.graph = oracle.csr_rows(H)
    rp, col = oracle_sample.graph
    sigma = oracle.sigma_from_ebn0(a.ebn0 if ebn0 is None else ebn0, K_INFO / N_BITS)
    t0 = time.perf_counter()
    mu = oracle.channel_awgn(a.seed, first_frame, nframes, N_BITS, sigma)
    _, hard, iters, ok = oracle.sp_decode(rp, col, N_BITS, mu, a.iters, early_stop=not a.no_early_stop,
                                          nthreads=threads)
    errs = hard.sum(axis=1).astype(np.int64)
    dt = time.perf_counter() - t0
    counts = {"frames": nframes, "frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()),
              "iters_sum": int(np.asarray(iters).sum()), "undetected": int(((errs > 0) & (ok == 1)).sum())}
    return dt, counts


COUNT_KEYS = ("frames", "frame_errors", "bit_errors", "iters_sum", "undetected")


def cpu_baseline(a, pkg, code, stream, opts, first_frame: int) -> dict:
    """The FP64 oracle on the host cores, on the first frames of the first timed step (the same frame ids),
    in two forms: OpenMP over frames on every core, and one thread.  Its counts on those frames are put
    beside the GPU's counts on the same frames ("ber_match"), and again at 3.0 dB where frames fail."""
    threads = os.cpu_count() or 1
    n = max(threads, 16)
    dt, cnt = oracle_sample(a, n, threads, first_frame)
    while dt < a.cpu_seconds * 0.5 and n < 4096:
        n = int(min(4096, max(2 * n, n * a.cpu_seconds / max(dt, 1e-3))))
        n = max(threads, (n // threads) * threads)
        dt, cnt = oracle_sample(a, n, threads, first_frame)
    n1 = max(1, min(n, int(round(4.0 * n / max(dt, 1e-3) / threads))))
    dt1, cnt1 = oracle_sample(a, n1, 1, first_frame)

    def gpu_counts(first, frames, ebn0):
        r = pkg.ldpc_ber_sim(code.handle, ebn0, a.seed, first, frames, 1 << 60, a.gamma, opts, stream)
        return {k: int(r[k]) for k in COUNT_KEYS}

    match = []
    if a.msg == "f32" and a.codewords == "zero":  # the oracle leg decodes all-zero frames by FP64 sum-product
        g = gpu_counts(first_frame, n, a.ebn0)
        match.append({"ebn0_db": a.ebn0, "frames": f"{first_frame}..{first_frame + n - 1}", "gpu": g,
                      "oracle": cnt, "equal": all(g[k] == cnt[k] for k in COUNT_KEYS)})
        low = 3.0
        nl = max(threads, 2 * threads)
        _, cl = oracle_sample(a, nl, threads, first_frame, ebn0=low)
        gl = gpu_counts(first_frame, nl, low)
        match.append({"ebn0_db": low, "frames": f"{first_frame}..{first_frame + nl - 1}", "gpu": gl, "oracle": cl,
                      "equal": all(gl[k] == cl[k] for k in COUNT_KEYS)})
    return {"value": n * K_INFO / dt / 1e6, "unit": "Mbit/s", "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"frames {first_frame}..{first_frame + n - 1} of the first timed step ({n} frames: channel + "
                      f"FP64 sum-product, {cnt['iters_sum'] / n:.2f} mean iters) on {threads} host threads, "
                      f"{dt:.1f} s",
            "single_thread": {"value": n1 * K_INFO / dt1 / 1e6, "unit": "Mbit/s", "frames": n1, "seconds": dt1},
            "ber_match": match}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    # size each step to a few seconds of host work
    t, _ = oracle_sample(a, threads, threads, first_frame=1 << 52)
    per = max(threads, int(round(4.0 / max(t, 1e-3))) * threads)
    per = min(per, 2048)
    for w in range(a.warmup):
        oracle_sample(a, threads, threads, first_frame=(1 << 52) + (w + 1) * 4096)
    total_t, frames, iters = 0.0, 0, 0
    for s in range(a.steps):
        dt, cnt = oracle_sample(a, per, threads, first_frame=(1 << 53) + s * per)
        total_t += dt
        frames += per
        iters += cnt["iters_sum"]
    value = frames * K_INFO / total_t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_t / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "frames_per_step": per, "mean_iters": iters / frames},
            "cpu_baseline": {"value": value, "unit": "Mbit/s", "cores": threads, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": f"{per} frames per step, {a.steps} steps"},
            "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU
def run_ours(a):
    import torch

    import synth
    import paper_1204_0334_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    shifts = synth.qc_shifts(J, L, P_CIRC, seed=SHIFT_SEED)
    code = pkg.QCCode(shifts, P_CIRC)
    msg = {"f32": pkg.MSG_F32, "f16": pkg.MSG_F16, "i8": pkg.MSG_I8}[a.msg]
    algo = pkg.ALGO_MS if a.msg == "i8" else pkg.ALGO_SP
    opts = pkg.default_opts(max_iter=a.iters, early_stop=0 if a.no_early_stop else 1, algo=algo, msg=msg,
                            codewords=pkg.CODEWORDS_RANDOM if a.codewords == "random" else pkg.CODEWORDS_ZERO)
    s_msg = {"f32": 4, "f16": 2, "i8": 1}[a.msg]
    s_mu = 1 if a.msg == "i8" else 4
    from paper_1204_0334_gb300 import shard

    def step(i, o=opts):
        return pkg.ldpc_ber_sim(code.handle, a.ebn0, a.seed, shard.first_frame(rank, i, a.frames), a.frames, 1 << 60,
                                a.gamma, o, stream)

    for w in range(a.warmup):
        step(-1 - w)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    pkg.ldpc_profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    res = [step(i) for i in range(a.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    prof = pkg.ldpc_profile_read()
    pkg.ldpc_profile_enable(False)
    clk = clocks.stop()
    ms = shard.max_over_ranks(ms, dist, dev)
    tot = shard.merge_counts(res, dist, dev)
    frames, iters_sum, fe, be = tot["frames"], tot["iters_sum"], tot["frame_errors"], tot["bit_errors"]
    value = frames * K_INFO / (ms / 1e3) / 1e6

    # roofline of the check-node kernel: algorithmic bytes = read + write of every edge message of every
    # frame-iteration the algorithm runs (the iterations each frame needed)
    local_iters = sum(r["iters_sum"] for r in res)
    cn_bytes = 2.0 * E_EDGES * s_msg * local_iters
    cn_s = prof["cn_ms"] / 1e3
    traffic, traffic_src = None, "no ncu measurement of this kernel source and workload"
    meas = CN_DRAM_BYTES_PER_LAUNCH.get(a.msg)
    default_workload = (not a.no_early_stop and a.gamma == 4096 and a.ebn0 == 3.5 and a.iters == 30
                        and a.frames == 131072 and a.codewords == "zero")
    if meas and default_workload and meas[1] == kernel_source_hash():
        traffic, traffic_src = meas[0], f"ncu dram__bytes_read.sum + dram__bytes_write.sum, sources {meas[1]}"
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"bound": "hbm", "kernel": "cn_pipe_kernel (" + ("sum-product" if algo == pkg.ALGO_SP else "min-sum") + ")",
            "achieved": cn_bytes / cn_s / 1e9 if cn_s > 0 else None, "peak": peak, "unit": "GB/s",
            "frac": (cn_bytes / cn_s / 1e9) / peak if cn_s > 0 else None,
            "traffic": traffic,
            "traffic_source": traffic_src,
            "algorithmic_bytes_per_launch": cn_bytes / max(1, prof["cn_launches"]),
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback",
            "cn_launches": prof["cn_launches"], "cn_ms_avg": prof["cn_ms"] / max(1, prof["cn_launches"]),
            "vn_ms_avg": prof["vn_ms"] / max(1, prof["vn_launches"]),
            "path_bytes_per_frame_iter": 4 * E_EDGES * s_msg + N_BITS * s_mu + N_BITS // 8,
            "path_achieved_gbs": (4 * E_EDGES * s_msg + N_BITS * s_mu + N_BITS / 8) * local_iters / (ms / 1e3) / 1e9}
    line = {"metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i8" if a.msg == "i8" else "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "slots": a.gamma, "frames_per_step": a.frames,
                       "iters_cap": a.iters,
                       "early_stop": not a.no_early_stop, "ebn0_db": a.ebn0, "msg": a.msg,
                       "l2": "inputs larger than L2 (message store %.2f GB)" % (
                           E_EDGES * s_msg * a.gamma / 1e9)},
            "frames": frames, "mean_iters": iters_sum / frames, "fer": fe / frames, "ber": be / (frames * N_BITS),
            "frames_per_s": frames / (ms / 1e3), "roofline": roof, "clocks": clk,
            "gpu_launches": prof["launches"]}

    if not a.no_variants:
        line["variants"] = variants(a, pkg, code, stream, opts)
    if not a.no_e2e:
        line["e2e"] = e2e(a, pkg, code, stream, opts)
    if not a.no_variants:
        # the library's slot-count autotuner on the same code and options (the headline keeps its slots)
        line["autotune"] = pkg.ldpc_tune_slots(code.handle, a.ebn0, a.seed, opts, stream)
    if not a.no_ldpccc:
        line["ldpccc"] = ldpccc_bench(a, pkg, stream)
        line["ldpccc_tanner"] = ldpccc_bench(a, pkg, stream, tanner=True)
    if not a.no_batch:
        line["hetero_batch"] = batch_bench(a, pkg, stream)
    if not a.no_noms:
        line["noms_training"] = noms_training_bench(a, pkg, code, stream)
    if not a.no_paper:
        line["paper_workloads"] = paper_workloads_bench(a, pkg, stream)
    if not a.no_sparse:
        line["general_code"] = sparse_bench(a, pkg, code, stream)
    roof.update(bandwidth_probes(pkg, stream))
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, pkg, code, stream, opts, shard.first_frame(rank, 0, a.frames))
    if rank == 0:
        print(json.dumps(line), flush=True)
    code.close()
    if dist:
        dist.destroy_process_group()


def bandwidth_probes(pkg, stream) -> dict:
    """This library's streaming probe: an L2-resident read (32 MB buffer, the peak for L2 byte rates) and an
    HBM copy of 2 GB (read + write bytes; beside MEASURED_PEAKS' copy figure)."""
    import torch

    small = torch.empty(32 << 20, dtype=torch.uint8, device="cuda")
    small.random_(0, 255)
    sink = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    l2 = pkg.ldpc_bandwidth_probe(small, sink, 2000, 0, stream)
    big = torch.empty(2 << 30, dtype=torch.uint8, device="cuda")
    dst = torch.empty_like(big)
    hbm = pkg.ldpc_bandwidth_probe(big, dst, 5, 1, stream)
    del big, dst
    return {"l2_probe_gbs": l2, "l2_probe": "ld.global.cg read sweeps of a 32 MB buffer (L2-resident)",
            "hbm_probe_gbs": hbm, "hbm_probe": "copy of 2 GB (read + write bytes)"}


def variants(a, pkg, code, stream, opts) -> dict:
    """Secondary figures on the same batch (not the headline): other message types, no early stop."""
    import torch

    out = {}
    cases = [("f32_fixed30", dict(early_stop=0, algo=pkg.ALGO_SP, msg=pkg.MSG_F32)),
             ("f16_early_stop", dict(early_stop=1, algo=pkg.ALGO_SP, msg=pkg.MSG_F16)),
             ("i8_minsum_early_stop", dict(early_stop=1, algo=pkg.ALGO_MS, msg=pkg.MSG_I8)),
             ("i8_minsum_fixed30", dict(early_stop=0, algo=pkg.ALGO_MS, msg=pkg.MSG_I8)),
             # random codewords encoded on the device (errors over the information bits)
             ("f32_random_codewords", dict(early_stop=1, algo=pkg.ALGO_SP, msg=pkg.MSG_F32,
                                           codewords=pkg.CODEWORDS_RANDOM))]
    for name, kw in cases:
        o = pkg.default_opts(max_iter=a.iters, **kw)
        base = (7 << 44)
        pkg.ldpc_ber_sim(code.handle, a.ebn0, a.seed, base, a.frames, 1 << 60, a.gamma, o, stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 3
        ev0.record(stream)
        rs = [pkg.ldpc_ber_sim(code.handle, a.ebn0, a.seed, base + (i + 1) * a.frames, a.frames, 1 << 60, a.gamma,
                               o, stream) for i in range(k)]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        fr = sum(r["frames"] for r in rs)
        out[name] = {"value": fr * K_INFO / (ms / 1e3) / 1e6, "unit": "Mbit/s", "ms_per_step": ms / k,
                     "mean_iters": sum(r["iters_sum"] for r in rs) / fr,
                     "fer": sum(r["frame_errors"] for r in rs) / fr}
    return out


def ldpccc_bench(a, pkg, stream, tanner=False) -> dict:
    """Pipelined LDPCCC decoder (secondary workload): 3x6 QC base, p = 128, I = 30 processors, 1024 streams,
    Eb/N0 2.0 dB; frames generated on the device, then decoded window by window.  Sec. II-D unwrapping
    (Lambda = 3, c = 256, b = 128) or, with tanner, the time-invariant code with delays D^a (frames of 128
    instants, c = 768, b = 384, memory up to 127 instants)."""
    import torch

    import synth

    J_, L_, p_, I_, g_ = 3, 6, 128, 30, 1024
    cc = pkg.LDPCCC(synth.qc_shifts(J_, L_, p_, seed=3), p_, I_, g_, tanner=tanner)
    T = 80 if tanner else 200
    llr = cc.channel(2.0, a.seed, 0, T)
    hard = torch.empty((g_, T, cc.c), dtype=torch.uint8, device="cuda")
    pkg.ldpccc_decode_window(cc.handle, llr, 30.0, hard, None, stream)  # fills the pipeline
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    windows = 3
    decided = 0
    ev0.record(stream)
    for w in range(windows):
        pkg.ldpccc_channel(cc.handle, 2.0, a.seed, T * (w + 1), llr, stream)
        _, n = pkg.ldpccc_decode_window(cc.handle, llr, 30.0, hard, None, stream)
        decided += n
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    errs = int(hard[:, :decided // windows].sum().item())
    cc.close()
    slot_bytes = I_ * (4 * J_ * cc.c * 4 + cc.c * 4) + cc.c // 8  # per stream per slot: edges r/w twice, mu
    name = ("time-invariant LDPCCC, delays from 3x6 QC shifts, p=128 (frames of 128 instants: c=768, b=384, ms=1)"
            if tanner else "LDPCCC from 3x6 QC, p=128 (c=256, b=128, ms=2)")
    return {"workload": name + ", I=30, 1024 streams, 2.0 dB",
            "value": g_ * decided * cc.b / (ms / 1e3) / 1e6, "unit": "Mbit/s", "ms_per_slot": ms / (windows * T),
            "achieved_gbs": g_ * slot_bytes * windows * T / (ms / 1e3) / 1e9,
            "bit_errors_last_window": errs}


def noms_training_bench(a, pkg, code, stream) -> dict:
    """One training step of the learned min-sum on the headline code: ldpc_noms_forward + ldpc_noms_backward on
    1024 frames (3.5 dB), 10 unrolled iterations, FP16 saved messages, a checkpoint every 2 iterations."""
    import torch

    B, T, ck = 1024, 10, 2
    llr = torch.empty((B, code.N), dtype=torch.float32, device="cuda")
    pkg.ldpc_channel(code.handle, 3.5, a.seed, 1 << 45, llr, stream)
    prm = torch.empty((T, J * L, 2), dtype=torch.float32, device="cuda")
    prm[..., 0] = 0.8
    prm[..., 1] = 0.1
    grad = torch.zeros_like(prm)
    for _ in range(2):
        pkg.ldpc_noms_forward(code.handle, llr, prm, pkg.MSG_F16, ck, 30.0, False, stream)
        pkg.ldpc_noms_backward(code.handle, prm, grad, stream)
    torch.cuda.synchronize()
    k = 5
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3 * k)]
    for i in range(k):
        evs[3 * i].record(stream)
        pkg.ldpc_noms_forward(code.handle, llr, prm, pkg.MSG_F16, ck, 30.0, False, stream)
        evs[3 * i + 1].record(stream)
        pkg.ldpc_noms_backward(code.handle, prm, grad, stream)
        evs[3 * i + 2].record(stream)
    torch.cuda.synchronize()
    fwd = sum(evs[3 * i].elapsed_time(evs[3 * i + 1]) for i in range(k)) / k
    bwd = sum(evs[3 * i + 1].elapsed_time(evs[3 * i + 2]) for i in range(k)) / k
    # canonical forward bytes per frame-iteration: FP16 messages read + written in both passes, channel LLRs
    fwd_bytes = B * T * (4 * E_EDGES * 2 + N_BITS * 4)
    peak = load_peaks().get("hbm_gbs", 6800.0)
    return {"workload": "learned min-sum training step, n=18360, 1024 frames, 10 iterations, FP16, checkpoint every 2",
            "frames_per_s": B / ((fwd + bwd) / 1e3), "fwd_ms": fwd, "bwd_ms": bwd, "bwd_over_fwd": bwd / fwd,
            "fwd_achieved_gbs": fwd_bytes / (fwd / 1e3) / 1e9, "fwd_frac": fwd_bytes / (fwd / 1e3) / 1e9 / peak}


# the paper's own workloads (Sec. V, tables "newdectime" and "dectime_ldpccc"): GTX460 time per
# codeword / frame in ms, for context beside this GPU's
PAPER_BLOCK_MS = {422: 2.12, 632: 2.9, 768: 3.4, 1024: 4.5}
PAPER_LDPCCC_MS = {422: 0.23, 632: 0.31, 768: 0.38, 1024: 0.48}


def paper_workloads_bench(a, pkg, stream) -> dict:
    """Codes A-D (4x24, p = 422 .. 1024, seeded shifts) at 3.2 dB with 30 iterations (no early stop) in 4096 slots,
    and their LDPCCCs A'-D' (Lambda = 4) at 3.1 dB with I = 20 processors for 1024 streams: time per codeword /
    per frame on this GPU beside the paper's GTX460 figures (context, not a target)."""
    import torch

    import synth

    out = {}
    for p_, ms_paper in PAPER_BLOCK_MS.items():
        code = pkg.QCCode(synth.qc_shifts(4, 24, p_, seed=7), p_)
        o = pkg.default_opts(max_iter=30, early_stop=0)
        frames = 16384
        pkg.ldpc_ber_sim(code.handle, 3.2, a.seed, 0, 4096, 1 << 60, 4096, o, stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        r = pkg.ldpc_ber_sim(code.handle, 3.2, a.seed, 1 << 20, frames, 1 << 60, 4096, o, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        us = ms * 1e3 / r["frames"]
        out[f"block_p{p_}"] = {"us_per_codeword": us, "mbit_s": r["frames"] * code.K / (ms / 1e3) / 1e6,
                               "fer": r["frame_errors"] / r["frames"], "paper_gtx460_us": ms_paper * 1e3,
                               "ratio": ms_paper * 1e3 / us}
        code.close()
    for p_, ms_paper in PAPER_LDPCCC_MS.items():
        g, T = 1024, 32
        cc = pkg.LDPCCC(synth.qc_shifts(4, 24, p_, seed=7), p_, 20, g)
        llr = torch.empty((g, T, cc.c), dtype=torch.float32, device="cuda")
        hard = torch.empty((g, T, cc.c), dtype=torch.uint8, device="cuda")
        # fill the pipeline (I * Lambda = 80 frames) so that every timed slot decides a frame
        fill = (20 * cc.Lambda + T - 1) // T + 1
        for w in range(fill):
            pkg.ldpccc_channel(cc.handle, 3.1, a.seed, T * w, llr, stream)
            pkg.ldpccc_decode_window(cc.handle, llr, 30.0, hard, None, stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        decided = 0
        for w in range(fill, fill + 2):
            pkg.ldpccc_channel(cc.handle, 3.1, a.seed, T * w, llr, stream)
            _, n = pkg.ldpccc_decode_window(cc.handle, llr, 30.0, hard, None, stream)
            decided += n
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        us = ms * 1e3 / (decided * g)
        out[f"ldpccc_p{p_}"] = {"us_per_frame": us, "mbit_s": decided * g * cc.b / (ms / 1e3) / 1e6,
                                "paper_gtx460_us": ms_paper * 1e3, "ratio": ms_paper * 1e3 / us}
        cc.close()
    return out


def batch_bench(a, pkg, stream) -> dict:
    """64 seeded QC codes (3x6 .. 4x24, p 32..765), 1..4096 frames each (log-uniform), FP16 messages, 30 iterations
    with early stop, one shared persistent iteration loop per call (CUDA graph), Eb/N0 3.0 dB, device channel."""
    import torch

    import synth

    mixed = synth.mixed_codes(64, seed=4)
    counts = [int(g) for g in synth.frame_counts(64, seed=4)]
    codes = [pkg.QCCode(sh, p) for (J, L, p, sh) in mixed]
    o = pkg.default_opts(max_iter=30, early_stop=1, msg=pkg.MSG_F16)
    b = pkg.ldpc_batch_create(codes, counts, o)
    llrs = []
    for i, (c, g) in enumerate(zip(codes, counts)):
        x = torch.empty((g, c.N), dtype=torch.float32, device="cuda")
        pkg.ldpc_channel(c.handle, 3.0, a.seed, i << 20, x, stream)
        llrs.append(x)
    its = [torch.empty(g, dtype=torch.int32, device="cuda") for g in counts]
    for _ in range(2):  # tuning + eager run, then the graph capture
        pkg.ldpc_batch_decode(b, llrs, None, its, None, stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = 5
    ev0.record(stream)
    for _ in range(k):
        pkg.ldpc_batch_decode(b, llrs, None, its, None, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / k
    info_bits = sum(c.K * g for c, g in zip(codes, counts))
    it_sums = [float(t.float().sum()) for t in its]
    mean_it = sum(it_sums) / sum(counts)
    # canonical bytes: per frame-iteration 4*E*2 (FP16 messages) + N*4 (channel LLRs) + N/8 (hard bits)
    path_bytes = sum(s_ * (8 * c.E + 4 * c.N + c.N / 8) for c, s_ in zip(codes, it_sums))

    info = pkg.ldpc_batch_info(b)
    moved = sum(pkg.ldpc_batch_moved(b, len(codes)))
    # one decode's phase boundaries (30 iterations x tiles, syndrome, check, variable pass) as graph
    # launches against grid barriers of one cooperative kernel, both without work
    sync = pkg.ldpc_sync_probe(120, 100)
    comp = pkg.ldpc_batch_compaction(b)
    pkg.ldpc_batch_destroy(b)
    peak = load_peaks().get("hbm_gbs", 6800.0)
    return {"workload": "64 QC codes 3x6..4x24, p 32..765, %d frames total (1..4096 per code), FP16, 30 iters "
                        "early stop, 3.0 dB" % sum(counts),
            "value": info_bits / (ms / 1e3) / 1e6, "unit": "Mbit/s", "ms_per_batch": ms, "mean_iters": mean_it,
            "path_achieved_gbs": path_bytes / (ms / 1e3) / 1e9, "path_frac": path_bytes / (ms / 1e3) / 1e9 / peak,
            "tile_rows": info["tile_rows"], "tile_groups": info["tile_groups"],
            "frames_compacted": moved, "compaction_after_iter": comp["after_iter"],
            "compaction_tune_ms": comp["tune_ms"],
            "phase_boundary_us": {"graph": sync["graph_us"], "cooperative": sync["cooperative_us"],
                                  "boundaries_per_decode": 120}}


def sparse_bench(a, pkg, qc, stream) -> dict:
    """General (index-table) decoder on a random code of the headline's shape (n = 18360, M = 3060,
    column weight 4, row weight 24), 4096 frames of the device channel at the bench's Eb/N0, 30 fixed
    iterations, FP32, through ldpc_decode -- and the QC decoder on the same frame ids for comparison."""
    import numpy as np
    import torch

    import synth

    rp, col = synth.random_ldpc(N_BITS, J * P_CIRC, seed=11, var_degrees=(4,))
    sc = pkg.SparseCode(rp, col, N_BITS)
    g = 4096
    out = {"workload": "random code n=18360, M=3060, column weight 4 (rows %d..%d), 4096 frames, 30 fixed iterations, "
                       "FP32, %.2f dB" % (int(np.diff(rp).min()), int(np.diff(rp).max()), a.ebn0)}
    for name, c in (("general", sc), ("qc", qc)):
        llr = torch.empty((g, N_BITS), dtype=torch.float32, device="cuda")
        pkg.ldpc_channel(c.handle, a.ebn0, a.seed, 1 << 44, llr, stream)
        hard = torch.empty((g, N_BITS), dtype=torch.uint8, device="cuda")
        o = pkg.default_opts(max_iter=30, early_stop=0)
        pkg.ldpc_decode(c.handle, llr, o, None, hard, None, None, stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 3
        ev0.record(stream)
        for _ in range(k):
            pkg.ldpc_decode(c.handle, llr, o, None, hard, None, None, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / k
        path = 30 * g * (4 * c.E * 4 + N_BITS * 4 + N_BITS / 8)
        out[name] = {"value": g * K_INFO / (ms / 1e3) / 1e6, "unit": "Mbit/s", "ms_per_decode": ms,
                     "path_achieved_gbs": path / (ms / 1e3) / 1e9,
                     "frame_errors": int((hard.sum(dim=1) > 0).sum().item())}
    sc.close()
    return out


def e2e(a, pkg, code, stream, opts) -> dict:
    """Same metric through ldpc_decode with pinned HOST buffers: one call per step on the step's frames
    (--frames, at least 2 x slots so that they stream; the LLRs of the call read from host memory, the
    hard decisions, iteration counts and ok flags written back to host memory, inside the timed region;
    with early stop the frames stream through the slots)."""
    import torch

    gamma = max(a.frames, 2 * a.gamma)
    llr_dev = torch.empty((gamma, code.N), dtype=torch.float32, device="cuda")
    pkg.ldpc_channel(code.handle, a.ebn0, a.seed, 3 << 44, llr_dev, stream)
    llr = llr_dev.cpu().pin_memory()
    del llr_dev
    hard = torch.empty((gamma, code.N), dtype=torch.uint8).pin_memory()
    iters = torch.empty(gamma, dtype=torch.int32).pin_memory()
    ok = torch.empty(gamma, dtype=torch.int32).pin_memory()
    o = opts
    pkg.ldpc_decode(code.handle, llr, o, None, hard, iters, ok, stream)
    torch.cuda.synchronize()
    k = 3
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(k):
        pkg.ldpc_decode(code.handle, llr, o, None, hard, iters, ok, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    return {"value": gamma * k * K_INFO / (ms / 1e3) / 1e6, "unit": "Mbit/s",
            "h2d_bytes_per_step": gamma * code.N * 4, "d2h_bytes_per_step": gamma * code.N + 2 * gamma * 4,
            "ms_per_step": ms / k, "frames_per_step": gamma, "mean_iters": float(iters.float().mean()),
            "call": "ldpc_decode(pinned host llr [gamma][N] f32 -> pinned host hard [gamma][N] u8, iters, ok)"}


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
