"""GPU parity of the pipelined LDPCCC window decoder (Algorithm 2) against the CPU oracle.

The oracle runs Algorithm 2 slot by slot on the explicitly unwrapped H (Sec. II-D);
the GPU decoder is fed the same frames, in one or several windows.  Tolerances as
for the block decoder: posteriors within 1e-4 * max(1, |oracle|), or within 16x the
oracle's own response to a one-ulp change of its FP32 input and never beyond
2e-3 * max(1, |oracle|); hard decisions equal wherever |oracle| >= 1e-3.  The frames
and posteriors that needed the second arm are recorded in the test summary.
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import record_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL, SENS, CEIL = 1e-4, 16.0, 2e-3


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_0334_gb300 as p

    p.lib()
    return p


def run_gpu(pkg, shifts, p, I, mu, windows, tanner=False):
    """mu: [gamma][T][c] numpy; windows: list of window lengths summing to T."""
    g, T, c = mu.shape
    cc = pkg.LDPCCC(shifts, p, I, g, tanner=tanner)
    assert cc.c == c
    hard = np.zeros((g, T, c), dtype=np.uint8)
    post = np.zeros((g, T, c), dtype=np.float32)
    decided = np.zeros(T, dtype=bool)
    t = 0
    for w in windows:
        x = torch.from_numpy(np.ascontiguousarray(mu[:, t:t + w])).cuda()
        first, n, h, pst = cc.window(x)
        if n:
            hard[:, first:first + n] = h.cpu().numpy()
            post[:, first:first + n] = pst.cpu().numpy()
            decided[first:first + n] = True
        t += w
    cc.close()
    return hard, post, decided


def run_oracle(shifts, p, I, mu, tanner=False):
    g, T, c = mu.shape
    Hc, geo = (oracle.ldpccc_tanner if tanner else oracle.ldpccc_unwrap)(shifts, p, T)
    po, ho, dec, _ = oracle.ldpccc_decode(Hc, geo, T, I, mu.reshape(g, T * c), nthreads=8)
    return Hc, geo, po.reshape(g, T, c), ho.reshape(g, T, c), dec


def compare(shifts, p, I, mu, hard, post, decided, label, tanner=False):
    Hc, geo, po, ho, dec = run_oracle(shifts, p, I, mu, tanner)
    g, T, c = mu.shape
    assert np.array_equal(dec[0].astype(bool), decided), label
    sel = decided
    dev = np.abs(post[:, sel].astype(np.float64) - po[:, sel])
    rel = dev / np.maximum(1.0, np.abs(po[:, sel]))
    arm_f = arm_e = 0
    if rel.max() > REL:
        # conditioning arm: the oracle's response to a one-ulp change of its input
        rng = np.random.default_rng(5)
        up = rng.integers(0, 2, size=mu.shape).astype(bool)
        m2 = np.where(up, np.nextafter(mu, np.float32(np.inf)), np.nextafter(mu, np.float32(-np.inf)))
        _, _, p2, _, _ = run_oracle(shifts, p, I, m2.astype(np.float32), tanner)
        resp = np.abs(p2[:, sel] - po[:, sel]).max(axis=2, keepdims=True)
        allowed = np.maximum(REL * np.maximum(1.0, np.abs(po[:, sel])), SENS * resp)
        assert (dev <= allowed).all(), f"{label}: deviation {dev.max():.3e}"
        assert rel.max() <= CEIL, f"{label}: relative deviation {rel.max():.3e} beyond the ceiling {CEIL}"
        arm_f = int((rel > REL).any(axis=2).sum())
        arm_e = int((rel > REL).sum())
    record_parity(f"LDPCCC {label}", frames=int(g * sel.sum()), arm_frames=arm_f, arm_elems=arm_e,
                  elems=int(rel.size), max_rel=float(rel.max()))
    sure = np.abs(po[:, sel]) >= 1e-3
    assert np.array_equal(hard[:, sel][sure], ho[:, sel][sure]), label
    return rel.max()


@pytest.mark.parametrize("J,L,p,I,gamma,T,windows,ebn0", [
    (3, 6, 16, 5, 40, 60, [60], 1.5),          # Lambda = 3, ragged packages (40 streams)
    (4, 8, 8, 3, 33, 50, [17, 25, 8], 2.0),    # Lambda = 4, three windows (continuity)
    (3, 7, 11, 4, 32, 30, [30], 2.0),          # Lambda = 1: frames decode independently
    (2, 6, 20, 6, 64, 70, [1, 69], 1.5),       # Lambda = 2, a one-frame window first
    (4, 24, 7, 3, 32, 30, [30], 3.5),          # Lambda = 4, rows of 24 edges (the paper's A'-D' shape)
])
def test_ldpccc_matches_oracle(pkg, J, L, p, I, gamma, T, windows, ebn0):
    shifts = synth.qc_shifts(J, L, p, seed=J * 100 + L)
    c = (L // np.gcd(J, L)) * p
    mu = synth.gaussian_llrs(gamma, T * c, seed=T, ebn0_db=ebn0, rate=1 - J / L).reshape(gamma, T, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, windows)
    compare(shifts, p, I, mu, hard, post, decided, f"{J}x{L} p={p} I={I}")


def test_ldpccc_zero_blocks(pkg):
    J, L, p, I = 4, 8, 9, 3
    shifts = synth.qc_shifts(J, L, p, seed=77, zero_blocks=5)
    c = (L // 4) * p
    mu = synth.gaussian_llrs(32, 40 * c, seed=3, ebn0_db=2.0, rate=0.5).reshape(32, 40, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, [40])
    compare(shifts, p, I, mu, hard, post, decided, "zero blocks")


def test_ldpccc_reset_restarts_stream(pkg):
    J, L, p, I = 3, 6, 8, 3
    shifts = synth.qc_shifts(J, L, p, seed=5)
    c = 2 * p
    mu = synth.gaussian_llrs(32, 30 * c, seed=9, ebn0_db=2.0, rate=0.5).reshape(32, 30, c)
    cc = pkg.LDPCCC(shifts, p, I, 32)
    x = torch.from_numpy(mu).cuda()
    a = cc.window(x)
    pkg.ldpccc_reset(cc.handle)
    b = cc.window(x)
    assert a[0] == b[0] == 0 and a[1] == b[1] == 30 - I * 3 + 1
    assert torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])
    cc.close()


def test_ldpccc_full_size_sampled(pkg):
    """3x6, p = 128 (c = 256, b = 128, Lambda = 3, ms = 2), I = 30 processors, 1024 streams:
    two sampled streams against the oracle over 300 frames."""
    J, L, p, I, g, T = 3, 6, 128, 30, 1024, 300
    shifts = synth.qc_shifts(J, L, p, seed=3)
    c = 256
    mu = synth.gaussian_llrs(g, T * c, seed=11, ebn0_db=2.0, rate=0.5).reshape(g, T, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, [120, 180])
    assert decided.sum() == T - I * 3 + 1
    idx = [0, 777]
    compare(shifts, p, I, mu[idx], hard[idx], post[idx], decided, "cfg3 sampled")


def test_ldpccc_channel_matches_oracle(pkg):
    """Stream s, frame f draws Philox counter (n/4, f, s, 1): the oracle's channel with frame id s*2^32 + f, tag 1."""
    J, L, p, I, g = 3, 6, 20, 2, 40
    cc = pkg.LDPCCC(synth.qc_shifts(J, L, p, seed=1), p, I, g)
    out = cc.channel(2.5, seed=123, first_frame=7, T=5).cpu().numpy().astype(np.float64)
    assert out.shape[1:] == (5, cc.c)
    sigma = oracle.sigma_from_ebn0(2.5, cc.b / cc.c)
    for s in (0, 17, 39):
        mu = oracle.channel_awgn(123, (s << 32) + 7, 5, cc.c, sigma, tag=1)
        assert np.array_equal(out[s], mu.astype(np.float64))  # the generator's binary32 bits
    cc.close()


# --------------------------------------------------------------------------
# time-invariant code with delays D^{a_jl} (frames of p instants, ms = 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("J,L,p,I,gamma,T,windows,ebn0,zb", [
    (3, 6, 16, 5, 40, 40, [40], 1.5, 0),         # ragged packages (40 streams)
    (4, 8, 8, 3, 33, 30, [11, 19], 2.0, 0),      # two windows (continuity)
    (4, 8, 9, 3, 32, 25, [25], 2.0, 5),          # zero blocks
    (2, 6, 20, 6, 64, 40, [1, 39], 1.5, 0),      # a one-frame window first
    (4, 24, 7, 3, 32, 20, [20], 3.5, 0),         # rows of 24 edges
])
def test_tanner_ldpccc_matches_oracle(pkg, J, L, p, I, gamma, T, windows, ebn0, zb):
    shifts = synth.qc_shifts(J, L, p, seed=J * 10 + L + zb, zero_blocks=zb)
    c = L * p
    mu = synth.gaussian_llrs(gamma, T * c, seed=T + 1, ebn0_db=ebn0, rate=1 - J / L).reshape(gamma, T, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, windows, tanner=True)
    compare(shifts, p, I, mu, hard, post, decided, f"tanner {J}x{L} p={p} I={I}", tanner=True)


def test_tanner_ldpccc_dims_and_zero_delays(pkg):
    """Dimensions of the time-invariant code; all delays 0 gives ms = 0 (frames decode independently),
    decided one slot after I - 1 further frames, as the oracle's block decoding."""
    shifts = synth.qc_shifts(3, 6, 16, seed=2)
    cc = pkg.LDPCCC(shifts, 16, 4, 32, tanner=True)
    assert (cc.c, cc.b, cc.ms, cc.Lambda) == (96, 48, 1, 1)
    cc.close()
    z = np.zeros((3, 6), dtype=np.int64)
    mu = synth.gaussian_llrs(32, 12 * 30, seed=7, ebn0_db=2.0, rate=0.5).reshape(32, 12, 30)
    hard, post, decided = run_gpu(pkg, z, 5, 4, mu, [12], tanner=True)
    assert decided.sum() == 12 - 4 + 1
    compare(z, 5, 4, mu, hard, post, decided, "tanner zero delays", tanner=True)


def test_tanner_ldpccc_full_size_sampled(pkg):
    """3x6 base, p = 128 delays (memory up to 127 instants; frames of 128 instants, c = 768), I = 30
    processors, 1024 streams: two sampled streams against the oracle over 100 frames."""
    J, L, p, I, g, T = 3, 6, 128, 30, 1024, 100
    shifts = synth.qc_shifts(J, L, p, seed=3)
    c = L * p
    mu = synth.gaussian_llrs(g, T * c, seed=12, ebn0_db=2.0, rate=0.5).reshape(g, T, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, [40, 60], tanner=True)
    assert decided.sum() == T - I * 2 + 1
    idx = [0, 901]
    compare(shifts, p, I, mu[idx], hard[idx], post[idx], decided, "tanner cfg3 sampled", tanner=True)


def test_tanner_ldpccc_single_processor_single_stream(pkg):
    """I = 1 (each frame gets one iteration, decided one frame later) and a single stream (one lane of one
    package), fed one frame per window."""
    J, L, p, I, T = 3, 6, 12, 1, 9
    shifts = synth.qc_shifts(J, L, p, seed=21)
    c = L * p
    mu = synth.gaussian_llrs(1, T * c, seed=5, ebn0_db=2.5, rate=0.5).reshape(1, T, c)
    hard, post, decided = run_gpu(pkg, shifts, p, I, mu, [1] * T, tanner=True)
    assert decided.sum() == T - I * 2 + 1
    compare(shifts, p, I, mu, hard, post, decided, "tanner I=1 one stream", tanner=True)
