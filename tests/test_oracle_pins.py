"""Pins for the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU.  None of them compares the oracle with
itself: each checks it against a printed table of the paper, a closed form,
brute force over all codewords, an invariant of BP, or a textbook special case.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import (TREE_BASES, brute_force_llr, brute_force_maxlog, random_codeword, read_sections,
                     syndrome)


# ---------------------------------------------------------------- graph, Sec. IV-A
def test_edge_order_matches_paper_example():
    """Eq. (simpleH): edges numbered row by row, left to right; eq. (LUT_c), eq. (LUT_v)."""
    g = read_sections("simple_H_edges.txt")
    H = np.array(g["H"], dtype=np.uint8)
    row_ptr, col = oracle.csr_rows(H)
    lut_c = [list(range(row_ptr[m], row_ptr[m + 1])) for m in range(H.shape[0])]
    assert lut_c == g["LUT_c"]
    vptr, vedge = oracle.variable_edges(row_ptr, col, H.shape[1])
    lut_v = [list(vedge[vptr[n]:vptr[n + 1]]) for n in range(H.shape[1])]
    assert lut_v == g["LUT_v"]
    # package p_01 first, then p_03, p_04, p_07, p_10 ... (Example in Sec. IV-A)
    assert list(zip(np.repeat(np.arange(4), np.diff(row_ptr))[:5], col[:5])) == [(0, 1), (0, 3), (0, 4), (0, 7),
                                                                                 (1, 0)]


def test_circulant_shift_direction():
    """P^a is the identity with its columns shifted cyclically right a times (Sec. II-A)."""
    P1 = oracle.circulant(1, 3)
    I3 = np.eye(3, dtype=np.uint8)
    assert np.array_equal(P1, np.roll(I3, 1, axis=1))
    assert np.array_equal(P1, [[0, 1, 0], [0, 0, 1], [1, 0, 0]])
    assert not oracle.circulant(-1, 4).any()


def test_qc_code_dimensions_match_codes_table():
    """Table of codes A-D: c x (c-b) and the number of edges E = J L p (Sec. IV-B-1)."""
    rows = read_sections("codes_table.txt")[None]
    for name, J, L, p, c, cb, edges in rows:
        geo = oracle.ldpccc_geometry(J, L, p)
        assert (geo["c"], geo["cb"]) == (c, cb)
        shifts = synth.qc_shifts(J, L, p, seed=7, avoid_4cycles=False)
        H = oracle.qc_parity_check(shifts, p)
        assert H.shape == (J * p, L * p)
        assert int(H.sum()) == edges == J * L * p
        assert (H.sum(axis=0) == J).all() and (H.sum(axis=1) == L).all()  # regular (w_c, w_r) = (J, L)
        assert abs(oracle.design_rate(shifts) - 5 / 6) < 1e-12


# ---------------------------------------------------------------- generator and channel
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the generator (Salmon et al., SC'11)."""
    kat = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in kat:
        assert tuple(int(x) for x in oracle.philox4x32_10(ctr, key)) == want


def test_channel_llr_statistics():
    """mu = 2y/sigma^2 with y ~ N(1, sigma^2): mean 2/sigma^2, variance 4/sigma^2 (Sec. II-B)."""
    sigma = oracle.sigma_from_ebn0(2.0, 0.5)
    mu, g = oracle.channel_awgn(seed=11, first_frame=0, nfr=64, N=4096, sigma=sigma, return_g=True)
    n = mu.size
    m, v = mu.mean(), mu.var()
    assert abs(m - 2 / sigma**2) < 5 * math.sqrt(4 / sigma**2 / n)
    assert abs(v / (4 / sigma**2) - 1) < 5 * math.sqrt(2 / n)
    assert abs(g.mean()) < 5 / math.sqrt(n) and abs(g.std() - 1) < 5 / math.sqrt(2 * n)
    # uncoded BER of hard decisions on mu equals Q(1/sigma)
    ber = (mu < 0).mean()
    q = 0.5 * math.erfc(1 / sigma / math.sqrt(2))
    assert abs(ber - q) < 5 * math.sqrt(q * (1 - q) / n)


def _all_uniform_numerators():
    """v = 2 floor(w / 2^9) + 1 for every 32-bit word w: all odd v in (0, 2^24); u = v 2^-24."""
    return (2 * np.arange(1 << 23, dtype=np.uint64) + 1).astype(np.uint32)


def test_channel_ln_all_inputs():
    """The generator's binary32 ln against float64 log on every uniform it can draw: <= 1 ulp."""
    v = _all_uniform_numerators()
    u = (v.astype(np.float64) * 2.0 ** -24).astype(np.float32)
    assert np.array_equal(u.astype(np.float64), v.astype(np.float64) * 2.0 ** -24)  # exact in binary32
    got = oracle.ln_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert (np.abs(got - ref) / ulp).max() <= 1.0
    assert got.max() < 0  # every uniform is below 1: -2 ln u > 0 under the square root


def test_channel_sincos_all_inputs():
    """sin and cos of 2 pi u against float64 on every uniform it can draw: <= 2 ulp of each value
    (float64 sin(2 pi u) is itself exact to ~1e-15 absolute, far below the bound), and the
    quadrant signs are right."""
    v = _all_uniform_numerators()
    s, c = oracle.sincos2pi_f32(v)
    ang = 2 * np.pi * (v.astype(np.float64) * 2.0 ** -24)
    for got, ref in ((s, np.sin(ang)), (c, np.cos(ang))):
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        err = np.abs(got.astype(np.float64) - ref)
        assert (err / ulp).max() <= 2.0
        assert np.array_equal(np.sign(got), np.sign(ref))


def test_channel_matches_double_precision_box_muller():
    """The binary32 generator against Box-Muller in float64 on the same Philox words: every LLR within
    the bound its operations allow (g: <= 4 ulp relative from ln, sqrt, cos/sin and the product; then
    the fused sigma*g + x and the product with s2, each half an ulp, and s2's own rounding)."""
    sigma = oracle.sigma_from_ebn0(1.5, 0.5)
    seed, first, nfr, N = 3, 1 << 33, 3, 1000
    mu, g = oracle.channel_awgn(seed, first, nfr, N, sigma, return_g=True)
    g64 = np.zeros((nfr, N))
    for f in range(nfr):
        F = first + f
        for q in range(N // 4):
            w = oracle.philox4x32_10((q, F & 0xFFFFFFFF, F >> 32, 0), (seed & 0xFFFFFFFF, seed >> 32))
            for pr in range(2):
                u0 = (2.0 * (int(w[2 * pr]) >> 9) + 1.0) * 2.0 ** -24
                u1 = (2.0 * (int(w[2 * pr + 1]) >> 9) + 1.0) * 2.0 ** -24
                rho = math.sqrt(-2.0 * math.log(u0))
                g64[f, 4 * q + 2 * pr] = rho * math.cos(2 * math.pi * u1)
                g64[f, 4 * q + 2 * pr + 1] = rho * math.sin(2 * math.pi * u1)
    eps = 2.0 ** -24
    assert np.all(np.abs(g - g64) <= 4 * eps * np.abs(g64) + 1e-12)
    mu64 = 2.0 * (1.0 + sigma * g64) / sigma ** 2
    s2 = 2.0 / sigma ** 2
    tol = s2 * (4 * eps * sigma * np.abs(g64) + eps * np.abs(1 + sigma * g64)) + 2 * eps * np.abs(mu64) + 1e-12
    assert np.all(np.abs(mu.astype(np.float64) - mu64) <= tol)


def test_channel_counter_partition_invariance():
    """Frame F's noise depends only on (seed, F, bit): any split of the frame range gives the same values."""
    sigma = 0.8
    a = oracle.channel_awgn(5, 100, 6, 130, sigma)
    b = np.concatenate([oracle.channel_awgn(5, 100, 2, 130, sigma), oracle.channel_awgn(5, 102, 4, 130, sigma)])
    assert np.array_equal(a, b)
    c = oracle.channel_awgn(6, 100, 6, 130, sigma)
    assert not np.array_equal(a, c)


# ---------------------------------------------------------------- sum-product, Algorithm 1
def _tree_code(name, p=1):
    H = oracle.qc_parity_check(np.array(TREE_BASES[name]), p)
    rp, col = oracle.csr_rows(H)
    return H, rp, col


@pytest.mark.parametrize("name", sorted(TREE_BASES))
def test_sp_exact_on_cycle_free_graphs(name):
    """BP on a cycle-free Tanner graph returns the exact a-posteriori LLRs (brute force over all codewords)."""
    H, rp, col = _tree_code(name)
    rng = np.random.default_rng(3)
    for trial in range(4):
        mu = rng.normal(1.0, 1.5, size=H.shape[1]).astype(np.float32)
        post, hard, iters, ok = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=12)
        want = brute_force_llr(H, mu)
        assert np.allclose(post[0], want, rtol=0, atol=1e-10), (name, trial)
        assert np.array_equal(hard[0], (want < 0).astype(np.uint8))


def test_sp_exact_on_lifted_tree():
    """A tree lifted by p x p circulants is a forest of p trees: BP stays exact (N = 21 brute force)."""
    H, rp, col = _tree_code("path3", p=3)
    mu = np.random.default_rng(4).normal(0.8, 1.2, size=H.shape[1]).astype(np.float32)
    post = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=10)[0][0]
    assert np.allclose(post, brute_force_llr(H, mu), atol=1e-10)


def test_single_parity_check_closed_form():
    """Eq. (bphs) on one check: alpha_n = 2 atanh(prod_{n' != n} tanh(mu_n'/2)); post = mu + alpha."""
    d = 6
    H = np.ones((1, d), dtype=np.uint8)
    rp, col = oracle.csr_rows(H)
    mu = np.array([1.3, -0.4, 2.2, 0.7, -3.1, 5.0], dtype=np.float32)
    post = oracle.sp_decode(rp, col, d, mu, max_iter=1)[0][0]
    m = mu.astype(np.float64)
    for n in range(d):
        prod = np.prod([math.tanh(m[k] / 2) for k in range(d) if k != n])
        assert abs(post[n] - (m[n] + 2 * math.atanh(prod))) < 1e-12


def test_repetition_code_posterior_is_sum():
    """A length-5 repetition code (path of degree-2 checks): every posterior equals sum(mu)."""
    H, rp, col = _tree_code("rep5")
    mu = np.array([0.5, -1.25, 2.0, 0.75, -0.5], dtype=np.float32)
    post = oracle.sp_decode(rp, col, 5, mu, max_iter=6)[0][0]
    assert np.allclose(post, mu.astype(np.float64).sum(), atol=1e-12)


def test_phi_form_equals_tanh_form():
    """The phi-form used by the oracle equals the literal tanh/atanh form of eq. (bphs) away from clipping."""
    shifts = synth.qc_shifts(3, 6, 16, seed=1)
    H = oracle.qc_parity_check(shifts, 16)
    rp, col = oracle.csr_rows(H)
    mu = synth.gaussian_llrs(8, H.shape[1], seed=2, ebn0_db=0.0, rate=0.5)
    mu = np.clip(mu, -6, 6)
    a = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=3, form="phi", clip=1e9)[0]
    b = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=3, form="tanh", clip=1e9)[0]
    assert np.max(np.abs(a - b)) < 1e-9


def test_noiseless_fixed_point():
    """A noiseless all-zero frame satisfies every check after the first iteration."""
    shifts = synth.qc_shifts(4, 24, 31, seed=3)
    H = oracle.qc_parity_check(shifts, 31)
    rp, col = oracle.csr_rows(H)
    mu = np.full((2, H.shape[1]), 8.0, dtype=np.float32)
    post, hard, iters, ok = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=30, early_stop=True)
    assert (iters == 1).all() and (ok == 1).all() and not hard.any()
    # every check sees 23 equal inputs: alpha = 2 atanh(tanh(4)^23), posterior = mu + 4 alpha
    alpha = 2 * math.atanh(math.tanh(4.0) ** 23)
    assert np.allclose(post, 8.0 + 4 * alpha, atol=1e-12)


def test_channel_symmetry_with_nonzero_codeword():
    """BP commutes with the sign flip of a codeword: decode(mu * x(c)) = decode(mu) * x(c)."""
    shifts = synth.qc_shifts(3, 6, 8, seed=9)
    H = oracle.qc_parity_check(shifts, 8)
    rp, col = oracle.csr_rows(H)
    N = H.shape[1]
    mu = synth.gaussian_llrs(4, N, seed=5, ebn0_db=1.0, rate=0.5)
    cw = random_codeword(H, seed=6)
    assert not syndrome(H, cw).any() and cw.any()
    x = (1 - 2 * cw.astype(np.float32))
    pa, ha, ia, oa = oracle.sp_decode(rp, col, N, mu, max_iter=7)
    pb, hb, ib, ob = oracle.sp_decode(rp, col, N, mu * x, max_iter=7)
    assert np.allclose(pb, pa * x, atol=1e-12)
    assert np.array_equal(oa, ob)


def test_converged_frames_satisfy_all_checks():
    """ok = 1 exactly when H c_hat = 0; early stop freezes at the first such iteration."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    H = oracle.qc_parity_check(shifts, 64)
    rp, col = oracle.csr_rows(H)
    mu = synth.gaussian_llrs(32, H.shape[1], seed=1, ebn0_db=1.5, rate=0.5)
    post, hard, iters, ok = oracle.sp_decode(rp, col, H.shape[1], mu, max_iter=30, early_stop=True)
    for f in range(32):
        s = syndrome(H, hard[f]).any()
        assert ok[f] == (0 if s else 1)
        if ok[f]:
            # no earlier iteration satisfied the checks
            if iters[f] > 1:
                h2 = oracle.sp_decode(rp, col, H.shape[1], mu[f], max_iter=iters[f] - 1)[1][0]
                assert syndrome(H, h2).any()
            full = oracle.sp_decode(rp, col, H.shape[1], mu[f], max_iter=iters[f])
            assert np.array_equal(full[0][0], post[f])
        else:
            assert iters[f] == 30
    assert ok.sum() > 16


def test_empty_extrinsic_set_and_degree_one_check():
    """A degree-1 check sends +clip (empty product = 1); the posterior then carries it."""
    H = np.array([[1, 0], [1, 1]], dtype=np.uint8)
    rp, col = oracle.csr_rows(H)
    mu = np.array([-2.0, 1.0], dtype=np.float32)
    post = oracle.sp_decode(rp, col, 2, mu, max_iter=1, clip=30.0)[0][0]
    # variable 0: mu + alpha(deg-1 check: +30) + alpha(check 2: mu_1 = 1.0 after one step)
    assert abs(post[0] - max(-30, min(30, -2.0 + 30.0 + 1.0))) < 1e-12


def test_frames_are_independent():
    shifts = synth.qc_shifts(3, 6, 16, seed=2)
    H = oracle.qc_parity_check(shifts, 16)
    rp, col = oracle.csr_rows(H)
    mu = synth.gaussian_llrs(6, H.shape[1], seed=8, ebn0_db=1.0, rate=0.5)
    a = oracle.sp_decode(rp, col, H.shape[1], mu, 9)[0]
    perm = np.array([3, 1, 5, 0, 2, 4])
    b = oracle.sp_decode(rp, col, H.shape[1], mu[perm], 9, nthreads=3)[0]
    assert np.array_equal(a[perm], b)


# ---------------------------------------------------------------- integer min-sum
@pytest.mark.parametrize("name", sorted(TREE_BASES))
def test_min_sum_is_max_log_on_trees(name):
    """On a cycle-free graph min-sum returns the max-log a-posteriori values (integer brute force)."""
    H, rp, col = _tree_code(name)
    rng = np.random.default_rng(12)
    for trial in range(4):
        mu = (rng.integers(-12, 13, size=H.shape[1]) * 0.25).astype(np.float32)  # exact on the F=2 grid
        q = oracle.quantize(mu, 2).astype(np.int64)
        assert np.array_equal(q, np.round(mu * 4).astype(np.int64))
        post, hard, _, _ = oracle.ms_decode(rp, col, H.shape[1], mu, max_iter=12)
        assert np.array_equal(post[0].astype(np.int64), brute_force_maxlog(H, q)), (name, trial)


def test_quantizer_rounding_and_saturation():
    """q = clamp(round-half-even(mu * 4), -127, 127)."""
    mu = np.array([0.125, 0.375, -0.125, -0.375, 31.75, 40.0, -40.0, 0.0, 1.1], dtype=np.float32)
    assert oracle.quantize(mu, 2).tolist() == [0, 2, 0, -2, 127, 127, -127, 0, 4]


def test_min_sum_saturates_messages():
    """Variable-to-check messages saturate at +-127; the posterior is the unsaturated sum."""
    H = np.ones((3, 2), dtype=np.uint8)  # three degree-2 checks on the same two bits
    rp, col = oracle.csr_rows(H)
    mu = np.array([30.0, 30.0], dtype=np.float32)  # q = 120
    post = oracle.ms_decode(rp, col, 2, mu, max_iter=2)[0][0]
    # iteration 1: alpha = 120 on each edge; beta = clamp(120 + 240) = 127
    # iteration 2: alpha = 127; post = 120 + 3 * 127
    assert post.tolist() == [120 + 3 * 127] * 2


# ---------------------------------------------------------------- LDPCCC, Sec. II-D, II-E, IV-B
def _label_of(block, subs):
    for lab, s in enumerate(subs):
        if block.shape == s.shape and (block != s).nnz == 0:
            return lab
    return None


def test_ldpccc_label_tables_match_paper():
    """Eqs. (lut_c_ldpccc), (lut_v_ldpccc): sub-block labels seen by each check-layer / frame type (Lambda=4)."""
    g = read_sections("ldpccc_luts_lambda4.txt")
    J, L, p = 4, 24, 5
    shifts = synth.qc_shifts(J, L, p, seed=21)
    T = 12
    Hc, geo = oracle.ldpccc_unwrap(shifts, p, T)
    lam, c, cb, ms = geo["Lambda"], geo["c"], geo["cb"], geo["ms"]
    assert (lam, ms) == (4, 3)
    import scipy.sparse as sp
    HQ = sp.csr_matrix(oracle.qc_parity_check(shifts, p))
    subs = [HQ[i * cb:(i + 1) * cb, j * c:(j + 1) * c] for i in range(lam) for j in range(lam)]
    lut_c, lut_v = [], []
    for R in range(ms, ms + lam):  # one layer of each type, past start-up
        lut_c.append([_label_of(Hc[R * cb:(R + 1) * cb, F * c:(F + 1) * c], subs) for F in range(R - ms, R + 1)])
    lut_c = [lut_c[(k - ms) % lam] for k in range(lam)]  # row k = layer type k
    for F in range(lam, 2 * lam):
        lut_v.append([_label_of(Hc[R * cb:(R + 1) * cb, F * c:(F + 1) * c], subs) for R in range(F, F + ms + 1)])
    lut_v = [lut_v[(k - lam) % lam] for k in range(lam)]
    assert lut_c == g["LUT_c"]
    assert lut_v == g["LUT_v"]


def test_ldpccc_structure():
    """Regular (ms, J, K) past start-up, period T = Lambda, and H^L + H^U reassembles H_QC (Sec. II-C, II-D)."""
    import scipy.sparse as sp
    J, L, p = 3, 6, 7
    shifts = synth.qc_shifts(J, L, p, seed=4)
    T = 10
    Hc, geo = oracle.ldpccc_unwrap(shifts, p, T)
    lam, c, cb, ms = geo["Lambda"], geo["c"], geo["cb"], geo["ms"]
    assert (lam, ms, c, cb) == (3, 2, 2 * p, p)
    rw = np.asarray(Hc.sum(axis=1)).ravel()
    cw = np.asarray(Hc.sum(axis=0)).ravel()
    assert (rw[ms * cb:] == L).all() and (rw[:ms * cb] < L).all()
    assert (cw[: (T - ms) * c] == J).all()
    # period Lambda
    blk = lambda R, F: Hc[R * cb:(R + 1) * cb, F * c:(F + 1) * c].toarray()
    for R in range(ms, T - lam):
        for d in range(ms + 1):
            assert np.array_equal(blk(R, R - d), blk(R + lam, R + lam - d))
    # sum of the Lambda x Lambda window starting at layer lam reassembles H_QC
    HQ = oracle.qc_parity_check(shifts, p)
    rebuilt = np.zeros_like(HQ)
    for a in range(lam):
        for d in range(ms + 1):
            R = lam + a
            F = R - d
            b = F % lam
            rebuilt[a * cb:(a + 1) * cb, b * c:(b + 1) * c] |= blk(R, F).astype(np.uint8)
    assert np.array_equal(rebuilt, HQ)


def test_ldpccc_schedule_matches_narrative():
    """Slots 0, 3, 4 and the first decision, Sec. IV-B-2 (Lambda = 4, ms = 3)."""
    J, L, p, I = 4, 8, 3, 3
    shifts = synth.qc_shifts(J, L, p, seed=5)
    T = 20
    Hc, geo = oracle.ldpccc_unwrap(shifts, p, T)
    mu = np.full(T * geo["c"], 3.0, dtype=np.float32)
    _, _, decided, log = oracle.ldpccc_decode(Hc, geo, T, I, mu, log_cap=10000)
    ev = {}
    for t, kind, idx, proc in log.tolist():
        ev.setdefault(t, []).append((kind, idx, proc))
    assert ev[0] == [(0, 0, 1), (1, 0, 1)]  # v0 enters, c0 updated, nothing else
    assert ev[1] == [(0, 1, 1), (1, 1, 1)]
    assert ev[3] == [(0, 3, 1), (1, 3, 1), (2, 0, 1)]  # after c3, v0 is updated
    assert ev[4] == [(0, 4, 1), (1, 4, 1), (1, 0, 2), (2, 1, 1)]  # c4 and c0; v1 leaves processor 1
    first_decision = min(t for t, k, i, _ in log.tolist() if k == 3)
    assert first_decision == I * 4 - 1
    assert decided[0].sum() == T - I * 4 + 1
    # the first check layer holds edges to frame 0 only
    assert Hc[0:geo["cb"], geo["c"]:].nnz == 0


def test_ldpccc_lambda1_is_block_decoding():
    """gcd(J, L) = 1: frames decouple (ms = 0) and I processors equal I iterations of Algorithm 1."""
    J, L, p, I = 3, 7, 11, 5
    shifts = synth.qc_shifts(J, L, p, seed=8)
    T = 12
    Hc, geo = oracle.ldpccc_unwrap(shifts, p, T)
    assert geo["Lambda"] == 1 and geo["ms"] == 0
    c = geo["c"]
    mu = synth.gaussian_llrs(1, T * c, seed=9, ebn0_db=1.5, rate=1 - J / L)[0]
    post, hard, decided, _ = oracle.ldpccc_decode(Hc, geo, T, I, mu)
    H = oracle.qc_parity_check(shifts, p)
    rp, col = oracle.csr_rows(H)
    frames = mu.reshape(T, c)
    bp, bh, _, _ = oracle.sp_decode(rp, col, c, frames, max_iter=I)
    nd = T - I + 1
    assert decided[0].sum() == nd
    assert np.allclose(post[0].reshape(T, c)[:nd], bp[:nd], atol=1e-12)
    assert np.array_equal(hard[0].reshape(T, c)[:nd], bh[:nd])


def test_ldpccc_noiseless_stream_decodes_to_zero():
    J, L, p, I = 3, 6, 8, 4
    shifts = synth.qc_shifts(J, L, p, seed=1)
    T = 30
    Hc, geo = oracle.ldpccc_unwrap(shifts, p, T)
    mu = np.full((2, T * geo["c"]), 5.0, dtype=np.float32)
    post, hard, decided, _ = oracle.ldpccc_decode(Hc, geo, T, I, mu)
    assert decided.sum() == 2 * (T - I * 3 + 1)
    assert not hard.any()


def test_codeword_enumeration_helper():
    """The null-space enumeration used by brute force agrees with exhaustive search (eq. ldpcc example H)."""
    from helpers import codewords, codewords_exhaustive
    H = np.array(read_sections("irregular_H_example.txt")[None], dtype=np.uint8)
    a = {tuple(r) for r in codewords(H)}
    b = {tuple(r) for r in codewords_exhaustive(H)}
    assert a == b and len(a) == 2 ** (10 - np.linalg.matrix_rank(H))  # rank over GF(2) = rank over R here


def test_sp_on_paper_irregular_example_with_cycles():
    """Eq. (ldpcc) H has cycles: BP is not exact, but hard decisions of a clean frame are right and ok=1."""
    H = np.array(read_sections("irregular_H_example.txt")[None], dtype=np.uint8)
    rp, col = oracle.csr_rows(H)
    from helpers import codewords
    C = codewords(H)
    cw = C[len(C) // 2]
    mu = (4.0 * (1 - 2 * cw)).astype(np.float32)
    mu[3] = -mu[3] * 0.25  # one weak wrong bit
    post, hard, iters, ok = oracle.sp_decode(rp, col, 10, mu, max_iter=20, early_stop=True)
    assert ok[0] == 1 and np.array_equal(hard[0], cw.astype(np.uint8))


# ---------------------------------------------------------------- learned normalized/offset min-sum
def _qc(J, L, p, seed):
    shifts = synth.qc_shifts(J, L, p, seed=seed)
    H = oracle.qc_parity_check(shifts, p)
    rp, col = oracle.csr_rows(H)
    return H, rp, col, oracle.circulant_index(rp, col, p, L)


def test_noms_with_unit_weight_is_min_sum():
    """w = 1, o = 0 reduces the NOMS rule to plain min-sum: equal to the integer oracle on the LLR grid."""
    H, rp, col, cb = _qc(3, 6, 16, 4)
    N = H.shape[1]
    mu = synth.integer_llrs(6, N, seed=2, lo=-12, hi=12, scale=0.25)
    T = 4
    params = np.zeros((T, 18, 2))
    params[:, :, 0] = 1.0
    _, post, _ = oracle.noms(rp, col, cb, N, mu, T, params, clip=31.75)
    mpost = oracle.ms_decode(rp, col, N, mu, T)[0]
    assert np.array_equal(post, mpost * 0.25)


def test_noms_single_check_hand_values():
    """One check of degree 5 (each edge its own circulant), one iteration, (w, o) != (1, 0).

    alpha_e = sign * max(w * m - o, 0) with m the smallest |beta| over the other edges and sign
    the product of their signs; post_v = mu_v + alpha_e.  Worked by hand:
      e0: others (-0.5, 2, -3, 0.75): m = 0.5, sign +, 0.8*0.5 - 0.1 = 0.3     -> post 1.8
      e1: others (1.5, 2, -3, 0.75):  m = 0.75, sign -, 0.5*0.75 - 0.3 = 0.075 -> post -0.575
      e2: others (1.5, -0.5, -3, 0.75): m = 0.5, +, 1.0*0.5 - 0.6 < 0 -> alpha 0 -> post 2.0
      e3: others (1.5, -0.5, 2, 0.75): m = 0.5, -, 0.9*0.5 - 0 = 0.45         -> post -3.45
      e4: others (1.5, -0.5, 2, -3):   m = 0.5, +, 0.7*0.5 - 0.2 = 0.15        -> post 0.9
    (w * max(m - o, 0) would give 0.32 on e0; sign * (w m - o) without the max -0.1 on e2.)
    """
    rp = np.array([0, 5], dtype=np.int32)
    col = np.arange(5, dtype=np.int32)
    cb = np.arange(5, dtype=np.int32)
    mu = np.array([[1.5, -0.5, 2.0, -3.0, 0.75]], dtype=np.float32)
    params = np.array([[[0.8, 0.1], [0.5, 0.3], [1.0, 0.6], [0.9, 0.0], [0.7, 0.2]]])
    loss, post, _ = oracle.noms(rp, col, cb, 5, mu, 1, params)
    want = np.array([1.8, -0.575, 2.0, -3.45, 0.9])
    assert np.allclose(post[0], want, rtol=0, atol=1e-12), post
    # loss: mean of softplus(-post) over the five bits of the single iteration
    assert abs(loss - np.mean(np.log1p(np.exp(-want)))) <= 1e-12
    # a tie in the minimum (|1.0| twice) and a zero input: e2 sees m = 1.0 from either tied edge
    mu2 = np.array([[1.0, -1.0, 2.0, 0.0, -2.5]], dtype=np.float32)
    ones = np.zeros((1, 5, 2))
    ones[..., 0] = 0.5
    ones[..., 1] = 0.125
    _, post2, _ = oracle.noms(rp, col, cb, 5, mu2, 1, ones)
    # every edge but e3 has the zero input among its others: m = 0, 0.5*0 - 0.125 < 0 -> alpha 0;
    # e3: others (1, -1, 2, -2.5): m = 1, sign + (two negatives), 0.5 - 0.125 = 0.375
    assert np.allclose(post2[0], [1.0, -1.0, 2.0, 0.375, -2.5], rtol=0, atol=1e-12), post2


def test_noms_two_checks_two_iterations_hand_values():
    """Two checks sharing variable 2 (base [[0,0,0,-1,-1],[-1,-1,0,0,0]], p = 1), two iterations with
    different parameter rows: pins the extrinsic variable rule, which row each iteration uses, and the
    circulant index j*L + l.  Worked by hand (all values exact in binary):
      iteration 1, (w, o) = (0.75, 0.125) everywhere:
        c0 on (2, -1.25, 0.5): alpha = (-0.25, +0.25, -0.8125)
        c1 on (0.5, 1.75, -3):  alpha = (-1.1875, -0.25, +0.25)
        beta(c0, v2) = 0.5 - 1.1875 = -0.6875, beta(c1, v2) = 0.5 - 0.8125 = -0.3125
        post = (1.75, -1.0, -1.5, 1.5, -2.75)
      iteration 2, (w, o) = (0.625, 0.0625) on circulant 0, (0.5, 0.25) elsewhere:
        c0 on (2, -1.25, -0.6875): alpha = (+0.3671875, -0.09375, -0.375)
        c1 on (-0.3125, 1.75, -3): alpha = (-0.625, 0, 0)   (0.5 * 0.3125 - 0.25 < 0)
        post = (2.3671875, -1.34375, -0.5, 1.75, -3.0)
    """
    H = oracle.qc_parity_check([[0, 0, 0, -1, -1], [-1, -1, 0, 0, 0]], 1)
    rp, col = oracle.csr_rows(H)
    cb = oracle.circulant_index(rp, col, 1, 5)
    assert cb.tolist() == [0, 1, 2, 7, 8, 9]
    mu = np.array([[2.0, -1.25, 0.5, 1.75, -3.0]], dtype=np.float32)
    params = np.zeros((2, 10, 2))
    params[0, :, :] = (0.75, 0.125)
    params[1, :, :] = (0.5, 0.25)
    params[1, 0, :] = (0.625, 0.0625)
    post1 = np.array([1.75, -1.0, -1.5, 1.5, -2.75])
    post2 = np.array([2.3671875, -1.34375, -0.5, 1.75, -3.0])
    _, p1, _ = oracle.noms(rp, col, cb, 5, mu, 1, params[:1])
    assert np.array_equal(p1[0], post1), p1
    loss, p2, _ = oracle.noms(rp, col, cb, 5, mu, 2, params)
    assert np.array_equal(p2[0], post2), p2
    assert abs(loss - np.mean(np.log1p(np.exp(-np.concatenate([post1, post2]))))) <= 1e-12


def test_binary16_rounding_matches_numpy_float16():
    """The FP16-message variant's storage rounding against numpy's own binary16 conversion (round to
    nearest even), over normals, subnormals, ties and the overflow edge."""
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.normal(0, 8, 100000), rng.normal(0, 1e-5, 20000), rng.uniform(-30, 30, 50000),
                        [0.0, -0.0, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 2.0 ** -24 * 1.5, 2.0 ** -25,
                         65504.0, 65519.0, 65520.0, -70000.0]])
    with np.errstate(over="ignore"):  # 65520 and beyond round to infinity, as intended
        want = x.astype(np.float16).astype(np.float64)
    got = oracle.round_half(x)
    assert np.array_equal(got, want)


def test_noms_fp16_variant_rounds_stored_messages():
    """With binary16 storage the check messages and the later iterations' variable messages are rounded
    (the first check step reads the FP32 channel LLRs): on the hand-worked two-check example every value
    is a multiple of 2^-7, exact in binary16, so the result equals the unrounded one."""
    H = oracle.qc_parity_check([[0, 0, 0, -1, -1], [-1, -1, 0, 0, 0]], 1)
    rp, col = oracle.csr_rows(H)
    cb = oracle.circulant_index(rp, col, 1, 5)
    mu = np.array([[2.0, -1.25, 0.5, 1.75, -3.0]], dtype=np.float32)
    params = np.zeros((2, 10, 2))
    params[0, :, :] = (0.75, 0.125)
    params[1, :, :] = (0.5, 0.25)
    params[1, 0, :] = (0.625, 0.0625)
    a = oracle.noms(rp, col, cb, 5, mu, 2, params)
    b = oracle.noms(rp, col, cb, 5, mu, 2, params, store16=True)
    assert np.array_equal(a[1], b[1]) and a[0] == b[0]
    # an input whose second-iteration messages are not binary16 values changes
    mu2 = np.array([[2.0, -1.2345678, 0.5, 1.75, -3.0]], dtype=np.float32)
    c = oracle.noms(rp, col, cb, 5, mu2, 2, params)
    e = oracle.noms(rp, col, cb, 5, mu2, 2, params, store16=True)
    assert not np.array_equal(c[1], e[1]) and np.allclose(c[1], e[1], atol=2e-3)


def test_noms_check_messages_are_clipped():
    """With w > 1 a saturated input can push w * m - o past the clip: alpha is clipped at +-clip like
    every other message, and the gradient of a clipped alpha is zero.  One check of degree 3, each edge
    its own circulant, (w, o) = (1.5, 1), clip 30, one iteration; by hand:
      e0: others (30, -25): m = 25, sign -, 1.5*25 - 1 = 36.5 -> clipped to 30 -> post 20 - 30 = -10
      e1: others (20, -25): m = 20, sign -, 1.5*20 - 1 = 29                    -> post 30 - 29 = 1
      e2: others (20, 30):  m = 20, sign +, 29                                 -> post -25 + 29 = 4
    (without the clip e0 would end at -16.5).  loss = mean softplus(-post); d loss / d (w, o) of edge
    e1 = (1/3) sigmoid(-post) * (-d post / d (w, o)), with d post1 / d w1 = -20, d post1 / d o1 = +1;
    edge e0's circulant gets none; a central difference of the loss agrees."""
    rp = np.array([0, 3], dtype=np.int32)
    col = np.arange(3, dtype=np.int32)
    cb = np.arange(3, dtype=np.int32)
    mu = np.array([[20.0, 30.0, -25.0]], dtype=np.float32)
    params = np.tile(np.array([1.5, 1.0]), (1, 3, 1))
    loss, post, grad = oracle.noms(rp, col, cb, 3, mu, 1, params, want_grad=True, clip=30.0)
    want = np.array([-10.0, 1.0, 4.0])
    assert np.allclose(post[0], want, rtol=0, atol=1e-12), post
    assert abs(loss - np.mean(np.log1p(np.exp(-want)))) <= 1e-12
    sig = lambda x: 1.0 / (1.0 + np.exp(-x))
    assert np.allclose(grad[0, 0], 0.0, atol=1e-15), grad
    assert abs(grad[0, 1, 0] - sig(-1.0) * 20.0 / 3.0) <= 1e-12, grad
    assert abs(grad[0, 1, 1] - (-sig(-1.0) / 3.0)) <= 1e-12, grad
    # e2's alpha feeds post2 = 4: d post2 / d w2 = +20, d post2 / d o2 = -1
    assert abs(grad[0, 2, 0] - (-sig(-4.0) * 20.0 / 3.0)) <= 1e-12, grad
    h = 1e-6
    for c in range(3):
        for k in range(2):
            pp, pm = params.copy(), params.copy()
            pp[0, c, k] += h
            pm[0, c, k] -= h
            fd = (oracle.noms(rp, col, cb, 3, mu, 1, pp, clip=30.0)[0]
                  - oracle.noms(rp, col, cb, 3, mu, 1, pm, clip=30.0)[0]) / (2 * h)
            assert abs(fd - grad[0, c, k]) <= 1e-7, (c, k, fd, grad[0, c, k])


def test_noms_gradient_matches_finite_differences():
    """Hand-written reverse mode against central differences of the FP64 loss (away from ties and kinks)."""
    H, rp, col, cb = _qc(3, 6, 8, 5)
    N = H.shape[1]
    mu = synth.gaussian_llrs(3, N, seed=6, ebn0_db=1.0, rate=0.5)
    T = 3
    rng = np.random.default_rng(7)
    params = np.stack([rng.uniform(0.6, 1.0, (T, 18)), rng.uniform(0.0, 0.5, (T, 18))], axis=-1)
    loss, _, grad = oracle.noms(rp, col, cb, N, mu, T, params, want_grad=True)
    h = 1e-6
    idx = [(0, 0, 0), (0, 5, 1), (1, 7, 0), (1, 17, 1), (2, 3, 0), (2, 11, 1), (0, 12, 0), (2, 0, 1)]
    for t, c, k in idx:
        pp, pm = params.copy(), params.copy()
        pp[t, c, k] += h
        pm[t, c, k] -= h
        fd = (oracle.noms(rp, col, cb, N, mu, T, pp)[0] - oracle.noms(rp, col, cb, N, mu, T, pm)[0]) / (2 * h)
        assert abs(fd - grad[t, c, k]) <= 1e-6 * max(1e-3, abs(fd)), (t, c, k, fd, grad[t, c, k])
    assert np.abs(grad).max() > 0


# --------------------------------------------------------------------------
# Systematic encoder (the transmitted codewords of Sec. V)
# --------------------------------------------------------------------------
def _span_rank(vectors) -> int:
    """GF(2) rank by brute force: the span of r independent vectors has 2^r elements."""
    span = {0}
    for v in vectors:
        span |= {x ^ v for x in span}
    return len(span).bit_length() - 1


def _small_parity_checks():
    rng = np.random.default_rng(31)
    Hs = [(rng.random((5, 10)) < 0.4).astype(np.uint8)]
    Hs.append(oracle.qc_parity_check(synth.qc_shifts(2, 4, 3, seed=3), 3))  # rank-deficient (2 block rows)
    H = (rng.random((4, 11)) < 0.5).astype(np.uint8)
    H[2] = 0                    # an empty check
    H[:, 7] = H[:, 9]           # two equal columns
    H[:, 10] = 0                # a variable in no check
    Hs.append(H)
    Hs.append(np.array(read_sections("irregular_H_example.txt")[None], dtype=np.uint8))
    return Hs


@pytest.mark.parametrize("case", range(4))
def test_encoder_matches_brute_force(case):
    """Information set by its definition (column n is parity iff it raises the rank of the columns to its
    right), k = N - rank, and encoding is the bijection onto the null space with c[info] = u."""
    from helpers import codewords_exhaustive
    H = _small_parity_checks()[case]
    M, N = H.shape
    enc = oracle.Encoder(H)
    cols = [sum(int(H[m, n]) << m for m in range(M)) for n in range(N)]
    parity = [n for n in range(N) if _span_rank(cols[n:]) > _span_rank(cols[n + 1:])]
    assert list(enc.parity) == parity
    assert list(enc.info) == [n for n in range(N) if n not in parity]
    C = {tuple(r) for r in codewords_exhaustive(H)}
    assert len(C) == 2 ** enc.k and enc.k == N - _span_rank(cols)
    U = np.array([[(x >> j) & 1 for j in range(enc.k)] for x in range(2 ** enc.k)], dtype=np.uint8)
    c = enc.encode(U)
    assert np.array_equal(c[:, enc.info], U)
    assert {tuple(r) for r in c} == C


def test_encoder_on_qc_code_rank_and_checks():
    """A J x L QC code with every block present has rank at most J p - (J - 1) (each block row sums to the
    all-ones row); encoded words of the 3 x 6, p = 64 code satisfy every check."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    H = oracle.qc_parity_check(shifts, 64)
    enc = oracle.Encoder(H)
    assert enc.rank <= 3 * 64 - 2 and enc.k == 384 - enc.rank
    u = (np.random.default_rng(4).random((6, enc.k)) < 0.5).astype(np.uint8)
    c = enc.encode(u)
    assert not syndrome(H, c).any() and np.array_equal(c[:, enc.info], u)


def test_channel_with_codeword_shifts_by_bpsk_symbol():
    """Sec. II-B with x = 1 - 2c: a one bit moves y by -2, so mu(c) = mu(0) - 4 c / sigma^2 (same noise)."""
    N, nfr, sigma = 37, 3, 0.8
    cw = (np.random.default_rng(2).random((nfr, N)) < 0.5).astype(np.uint8)
    m0, g0 = oracle.channel_awgn(9, 100, nfr, N, sigma, return_g=True)
    m1, g1 = oracle.channel_awgn(9, 100, nfr, N, sigma, return_g=True, cw=cw)
    assert np.array_equal(g0, g1)
    x = 1.0 - 2.0 * cw.astype(np.float64)
    # the generator's binary32 steps: s2 * fma(sigma, g, x); sigma * g is exact in float64 and
    # the float64 sum then rounds once more than a fused add, which these 111 values never expose
    sf, s2 = np.float32(sigma), np.float32(2.0 / (sigma * sigma))
    y = (np.float64(sf) * g0 + x).astype(np.float32)
    want = (s2 * y).astype(np.float32)
    assert np.array_equal(m1, want)
    assert np.allclose(m1.astype(np.float64) - m0, -4.0 * cw.astype(np.float64) / sigma**2, atol=1e-5)


# --------------------------------------------------------------------------
# Time-invariant LDPCCC with delays D^{a_jl} (the Tanner unwrapping of a QC base)
# --------------------------------------------------------------------------
def test_tanner_ldpccc_folds_to_qc_code():
    """Reading every bit instant modulo p (tail-biting one frame) turns a complete check layer into the
    QC code whose circulants have the negated shifts: check tau of block row j meets bit tau - a."""
    J, L, p, T = 3, 6, 16, 5
    shifts = synth.qc_shifts(J, L, p, seed=12, zero_blocks=2)
    Hc, geo = oracle.ldpccc_tanner(shifts, p, T)
    c, cb = geo["c"], geo["cb"]
    assert (c, cb, geo["ms"], geo["delay"]) == (L * p, J * p, 1, int(shifts.max()))
    neg = np.where(shifts >= 0, (-shifts) % p, -1)
    want = oracle.qc_parity_check(neg, p)
    for F in range(1, T):  # layer 0 lacks the edges to instants before 0
        layer = Hc[F * cb:(F + 1) * cb].tocoo()
        folded = np.zeros((cb, c), dtype=np.uint8)
        folded[layer.row, layer.col % c] = 1
        assert np.array_equal(folded, want)
        assert layer.col.min() >= (F - 1) * c and layer.col.max() < (F + 1) * c  # memory one frame


def test_tanner_ldpccc_delays_are_the_shifts():
    """Check j at instant t involves bit l at instant t - a_jl: the instant differences of each row are the
    row's shifts, so the syndrome-former memory in instants is the largest shift."""
    J, L, p, T = 3, 6, 16, 4
    shifts = synth.qc_shifts(J, L, p, seed=3)
    Hc, geo = oracle.ldpccc_tanner(shifts, p, T)
    c, cb = geo["c"], geo["cb"]
    for row in range(cb * T):
        F, rem = divmod(row, cb)
        j, tau = divmod(rem, p)
        t = F * p + tau
        cols = Hc.indices[Hc.indptr[row]:Hc.indptr[row + 1]]
        got = sorted((int(col % c) // p, t - ((col // c) * p + (col % c) % p)) for col in cols)
        want = sorted((l, int(shifts[j, l])) for l in range(L) if shifts[j, l] >= 0 and t - shifts[j, l] >= 0)
        assert got == want
    assert geo["delay"] == int(shifts.max())


def test_tanner_ldpccc_zero_delays_is_block_decoding():
    """All delays 0: frames decouple (ms = 0) and I processors equal I iterations of Algorithm 1 on the
    block code with identity circulants."""
    J, L, p, I, T = 3, 6, 5, 4, 10
    shifts = np.zeros((J, L), dtype=np.int64)
    Hc, geo = oracle.ldpccc_tanner(shifts, p, T)
    assert geo["ms"] == 0
    c = geo["c"]
    mu = synth.gaussian_llrs(1, T * c, seed=4, ebn0_db=2.0, rate=0.5)[0]
    post, hard, decided, _ = oracle.ldpccc_decode(Hc, geo, T, I, mu)
    rp, col = oracle.csr_rows(oracle.qc_parity_check(shifts, p))
    bp, bh, _, _ = oracle.sp_decode(rp, col, c, mu.reshape(T, c), max_iter=I)
    nd = T - I + 1
    assert decided[0].sum() == nd
    assert np.allclose(post[0].reshape(T, c)[:nd], bp[:nd], atol=1e-12)
    assert np.array_equal(hard[0].reshape(T, c)[:nd], bh[:nd])


def test_tanner_ldpccc_noiseless_stream_decodes_to_zero():
    J, L, p, I, T = 3, 6, 8, 4, 20
    shifts = synth.qc_shifts(J, L, p, seed=1)
    Hc, geo = oracle.ldpccc_tanner(shifts, p, T)
    mu = np.full((2, T * geo["c"]), 5.0, dtype=np.float32)
    post, hard, decided, _ = oracle.ldpccc_decode(Hc, geo, T, I, mu)
    assert decided.sum() == 2 * (T - I * 2 + 1)
    assert not hard.any()
