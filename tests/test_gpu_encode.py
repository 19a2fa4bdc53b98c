"""GPU parity of the systematic encoder and of the simulation with random codewords (through the C-ABI).

Encoding is bit work: information sets, codewords and information bits are compared bit-exactly with
the oracle (its own greedy column basis and Philox).  The channel of a codeword is the generator's
binary32 arithmetic on the same noise: bit-exact against the oracle.  The simulation with
random codewords is compared with the batch path on the same frames (random_codewords ->
channel_codewords -> decode, errors over the information positions): exact counts for FP32
sum-product and integer min-sum.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_0334_gb300 as p

    p.lib()
    return p


def _codes(pkg):
    """(name, code object, sparse H) for a QC code, a QC code with zero blocks and a general code."""
    out = []
    for name, (J, L, p, seed, zb) in {"qc_3x6_p64": (3, 6, 64, 1, 0), "qc_4x12_p40_zero_blocks": (4, 12, 40, 7, 5)}.items():
        shifts = synth.qc_shifts(J, L, p, seed=seed, zero_blocks=zb)
        out.append((name, pkg.QCCode(shifts, p), sp.csr_matrix(oracle.qc_parity_check(shifts, p))))
    rp, col = synth.random_ldpc(600, 300, seed=5)
    H = sp.csr_matrix((np.ones(len(col), dtype=np.uint8), col, rp), shape=(300, 600))
    out.append(("general_600x300", pkg.SparseCode(rp, col, 600), H))
    return out


def _syndrome(H, c):
    return (H.astype(np.int64) @ c.T.astype(np.int64)) % 2


def test_encode_matches_oracle(pkg):
    """ldpc_encode of seeded information bits equals the oracle's systematic encoder bit for bit, over
    several groups of 32 frames with a ragged last group."""
    rng = np.random.default_rng(11)
    for name, code, H in _codes(pkg):
        enc = oracle.Encoder(H)
        k, pos = code.info_set()
        assert k == enc.k and np.array_equal(pos, enc.info), name
        for gamma in (1, 70):
            u = (rng.random((gamma, k)) < 0.5).astype(np.uint8)
            # bytes other than 0/1: only bit 0 counts
            ub = u | (rng.integers(0, 128, size=u.shape).astype(np.uint8) << 1)
            cw = code.encode(torch.from_numpy(ub).cuda()).cpu().numpy()
            want = enc.encode(u)
            assert np.array_equal(cw, want), name
            assert not _syndrome(H, cw).any()


def test_random_codewords_match_oracle(pkg):
    """Information bits are the oracle's Philox draws (counter word 3 = 1) and the codewords its encoding,
    for frame ids across the 2^32 boundary of the counter."""
    for name, code, H in _codes(pkg)[:2]:
        enc = oracle.Encoder(H)
        for first, gamma in ((0, 33), ((1 << 32) - 7, 40)):
            info, cw = code.random_codewords(seed=(5 << 32) + 3, first_frame=first, gamma=gamma)
            u = oracle.info_bits((5 << 32) + 3, first, gamma, enc.k)
            assert np.array_equal(info.cpu().numpy(), u), name
            assert np.array_equal(cw.cpu().numpy(), enc.encode(u)), name


def test_random_codewords_full_size(pkg):
    """n = 18360 (4 x 24, p = 765), the bench's code: information set equal to the oracle's, every codeword
    satisfies all 3060 checks, carries the oracle's information bits, and is about half ones."""
    shifts = synth.qc_shifts(4, 24, 765, seed=2)
    code = pkg.QCCode(shifts, 765)
    H = sp.csr_matrix(oracle.qc_parity_check(shifts, 765))
    enc = oracle.Encoder(H, track=False)
    k, pos = code.info_set()
    assert k == enc.k == 15303 and np.array_equal(pos, enc.info)
    info, cw = code.random_codewords(seed=9, first_frame=1000, gamma=96)
    c = cw.cpu().numpy()
    assert not _syndrome(H, c).any()
    assert np.array_equal(c[:, pos], oracle.info_bits(9, 1000, 96, k)[:, :])
    assert np.array_equal(info.cpu().numpy(), c[:, pos])
    assert abs(c.mean() - 0.5) < 0.01


def test_channel_codewords_matches_oracle(pkg):
    """mu = 2 (x + sigma g) / sigma^2 with x = 1 - 2c on the all-zero channel's noise g: the oracle's
    implementation of the generator, bit for bit."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    _, cw = code.random_codewords(seed=3, first_frame=17, gamma=50)
    for ebn0, first in [(2.0, 0), (4.5, 123456789012)]:
        out = code.channel_codewords(ebn0, 77, first, cw).cpu().numpy().astype(np.float64)
        sigma = oracle.sigma_from_ebn0(ebn0, 0.5)
        c = cw.cpu().numpy()
        mu = oracle.channel_awgn(77, first, 50, code.N, sigma, cw=c)
        assert np.array_equal(out, mu.astype(np.float64))  # the generator's binary32 bits
        # the all-zero word reproduces ldpc_channel exactly
        z = code.channel_codewords(ebn0, 77, first, torch.zeros_like(cw)).cpu().numpy()
        assert np.array_equal(z, code.channel(ebn0, 77, first, 50).cpu().numpy())


def _batch_counts_cw(pkg, code, ebn0, seed, first, frames, **kw):
    k, pos = code.info_set()
    _, cw = code.random_codewords(seed, first, frames, want_info=False)
    llr = code.channel_codewords(ebn0, seed, first, cw)
    _, hard, iters, ok = code.decode(llr, want_post=False, **kw)
    pos_t = torch.from_numpy(pos.astype(np.int64)).cuda()
    errs = (hard[:, pos_t] != cw[:, pos_t]).sum(dim=1).cpu().numpy().astype(np.int64)
    okn = ok.cpu().numpy()
    return {"frames": frames, "frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()),
            "iters_sum": int(iters.cpu().numpy().sum()), "undetected": int(((errs > 0) & (okn == 1)).sum())}


@pytest.mark.parametrize("case", ["sp_f32", "ms_i8", "ragged_slots", "high_frame_ids"])
def test_ber_sim_random_codewords_equals_batch(pkg, case):
    """The continuous simulation with random codewords counts exactly what the batch path counts on the
    same frames: same codewords, same channel, same decisions, errors over the information bits."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    algo, msg, max_iter, early = pkg.ALGO_SP, pkg.MSG_F32, 12, True
    frames, first, gamma, ebn0 = 400, 3, 128, 1.5
    if case == "ms_i8":
        algo, msg, max_iter, early = pkg.ALGO_MS, pkg.MSG_I8, 15, True
    elif case == "ragged_slots":
        gamma = 100
    elif case == "high_frame_ids":
        first = (1 << 32) - 50
    res = code.ber_sim(ebn0, seed=21, first_frame=first, max_frames=frames, target_frame_errors=10 ** 9,
                       gamma=gamma, max_iter=max_iter, early_stop=int(early), algo=algo, msg=msg,
                       codewords=pkg.CODEWORDS_RANDOM)
    want = _batch_counts_cw(pkg, code, ebn0, 21, first, frames, max_iter=max_iter, early_stop=early, algo=algo,
                            msg=msg)
    for key, v in want.items():
        assert res[key] == v, (key, res[key], v)
    assert want["frame_errors"] > 0


def test_ber_sim_random_codewords_matches_oracle(pkg):
    """Oracle channel of the oracle's codewords + FP64 decoding, errors over the information positions:
    the same counts as the device simulation (the channel is bit-exact, so every count agrees)."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    H = oracle.qc_parity_check(shifts, 64)
    rp, col = oracle.csr_rows(H)
    code = pkg.QCCode(shifts, 64)
    enc = oracle.Encoder(H)
    sigma = oracle.sigma_from_ebn0(1.75, 0.5)
    res = code.ber_sim(1.75, seed=5, first_frame=10, max_frames=300, target_frame_errors=10 ** 9, gamma=128,
                       max_iter=20, early_stop=1, codewords=pkg.CODEWORDS_RANDOM)
    cw = enc.encode(oracle.info_bits(5, 10, 300, enc.k))
    mu = oracle.channel_awgn(5, 10, 300, code.N, sigma, cw=cw)
    po, ho, io, oo = oracle.sp_decode(rp, col, code.N, mu, 20, early_stop=True, nthreads=8)
    errs = (ho[:, enc.info] != cw[:, enc.info]).sum(axis=1)
    want = {"frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()), "iters_sum": int(io.sum()),
            "undetected": int(((errs > 0) & (oo == 1)).sum())}
    for key, v in want.items():
        assert res[key] == v, (key, res[key], v)
    assert want["frame_errors"] > 0


def test_random_codewords_same_statistics_as_all_zero(pkg):
    """Channel symmetry (BP commutes with a codeword's sign flip): the frame error rate with random
    codewords equals the all-zero one's; 8192 frames each at 1.5 dB agree within 4 standard errors."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    kw = dict(max_frames=8192, target_frame_errors=10 ** 9, gamma=1024, max_iter=20, early_stop=1)
    z = code.ber_sim(1.5, seed=2, **kw)
    r = code.ber_sim(1.5, seed=3, codewords=pkg.CODEWORDS_RANDOM, **kw)
    pz, pr = z["frame_errors"] / 8192, r["frame_errors"] / 8192
    se = np.sqrt(pz * (1 - pz) / 8192 + pr * (1 - pr) / 8192)
    assert 0.01 < pz < 0.9 and abs(pz - pr) < 4 * se


def test_encoder_argument_errors(pkg):
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    k, _ = code.info_set()
    cw = torch.empty((4, code.N), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_encode(code.handle, None, cw)
    assert e.value.status == 1
    host = torch.zeros((4, k), dtype=torch.uint8)
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_encode(code.handle, host, cw)
    assert e.value.status == 1 and "device" in str(e.value)


@pytest.mark.parametrize("case", ["noms_f32", "noms_f16", "sp_f16"])
def test_ber_sim_random_codewords_other_decoders(pkg, case):
    """Random codewords with the learned min-sum (per-iteration parameter rows) and with FP16 storage (two
    frames per lane word): FP32 exactly the batch path's counts; FP16 statistically (the batch decoder's first
    check pass reads the FP32 channel LLRs, the continuous one their FP16 rounding)."""
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    T, frames, gamma, ebn0, seed, first = 9, 900, 128, 1.75, 31, 7
    msg = pkg.MSG_F16 if case.endswith("f16") else pkg.MSG_F32
    kw = dict(max_iter=T, early_stop=1, msg=msg)
    prm = None
    if case.startswith("noms"):
        rng = np.random.default_rng(4)
        p = np.stack([rng.uniform(0.7, 1.0, size=(T, 18)), rng.uniform(0.0, 0.3, size=(T, 18))], axis=-1)
        prm = torch.from_numpy(p.astype(np.float32)).cuda()
        kw["algo"] = pkg.ALGO_NOMS
    o = pkg.default_opts(codewords=pkg.CODEWORDS_RANDOM, **kw)
    if prm is not None:
        o.noms_params = prm.data_ptr()
    res = pkg.ldpc_ber_sim(code.handle, ebn0, seed, first, frames, 10 ** 9, gamma, o)
    k, pos = code.info_set()
    _, cw = code.random_codewords(seed, first, frames, want_info=False)
    llr = code.channel_codewords(ebn0, seed, first, cw)
    hard = torch.empty((frames, code.N), dtype=torch.uint8, device="cuda")
    iters = torch.empty(frames, dtype=torch.int32, device="cuda")
    ok = torch.empty(frames, dtype=torch.int32, device="cuda")
    ob = pkg.default_opts(**kw)
    if prm is not None:
        ob.noms_params = prm.data_ptr()
    pkg.ldpc_decode(code.handle, llr, ob, None, hard, iters, ok)
    pos_t = torch.from_numpy(pos.astype(np.int64)).cuda()
    errs = (hard[:, pos_t] != cw[:, pos_t]).sum(dim=1).cpu().numpy().astype(np.int64)
    okn = ok.cpu().numpy()
    want = {"frames": frames, "frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()),
            "iters_sum": int(iters.cpu().numpy().sum()), "undetected": int(((errs > 0) & (okn == 1)).sum())}
    assert 0 < want["frame_errors"] < frames
    if msg == pkg.MSG_F32:
        for key, v in want.items():
            assert res[key] == v, (key, res[key], v)
    else:
        assert res["frames"] == frames
        assert abs(res["frame_errors"] - want["frame_errors"]) <= max(3, 0.05 * want["frame_errors"])
        assert abs(res["iters_sum"] - want["iters_sum"]) <= 0.03 * want["iters_sum"]


def test_ber_sim_random_codewords_ragged_length(pkg):
    """N = 162 (3 x 6, p = 27): codeword rows end inside a 32-bit word and inside a group of four
    channel values; the continuous simulation still counts exactly what the batch path counts."""
    shifts = synth.qc_shifts(3, 6, 27, seed=6)
    code = pkg.QCCode(shifts, 27)
    assert code.N % 32 and code.N % 4
    res = code.ber_sim(1.25, seed=8, first_frame=11, max_frames=500, target_frame_errors=10 ** 9, gamma=96,
                       max_iter=10, early_stop=1, codewords=pkg.CODEWORDS_RANDOM)
    want = _batch_counts_cw(pkg, code, 1.25, 8, 11, 500, max_iter=10, early_stop=True)
    for key, v in want.items():
        assert res[key] == v, (key, res[key], v)
    assert want["frame_errors"] > 0


def test_encoder_dimension_zero(pkg):
    """H = I (a general code with one check per variable): k = 0, the only codeword is zero."""
    N = 40
    code = pkg.SparseCode(np.arange(N + 1), np.arange(N), N)
    k, pos = code.info_set()
    assert k == 0 and pos.size == 0
    cw = torch.full((5, N), 7, dtype=torch.uint8, device="cuda")
    pkg.ldpc_encode(code.handle, None, cw)
    assert not cw.any()
    info, cw2 = code.random_codewords(seed=1, first_frame=0, gamma=3)
    assert info is None and not cw2.any()
