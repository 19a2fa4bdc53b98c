"""GPU parity of the learned normalized/offset min-sum: inference, loss, and the
hand-written backward pass against the FP64 oracle gradient; checkpointing; and
what training gains over plain min-sum (the same rule with w = 1, o = 0)."""
import numpy as np
import pytest

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


def setup(J, L, p, seed):
    shifts = synth.qc_shifts(J, L, p, seed=seed)
    H = oracle.qc_parity_check(shifts, p)
    rp, col = oracle.csr_rows(H)
    return shifts, rp, col, oracle.circulant_index(rp, col, p, L)


def rand_params(T, ncirc, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.6, 1.0, (T, ncirc)), rng.uniform(0.0, 0.6, (T, ncirc))], axis=-1).astype(
        np.float32)


def test_noms_inference_matches_oracle(pkg):
    shifts, rp, col, cb = setup(4, 12, 31, 3)
    code = pkg.QCCode(shifts, 31)
    T = 8
    prm = rand_params(T, 48, 1)
    mu = synth.gaussian_llrs(100, code.N, seed=4, ebn0_db=2.5, rate=2 / 3)
    o = pkg.default_opts(max_iter=T, algo=pkg.ALGO_NOMS, msg=pkg.MSG_F32)
    prm_d = torch.from_numpy(prm).cuda()
    o.noms_params = prm_d.data_ptr()
    post = torch.empty((100, code.N), device="cuda")
    hard = torch.empty((100, code.N), dtype=torch.uint8, device="cuda")
    pkg.ldpc_decode(code.handle, torch.from_numpy(mu).cuda(), o, post, hard)
    _, po, _ = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), nthreads=8)
    po = np.clip(po, -30, 30)
    p = post.cpu().numpy()
    assert np.max(np.abs(p - po) / np.maximum(1, np.abs(po))) < 1e-4
    sure = np.abs(po) > 1e-3
    assert np.array_equal(hard.cpu().numpy()[sure], (po < 0)[sure])


# rows of 6 edges (padded to 8: the general kernels) and full rows of 8 and 24 edges (the kernels
# for codes whose base matrix has no zero block and whose row degree fills the template)
SHAPES = [(3, 6, 32), (4, 8, 16), (4, 24, 11)]


@pytest.mark.parametrize("J,L,p", SHAPES)
@pytest.mark.parametrize("msg,ckpt", [(0, 1), (0, 3)])
def test_noms_loss_and_gradient_match_oracle(pkg, msg, ckpt, J, L, p):
    shifts, rp, col, cb = setup(J, L, p, 2)
    code = pkg.QCCode(shifts, p)
    T, B = 5, 70
    prm = rand_params(T, J * L, 3)
    mu = synth.gaussian_llrs(B, code.N, seed=5, ebn0_db=1.5 + 0.5 * (L > 8), rate=1 - J / L)
    prm_d = torch.from_numpy(prm).cuda()
    loss, post = pkg.ldpc_noms_forward(code.handle, torch.from_numpy(mu).cuda(), prm_d, msg, ckpt, 30.0, True)
    grad = torch.zeros_like(prm_d)
    pkg.ldpc_noms_backward(code.handle, prm_d, grad)
    lo, po, go = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), want_grad=True, nthreads=8)
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(post.cpu().numpy() - po) / np.maximum(1, np.abs(po))) < 1e-4
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(go).max()
    # element by element: within 1e-3 of each gradient entry (entries below 1e-3 of the largest
    # measured against that floor); measured 8e-5
    rel = np.abs(g - go) / np.maximum(np.abs(go), 1e-3 * scale)
    assert rel.max() <= 1e-3, (rel.max(), scale)


def test_noms_checkpointing_does_not_change_gradients(pkg):
    shifts, rp, col, cb = setup(4, 8, 16, 6)
    code = pkg.QCCode(shifts, 16)
    T = 7
    prm_d = torch.from_numpy(rand_params(T, 32, 8)).cuda()
    llr = torch.from_numpy(synth.gaussian_llrs(96, code.N, seed=9, ebn0_db=2.0, rate=0.5)).cuda()
    out = []
    for k in (1, 2, 3, 7):
        loss, _ = pkg.ldpc_noms_forward(code.handle, llr, prm_d, 0, k, 30.0)
        g = torch.zeros_like(prm_d)
        pkg.ldpc_noms_backward(code.handle, prm_d, g)
        out.append((float(loss), g.cpu().numpy()))
    for lk, gk in out[1:]:
        assert lk == out[0][0]
        # same values up to the order of the float atomic sums of the parameter gradients
        assert np.allclose(gk, out[0][1], rtol=1e-5, atol=1e-6 * np.abs(out[0][1]).max())


@pytest.mark.parametrize("J,L,p", SHAPES)
def test_noms_fp16_storage_gradient(pkg, J, L, p):
    """FP16 storage of the messages against the oracle of the same variant (the stored alpha and beta
    rounded to binary16, its forward in binary32 so that both sides round the same values and pick the
    same arg-min edges): loss and gradient element by element.  Against the unrounded FP64 oracle the min-sum
    gradient jumps wherever rounding changes the arg-min edge, so that comparison is not element-wise."""
    shifts, rp, col, cb = setup(J, L, p, 2)
    code = pkg.QCCode(shifts, p)
    T, B = 5, 70  # two packages of 64 frames, the second with 6
    prm = rand_params(T, J * L, 4)
    mu = synth.gaussian_llrs(B, code.N, seed=6, ebn0_db=1.5 + 0.5 * (L > 8), rate=1 - J / L)
    prm_d = torch.from_numpy(prm).cuda()
    loss, _ = pkg.ldpc_noms_forward(code.handle, torch.from_numpy(mu).cuda(), prm_d, pkg.MSG_F16, 2, 30.0)
    grad = torch.zeros_like(prm_d)
    pkg.ldpc_noms_backward(code.handle, prm_d, grad)
    lo, _, go = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), want_grad=True, nthreads=8,
                            store16=True)
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo)
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.abs(g - go) / np.maximum(np.abs(go), 1e-3 * np.abs(go).max())
    print(f"FP16 gradient: largest element-wise relative deviation {rel.max():.2e}")
    assert rel.max() <= 1e-3, rel.max()


@pytest.mark.parametrize("msg", [0, 1])
def test_noms_gradient_with_zero_blocks(pkg, msg):
    """A base matrix with zero blocks (rows of 8 slots with some absent, columns of 2 to 4 edges):
    loss and gradient against the oracle (FP16 against its binary16 variant), element by element."""
    J, L, p = 4, 8, 16
    shifts = synth.qc_shifts(J, L, p, seed=6, zero_blocks=5)
    H = oracle.qc_parity_check(shifts, p)
    rp, col = oracle.csr_rows(H)
    cb = oracle.circulant_index(rp, col, p, L)
    assert (np.asarray(shifts) < 0).sum() == 5
    code = pkg.QCCode(shifts, p)
    T, B = 4, 70
    prm = rand_params(T, J * L, 13)
    mu = synth.gaussian_llrs(B, code.N, seed=14, ebn0_db=1.5, rate=0.5)
    prm_d = torch.from_numpy(prm).cuda()
    loss, post = pkg.ldpc_noms_forward(code.handle, torch.from_numpy(mu).cuda(), prm_d, msg, 2, 30.0, True)
    grad = torch.zeros_like(prm_d)
    pkg.ldpc_noms_backward(code.handle, prm_d, grad)
    lo, po, go = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), want_grad=True, nthreads=8,
                             store16=bool(msg))
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(post.cpu().numpy() - po) / np.maximum(1, np.abs(po))) < 1e-4
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.abs(g - go) / np.maximum(np.abs(go), 1e-3 * np.abs(go).max())
    # circulants of zero blocks have no edges: no gradient on either side
    zb = (np.asarray(shifts).reshape(-1) < 0)
    assert np.all(g[:, zb, :] == 0.0) and np.all(go[:, zb, :] == 0.0)
    assert rel.max() <= 1e-3, rel.max()


def test_noms_fp16_gradient_ten_iterations(pkg):
    """The training configuration's depth (10 unrolled iterations, a checkpoint every 2) on a code with
    full rows of 24 edges, FP16 messages against the oracle's binary16 variant, element by element."""
    J, L, p = 4, 24, 31
    shifts, rp, col, cb = setup(J, L, p, 7)
    code = pkg.QCCode(shifts, p)
    T, B = 10, 64
    prm = rand_params(T, J * L, 9)
    mu = synth.gaussian_llrs(B, code.N, seed=10, ebn0_db=3.0, rate=1 - J / L)
    prm_d = torch.from_numpy(prm).cuda()
    loss, _ = pkg.ldpc_noms_forward(code.handle, torch.from_numpy(mu).cuda(), prm_d, pkg.MSG_F16, 2, 30.0)
    grad = torch.zeros_like(prm_d)
    pkg.ldpc_noms_backward(code.handle, prm_d, grad)
    lo, _, go = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), want_grad=True, nthreads=8,
                            store16=True)
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo)
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.abs(g - go) / np.maximum(np.abs(go), 1e-3 * np.abs(go).max())
    assert rel.max() <= 1e-3, rel.max()


@pytest.mark.parametrize("msg", [0, 1])
def test_noms_gradient_with_clipped_check_messages(pkg, msg):
    """Weights above 1 and a low clip: w * m - o often exceeds the clip, so alpha is clipped and its
    gradient is zero there.  Loss, posteriors and the gradient against the oracle (FP16 storage
    against its binary16 variant), element by element."""
    J, L, p = 4, 8, 16
    shifts, rp, col, cb = setup(J, L, p, 5)
    code = pkg.QCCode(shifts, p)
    T, B, clip = 4, 64, 6.0
    rng = np.random.default_rng(11)
    prm = np.stack([rng.uniform(1.0, 1.6, (T, J * L)), rng.uniform(0.0, 0.3, (T, J * L))], axis=-1).astype(
        np.float32)
    mu = synth.gaussian_llrs(B, code.N, seed=12, ebn0_db=3.0, rate=0.5)
    prm_d = torch.from_numpy(prm).cuda()
    loss, post = pkg.ldpc_noms_forward(code.handle, torch.from_numpy(mu).cuda(), prm_d, msg, 2, clip, True)
    grad = torch.zeros_like(prm_d)
    pkg.ldpc_noms_backward(code.handle, prm_d, grad)
    lo, po, go = oracle.noms(rp, col, cb, code.N, mu, T, prm.astype(np.float64), clip=clip, want_grad=True,
                             nthreads=8, store16=bool(msg))
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo)
    assert np.max(np.abs(post.cpu().numpy() - po) / np.maximum(1, np.abs(po))) < 1e-4
    # the messages saturate (a posterior of at least 2 * clip needs several inputs at the clip, and with
    # w > 1 and inputs at the clip w * m - o exceeds it)
    assert np.mean(np.abs(po) >= 2 * clip) > 0.1
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.abs(g - go) / np.maximum(np.abs(go), 1e-3 * np.abs(go).max())
    assert rel.max() <= 1e-3, rel.max()


def test_parameters_must_be_8_byte_aligned(pkg):
    """The kernels read (w, o) as pairs: a parameter pointer 4 bytes past an 8-byte boundary is refused
    before any launch, for training and for inference."""
    code = pkg.QCCode(synth.qc_shifts(3, 6, 8, seed=1), 8)
    store = torch.ones(3 * 18 * 2 + 1, device="cuda")
    prm = store[1:].view(3, 18, 2)
    assert prm.data_ptr() % 8 == 4
    llr = torch.from_numpy(synth.gaussian_llrs(32, code.N, seed=1, ebn0_db=2.0, rate=0.5)).cuda()
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_noms_forward(code.handle, llr, prm, 0, 1, 30.0)
    o = pkg.default_opts(max_iter=3, algo=pkg.ALGO_NOMS, msg=pkg.MSG_F32)
    o.noms_params = prm.data_ptr()
    post = torch.empty((32, code.N), device="cuda")
    hard = torch.empty((32, code.N), dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_decode(code.handle, llr, o, post, hard)


def test_backward_requires_forward(pkg):
    code = pkg.QCCode(synth.qc_shifts(3, 6, 8, seed=1), 8)
    prm = torch.ones((3, 18, 2), device="cuda")
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_noms_backward(code.handle, prm, torch.zeros_like(prm))


def test_training_gains_over_plain_min_sum(pkg):
    """A short training run (the simulator's own frames, Eb/N0 ~ U[2.5, 4.5]) lowers the loss and the
    trained decoder makes fewer bit errors than the untrained rule (w = 1, o = 0, plain min-sum)."""
    from paper_1204_0334_gb300 import noms

    shifts = synth.qc_shifts(4, 24, 128, seed=2)
    code = pkg.QCCode(shifts, 128)
    T = 10
    p0 = noms.init_params(T, 96)
    params, losses = noms.train_noms(code, T=T, steps=60, batch=512, ebn0=(2.5, 4.5), lr=0.03, seed=3,
                                     msg=pkg.MSG_F16, ckpt_every=2, params=p0)
    assert np.mean(losses[-10:]) < 0.8 * np.mean(losses[:5])
    base = noms.ber(code, p0, 3.5, frames=8192)
    trained = noms.ber(code, params, 3.5, frames=8192)
    assert trained["bit_errors"] < 0.5 * base["bit_errors"], (trained, base)


@pytest.mark.parametrize("msg,exact", [("f32", True), ("f16", False)])
def test_noms_ber_sim_equals_batch_decode(pkg, msg, exact):
    """The continuous simulation runs frames at different iterations side by side; each frame must still
    use the parameter row of its own iteration: counts equal those of the batch decoder on the same
    channel frames (FP16: statistically, the batch decoder's first pass reads the FP32 channel LLRs)."""
    shifts, rp, col, cb = setup(3, 6, 64, 1)
    code = pkg.QCCode(shifts, 64)
    T, frames, gamma, ebn0, seed, first = 9, 900, 128, 1.75, 31, 7
    prm = torch.from_numpy(rand_params(T, 18, 4)).cuda()
    M = pkg.MSG_F32 if msg == "f32" else pkg.MSG_F16
    o = pkg.default_opts(max_iter=T, early_stop=1, algo=pkg.ALGO_NOMS, msg=M)
    o.noms_params = prm.data_ptr()
    res = pkg.ldpc_ber_sim(code.handle, ebn0, seed, first, frames, 10 ** 9, gamma, o)
    llr = code.channel(ebn0, seed, first, frames)
    hard = torch.empty((frames, code.N), dtype=torch.uint8, device="cuda")
    iters = torch.empty(frames, dtype=torch.int32, device="cuda")
    ok = torch.empty(frames, dtype=torch.int32, device="cuda")
    pkg.ldpc_decode(code.handle, llr, o, None, hard, iters, ok)
    errs = hard.sum(dim=1).cpu().numpy().astype(np.int64)
    okn = ok.cpu().numpy()
    want = {"frames": frames, "frame_errors": int((errs > 0).sum()), "bit_errors": int(errs.sum()),
            "iters_sum": int(iters.cpu().numpy().sum()), "undetected": int(((errs > 0) & (okn == 1)).sum())}
    assert 0 < want["frame_errors"] < frames
    if exact:
        for k, v in want.items():
            assert res[k] == v, (k, res[k], v)
    else:
        assert res["frames"] == frames
        assert abs(res["frame_errors"] - want["frame_errors"]) <= max(3, 0.05 * want["frame_errors"])
        assert abs(res["iters_sum"] - want["iters_sum"]) <= 0.03 * want["iters_sum"]
