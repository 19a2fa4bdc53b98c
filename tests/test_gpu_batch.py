"""Heterogeneous batches: many codes with uneven frame counts in one shared
iteration loop (persistent launches over tiles, CUDA-graph replay, autotuned
tile sizes) give exactly the per-code decoder's results, which the oracle pins."""
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


def batch_vs_single(pkg, specs, opts_kw, seeds, ebn0=2.0, compaction=None):
    """specs: list of (J, L, p, gamma, shift seed).  Runs the batch once per seed and compares every
    code's hard decisions, iteration counts and ok flags with a per-code ldpc_decode."""
    codes = [pkg.QCCode(synth.qc_shifts(J, L, p, seed=s), p) for J, L, p, g, s in specs]
    gammas = [g for _, _, _, g, _ in specs]
    o = pkg.default_opts(**opts_kw)
    b = pkg.ldpc_batch_create(codes, gammas, o)
    if compaction is not None:
        pkg.ldpc_batch_set_compaction(b, compaction)
    moved = []
    for seed in seeds:
        llrs = [torch.from_numpy(synth.gaussian_llrs(g, c.N, seed=seed + i, ebn0_db=ebn0, rate=1 - J / L)).cuda()
                for i, (c, (J, L, p, g, s)) in enumerate(zip(codes, specs))]
        hards = [torch.empty((g, c.N), dtype=torch.uint8, device="cuda") for c, g in zip(codes, gammas)]
        its = [torch.empty(g, dtype=torch.int32, device="cuda") for g in gammas]
        oks = [torch.empty(g, dtype=torch.int32, device="cuda") for g in gammas]
        pkg.ldpc_batch_decode(b, llrs, hards, its, oks)
        moved.append(sum(pkg.ldpc_batch_moved(b, len(codes))))
        for c, llr, h, it, ok in zip(codes, llrs, hards, its, oks):
            _, h1, it1, ok1 = c.decode(llr, want_post=False, **{k: v for k, v in opts_kw.items()
                                                                 if k in ("max_iter", "early_stop", "algo", "msg")})
            assert torch.equal(h, h1) and torch.equal(it, it1) and torch.equal(ok, ok1)
    info = pkg.ldpc_batch_info(b)
    info["moved"] = moved
    pkg.ldpc_batch_destroy(b)
    return codes, info


@pytest.mark.parametrize("opts_kw", [dict(max_iter=20, early_stop=1, msg=1),
                                     dict(max_iter=12, early_stop=0, msg=0),
                                     dict(max_iter=15, early_stop=1, algo=1, msg=2)])
def test_batch_equals_per_code_decode(pkg, opts_kw):
    specs = [(3, 6, 32, 1, 1), (4, 8, 37, 70, 2), (3, 12, 50, 33, 3), (4, 24, 128, 129, 4), (3, 9, 16, 5, 5),
             (4, 16, 64, 300, 6)]
    # three calls: the tuned eager run, the capture run, a graph replay
    _, info = batch_vs_single(pkg, specs, opts_kw, seeds=[10, 20, 30])
    assert info["tile_rows"] in (16, 64, 256) and all(t > 0 for t in info["tune_ms"])
    if not opts_kw.get("early_stop"):
        assert not any(info["moved"])  # compaction only with early stop


@pytest.mark.parametrize("opts_kw", [dict(max_iter=25, early_stop=1, msg=0),
                                     dict(max_iter=25, early_stop=1, msg=1),
                                     dict(max_iter=25, early_stop=1, algo=1, msg=2)])
def test_batch_compaction_equals_per_code_decode(pkg, opts_kw):
    """Frame-level compaction after iteration 8 (FP32, FP16 and int8 storage): the frames still running
    move to each code's second package area and their results still equal the per-code decoder's."""
    specs = [(3, 6, 40, 200, 11), (4, 8, 37, 150, 12), (3, 12, 50, 96, 13), (4, 24, 64, 70, 14), (3, 9, 16, 3, 15)]
    _, info = batch_vs_single(pkg, specs, opts_kw, seeds=[50, 60, 70], ebn0=2.75, compaction=8)
    assert all(m > 0 for m in info["moved"]), info["moved"]


def test_batch_matches_oracle(pkg):
    specs = [(3, 6, 16, 40, 7), (4, 8, 8, 9, 8)]
    codes = [pkg.QCCode(synth.qc_shifts(J, L, p, seed=s), p) for J, L, p, g, s in specs]
    o = pkg.default_opts(max_iter=25, early_stop=1, msg=0)
    b = pkg.ldpc_batch_create(codes, [g for *_, g, _ in specs], o)
    mus = [synth.gaussian_llrs(g, c.N, seed=40 + i, ebn0_db=2.0, rate=0.5) for i, (c, (_, _, _, g, _)) in
           enumerate(zip(codes, specs))]
    hards = [torch.empty((m.shape[0], c.N), dtype=torch.uint8, device="cuda") for c, m in zip(codes, mus)]
    its = [torch.empty(m.shape[0], dtype=torch.int32, device="cuda") for m in mus]
    oks = [torch.empty(m.shape[0], dtype=torch.int32, device="cuda") for m in mus]
    pkg.ldpc_batch_decode(b, [torch.from_numpy(m).cuda() for m in mus], hards, its, oks)
    for (J, L, p, g, s), c, m, h, it, ok in zip(specs, codes, mus, hards, its, oks):
        H = oracle.qc_parity_check(synth.qc_shifts(J, L, p, seed=s), p)
        rp, col = oracle.csr_rows(H)
        po, ho, io, oo = oracle.sp_decode(rp, col, c.N, m, 25, early_stop=True, nthreads=8)
        sure = np.abs(po) >= 1e-3
        assert np.array_equal(h.cpu().numpy()[sure], ho[sure])
        assert np.array_equal(it.cpu().numpy(), io) and np.array_equal(ok.cpu().numpy(), oo)
    pkg.ldpc_batch_destroy(b)


def test_mixed_64_code_batch(pkg):
    """64 seeded codes (3x6 .. 4x24, p 32..765, n 192..18360), 1..4096 frames each (log-uniform),
    FP16 messages, early stop: batch results equal per-code decodes."""
    mixed = synth.mixed_codes(64, seed=4)
    counts = synth.frame_counts(64, seed=4)
    specs = [(J, L, p, int(g), 0) for (J, L, p, sh), g in zip(mixed, counts)]
    codes = [pkg.QCCode(sh, p) for (J, L, p, sh) in mixed]
    o = pkg.default_opts(max_iter=30, early_stop=1, msg=1)
    b = pkg.ldpc_batch_create(codes, [int(g) for g in counts], o)
    pkg.ldpc_batch_set_compaction(b, 12)
    llrs = [torch.from_numpy(synth.gaussian_llrs(int(g), c.N, seed=100 + i, ebn0_db=3.0, rate=1 - J / L)).cuda()
            for i, (c, (J, L, p, g, s)) in enumerate(zip(codes, specs))]
    for rep in range(2):
        hards = [torch.empty((l.shape[0], c.N), dtype=torch.uint8, device="cuda") for c, l in zip(codes, llrs)]
        its = [torch.empty(l.shape[0], dtype=torch.int32, device="cuda") for l in llrs]
        pkg.ldpc_batch_decode(b, llrs, hards, its, None)
    moved = pkg.ldpc_batch_moved(b, 64)
    assert sum(moved) > 0
    checked = set(range(0, 64, 7)) | {i for i in range(64) if moved[i]}  # every compacted code too
    for i in sorted(checked):
        _, h1, it1, _ = codes[i].decode(llrs[i], max_iter=30, early_stop=True, msg=1, want_post=False)
        assert torch.equal(hards[i], h1) and torch.equal(its[i], it1)
    pkg.ldpc_batch_destroy(b)


def test_phase_boundary_probe(pkg):
    """The synchronization probe behind the graph-versus-cooperative-loop reading: both forms run and
    report a positive cost per boundary, and bad arguments are refused."""
    r = pkg.ldpc_sync_probe(40, 5)
    assert 0.0 < r["graph_us"] < 1e3 and 0.0 < r["cooperative_us"] < 1e3, r
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_sync_probe(0, 5)
