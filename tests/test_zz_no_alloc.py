"""The allocation-free decode entry point, for callers that cannot allocate device
memory (captured streams, real-time loops, pre-reserved device memory): its results
must equal those of the ordinary ldpc_decode on the same inputs, on two calls in a
row (the second call starts from the scratch the first one left behind).

Covered: QC codes with sum-product over FP32 and FP16 message storage and integer
min-sum, and a general (index-table) code, which is also checked against the FP64
oracle directly.

This file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_0334_gb300 as p

    p.lib()
    return p


def _run(pkg, fn, code, llr, opts):
    g = llr.shape[0]
    post = torch.empty((g, code.N), dtype=torch.float32, device="cuda")
    hard = torch.empty((g, code.N), dtype=torch.uint8, device="cuda")
    iters = torch.empty(g, dtype=torch.int32, device="cuda")
    ok = torch.empty(g, dtype=torch.int32, device="cuda")
    fn(code.handle, llr, opts, post, hard, iters, ok)
    torch.cuda.synchronize()
    return post.cpu().numpy(), hard.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()


def _same(a, b):
    """The two entry points run the same kernels on the same inputs: equal results."""
    pa, ha, ia, oa = a
    pb, hb, ib, ob = b
    assert np.max(np.abs(pa - pb) / np.maximum(1.0, np.abs(pb))) <= REL
    assert np.array_equal(ha, hb) and np.array_equal(ia, ib) and np.array_equal(oa, ob)


@pytest.mark.parametrize("msg", ["F32", "F16"])
def test_noalloc_decode_matches_decode_twice(pkg, msg):
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    m = pkg.MSG_F32 if msg == "F32" else pkg.MSG_F16
    # first call: early stop, 100 frames; second call: fewer frames, fixed iterations
    cases = [(100, 11, 2.0, dict(max_iter=30, early_stop=1)), (40, 12, 1.5, dict(max_iter=20, early_stop=0))]
    for g, seed, ebn0, kw in cases:
        llr = torch.from_numpy(synth.gaussian_llrs(g, code.N, seed=seed, ebn0_db=ebn0, rate=0.5)).cuda()
        o = pkg.default_opts(msg=m, **kw)
        _same(_run(pkg, pkg.ldpc_decode_noalloc, code, llr, o), _run(pkg, pkg.ldpc_decode, code, llr, o))
    # integer min-sum through the same scratch
    llr = torch.from_numpy(synth.gaussian_llrs(70, code.N, seed=13, ebn0_db=2.0, rate=0.5)).cuda()
    o = pkg.default_opts(max_iter=15, early_stop=1, algo=pkg.ALGO_MS, msg=pkg.MSG_I8)
    _same(_run(pkg, pkg.ldpc_decode_noalloc, code, llr, o), _run(pkg, pkg.ldpc_decode, code, llr, o))
    code.close()


def test_noalloc_general_code_matches_decode_and_oracle(pkg):
    """A code given by its index tables (ldpc_code_create_sparse), sum-product and integer
    min-sum, two calls in a row; also against the FP64 oracle (FP32 within the tolerance of the
    block-code tests, min-sum bit-exact)."""
    from test_gpu_qc import _cmp_sp

    N, M = 400, 200
    rp, col = synth.random_ldpc(N, M, seed=N + M)
    code = pkg.SparseCode(rp, col, N)
    for g, seed, iters, es in ((70, 5, 10, 0), (33, 6, 20, 1)):
        mu = synth.gaussian_llrs(g, N, seed=seed, ebn0_db=2.0, rate=1 - M / N)
        llr = torch.from_numpy(mu).cuda()
        o = pkg.default_opts(max_iter=iters, early_stop=es)
        got = _run(pkg, pkg.ldpc_decode_noalloc, code, llr, o)
        _same(got, _run(pkg, pkg.ldpc_decode, code, llr, o))
        ref = oracle.sp_decode(rp, col, N, mu, iters, early_stop=bool(es), nthreads=8)
        t = [torch.from_numpy(x) for x in got]
        _cmp_sp(*t, ref, f"noalloc sparse it={iters}", strict_all=iters <= 10,
                sens=(rp, col, N, mu, iters, bool(es)))
    mu = synth.integer_llrs(50, N, seed=4, lo=-200, hi=200, scale=0.25)
    llr = torch.from_numpy(mu).cuda()
    o = pkg.default_opts(max_iter=12, early_stop=1, algo=pkg.ALGO_MS, msg=pkg.MSG_I8)
    for _ in range(2):
        post, hard, it, ok = _run(pkg, pkg.ldpc_decode_noalloc, code, llr, o)
        po, ho, io, oo = oracle.ms_decode(rp, col, N, mu, 12, early_stop=True)
        assert np.array_equal(post, po.astype(np.float32) * 0.25)
        assert np.array_equal(hard, ho) and np.array_equal(it, io) and np.array_equal(ok, oo)
    code.close()


def test_noalloc_rejects_requests_beyond_its_scratch(pkg):
    code = pkg.QCCode(synth.qc_shifts(4, 24, 765, seed=2), 765)
    llr = torch.zeros((1000, code.N), dtype=torch.float32, device="cuda")  # about 440 MB of workspace
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_decode_noalloc(code.handle, llr, pkg.default_opts())
    assert e.value.status == 1 and "scratch" in str(e.value)
    code.close()
