"""The allocation-free decode entry point, for callers that cannot allocate device
memory (captured streams, real-time loops, pre-reserved device memory): its results
must equal those of the ordinary ldpc_decode on the same inputs, on two calls in a
row (the second call starts from the scratch the first one left behind).

This file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import numpy as np
import pytest

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
    pa, ha, ia, oa = a
    pb, hb, ib, ob = b
    assert np.max(np.abs(pa - pb) / np.maximum(1.0, np.abs(pb))) <= REL
    assert np.array_equal(ha, hb) and np.array_equal(ia, ib) and np.array_equal(oa, ob)


def test_noalloc_decode_matches_decode_twice(pkg):
    shifts = synth.qc_shifts(3, 6, 64, seed=1)
    code = pkg.QCCode(shifts, 64)
    # first call: early stop, 100 frames; second call: fewer frames, fixed iterations
    cases = [(100, 11, 2.0, dict(max_iter=30, early_stop=1)), (40, 12, 1.5, dict(max_iter=20, early_stop=0))]
    for g, seed, ebn0, kw in cases:
        llr = torch.from_numpy(synth.gaussian_llrs(g, code.N, seed=seed, ebn0_db=ebn0, rate=0.5)).cuda()
        o = pkg.default_opts(**kw)
        _same(_run(pkg, pkg.ldpc_decode_noalloc, code, llr, o), _run(pkg, pkg.ldpc_decode, code, llr, o))
    # integer min-sum through the same scratch
    llr = torch.from_numpy(synth.gaussian_llrs(70, code.N, seed=13, ebn0_db=2.0, rate=0.5)).cuda()
    o = pkg.default_opts(max_iter=15, early_stop=1, algo=pkg.ALGO_MS, msg=pkg.MSG_I8)
    _same(_run(pkg, pkg.ldpc_decode_noalloc, code, llr, o), _run(pkg, pkg.ldpc_decode, code, llr, o))
    code.close()


def test_noalloc_rejects_requests_beyond_its_scratch(pkg):
    code = pkg.QCCode(synth.qc_shifts(4, 24, 765, seed=2), 765)
    llr = torch.zeros((1000, code.N), dtype=torch.float32, device="cuda")  # about 440 MB of workspace
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_decode_noalloc(code.handle, llr, pkg.default_opts())
    assert e.value.status == 1 and "scratch" in str(e.value)
    code.close()
