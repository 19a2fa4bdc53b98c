"""General (index-table) LDPC codes: the pipelined passes with table-driven copy stages
against the FP64 oracle (which takes any H), and a QC code given as a plain sparse matrix
against the QC decoder.  Tolerances as in test_gpu_qc."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_qc import _cmp_sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_0334_gb300 as p

    p.lib()
    return p


@pytest.mark.parametrize("N,M,degs,gamma", [(400, 200, (2, 3, 3, 4, 6), 70), (1200, 300, (3, 3, 4), 40),
                                             (151, 100, (2, 2, 3, 8), 33)])
def test_sparse_sum_product_matches_oracle(pkg, N, M, degs, gamma):
    rp, col = synth.random_ldpc(N, M, seed=N + M, var_degrees=degs)
    code = pkg.SparseCode(rp, col, N)
    assert (code.N, code.M, code.E) == (N, M, len(col))
    mu = synth.gaussian_llrs(gamma, N, seed=5, ebn0_db=2.0, rate=1 - M / N)
    for iters, es in ((10, False), (30, True)):
        post, hard, it, ok = code.decode(torch.from_numpy(mu).cuda(), max_iter=iters, early_stop=es)
        ref = oracle.sp_decode(rp, col, N, mu, iters, early_stop=es, nthreads=8)
        _cmp_sp(post, hard, it, ok, ref, f"sparse N={N}", strict_all=iters <= 10,
                sens=(rp, col, N, mu, iters, es))


def test_sparse_min_sum_bit_exact(pkg):
    N, M = 500, 250
    rp, col = synth.random_ldpc(N, M, seed=9)
    code = pkg.SparseCode(rp, col, N)
    mu = synth.integer_llrs(70, N, seed=4, lo=-200, hi=200, scale=0.25)
    post, hard, iters, ok = code.decode(torch.from_numpy(mu).cuda(), max_iter=12, early_stop=True, algo=pkg.ALGO_MS)
    po, ho, io, oo = oracle.ms_decode(rp, col, N, mu, 12, early_stop=True)
    assert np.array_equal(post.cpu().numpy(), po.astype(np.float32) * 0.25)
    assert np.array_equal(hard.cpu().numpy(), ho)
    assert np.array_equal(iters.cpu().numpy(), io) and np.array_equal(ok.cpu().numpy(), oo)


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_qc_code_as_sparse_matrix_equals_qc_decoder(pkg, msg):
    """The same H through both addressing schemes: identical decisions, iterations and ok flags (FP32:
    identical posteriors too -- same arithmetic in the same order)."""
    shifts = synth.qc_shifts(4, 12, 31, seed=6)
    rp, col = oracle.csr_rows(oracle.qc_parity_check(shifts, 31))
    qc = pkg.QCCode(shifts, 31)
    sc = pkg.SparseCode(rp, col, qc.N)
    M = pkg.MSG_F32 if msg == "f32" else pkg.MSG_F16
    llr = torch.from_numpy(synth.gaussian_llrs(100, qc.N, seed=8, ebn0_db=2.5, rate=2 / 3)).cuda()
    a = qc.decode(llr, max_iter=20, early_stop=True, msg=M)
    b = sc.decode(llr, max_iter=20, early_stop=True, msg=M)
    if msg == "f32":
        assert torch.equal(a[0], b[0])
        assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])
    else:
        # FP16: the QC decoder's first check pass reads the FP32 channel LLRs, the general one
        # their FP16 transformed rounding; decisions agree on almost every frame
        same = (a[1] == b[1]).all(dim=1).float().mean().item()
        assert same >= 0.9, same


def test_sparse_unsupported_calls(pkg):
    rp, col = synth.random_ldpc(64, 32, seed=1)
    code = pkg.SparseCode(rp, col, 64)
    with pytest.raises(pkg.LdpcError) as e:
        code.ber_sim(2.0, max_frames=64, gamma=64)
    assert e.value.status == 5
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_batch_create([code], [8], pkg.default_opts())
    assert e.value.status == 5
