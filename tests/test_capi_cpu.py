"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/*.h declares, and rejects bad arguments before touching a device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1204_0334_gb300 import build as b

    path = b.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ldpc\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ldpc_code_create", "ldpc_decode", "ldpc_channel", "ldpc_ber_sim"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_1204_0334_gb300 as pkg

    assert set(pkg.exported_names()) <= set(declared_functions())
    assert set(declared_functions()) <= set(pkg.exported_names())


def test_validation_without_a_device(lib):
    import paper_1204_0334_gb300 as pkg

    pkg.lib()
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_code_create(np.array([[0, 64]]), 64)  # shift out of [0, p)
    assert e.value.status == 1 and "shift" in str(e.value)
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_code_create(np.array([[-2, 0]]), 64)
    with pytest.raises(pkg.LdpcError):
        pkg.ldpc_code_create(np.zeros((2, 40), dtype=np.int32), 8)  # L > 32
    h = pkg.ldpc_code_create(np.array([[0, 1, -1], [2, -1, 3]]), 5)
    d = pkg.ldpc_code_dims(h)
    assert d == {"N": 15, "M": 10, "E": 20, "K": 5}
    o = pkg.default_opts()
    assert (o.max_iter, o.algo, o.msg, o.clip, o.frac_bits) == (30, 0, 0, 30.0, 2)
    pkg.ldpc_code_destroy(h)
    assert lib.ldpc_status_str(1) is not None


def test_ldpccc_rejects_sizes_beyond_32_bit_indexing(lib):
    """The window decoder indexes 128-byte package lines with 32-bit integers: a ring of
    I * Lambda frames of ceil(gamma / 32) packages with J * c edges each must stay below 2^31
    lines, and the request is refused before any device memory is touched."""
    import paper_1204_0334_gb300 as pkg

    pkg.lib()
    shifts = np.array([[0, 1, 2, 3, 4, 5], [1, 2, 3, 4, 5, 0], [2, 3, 4, 5, 0, 1]])
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpccc_create(shifts, 4096, 4000, 1 << 20)  # 12000 * 32768 * 3 * 8192 lines
    assert e.value.status == 1 and "2^31" in str(e.value)
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpccc_create(shifts, 64, 0, 32)  # no processors
    assert e.value.status == 1


def test_sparse_code_validation_without_a_device(lib):
    """Malformed compressed-row input is refused before any device memory is touched."""
    import paper_1204_0334_gb300 as pkg

    pkg.lib()
    cases = [([1, 2], [0], 4),                  # row_ptr[0] != 0
             ([0, 2, 3], [1, 0, 2], 4),         # columns not increasing within a row
             ([0, 2, 4], [0, 1, 2, 9], 4),      # column out of range
             ([0, 2, 2], [0, 1], 4),            # empty row
             ([0, 33], list(range(33)), 40)]    # row degree above 32
    for rp, col, N in cases:
        with pytest.raises(pkg.LdpcError) as e:
            pkg.ldpc_code_create_sparse(rp, col, N)
        assert e.value.status == 1, (rp, col)
    # a column of degree 9
    rp = [2 * m for m in range(10)]
    col = [c for m in range(9) for c in (0, m + 1)]
    with pytest.raises(pkg.LdpcError) as e:
        pkg.ldpc_code_create_sparse(rp, col, 12)
    assert e.value.status == 1 and "degree" in str(e.value)


@pytest.mark.parametrize("J,L,p,seed,zero_blocks", [(3, 6, 64, 1, 0), (4, 24, 32, 3, 0), (4, 12, 40, 7, 5),
                                                    (4, 24, 765, 2, 0)])
def test_information_set_matches_oracle(lib, J, L, p, seed, zero_blocks):
    """The encoder's information set is built on the host (no device memory): it equals the oracle's
    greedy right-to-left column basis complement, including the rank deficiency of QC codes and zero
    blocks, up to the full 4 x 24, p = 765 code."""
    import scipy.sparse as sp

    import oracle
    import paper_1204_0334_gb300 as pkg

    shifts = synth.qc_shifts(J, L, p, seed=seed, zero_blocks=zero_blocks)
    h = pkg.ldpc_code_create(shifts, p)
    try:
        k, pos = pkg.ldpc_code_info_set(h)
    finally:
        pkg.ldpc_code_destroy(h)
    enc = oracle.Encoder(sp.csr_matrix(oracle.qc_parity_check(shifts, p)), track=False)
    assert k == enc.k >= L * p - J * p
    assert np.array_equal(pos, enc.info)


def test_codeword_options_validated(lib):
    import paper_1204_0334_gb300 as pkg

    pkg.lib()
    o = pkg.default_opts()
    assert o.codewords == pkg.CODEWORDS_ZERO and list(o.reserved) == [0, 0, 0]
    h = pkg.ldpc_code_create(np.array([[0, 1, 2, 3], [1, 3, 0, 2]]), 8)
    try:
        for bad in (dict(codewords=2), dict(codewords=-1)):
            with pytest.raises(pkg.LdpcError) as e:
                pkg.ldpc_ber_sim(h, 2.0, 1, 0, 64, 10, 64, pkg.default_opts(**bad), stream=0)
            assert e.value.status == 1 and "codewords" in str(e.value)
    finally:
        pkg.ldpc_code_destroy(h)


def test_encoder_calls_reject_bad_arguments_without_a_device(lib):
    """The encoder entry points refuse null handles, empty batches and a non-finite Eb/N0 before any device
    memory is touched."""
    import paper_1204_0334_gb300 as pkg

    L = pkg.lib()
    k = ctypes.c_int64()
    assert L.ldpc_code_info_set(None, ctypes.byref(k), None) == 1
    dummy = ctypes.c_void_p(16)
    assert L.ldpc_encode(None, dummy, 4, dummy, None) == 1
    assert L.ldpc_random_codewords(None, 1, 0, 4, None, dummy, None) == 1
    h = pkg.ldpc_code_create(np.array([[0, 1, 2, 3], [1, 3, 0, 2]]), 8)
    try:
        assert L.ldpc_encode(h, dummy, 0, dummy, None) == 1          # gamma < 1
        assert L.ldpc_encode(h, dummy, 4, None, None) == 1           # no output
        assert L.ldpc_random_codewords(h, 1, 0, 0, None, dummy, None) == 1
        assert L.ldpc_channel_codewords(h, float("nan"), 1, 0, 4, dummy, dummy, None) == 1
        assert L.ldpc_channel_codewords(h, 2.0, 1, 0, 4, None, dummy, None) == 1
        assert L.ldpccc_create_tanner(None, 3, 6, 8, 2, 4, ctypes.byref(ctypes.c_void_p())) == 1
    finally:
        pkg.ldpc_code_destroy(h)


def test_bench_reference_arm_line(lib):
    """bench.py --impl reference times the FP64 oracle on the host cores and prints one JSON line with the
    contract's keys (a short run: one step of a small sample)."""
    import json
    import subprocess
    import sys

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
