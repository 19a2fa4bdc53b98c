"""Plain CPU oracle for the BP decoders of Zhao & Lau (arXiv 1204.0334).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path in ``paper_1204_0334_gb300``; neither imports the other.

The arithmetic lives in ``oracle.c`` (double precision, one frame at a time,
the steps of Algorithm 1 / Algorithm 2 in the paper's order).  This module
holds the definitional pieces that are plain matrix constructions:

* ``qc_parity_check``  -- H of a QC-LDPC code, eq. (qcH): block (j, l) is the
  p x p identity with its columns shifted cyclically right a_jl times
  (row r has its one in column (r + a_jl) mod p); a_jl = -1 is the zero block
  (Sec. IV-B-1 footnote on shift numbers).
* ``csr_rows``         -- the edge order of the message store H: row by row,
  left to right (Sec. IV-A).
* ``ldpccc_unwrap``    -- H of the LDPC convolutional code derived from a QC
  base by the three steps of Sec. II-D (partition into Lambda x Lambda
  sub-blocks, split into lower / strictly-upper parts, unwrap and repeat).
* ``ldpccc_tanner``    -- H of the time-invariant LDPCCC with delays D^{a_jl}
  (the other unwrapping Sec. II-D cites): check j at instant t meets bit l at
  instant t - a_jl.
* ``Encoder``          -- the systematic encoder of the transmitted codewords
  (Sec. V): information set = complement of the greedy right-to-left column
  basis of H, codeword = the unique null-space word with those bits.
* ``info_bits``        -- the information bits a frame id draws from Philox.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None


_LIB32_PATH = os.path.join(_HERE, "_oracle_f32.so")
_lib32 = None


def build(force: bool = False) -> str:
    """Compile oracle.c into shared libraries next to it (gcc, OpenMP): the FP64 oracle, and
    the same source with the sum-product / LDPCCC real type set to binary32 (a diagnostic)."""
    for path, extra in ((_LIB_PATH, []), (_LIB32_PATH, ["-DOR_REAL_FLOAT"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC"] + extra + [_SRC, "-o", tmp,
                                                                                                 "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, path)
    return _LIB_PATH


def _declare(lib):
    P = ctypes.c_void_p
    i32, u32, u64, f64 = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
    lib.or_philox4x32_10.argtypes = [P, P, P]
    lib.or_philox4x32_10.restype = None
    lib.or_channel_awgn.argtypes = [u64, u64, i32, i32, f64, u32, P, P]
    lib.or_channel_awgn.restype = None
    lib.or_channel_awgn_cw.argtypes = [u64, u64, i32, i32, f64, u32, P, P, P]
    lib.or_channel_awgn_cw.restype = None
    lib.or_ln_f32_array.argtypes = [P, P, ctypes.c_int64]
    lib.or_ln_f32_array.restype = None
    lib.or_sincos2pi_f32_array.argtypes = [P, P, P, ctypes.c_int64]
    lib.or_sincos2pi_f32_array.restype = None
    lib.or_variable_edges.argtypes = [i32, i32, P, P, P, P]
    lib.or_sp_decode.argtypes = [i32, i32, P, P, i32, P, i32, i32, f64, i32, P, P, P, P, i32]
    lib.or_ms_decode.argtypes = [i32, i32, P, P, i32, P, i32, i32, i32, P, P, P, P, i32]
    lib.or_quantize.argtypes = [P, i32, i32, P]
    lib.or_noms.argtypes = [i32, i32, P, P, P, i32, P, i32, P, i32, f64, P, P, i32, i32]
    lib.or_round_half_array.argtypes = [P, P, ctypes.c_int64]
    lib.or_round_half_array.restype = None
    lib.or_noms.restype = f64
    lib.or_ldpccc_decode.argtypes = [i32, i32, P, P, i32, i32, i32, i32, i32, i32, P, f64, P, P, P,
                                     P, i32, P, i32]
    return lib


def _load(real: int = 64):
    """The FP64 oracle (real = 64), or the binary32 diagnostic build (real = 32)."""
    global _lib, _lib32
    if real == 32:
        if _lib32 is None:
            build()
            _lib32 = _declare(ctypes.CDLL(_LIB32_PATH))
        return _lib32
    if _lib is None:
        build()
        _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Code construction (Sec. II-A, eq. qcH) and the edge order (Sec. IV-A)
# --------------------------------------------------------------------------
def circulant(a: int, p: int) -> np.ndarray:
    """P^a: the p x p identity with its columns shifted cyclically right a times.

    Row r holds its one in column (r + a) mod p.  a = -1 gives the zero matrix.
    """
    P = np.zeros((p, p), dtype=np.uint8)
    if a >= 0:
        for r in range(p):
            P[r, (r + a) % p] = 1
    return P


def qc_parity_check(shifts, p: int) -> np.ndarray:
    """Dense H = [P^{a_jl}] of a (J, L) QC-LDPC code, eq. (qcH)."""
    shifts = np.asarray(shifts, dtype=np.int64)
    J, L = shifts.shape
    return np.block([[circulant(int(shifts[j, l]), p) for l in range(L)] for j in range(J)])


def csr_rows(H) -> tuple[np.ndarray, np.ndarray]:
    """Edges of H row by row, left to right: (row_ptr[M+1], col[E]) as int32."""
    import scipy.sparse as sp

    Hc = sp.csr_matrix(H)
    Hc.sort_indices()
    return Hc.indptr.astype(np.int32), Hc.indices.astype(np.int32)


def variable_edges(row_ptr, col, N: int):
    """LUT_v of Sec. IV-A: for each variable, its edge indices (ascending)."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    M = len(row_ptr) - 1
    vptr = np.zeros(N + 1, dtype=np.int32)
    vedge = np.zeros(max(int(row_ptr[-1]), 1), dtype=np.int32)
    if lib.or_variable_edges(M, N, _p(row_ptr), _p(col), _p(vptr), _p(vedge)) != 0:
        raise RuntimeError("or_variable_edges failed")
    return vptr, vedge[: int(row_ptr[-1])]


def design_rate(shifts) -> float:
    """R = 1 - M/N counted over the non-zero block structure (the bound of Sec. II-A)."""
    shifts = np.asarray(shifts)
    J, L = shifts.shape
    return 1.0 - J / L


def sigma_from_ebn0(ebn0_db: float, rate: float) -> float:
    """Noise std for unit-energy BPSK: Es = 1, Eb = Es / R, sigma^2 = N0/2."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


# --------------------------------------------------------------------------
# LDPC convolutional code derived from a QC base (Sec. II-D)
# --------------------------------------------------------------------------
def ldpccc_geometry(J: int, L: int, p: int) -> dict:
    lam = math.gcd(J, L)
    return {"Lambda": lam, "ms": lam - 1, "c": (L // lam) * p, "cb": (J // lam) * p, "b": ((L - J) // lam) * p}


def ldpccc_unwrap(shifts, p: int, T: int):
    """H_[0,T) of the derived LDPCCC as a sparse CSR matrix (T*cb x T*c).

    Step 1: partition H_QC into Lambda x Lambda sub-blocks H_{i,j}.
    Step 2: H^L keeps the sub-blocks on and below the diagonal, H^U the ones
            strictly above it.
    Step 3: paste H^U below H^L (H_base = [H^L; H^U]) and repeat H_base down
            the diagonal, one copy every Lambda sub-block rows / columns.
    The result is cut to the first T check layers and T frames.
    """
    import scipy.sparse as sp

    shifts = np.asarray(shifts, dtype=np.int64)
    J, L = shifts.shape
    geo = ldpccc_geometry(J, L, p)
    lam, c, cb = geo["Lambda"], geo["c"], geo["cb"]
    H = sp.csr_matrix(qc_parity_check(shifts, p))
    # step 1
    sub = [[H[i * cb:(i + 1) * cb, j * c:(j + 1) * c] for j in range(lam)] for i in range(lam)]
    zero = sp.csr_matrix((cb, c), dtype=np.uint8)
    # step 2
    HL = sp.bmat([[sub[i][j] if j <= i else zero for j in range(lam)] for i in range(lam)], format="csr")
    HU = sp.bmat([[sub[i][j] if j > i else zero for j in range(lam)] for i in range(lam)], format="csr")
    # step 3
    Hbase = sp.vstack([HL, HU], format="coo")
    rows, cols = [], []
    copies = (T + lam - 1) // lam + 1
    for k in range(copies):
        r = Hbase.row + k * lam * cb
        cc = Hbase.col + k * lam * c
        keep = (r < T * cb) & (cc < T * c)
        rows.append(r[keep])
        cols.append(cc[keep])
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    Hc = sp.csr_matrix((np.ones(len(rows), dtype=np.uint8), (rows, cols)), shape=(T * cb, T * c))
    Hc.sort_indices()
    return Hc, geo


# --------------------------------------------------------------------------
# Generator and channel (Sec. II-B)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def ln_f32(u) -> np.ndarray:
    """The channel generator's binary32 natural logarithm of positive normal binary32 values."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float32)
    out = np.empty_like(u)
    lib.or_ln_f32_array(_p(u), _p(out), u.size)
    return out


def sincos2pi_f32(v) -> tuple[np.ndarray, np.ndarray]:
    """The channel generator's binary32 (sin, cos) of 2 pi v 2^-24 for odd v in (0, 2^24)."""
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.uint32)
    s = np.empty(v.shape, dtype=np.float32)
    c = np.empty(v.shape, dtype=np.float32)
    lib.or_sincos2pi_f32_array(_p(v), _p(s), _p(c), v.size)
    return s, c


def channel_awgn(seed: int, first_frame: int, nfr: int, N: int, sigma: float, tag: int = 0,
                 return_g: bool = False, cw=None):
    """mu[nfr][N] (float32) over BPSK/AWGN: the all-zero codeword, or cw[nfr][N] (0/1) when given."""
    lib = _load()
    mu = np.zeros((nfr, N), dtype=np.float32)
    g = np.zeros((nfr, N), dtype=np.float64) if return_g else None
    if cw is None:
        lib.or_channel_awgn(seed, first_frame, nfr, N, sigma, tag, _p(mu), _p(g) if return_g else None)
    else:
        c = np.ascontiguousarray(cw, dtype=np.uint8)
        assert c.shape == (nfr, N)
        lib.or_channel_awgn_cw(seed, first_frame, nfr, N, sigma, tag, _p(c), _p(mu), _p(g) if return_g else None)
    return (mu, g) if return_g else mu


# --------------------------------------------------------------------------
# Systematic encoding (the transmitted codewords of Sec. V)
# --------------------------------------------------------------------------
def _columns_as_ints(H) -> tuple[list[int], int, int]:
    """Column n of H as the integer sum over rows m with H[m, n] = 1 of 2^m."""
    import scipy.sparse as sp

    Hc = sp.csc_matrix(H)
    Hc.sort_indices()
    M, N = Hc.shape
    cols = []
    for n in range(N):
        v = 0
        for m, val in zip(Hc.indices[Hc.indptr[n]:Hc.indptr[n + 1]], Hc.data[Hc.indptr[n]:Hc.indptr[n + 1]]):
            if int(val) & 1:
                v ^= 1 << int(m)
        cols.append(v)
    return cols, M, N


class Encoder:
    """Systematic encoder of the code {c : H c = 0 over GF(2)}.

    Information set (a definition, not a search heuristic): scanning columns
    from n = N - 1 down to 0, column n is a PARITY position when it is not in
    the GF(2) span of the columns to its right, and an INFORMATION position
    otherwise.  The parity columns form a basis of H's column space, so
    k = N - rank(H) and, for every u in {0,1}^k, exactly one codeword c has
    c[info[j]] = u[j] (info in increasing order).

    Built by inserting the columns, right to left, into a GF(2) basis kept by
    leading row bit; each basis vector remembers which parity columns it is
    the sum of (only with ``track`` = True: needed to encode, not for the
    information set).
    """

    def __init__(self, H, track: bool = True):
        self.cols, self.M, self.N = _columns_as_ints(H)
        self.track = track
        self.basis: dict[int, tuple[int, int]] = {}
        parity = []
        for n in range(self.N - 1, -1, -1):
            v, comb = self.cols[n], (1 << n) if track else 0
            while v:
                lead = v.bit_length() - 1
                if lead not in self.basis:
                    break
                bv, bc = self.basis[lead]
                v ^= bv
                comb ^= bc
            if v:
                self.basis[v.bit_length() - 1] = (v, comb)
                parity.append(n)
        self.parity = np.array(sorted(parity), dtype=np.int64)
        is_par = np.zeros(self.N, dtype=bool)
        is_par[self.parity] = True
        self.info = np.nonzero(~is_par)[0].astype(np.int64)
        self.k = len(self.info)
        self.rank = len(self.parity)

    def encode(self, u) -> np.ndarray:
        """c[nfr][N] (uint8) for information bits u[nfr][k]: c[info] = u and H c = 0."""
        assert self.track, "built with track=False"
        u = np.atleast_2d(np.asarray(u, dtype=np.uint8))
        out = np.zeros((u.shape[0], self.N), dtype=np.uint8)
        for f in range(u.shape[0]):
            s = 0  # syndrome of the information part
            for j in np.nonzero(u[f] & 1)[0]:
                s ^= self.cols[int(self.info[j])]
            # s lies in the span of the parity columns: express it in the basis
            comb = 0
            while s:
                bv, bc = self.basis[s.bit_length() - 1]
                s ^= bv
                comb ^= bc
            out[f, self.info] = u[f] & 1
            n = 0
            while comb:
                if comb & 1:
                    out[f, n] = 1
                comb >>= 1
                n += 1
        return out


def info_bits(seed: int, first_frame: int, nfr: int, k: int) -> np.ndarray:
    """u[nfr][k] (uint8): information bit j of frame F is bit j mod 32 of word
    (j / 32) mod 4 of Philox4x32-10 at counter (j / 128, F_lo, F_hi, 1) under key
    (seed_lo, seed_hi) -- the channel's counters carry 0 in the last word."""
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    u = np.zeros((nfr, k), dtype=np.uint8)
    for f in range(nfr):
        F = first_frame + f
        for q in range((k + 127) // 128):
            w = philox4x32_10([q, F & 0xFFFFFFFF, (F >> 32) & 0xFFFFFFFF, 1], key)
            # bit j of the 128 = bit j mod 32 of word j / 32 (little-endian bytes, LSB first)
            bits = np.unpackbits(w.astype("<u4").view(np.uint8), bitorder="little")
            n = min(k, 128 * q + 128) - 128 * q
            u[f, 128 * q:128 * q + n] = bits[:n]
    return u


# --------------------------------------------------------------------------
# Decoders
# --------------------------------------------------------------------------
def sp_decode(row_ptr, col, N: int, mu, max_iter: int, early_stop: bool = False, clip: float = 30.0,
              form: str = "phi", nthreads: int = 1, real: int = 64):
    """Sum-product BP, Algorithm 1, double precision (real = 32: the same steps in binary32,
    a diagnostic of FP32 rounding, not a reference).

    Returns (post[nfr][N] float64, hard[nfr][N] uint8, iters[nfr], ok[nfr]).
    """
    lib = _load(real)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    if mu.ndim == 1:
        mu = mu[None, :]
    nfr = mu.shape[0]
    M = len(row_ptr) - 1
    post = np.zeros((nfr, N), dtype=np.float64)
    hard = np.zeros((nfr, N), dtype=np.uint8)
    iters = np.zeros(nfr, dtype=np.int32)
    ok = np.zeros(nfr, dtype=np.int32)
    f = {"phi": 0, "tanh": 1}[form]
    rc = lib.or_sp_decode(M, N, _p(row_ptr), _p(col), nfr, _p(mu), max_iter, int(early_stop), clip, f,
                          _p(post), _p(hard), _p(iters), _p(ok), nthreads)
    if rc != 0:
        raise ValueError("or_sp_decode rejected its arguments")
    return post, hard, iters, ok


def quantize(mu, frac_bits: int = 2) -> np.ndarray:
    lib = _load()
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    q = np.zeros(mu.shape, dtype=np.int8)
    lib.or_quantize(_p(mu), mu.size, frac_bits, _p(q))
    return q


def ms_decode(row_ptr, col, N: int, mu, max_iter: int, early_stop: bool = False, frac_bits: int = 2,
              nthreads: int = 1):
    """Integer min-sum.  Returns (post int32, hard uint8, iters, ok)."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    if mu.ndim == 1:
        mu = mu[None, :]
    nfr = mu.shape[0]
    M = len(row_ptr) - 1
    post = np.zeros((nfr, N), dtype=np.int32)
    hard = np.zeros((nfr, N), dtype=np.uint8)
    iters = np.zeros(nfr, dtype=np.int32)
    ok = np.zeros(nfr, dtype=np.int32)
    rc = lib.or_ms_decode(M, N, _p(row_ptr), _p(col), nfr, _p(mu), frac_bits, max_iter, int(early_stop),
                          _p(post), _p(hard), _p(iters), _p(ok), nthreads)
    if rc != 0:
        raise ValueError("or_ms_decode rejected its arguments")
    return post, hard, iters, ok


def ldpccc_decode(Hconv, geo: dict, T: int, I: int, mu, clip: float = 30.0, nthreads: int = 1,
                  log_cap: int = 0, real: int = 64):
    """Pipelined BP of Algorithm 2 over T slots (real = 32: the binary32 diagnostic build).

    mu is [nstreams][T*c] (or [T*c]).  Returns (post, hard, decided[nstreams][T], log) where
    post/hard are [nstreams][T*c]; frames F <= T - I*(ms+1) are decided.
    """
    lib = _load(real)
    row_ptr = np.ascontiguousarray(Hconv.indptr, dtype=np.int32)
    col = np.ascontiguousarray(Hconv.indices, dtype=np.int32)
    c, cb, ms = geo["c"], geo["cb"], geo["ms"]
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    if mu.ndim == 1:
        mu = mu[None, :]
    ns = mu.shape[0]
    N = T * c
    M = T * cb
    post = np.zeros((ns, N), dtype=np.float64)
    hard = np.zeros((ns, N), dtype=np.uint8)
    decided = np.zeros((ns, T), dtype=np.uint8)
    log = np.zeros((max(log_cap, 1), 4), dtype=np.int32)
    log_n = np.zeros(1, dtype=np.int32)
    rc = lib.or_ldpccc_decode(M, N, _p(row_ptr), _p(col), T, c, cb, ms, I, ns, _p(mu), clip, _p(post),
                              _p(hard), _p(decided), _p(log) if log_cap else None, log_cap, _p(log_n), nthreads)
    if rc < 0:
        raise ValueError("or_ldpccc_decode rejected its arguments")
    return post, hard, decided, log[: min(int(log_n[0]), log_cap)]


def ldpccc_tanner_geometry(shifts, p: int) -> dict:
    """Frames of p time instants: c = L p bits, J p checks per layer, memory 1 frame (0 if
    every delay is 0); "delay" is the largest shift, the code's memory in time instants."""
    shifts = np.asarray(shifts, dtype=np.int64)
    J, L = shifts.shape
    amax = int(shifts.max()) if (shifts >= 0).any() else 0
    return {"Lambda": 1, "ms": 1 if amax > 0 else 0, "c": L * p, "cb": J * p, "b": (L - J) * p, "delay": amax}


def ldpccc_tanner(shifts, p: int, T: int):
    """H_[0,T) of the time-invariant LDPCCC whose polynomial parity-check matrix has entries
    D^{a_jl} (a_jl = -1: no entry): check j at time instant t involves bit l at instant t - a_jl,
    instants before 0 do not exist.  Instant t = F p + tau belongs to frame F; bit (l, tau) of
    frame F is column F c + l p + tau, check (j, tau) of layer F is row F cb + j p + tau.
    """
    import scipy.sparse as sp

    shifts = np.asarray(shifts, dtype=np.int64)
    J, L = shifts.shape
    geo = ldpccc_tanner_geometry(shifts, p)
    c, cb = geo["c"], geo["cb"]
    rows, cols = [], []
    for j in range(J):
        for l in range(L):
            a = int(shifts[j, l])
            if a < 0:
                continue
            t = np.arange(T * p, dtype=np.int64)  # check instants
            tb = t - a                             # bit instants
            keep = tb >= 0
            t, tb = t[keep], tb[keep]
            rows.append((t // p) * cb + j * p + t % p)
            cols.append((tb // p) * c + l * p + tb % p)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    Hc = sp.csr_matrix((np.ones(len(rows), dtype=np.uint8), (rows, cols)), shape=(T * cb, T * c))
    Hc.sort_indices()
    return Hc, geo


def circulant_index(row_ptr, col, p: int, L: int) -> np.ndarray:
    """Circulant block j*L + l of every edge of a QC code (row m = j*p + r, column n = l*p + k)."""
    row_ptr = np.asarray(row_ptr)
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return ((rows // p) * L + (np.asarray(col) // p)).astype(np.int32)


def round_half(x) -> np.ndarray:
    """x rounded to the nearest binary16 value (ties to even), as float64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib.or_round_half_array(_p(x), _p(out), x.size)
    return out


def noms(row_ptr, col, cblk, N: int, mu, T: int, params, clip: float = 30.0, want_grad: bool = False,
         nthreads: int = 1, store16: bool = False):
    """Normalized/offset min-sum over T iterations with params [T][ncirc][2] = (w, o).

    Returns (loss, post^(T) [nfr][N], grad [T][ncirc][2] or None); loss is the mean over
    iterations, bits and frames of softplus(-posterior) (BCE against the all-zero codeword).
    store16: the FP16-message variant (the stored alpha and beta rounded to binary16); its forward
    runs in binary32 like the device's, so that each rounding and each arg-min is decided on the same
    value.
    """
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    cblk = np.ascontiguousarray(cblk, dtype=np.int32)
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    if mu.ndim == 1:
        mu = mu[None, :]
    params = np.ascontiguousarray(params, dtype=np.float64)
    assert params.shape[0] == T and params.shape[2] == 2
    ncirc = params.shape[1]
    nfr = mu.shape[0]
    post = np.zeros((nfr, N), dtype=np.float64)
    grad = np.zeros_like(params) if want_grad else None
    loss = lib.or_noms(len(row_ptr) - 1, N, _p(row_ptr), _p(col), _p(cblk), nfr, _p(mu), T, _p(params), ncirc,
                       clip, _p(post), _p(grad) if want_grad else None, nthreads, int(store16))
    return loss, post, grad
