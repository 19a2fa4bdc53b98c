"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws inputs only; it holds none of the decoders' arithmetic and
imports neither the oracle nor the CUDA package.

* ``qc_shifts``      -- a J x L matrix of circulant shifts, uniform in [0, p),
  drawn entry by entry so that no 4-cycle is formed where one can be avoided
  (a_{j1,l1} - a_{j1,l2} + a_{j2,l2} - a_{j2,l1} != 0 mod p).  The paper does
  not print the shifts of its codes A-D; seeded matrices of the same J, L, p
  stand in for them.
* ``gaussian_llrs``  -- frames of channel LLRs distributed as the BPSK/AWGN
  channel delivers them for the all-zero codeword (the consistent Gaussian
  N(m, 2m) with m = 4 R Eb/N0), drawn with numpy's PCG64.
* ``frame_counts``   -- log-uniform frame counts for mixed batches.
* ``mixed_codes``    -- the 64-code heterogeneous batch recipe.
"""
from __future__ import annotations

import math

import numpy as np


def qc_shifts(J: int, L: int, p: int, seed: int, zero_blocks: int = 0, avoid_4cycles: bool = True) -> np.ndarray:
    """Seeded shift matrix; ``zero_blocks`` entries are set to -1 (zero circulant)."""
    rng = np.random.default_rng([seed, J, L, p, 0x51F7])
    a = -np.ones((J, L), dtype=np.int32)
    for j in range(J):
        for l in range(L):
            best = int(rng.integers(0, p))
            if avoid_4cycles:
                for _ in range(64):
                    bad = False
                    for j2 in range(j):
                        for l2 in range(L):
                            if l2 == l or a[j2, l2] < 0 or a[j, l2] < 0 or a[j2, l] < 0:
                                continue
                            if (best - a[j, l2] + a[j2, l2] - a[j2, l]) % p == 0:
                                bad = True
                                break
                        if bad:
                            break
                    if not bad:
                        break
                    best = int(rng.integers(0, p))
            a[j, l] = best
    if zero_blocks:
        flat = rng.choice(J * L, size=zero_blocks, replace=False)
        for f in flat:
            a[f // L, f % L] = -1
        # keep every block column connected to at least one check
        for l in range(L):
            if np.all(a[:, l] < 0):
                a[int(rng.integers(0, J)), l] = int(rng.integers(0, p))
    return a


def ebn0_llr_mean(ebn0_db: float, rate: float) -> float:
    """Mean of the channel LLR for the all-zero codeword (unit-energy BPSK)."""
    return 4.0 * rate * 10.0 ** (ebn0_db / 10.0)


def gaussian_llrs(nfr: int, N: int, seed: int, ebn0_db: float, rate: float) -> np.ndarray:
    """float32 [nfr][N] LLRs, i.i.d. N(m, 2m), m = 4 R 10^(EbN0/10)."""
    m = ebn0_llr_mean(ebn0_db, rate)
    rng = np.random.default_rng([seed, nfr, N, 0xA3C5])
    return (m + math.sqrt(2.0 * m) * rng.standard_normal((nfr, N))).astype(np.float32)


def integer_llrs(nfr: int, N: int, seed: int, lo: int = -20, hi: int = 20, scale: float = 0.25) -> np.ndarray:
    """float32 LLRs on a coarse grid (many exact ties and zeros)."""
    rng = np.random.default_rng([seed, nfr, N, 0x7E5])
    return (rng.integers(lo, hi + 1, size=(nfr, N)) * scale).astype(np.float32)


def frame_counts(ncodes: int, seed: int, max_frames: int = 4096) -> np.ndarray:
    """floor(exp(U[0, ln max_frames])) in [1, max_frames]."""
    rng = np.random.default_rng([seed, ncodes, 0xF00D])
    return np.floor(np.exp(rng.uniform(0.0, math.log(max_frames), size=ncodes))).astype(np.int64).clip(1, max_frames)


def mixed_codes(ncodes: int, seed: int, p_min: int = 32, p_max: int = 765, n_min: int = 192, n_max: int = 18360):
    """(J, L, p, shifts) of a heterogeneous batch: rates 1/2..5/6, p log-uniform."""
    rng = np.random.default_rng([seed, ncodes, 0xC0DE])
    shapes = [(3, 6), (4, 8), (3, 9), (4, 12), (3, 12), (4, 16), (3, 18), (4, 24)]
    out = []
    for i in range(ncodes):
        J, L = shapes[int(rng.integers(0, len(shapes)))]
        p = int(math.floor(math.exp(rng.uniform(math.log(p_min), math.log(p_max)))))
        p = max(p_min, min(p, p_max))
        p = max(min(p, n_max // L), -(-n_min // L))
        out.append((J, L, p, qc_shifts(J, L, p, seed * 1000 + i)))
    return out


def random_ldpc(N: int, M: int, seed: int, var_degrees=(2, 3, 3, 4, 6), max_row: int = 32):
    """A random irregular LDPC code (inputs only): variable degrees drawn from var_degrees, edges
    matched to checks by the configuration model with check degrees as equal as possible, repeated
    edges and over-full rows redrawn.  Returns (row_ptr [M+1], col_idx [E]) of H in compressed-row
    form, columns increasing within each row; every check gets at least two variables."""
    rng = np.random.default_rng(seed)
    dv = rng.choice(np.asarray(var_degrees), size=N)
    for _ in range(100):
        rows = [set() for _ in range(M)]
        ok = True
        order = rng.permutation(N)
        for n in order:
            # the least-loaded checks first, random among equals
            load = np.array([len(r) for r in rows]) + rng.random(M)
            for m in np.argsort(load)[: int(dv[n])]:
                if len(rows[m]) >= max_row:
                    ok = False
                    break
                rows[m].add(int(n))
            if not ok:
                break
        if ok and all(len(r) >= 2 for r in rows):
            break
    row_ptr = np.zeros(M + 1, dtype=np.int32)
    cols = []
    for m, r in enumerate(rows):
        c = sorted(r)
        cols += c
        row_ptr[m + 1] = row_ptr[m] + len(c)
    return row_ptr, np.asarray(cols, dtype=np.int32)
