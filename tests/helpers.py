"""Test-side helpers: fixture parsing, GF(2) codeword enumeration and brute force.

Nothing here is shared with the CUDA path; brute force is the independent
pin for the oracle's belief propagation (exact marginals on cycle-free graphs).
"""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# parity figures of the GPU tests, printed in the pytest summary (conftest.py)
PARITY_RECORDS: list = []


def record_parity(label: str, **figures):
    """Keep one comparison's figures: frames, elements, frames/elements that needed the
    conditioning arm of the FP32 tolerance, largest relative deviation."""
    PARITY_RECORDS.append(dict(label=label, **figures))


def read_sections(name: str) -> dict:
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                out[cur] = []
                continue
            out.setdefault(cur, []).append([int(x) if x.lstrip("-").isdigit() else x for x in line.split()])
    return out


def codewords(H: np.ndarray) -> np.ndarray:
    """All c with H c = 0 over GF(2): every combination of a null-space basis (dimension <= 20)."""
    B = gf2_nullspace(H).astype(np.int64)
    k = B.shape[0]
    assert k <= 20
    coeff = np.array(list(itertools.product([0, 1], repeat=k)), dtype=np.int64).reshape(-1, k)
    C = (coeff @ B) % 2
    assert not ((C @ np.asarray(H, dtype=np.int64).T) % 2).any()
    return C


def codewords_exhaustive(H: np.ndarray) -> np.ndarray:
    """All c with H c = 0 by enumerating all 2^N words (N <= 16); checks ``codewords``."""
    H = np.asarray(H, dtype=np.int64)
    N = H.shape[1]
    assert N <= 16
    words = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.int64)
    return words[((words @ H.T) % 2 == 0).all(axis=1)]


def brute_force_llr(H: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Exact a-posteriori LLRs: P(c | y) ~ exp(sum_k mu_k x_k / 2), x = 1 - 2c."""
    C = codewords(H)
    X = 1 - 2 * C
    s = (X @ np.asarray(mu, dtype=np.float64)) / 2.0
    out = np.zeros(H.shape[1])
    for n in range(H.shape[1]):
        a = s[C[:, n] == 0]
        b = s[C[:, n] == 1]
        la = a.max() + np.log(np.exp(a - a.max()).sum())
        lb = b.max() + np.log(np.exp(b - b.max()).sum())
        out[n] = la - lb
    return out


def brute_force_maxlog(H: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Max-log a-posteriori values: (max_{c_n=0} sum q x - max_{c_n=1} sum q x) / 2."""
    C = codewords(H)
    X = 1 - 2 * C
    s = X @ np.asarray(q, dtype=np.int64)
    out = np.zeros(H.shape[1], dtype=np.int64)
    for n in range(H.shape[1]):
        d = s[C[:, n] == 0].max() - s[C[:, n] == 1].max()
        assert d % 2 == 0
        out[n] = d // 2
    return out


def gf2_nullspace(H: np.ndarray) -> np.ndarray:
    """Basis of {c : H c = 0} over GF(2) by Gaussian elimination (rows of the result)."""
    A = np.array(H, dtype=np.uint8) % 2
    M, N = A.shape
    pivots = []
    r = 0
    for c in range(N):
        rows = np.nonzero(A[r:, c])[0]
        if len(rows) == 0:
            continue
        pr = r + rows[0]
        A[[r, pr]] = A[[pr, r]]
        for rr in range(M):
            if rr != r and A[rr, c]:
                A[rr] ^= A[r]
        pivots.append(c)
        r += 1
        if r == M:
            break
    free = [c for c in range(N) if c not in pivots]
    basis = []
    for f in free:
        v = np.zeros(N, dtype=np.uint8)
        v[f] = 1
        for i, pc in enumerate(pivots):
            v[pc] = A[i, f]
        basis.append(v)
    return np.array(basis, dtype=np.uint8)


def random_codeword(H: np.ndarray, seed: int) -> np.ndarray:
    B = gf2_nullspace(H)
    rng = np.random.default_rng(seed)
    coeff = rng.integers(0, 2, size=B.shape[0]).astype(np.uint8)
    return (coeff @ B) % 2


def syndrome(H: np.ndarray, c: np.ndarray) -> np.ndarray:
    return (np.asarray(H, dtype=np.int64) @ np.asarray(c, dtype=np.int64).T) % 2


# Cycle-free Tanner graphs written as base matrices of shifts (-1 = zero block),
# so that they can be lifted with any circulant size p (a lifted tree is a forest).
TREE_BASES = {
    "path3": [[0, 0, 0, -1, -1, -1, -1], [-1, -1, 0, 0, 0, -1, -1], [-1, -1, -1, -1, 0, 0, 0]],
    "star": [[0, 0, 0, -1, -1, -1, -1], [0, -1, -1, 0, 0, -1, -1], [0, -1, -1, -1, -1, 0, 0]],
    "deg4": [[0, 0, 0, 0, -1, -1, -1, -1, -1], [-1, -1, -1, 0, 0, 0, -1, -1, -1],
             [-1, 0, -1, -1, -1, -1, 0, 0, 0]],
    "spc6": [[0, 0, 0, 0, 0, 0]],
    "rep5": [[0, 0, -1, -1, -1], [-1, 0, 0, -1, -1], [-1, -1, 0, 0, -1], [-1, -1, -1, 0, 0]],
}
