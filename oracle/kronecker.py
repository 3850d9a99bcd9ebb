"""The paper's Kronecker-product factorisation (Eq. 1) and its Table 1 operators.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 1 (Section 3) writes the general-radix decimation-in-time DFT of size
N = M*K as

    DFT_N = (DFT_K (x) I_M) . D^N_M . (I_K (x) DFT_M) . Pi^N_K .

The paper does not spell out Pi^N_K or the entries of D^N_M, and its Table 1
has typos. The readings taken here (each pinned by the dense-matrix test in
tests/test_oracle_kronecker.py):

* Pi^N_K gathers the K stride-K subsequences into contiguous blocks:
  y[b*M + t] = x[t*K + b] (b < K, t < M). In Table 1's notation this is
  Permute(M, N) (Y[i + M*j] = X[K*i + j]); the literal Permute(K, N) does not
  satisfy Eq. 1 whenever K != M.
* D^N_M is block diagonal: block b (< K), position t (< M) holds w_N^(b*t),
  w_N = exp(-2 pi i / N) for the forward transform.
* Table 1 "Mul" multiplies every entry (its printed bound i < m is a typo for
  the full length), "Permute" is a pure copy (the printed A* is a typo) and
  FusedPKIV moves whole k-element blocks.
* Slices in Table 1 are start:step:end with an inclusive end.
"""
from __future__ import annotations

import numpy as np


def omega(N: int, e, sign: int = -1):
    """w_N^e = exp(sign * 2 pi i e / N) with the exponent reduced exactly mod N."""
    e = np.asarray(e, dtype=np.int64) % N
    ang = 2.0 * np.pi * (e.astype(np.float64) / N)
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    """Dense DFT_n: entry (k, j) = w_n^(j*k)."""
    j = np.arange(n, dtype=np.int64)
    return omega(n, np.outer(j, j), sign)


# ---- Table 1 operators, as loops over the printed index sets --------------

def fused_mkiv(A: np.ndarray, n: int, X: np.ndarray) -> np.ndarray:
    """Y = (A_m (x) I_n) X: for i < n, Y[i : n : i+m*n-n] = A . X[same]."""
    m = A.shape[0]
    Y = np.empty(m * n, dtype=np.complex128)
    for i in range(n):
        idx = np.arange(i, i + m * n - n + 1, n)  # inclusive end
        Y[idx] = A @ X[idx]
    return Y


def fused_ikmv(A: np.ndarray, m: int, X: np.ndarray) -> np.ndarray:
    """Y = (I_m (x) A_n) X: for i < m, Y[i*n : 1 : i*n+n-1] = A . X[same]."""
    n = A.shape[0]
    Y = np.empty(m * n, dtype=np.complex128)
    for i in range(m):
        idx = np.arange(i * n, i * n + n - 1 + 1)  # inclusive end
        Y[idx] = A @ X[idx]
    return Y


def permute(m: int, mn: int, X: np.ndarray) -> np.ndarray:
    """Table 1 Permute(m, mn): Y[i + m*j] = X[n*i + j] for i < m, j < n (n = mn/m)."""
    n = mn // m
    Y = np.empty(mn, dtype=np.complex128)
    for i in range(m):
        for j in range(n):
            Y[i + m * j] = X[n * i + j]
    return Y


def fused_pkiv(m: int, mn: int, k: int, X: np.ndarray) -> np.ndarray:
    """(Pi^{mn}_m (x) I_k) X: k-element block n*i+j moves to block i+m*j."""
    n = mn // m
    Y = np.empty(mn * k, dtype=np.complex128)
    for i in range(m):
        for j in range(n):
            Y[k * (i + m * j): k * (i + m * j) + k] = X[k * (n * i + j): k * (n * i + j) + k]
    return Y


def mul(D: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Table 1 Mul(TwiddleCoe, X): Y[i] = D[i] * X[i] over the whole vector."""
    return D * X


# ---- Eq. 1 pieces -----------------------------------------------------------

def stride_permutation(N: int, K: int) -> np.ndarray:
    """Pi^N_K as a dense 0/1 matrix: (Pi x)[b*M + t] = x[t*K + b]."""
    M = N // K
    P = np.zeros((N, N))
    for b in range(K):
        for t in range(M):
            P[b * M + t, t * K + b] = 1.0
    return P


def twiddle_diagonal(N: int, M: int, sign: int = -1) -> np.ndarray:
    """Diagonal of D^N_M: entry b*M + t is w_N^(b*t) (b < N/M, t < M)."""
    K = N // M
    b = np.repeat(np.arange(K, dtype=np.int64), M)
    t = np.tile(np.arange(M, dtype=np.int64), K)
    return omega(N, b * t, sign)


def eq1_dense(N: int, K: int, sign: int = -1) -> np.ndarray:
    """The dense product (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K."""
    M = N // K
    left = np.kron(dft_matrix(K, sign), np.eye(M))
    D = np.diag(twiddle_diagonal(N, M, sign))
    inner = np.kron(np.eye(K), dft_matrix(M, sign))
    return left @ D @ inner @ stride_permutation(N, K)


def eq1_apply(x: np.ndarray, K: int, sign: int = -1) -> np.ndarray:
    """Apply Eq. 1 once to a vector with Table 1's sparse operators, in Eq. 1's order."""
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[0]
    M = N // K
    y = permute(M, N, x)                        # Pi^N_K (reading: Permute(M, N))
    y = fused_ikmv(dft_matrix(M, sign), K, y)   # I_K (x) DFT_M
    y = mul(twiddle_diagonal(N, M, sign), y)    # D^N_M
    return fused_mkiv(dft_matrix(K, sign), M, y)  # DFT_K (x) I_M
