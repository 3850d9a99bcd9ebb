"""Pins for the readings of Eq. 1 and Table 1 (stride permutation, twiddle diagonal).

Eq. 1 (Section 3): DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K, N = M K.
The paper leaves Pi^N_K and the entries of D^N_M implicit, so the readings in
oracle/kronecker.py are pinned here against the dense DFT matrix for every
factorisation N = K M <= 64.
"""
import numpy as np
import pytest

from oracle import kronecker as kr

FACTORISATIONS = [(N, K) for N in (2, 4, 6, 8, 12, 16, 32, 64) for K in range(1, N + 1) if N % K == 0]


@pytest.mark.parametrize("N,K", FACTORISATIONS)
@pytest.mark.parametrize("sign", [-1, 1])
def test_eq1_dense_equals_dft(N, K, sign):
    assert np.abs(kr.eq1_dense(N, K, sign) - kr.dft_matrix(N, sign)).max() < 1e-12


@pytest.mark.parametrize("N,K", FACTORISATIONS)
def test_eq1_with_table1_operators(N, K):
    rng = np.random.Generator(np.random.PCG64(N * 100 + K))
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    np.testing.assert_allclose(kr.eq1_apply(x, K), kr.dft_matrix(N) @ x, atol=1e-12)


def test_stride_permutation_is_table1_permute_m_n():
    for N, K in FACTORISATIONS:
        M = N // K
        x = np.arange(N).astype(complex)
        np.testing.assert_array_equal(kr.stride_permutation(N, K) @ x, kr.permute(M, N, x))


def test_literal_permute_k_n_fails_when_k_differs_from_m():
    """Reading Pi^N_K as Table 1's Permute(K, N) breaks Eq. 1 whenever K != M (and both > 1)."""
    for N, K in FACTORISATIONS:
        M = N // K
        if K == M or K == 1 or M == 1:  # both readings are the identity there
            continue
        P_literal = np.zeros((N, N))
        for i in range(K):
            for j in range(M):
                P_literal[i + K * j, M * i + j] = 1.0
        dense = (np.kron(kr.dft_matrix(K), np.eye(M)) @ np.diag(kr.twiddle_diagonal(N, M))
                 @ np.kron(np.eye(K), kr.dft_matrix(M)) @ P_literal)
        assert np.abs(dense - kr.dft_matrix(N)).max() > 1e-3, (N, K)


def test_hand_checked_n8_k2():
    """N = 8, K = 2: Pi gathers x0,x2,x4,x6 then x1,x3,x5,x7."""
    y = kr.permute(4, 8, np.arange(8).astype(complex)).real
    np.testing.assert_array_equal(y, [0, 2, 4, 6, 1, 3, 5, 7])
    d = kr.twiddle_diagonal(8, 4)
    np.testing.assert_allclose(d[:4], 1)
    np.testing.assert_allclose(d[4:], np.exp(-2j * np.pi * np.arange(4) / 8), atol=1e-15)


def test_fused_pkiv_moves_blocks():
    m, n, k = 2, 3, 4
    X = np.arange(m * n * k).astype(complex)
    Y = kr.fused_pkiv(m, m * n, k, X)
    for i in range(m):
        for j in range(n):
            np.testing.assert_array_equal(Y[k * (i + m * j): k * (i + m * j) + k],
                                          X[k * (n * i + j): k * (n * i + j) + k])
    # with k = 1 it is Permute(m, mn)
    np.testing.assert_array_equal(kr.fused_pkiv(m, m * n, 1, X[:6]), kr.permute(m, m * n, X[:6]))


def test_kronecker_loops_match_dense_kron():
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    X = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    np.testing.assert_allclose(kr.fused_mkiv(A, 3, X), np.kron(A, np.eye(3)) @ X, atol=1e-12)
    np.testing.assert_allclose(kr.fused_ikmv(A, 3, X), np.kron(np.eye(3), A) @ X, atol=1e-12)
