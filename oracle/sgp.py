"""Unmapped sparse-GP mean and variance (Eq. 1 and Eq. 2) and their lossless
mapping to the quadratic forms beta and gamma (Sec. V-B, "Mapped Sparse GP").

TEST INFRASTRUCTURE ONLY (part of the oracle).

Reading of the paper used here: the kernel is k_xi(d1, d2) = sigma^2 (d1 . d2)^xi
on normalized descriptors; the mean uses xi = 2 and the variance xi = 1.  In
Eq. 2 the prefactors sigma^2 and sigma^4 are written out explicitly, so k_1
there is read as the unscaled dot product (d1 . d2); with ||d|| = 1 this gives

    V(d) = sigma^2 - sigma^4 k^T K_SS^{-1} k,   k_s = d . d_s,
    gamma = sigma^2 I - sigma^4 D_S^T K_SS^{-1} D_S,

and for the mean

    eps(d) = sum_s sigma^2 (d . d_s)^2 alpha_s = d^T beta d,
    beta = sigma^2 sum_s alpha_s d_s d_s^T.
"""
from __future__ import annotations

import numpy as np


def sgp_mean(d, D_S, alpha, sig2):
    """Eq. 1, summed over the sparse set: sum_s sig2 (d . d_s)^2 alpha_s.
    d: [m, n_d] (rows unit norm), D_S: [n_S, n_d]."""
    k2 = sig2 * (d @ D_S.T) ** 2
    return k2 @ alpha


def sgp_variance(d, D_S, K_SS, sig2):
    """Eq. 2, summed over the sparse set: sig2 k1(d, d) - sig2^2 k^T K_SS^{-1} k
    with k1 the unscaled dot product (k1(d, d) = 1 for unit d)."""
    k1 = d @ D_S.T                                   # [m, n_S]
    sol = np.linalg.solve(K_SS, k1.T)               # [n_S, m]
    return sig2 * np.einsum("ij,ij->i", d, d) - sig2 ** 2 * np.einsum("ij,ji->i", k1, sol)


def mapped_beta(D_S, alpha, sig2):
    """beta = sig2 sum_s alpha_s d_s d_s^T (the reordering of Eq. 1)."""
    return sig2 * (D_S.T * alpha[None, :]) @ D_S


def mapped_gamma(D_S, K_SS, sig2):
    """gamma = sig2 I - sig2^2 D_S^T K_SS^{-1} D_S (the reordering of Eq. 2)."""
    n_d = D_S.shape[1]
    return sig2 * np.eye(n_d) - sig2 ** 2 * D_S.T @ np.linalg.solve(K_SS, D_S)


def quad(d, M):
    """d^T M d for each row of d."""
    return np.einsum("ij,jk,ik->i", d, M, d)
