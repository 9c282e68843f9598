"""Oracle RBF interpolation of sampled scalar fluxes (test infrastructure only).

The paper's interpolated initial guess (Sec. 5: "GMRES-DSA-Interp-IG") interpolates the high-fidelity scalar
fluxes of the sampled training parameters with radial basis functions; it does not state the kernel.  Reading
taken here: features x = (log sigma_s[R], sigma_a[R]) standardised by the samples' mean and standard deviation
(a feature with zero spread keeps scale 1), the polyharmonic cubic kernel phi(r) = r^3 with a degree-1
polynomial term, i.e. s(x) = sum_k lambda_k |x - x_k|^3 + c_0 + sum_i c_i x_i with
    [Phi  P] [lambda]   [F]
    [P^T  0] [  c   ] = [0],   Phi_kl = |x_k - x_l|^3,  P_k = (1, x_k),
solved once for all data columns F = [phi_1 ... phi_K]^T, and s evaluated directly from (lambda, c).
"""
from __future__ import annotations

import numpy as np


def features(sigma_s: np.ndarray, sigma_a: np.ndarray) -> np.ndarray:
    return np.concatenate([np.log(np.asarray(sigma_s, dtype=np.float64)), np.asarray(sigma_a, dtype=np.float64)],
                          axis=-1)


class Rbf:
    def __init__(self, sigma_s: np.ndarray, sigma_a: np.ndarray, solutions: np.ndarray):
        """sigma_s, sigma_a: [K][R] sampled parameters; solutions: [K][N] their scalar fluxes."""
        X = features(sigma_s, sigma_a)
        self.mean = X.mean(axis=0)
        sd = X.std(axis=0)
        self.scale = np.where(sd > 0, sd, 1.0)
        self.X = (X - self.mean) / self.scale
        K, d = self.X.shape
        Phi = np.linalg.norm(self.X[:, None, :] - self.X[None, :, :], axis=-1) ** 3
        P = np.concatenate([np.ones((K, 1)), self.X], axis=1)
        A = np.zeros((K + d + 1, K + d + 1))
        A[:K, :K] = Phi
        A[:K, K:] = P
        A[K:, :K] = P.T
        rhs = np.zeros((K + d + 1, solutions.shape[1]))
        rhs[:K] = solutions
        coef = np.linalg.solve(A, rhs)
        self.lam, self.c = coef[:K], coef[K:]

    def __call__(self, sigma_s: np.ndarray, sigma_a: np.ndarray) -> np.ndarray:
        """s(x) for one parameter point (sigma_s [R], sigma_a [R]) -> [N]."""
        x = (features(sigma_s, sigma_a) - self.mean) / self.scale
        g = np.linalg.norm(self.X - x[None, :], axis=1) ** 3
        return g @ self.lam + self.c[0] + x @ self.c[1:]
