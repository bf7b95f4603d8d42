"""Exact DMD of a whole snapshot matrix, written from its definition (TEST INFRASTRUCTURE ONLY).

Section 2.3: U^- = [u^0 .. u^{m-1}], U^+ = [u^1 .. u^m]; truncated SVD U^- = L S R^*;
A~_r = L^* U^+ R S^{-1}; A~_r = V Lambda V^{-1}; Phi = L V; u(t) = Phi Lambda^t Phi^+ u(0).
Column order (the paper stacks newest first) does not change any of these results.

This is the O(N m r) "from scratch" construction the online method avoids; it serves
as the brute-force check of the incremental oracle on tiny inputs.  The truncation
rule is the one the incremental oracle uses (sigma_i > tau sigma_1, at most r_max).
Phi^+ is taken literally with numpy.linalg.pinv, independently of the incremental
oracle's S * r_first shortcut.
"""
from __future__ import annotations

import numpy as np


class BatchDMD:
    def __init__(self, snapshots: np.ndarray, r_max: int, trunc_tol: float = 1e-10):
        """snapshots: (N, m+1) array whose column k is u^k."""
        X = np.asarray(snapshots, dtype=np.float64)
        self.Um = X[:, :-1]
        self.Up = X[:, 1:]
        Lf, sf, Rt = np.linalg.svd(self.Um, full_matrices=False)
        keep = int(np.count_nonzero(sf > trunc_tol * sf[0]))
        keep = max(1, min(keep, r_max))
        self.L = Lf[:, :keep]
        self.S = sf[:keep]
        self.R = Rt[:keep, :].T
        self.all_singular_values = sf
        self.Atilde = self.L.T @ self.Up @ self.R / self.S[None, :]
        self.lam, self.V = np.linalg.eig(self.Atilde)
        self.Phi = self.L @ self.V
        self.b = np.linalg.pinv(self.Phi) @ X[:, 0]

    def predict(self, ts) -> np.ndarray:
        ts = np.atleast_1d(np.asarray(ts, dtype=np.float64))
        cols = []
        for t in ts:
            lt = np.ones_like(self.lam) if t == 0 else np.where(
                self.lam != 0, np.exp(t * np.log(np.where(self.lam != 0, self.lam, 1))), 0)
            cols.append((self.Phi @ (lt * self.b)).real)
        return np.stack(cols, axis=1)

    def projector(self) -> np.ndarray:
        return self.L @ self.L.T


class BatchPairDMD:
    """Exact DMD of paired matrices X -> Y, from the definition (Sec. 2.3 with arbitrary
    pairs): truncated SVD X = L S R^T by LAPACK, A~_r = L^T Y R S^{-1}, and a prediction
    from a state u as Phi Lambda^t Phi^+ u with Phi^+ = pinv(Phi) taken literally."""

    def __init__(self, X: np.ndarray, Y: np.ndarray, r_max: int, trunc_tol: float = 1e-10):
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        Lf, sf, Rt = np.linalg.svd(X, full_matrices=False)
        keep = int(np.count_nonzero(sf > trunc_tol * sf[0]))
        keep = max(1, min(keep, r_max))
        self.L = Lf[:, :keep]
        self.S = sf[:keep]
        self.R = Rt[:keep, :].T
        self.Atilde = self.L.T @ Y @ self.R / self.S[None, :]
        self.lam, self.V = np.linalg.eig(self.Atilde)
        self.Phi = self.L @ self.V

    def predict_from(self, u, ts) -> np.ndarray:
        b = np.linalg.pinv(self.Phi) @ np.asarray(u, dtype=np.float64).reshape(-1)
        cols = []
        for t in np.atleast_1d(np.asarray(ts, dtype=np.float64)):
            lt = np.ones_like(self.lam) if t == 0 else np.where(
                self.lam != 0, np.exp(t * np.log(np.where(self.lam != 0, self.lam, 1))), 0)
            cols.append((self.Phi @ (lt * b)).real)
        return np.stack(cols, axis=1)
