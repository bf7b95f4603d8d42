"""Incremental online DMD in plain FP64 NumPy -- the oracle (TEST INFRASTRUCTURE ONLY).

Paper: Suh, Chung, Bremer, Choi, "Accelerating Flow Simulations using Online Dynamic
Mode Decomposition" (NeurIPS 2023 ML4PS), Section 2.3.  The paper gives the DMD
definitions and names the update (Brand's incremental SVD, "original version", with
O(Nr) per snapshot) but not its steps; the steps below are Brand's rank-1 column
append (M. Brand, Linear Algebra Appl. 415 (2006)) applied to the paper's matrices:

  U^- = [u^0 .. u^{m-1}] = L S R^T  (truncated SVD, rank r)
  U^+ = [u^1 .. u^m]                (paired column by column with U^-)
  A~_r = L^T U^+ R S^{-1}  (r x r),  A~_r = V Lambda V^{-1},  Phi = L V
  u(t) = Phi Lambda^{t} Phi^+ u(0)   (t in steps of Delta t)

State kept (never the snapshot history): L (N x r), S (r), M = L^T U^+ R (r x r),
the first and last rows of R, and the latest snapshot c.  Each new snapshot x adds the
column c to U^- and the column x to U^+.

Readings where the paper is silent (each listed in the design notes):
* orthogonalisation of the new column: classical Gram-Schmidt applied twice (CGS2);
* thresholds: a new direction enters iff rho > tau max(sigma_1, ||c||); after the core
  SVD, singular values sigma'_i <= tau sigma'_1 are dropped, then the rank is capped at
  r_max (the smallest go first);
* operator update: with j the new unit direction, the columns of U^+ other than x are
  columns of U^- (contiguous stream), so j^T U^+ R = rho r_last^T; hence
  M' = U'^T [[M, L^T x], [rho r_last^T, j^T x]] V';
* b = Phi^+ u^0 = V^{-1} L^T u^0 = V^{-1} (S * r_first), time counted from u^0;
* output x(t) = Re(Phi Lambda^t b) (conjugate pairs make the imaginary part rounding).

Every step is a separate function so a test can replace one of them by a deliberately
wrong variant and see a pin fail.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- single steps
def project(L: np.ndarray, c: np.ndarray, x: np.ndarray):
    """p = L^T c and w = L^T x (Sec. 2.3: matrix-vector products only)."""
    return L.T @ c, L.T @ x


def orthogonalise_cgs2(L: np.ndarray, c: np.ndarray, p: np.ndarray):
    """Residual of c against span(L), Gram-Schmidt applied twice.

    e = c - L p; s = L^T e; p <- p + s; e <- e - L s.  Returns (p, e).
    """
    e = c - L @ p
    s = L.T @ e
    return p + s, e - L @ s


def new_direction(e: np.ndarray, sigma1: float, cnorm: float, tau: float):
    """rho = ||e||; below tau * max(sigma_1, ||c||) the direction is treated as absent."""
    rho = float(np.linalg.norm(e))
    if rho <= tau * max(sigma1, cnorm):
        return 0.0, np.zeros_like(e)
    return rho, e / rho


def core_matrix(S: np.ndarray, p: np.ndarray, rho: float) -> np.ndarray:
    """K = [[diag(S), p], [0, rho]], so that [U^-, c] = [L, j] K blkdiag(R, 1)^T."""
    r = S.shape[0]
    K = np.zeros((r + 1, r + 1))
    K[:r, :r] = np.diag(S)
    K[:r, r] = p
    K[r, r] = rho
    return K


def core_svd_truncated(K: np.ndarray, tau: float, r_max: int):
    """SVD K = U' diag(sigma') V'^T (LAPACK), then keep sigma'_i > tau sigma'_1, <= r_max."""
    U1, sig, V1t = np.linalg.svd(K)
    keep = int(np.count_nonzero(sig > tau * sig[0])) if sig[0] > 0 else 0
    keep = max(1, min(keep, r_max))
    discarded = float(np.sum(sig[keep:] ** 2))
    return U1[:, :keep], sig[:keep], V1t.T[:, :keep], discarded


def rotate_basis(L: np.ndarray, j: np.ndarray, U1: np.ndarray) -> np.ndarray:
    """L' = [L, j] U'."""
    return np.hstack([L, j[:, None]]) @ U1


def operator_update(M, w, rho, r_last, gamma, U1, V1):
    """M' = U'^T [[M, w], [rho r_last^T, gamma]] V'  (M = L^T U^+ R, Sec. 2.3)."""
    r = M.shape[0]
    B = np.zeros((r + 1, r + 1))
    B[:r, :r] = M
    B[:r, r] = w
    B[r, :r] = rho * r_last
    B[r, r] = gamma
    return U1.T @ B @ V1


def right_rows_update(r_first, V1):
    """R' = blkdiag(R, 1) V': first row [r_first, 0] V', last row = V'[r, :]."""
    rf = np.append(r_first, 0.0) @ V1
    rl = V1[-1, :].copy()
    return rf, rl


# ---------------------------------------------------------------- the model
class OnlineDMDRef:
    """Online DMD with rank-1 updates (the oracle).  FP64 throughout."""

    def __init__(self, n: int, r_max: int, trunc_tol: float = 1e-10):
        if n < 1 or r_max < 1:
            raise ValueError("n and r_max must be positive")
        self.n = int(n)
        self.r_max = int(r_max)
        self.tau = float(trunc_tol)
        self.c = None          # latest snapshot (last column of U^+, next column of U^-)
        self.count = 0         # snapshots received so far
        self.L = None
        self.S = None
        self.M = None
        self.r_first = None
        self.r_last = None
        self.q = None          # L^T c
        self.discarded_sq = 0.0  # sum of squared singular values dropped so far
        self._eig = None

    # -- state
    @property
    def rank(self) -> int:
        return 0 if self.S is None else int(self.S.shape[0])

    def update(self, x) -> None:
        """Append snapshot x: U^- gains the previous snapshot c, U^+ gains x."""
        x = np.array(x, dtype=np.float64, copy=True).reshape(-1)
        if x.shape[0] != self.n:
            raise ValueError("snapshot length mismatch")
        self.count += 1
        self._eig = None
        if self.c is None:
            self.c = x
            return
        c = self.c
        if self.L is None:
            cn = float(np.linalg.norm(c))
            if cn == 0.0:
                # a zero column of U^- adds nothing to L S R^T; keep waiting
                self.c = x
                return
            L = (c / cn)[:, None]
            self.L = L
            self.S = np.array([cn])
            # c is u^0 iff this is the second snapshot; otherwise u^0 (and every
            # snapshot before c) was zero and its row of R is zero.
            self.r_first = np.array([1.0 if self.count == 2 else 0.0])
            self.r_last = np.array([1.0])
            w = L.T @ x
            self.M = w.reshape(1, 1).copy()
            self.q = w.copy()
            self.c = x
            return
        L, S = self.L, self.S
        p, w = project(L, c, x)
        p, e = orthogonalise_cgs2(L, c, p)
        rho, j = new_direction(e, float(S[0]), float(np.linalg.norm(c)), self.tau)
        gamma = float(j @ x)
        K = core_matrix(S, p, rho)
        U1, sig, V1, disc = core_svd_truncated(K, self.tau, self.r_max)
        self.discarded_sq += disc
        self.L = rotate_basis(L, j, U1)
        self.M = operator_update(self.M, w, rho, self.r_last, gamma, U1, V1)
        self.r_first, self.r_last = right_rows_update(self.r_first, V1)
        self.q = U1.T @ np.append(w, gamma)
        self.S = sig
        self.c = x

    # -- reduced operator and modes
    def reduced_operator(self) -> np.ndarray:
        """A~_r = L^T U^+ R S^{-1} = M diag(S)^{-1}."""
        return self.M / self.S[None, :]

    def eig(self):
        """(Lambda, V, b): A~_r = V Lambda V^{-1}, b = V^{-1} L^T u^0 = V^{-1}(S * r_first)."""
        if self.L is None:
            raise RuntimeError("no DMD yet: need two snapshots with a nonzero first one")
        if self._eig is None:
            lam, V = np.linalg.eig(self.reduced_operator())
            b = np.linalg.solve(V, self.S * self.r_first)
            self._eig = (lam, V, b)
        return self._eig

    @staticmethod
    def powers(lam: np.ndarray, t: float) -> np.ndarray:
        """Lambda^t on the principal branch (|lambda|^t e^{i t arg lambda}); 0^0 = 1."""
        lam = np.asarray(lam, dtype=np.complex128)
        if t == 0:
            return np.ones_like(lam)
        out = np.zeros_like(lam)
        nz = lam != 0
        out[nz] = np.exp(t * np.log(lam[nz]))
        return out

    def coefficients(self, ts) -> np.ndarray:
        """C[:, k] = V Lambda^{t_k} b, complex (r x len(ts))."""
        lam, V, b = self.eig()
        return np.stack([V @ (self.powers(lam, float(t)) * b) for t in ts], axis=1)

    def predict(self, ts) -> np.ndarray:
        """x(t_k) = Re(Phi Lambda^{t_k} b) = Re(L V Lambda^{t_k} b), shape (N, len(ts))."""
        ts = np.atleast_1d(np.asarray(ts, dtype=np.float64))
        return self.L @ self.coefficients(ts).real

    def predict_imag_max(self, ts) -> float:
        """Largest |Im| of the modal sum (rounding level for conjugate pairs)."""
        ts = np.atleast_1d(np.asarray(ts, dtype=np.float64))
        return float(np.max(np.abs(self.L @ self.coefficients(ts).imag)))

    def check(self, t: float, x_fom, tol: float = 1e-5):
        """Credibility check: relative L2 distance of the prediction to the FOM snapshot.

        err = ||x(t) - x_fom|| / ||x_fom||, pass = err <= tol (Sec. 2.2 uses the FOM
        residual; with the FOM state at hand the relative error is measured directly).
        A zero x_fom gives err = 0 if the prediction is zero too, else inf.
        """
        x_fom = np.asarray(x_fom, dtype=np.float64).reshape(-1)
        xp = self.predict([t])[:, 0]
        num = float(np.linalg.norm(xp - x_fom))
        den = float(np.linalg.norm(x_fom))
        if den == 0.0:
            err = 0.0 if num == 0.0 else float("inf")
        else:
            err = num / den
        return err, bool(err <= tol)
