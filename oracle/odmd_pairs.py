"""Online DMD over arbitrary snapshot pairs, in plain FP64 NumPy (TEST INFRASTRUCTURE ONLY).

Paper: Suh, Chung, Bremer, Choi, arXiv 2311.18715, Sec. 2 (hybrid workflow, Fig. 1) and
Sec. 2.3 (DMD).  The text of the workflow lets an accepted DMD prediction become the new
snapshot; the description of Fig. 1 updates the DMD with FOM results.  In the second
reading only FOM steps update the model, and each update is a pair (x, y) with
y = FOM(x): x is the state the FOM started from, which is a DMD state whenever the step
before it was accepted, so x need not be the previous pair's y.  Sec. 2.3's matrices
then become

  X = [x_1 .. x_m] = L S R^T   (truncated SVD, rank r)
  Y = [y_1 .. y_m]             (paired column by column with X)
  A~_r = L^T Y R S^{-1},  A~_r = V Lambda V^{-1},  Phi = L V

and a prediction starts from a given state u: u(t) = Phi Lambda^t Phi^+ u with
Phi^+ u = V^{-1} L^T u (L orthonormal), t in steps of Delta t after u.

The new column of X is added by Brand's rank-1 append exactly as in ``odmd_ref`` (its
step functions, looked up at call time).  What changes is the operator: with
non-contiguous pairs the projection of Y R on the new direction j is not rho r_last^T, so
this oracle keeps the tall product P = Y R (N x r), rotates it with the right factor of
the core SVD, P' = [P, y] V', and forms M = L^T P from its definition.

Parity status: pinned by ``tests/test_oracle_pairs.py`` against the batch DMD of the
pair matrices (LAPACK SVD of X, no truncation), against ``odmd_ref`` on contiguous pairs,
and against the exact operator of a low-rank linear map.
"""
from __future__ import annotations

import numpy as np

from . import odmd_ref as brand


def rotate_right_products(P: np.ndarray, y: np.ndarray, V1: np.ndarray) -> np.ndarray:
    """P' = Y' R' = [Y R, y] V'  (R' = blkdiag(R, 1) V')."""
    return np.hstack([P, y[:, None]]) @ V1


class OnlineDMDPairsRef:
    """Online DMD fed (x, y) pairs; FP64 throughout."""

    def __init__(self, n: int, r_max: int, trunc_tol: float = 1e-10):
        if n < 1 or r_max < 1:
            raise ValueError("n and r_max must be positive")
        self.n = int(n)
        self.r_max = int(r_max)
        self.tau = float(trunc_tol)
        self.pairs = 0       # pairs received (including those that added nothing)
        self.L = None        # N x r, orthonormal columns spanning the kept part of X
        self.S = None        # r singular values of X, descending
        self.P = None        # N x r, Y R
        self._eig = None

    @property
    def rank(self) -> int:
        return 0 if self.S is None else int(self.S.shape[0])

    def update(self, x, y) -> None:
        """Append the pair (x, y): X gains the column x, Y the column y."""
        x = np.array(x, dtype=np.float64, copy=True).reshape(-1)
        y = np.array(y, dtype=np.float64, copy=True).reshape(-1)
        if x.shape[0] != self.n or y.shape[0] != self.n:
            raise ValueError("snapshot length mismatch")
        self.pairs += 1
        self._eig = None
        if self.L is None:
            xn = float(np.linalg.norm(x))
            if xn == 0.0:
                return  # a zero column of X adds nothing to L S R^T (its row of R is zero)
            self.L = (x / xn)[:, None]
            self.S = np.array([xn])
            self.P = y[:, None].copy()  # R = [[1]]
            return
        L, S = self.L, self.S
        p = L.T @ x
        p, e = brand.orthogonalise_cgs2(L, x, p)
        rho, j = brand.new_direction(e, float(S[0]), float(np.linalg.norm(x)), self.tau)
        K = brand.core_matrix(S, p, rho)
        U1, sig, V1, _ = brand.core_svd_truncated(K, self.tau, self.r_max)
        self.L = brand.rotate_basis(L, j, U1)
        self.P = rotate_right_products(self.P, y, V1)
        self.S = sig

    def operator_products(self) -> np.ndarray:
        """M = L^T Y R = L^T P (r x r), from its definition."""
        return self.L.T @ self.P

    def reduced_operator(self) -> np.ndarray:
        """A~_r = L^T Y R S^{-1}."""
        return self.operator_products() / self.S[None, :]

    def eig(self):
        """(Lambda, V): A~_r = V Lambda V^{-1}."""
        if self.L is None:
            raise RuntimeError("no DMD yet: need a pair with a nonzero x")
        if self._eig is None:
            self._eig = np.linalg.eig(self.reduced_operator())
        return self._eig

    def step(self, u, t: int = 1) -> np.ndarray:
        """L A~^t L^T u for an integer t >= 0 (t products with A~, no eigensolve)."""
        if self.L is None:
            raise RuntimeError("no DMD yet: need a pair with a nonzero x")
        v = self.L.T @ np.asarray(u, dtype=np.float64).reshape(-1)
        A = self.reduced_operator()
        for _ in range(int(t)):
            v = A @ v
        return self.L @ v

    def predict_from(self, u, ts) -> np.ndarray:
        """Re(Phi Lambda^t V^{-1} L^T u) for each t (principal branch), shape (N, len(ts))."""
        lam, V = self.eig()
        b = np.linalg.solve(V, self.L.T @ np.asarray(u, dtype=np.float64).reshape(-1))
        cols = []
        for t in np.atleast_1d(np.asarray(ts, dtype=np.float64)):
            if t == 0:
                lt = np.ones_like(lam, dtype=np.complex128)
            else:
                lt = np.zeros_like(lam, dtype=np.complex128)
                nz = lam != 0
                lt[nz] = np.exp(t * np.log(lam[nz].astype(np.complex128)))
            cols.append((self.L @ (V @ (lt * b))).real)
        return np.stack(cols, axis=1)


def hybrid_fom_updates(fom, credible, u0, steps: int, r_max: int, trunc_tol: float = 1e-10):
    """The hybrid loop of Sec. 2 (Fig. 1) in the reading where only FOM steps update.

    At step k the model (if any) predicts u_k = L A~ L^T u_{k-1};
    ``credible(k, u_{k-1}, u_pred)`` decides whether it is kept (a residual of the FOM's
    system at step k depends on the state it starts from).  Otherwise ``fom(k, u_{k-1})``
    gives u_k and the pair (u_{k-1}, u_k) updates the model.  Returns (states
    (steps+1, N), FOM step indices, the model).
    """
    u0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    model = OnlineDMDPairsRef(u0.shape[0], r_max, trunc_tol)
    states = [u0]
    fom_steps = []
    for k in range(1, steps + 1):
        prev = states[-1]
        if model.rank > 0:
            pred = model.step(prev, 1)
            if credible(k, prev, pred):
                states.append(pred)
                continue
        nxt = np.asarray(fom(k, prev), dtype=np.float64).reshape(-1)
        model.update(prev, nxt)
        fom_steps.append(k)
        states.append(nxt)
    return np.stack(states), fom_steps, model
