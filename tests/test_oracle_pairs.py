"""Pins of the pair oracle (online DMD fed (x, y) pairs; the hybrid loop in the reading
where only FOM steps update), against what the mathematics fixes: the pseudo-inverse
form of the DMD operator, the batch DMD of the pair matrices, the snapshot-stream oracle
on contiguous pairs, and the exact operator of a low-rank linear map.  Planted mistakes
in the pair oracle's own step must trip at least one pin."""
import numpy as np
import pytest

import oracle.odmd_pairs as pairs
from oracle import BatchPairDMD, OnlineDMDPairsRef, OnlineDMDRef, hybrid_fom_updates


def _feed(X, Y, r_max, tau=1e-10):
    m = OnlineDMDPairsRef(X.shape[0], r_max, tau)
    for i in range(X.shape[1]):
        m.update(X[:, i], Y[:, i])
    return m


def _full_operator(m):
    """L A~ L^T: the DMD operator on the whole space, independent of the basis chosen."""
    return m.L @ m.reduced_operator() @ m.L.T


def _low_rank_map(n, lams, seed):
    """A = B W diag-blocks W^{-1} B^T: eigenvalues lams (real, or conjugate pairs given
    once as complex), B an n x k orthonormal basis; returns (A, B, W, lam_full)."""
    rng = np.random.default_rng(seed)
    blocks, lam_full = [], []
    for lam in lams:
        if np.iscomplex(lam):
            a, b = lam.real, lam.imag
            blocks.append(np.array([[a, -b], [b, a]]))
            lam_full += [lam, np.conj(lam)]
        else:
            blocks.append(np.array([[float(np.real(lam))]]))
            lam_full.append(complex(lam))
    k = sum(b.shape[0] for b in blocks)
    D = np.zeros((k, k))
    o = 0
    for b in blocks:
        D[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    W = rng.standard_normal((k, k)) + 3 * np.eye(k)
    B, _ = np.linalg.qr(rng.standard_normal((n, k)))
    C = W @ D @ np.linalg.inv(W)
    return B @ C @ B.T, B, C, np.array(lam_full)


def test_operator_equals_pseudo_inverse_form():
    """Without truncation L L^T = X X^+, so L A~ L^T = X X^+ Y X^+ (Sec. 2.3 with pairs),
    and the singular values are those of X."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((30, 10))
    Y = rng.standard_normal((30, 10))
    m = _feed(X, Y, r_max=12)
    assert m.rank == 10
    np.testing.assert_allclose(m.S, np.linalg.svd(X, compute_uv=False), rtol=1e-12)
    Xp = np.linalg.pinv(X)
    want = X @ Xp @ Y @ Xp
    assert np.max(np.abs(_full_operator(m) - want)) < 1e-11 * np.max(np.abs(want))


def test_predictions_equal_batch_pair_dmd():
    """Step and modal predictions from a state against the batch DMD of the pair matrices
    (LAPACK SVD, Phi^+ by pinv), integer and fractional horizons."""
    rng = np.random.default_rng(4)
    n, m_ = 40, 9
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    X = rng.standard_normal((n, m_))
    Y = A @ X + 0.05 * rng.standard_normal((n, m_))
    m = _feed(X, Y, r_max=20)
    B = BatchPairDMD(X, Y, r_max=20)
    u = X @ rng.standard_normal(m_)
    ts = [0.0, 1.0, 2.0, 2.5, 4.0]
    want = B.predict_from(u, ts)
    got = m.predict_from(u, ts)
    assert np.linalg.norm(got - want) < 1e-10 * np.linalg.norm(want)
    for t in (0, 1, 3):
        np.testing.assert_allclose(m.step(u, t), B.predict_from(u, [float(t)])[:, 0], rtol=0,
                                   atol=1e-10 * np.linalg.norm(u))


@pytest.mark.parametrize("r_max", [12, 40])
def test_contiguous_pairs_reduce_to_snapshot_stream(r_max):
    """Pairs (u^{k-1}, u^k) of one stream build the same X as the snapshot-stream oracle:
    same singular values and, where nothing is truncated (the stream has rank 12 and
    noise-free snapshots), the same operator L A~ L^T."""
    rng = np.random.default_rng(5)
    n, k, steps = 60, 12, 30
    A, Bq, _, _ = _low_rank_map(n, [0.99 * np.exp(0.2j), 0.97 * np.exp(0.5j), 0.95 * np.exp(0.9j),
                                    0.98 * np.exp(1.3j), 0.9 * np.exp(2.0j), 0.96 * np.exp(2.6j)], seed=6)
    U = np.empty((n, steps + 1))
    U[:, 0] = Bq @ rng.standard_normal(k)
    for t in range(steps):
        U[:, t + 1] = A @ U[:, t]
    ref = OnlineDMDRef(n, r_max)
    for t in range(steps + 1):
        ref.update(U[:, t])
    m = _feed(U[:, :-1], U[:, 1:], r_max)
    assert m.rank == ref.rank
    np.testing.assert_allclose(m.S, ref.S, rtol=0, atol=1e-12 * ref.S[0])
    full_ref = ref.L @ ref.reduced_operator() @ ref.L.T
    assert np.max(np.abs(_full_operator(m) - full_ref)) < 1e-10
    # and both equal the true map on its range
    assert np.max(np.abs(_full_operator(m) - A)) < 1e-9


def test_low_rank_map_recovered_from_scattered_pairs():
    """Pairs (x_i, A x_i) with x_i drawn at random in the range of A (no two consecutive):
    after as many pairs as the rank the eigenvalues are A's and integer and fractional
    steps from a state in the range are A^t u (principal branch for fractional t)."""
    lams = [0.995 * np.exp(0.3j), 0.9 * np.exp(1.1j), 0.8, -0.6]
    A, Bq, C, lam_full = _low_rank_map(50, lams, seed=7)
    k = Bq.shape[1]
    rng = np.random.default_rng(8)
    Xs = Bq @ rng.standard_normal((k, k + 3))
    m = _feed(Xs, A @ Xs, r_max=20)
    assert m.rank == k
    lam, _ = m.eig()
    for z in lam_full:
        assert np.min(np.abs(lam - z)) < 1e-10
    u = Bq @ rng.standard_normal(k)
    for t in (1, 2, 5):
        want = np.linalg.matrix_power(A, t) @ u
        assert np.linalg.norm(m.step(u, t) - want) < 1e-10 * np.linalg.norm(u)
    ev, W = np.linalg.eig(C)
    want = (Bq @ (W @ (np.exp(2.5 * np.log(ev.astype(complex))) * np.linalg.solve(W, Bq.T @ u)))).real
    got = m.predict_from(u, [2.5])[:, 0]
    assert np.linalg.norm(got - want) < 1e-10 * np.linalg.norm(u)


def test_hybrid_loop_updates_on_fom_steps_only():
    """The hybrid loop with FOM-only updates on a linear FOM whose state has a decaying
    component outside a rank-8 subspace; every fourth step calls the FOM even when the
    prediction is credible, so the model receives pairs whose x is a DMD state (not the
    previous pair's y).  Checked: FOM steps are exact and each adds one pair, credible
    steps are within the tolerance of the FOM, at least one pair is non-contiguous, and
    the final model equals the batch DMD of the recorded pairs."""
    n, tol, steps = 80, 1e-6, 120
    Ar, Bq, _, _ = _low_rank_map(n, [0.995 * np.exp(0.15j), 0.99 * np.exp(0.4j), 0.97 * np.exp(0.7j),
                                     0.96 * np.exp(1.0j)], seed=9)
    A = Ar + 0.3 * (np.eye(n) - Bq @ Bq.T)
    rng = np.random.default_rng(10)
    u0 = Bq @ rng.standard_normal(8) + 1e-3 * rng.standard_normal(n)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    states, fom_steps, model = hybrid_fom_updates(
        lambda k, u: A @ u, lambda k, prev, pred: k % 4 != 0 and rel(pred, A @ prev) <= tol, u0, steps, 30)
    assert states.shape == (steps + 1, n)
    assert model.pairs == len(fom_steps)
    for k in fom_steps:
        np.testing.assert_array_equal(states[k], A @ states[k - 1])
    accepted = [k for k in range(1, steps + 1) if k not in fom_steps]
    assert len(accepted) > 40
    for k in accepted:
        assert rel(states[k], A @ states[k - 1]) <= tol
    assert any(k - 1 in accepted for k in fom_steps)
    X = np.stack([states[k - 1] for k in fom_steps], axis=1)
    Y = np.stack([states[k] for k in fom_steps], axis=1)
    Bd = BatchPairDMD(X, Y, r_max=30)
    full_b = Bd.L @ Bd.Atilde @ Bd.L.T
    assert model.rank == Bd.S.shape[0]
    assert np.max(np.abs(_full_operator(model) - full_b)) < 1e-9 * np.max(np.abs(full_b))


# ------------------------------------------------------------ planted mistakes
PINS = [
    test_operator_equals_pseudo_inverse_form,
    test_predictions_equal_batch_pair_dmd,
    lambda: test_contiguous_pairs_reduce_to_snapshot_stream(12),
    test_low_rank_map_recovered_from_scattered_pairs,
]


def _mistakes():
    orig = pairs.rotate_right_products
    orig_update = pairs.OnlineDMDPairsRef.update

    def transposed(P, y, V1):
        return orig(P, y, V1.T if V1.shape[0] == V1.shape[1] else V1[::-1])

    def rows_reversed(P, y, V1):
        return orig(P, y, V1[::-1])

    def drop_y(P, y, V1):
        return orig(P, 0 * y, V1)

    def not_rotated(P, y, V1):
        return np.hstack([P, y[:, None]])[:, : V1.shape[1]]

    def pairs_x_with_x(self, x, y):
        return orig_update(self, x, x)

    return [("rotate_right_products", transposed), ("rotate_right_products", rows_reversed),
            ("rotate_right_products", drop_y), ("rotate_right_products", not_rotated),
            ("update", pairs_x_with_x)]


@pytest.mark.parametrize("idx", range(5))
def test_planted_mistake_in_pair_products_is_caught(idx, monkeypatch):
    name, bad = _mistakes()[idx]
    if name == "update":
        monkeypatch.setattr(pairs.OnlineDMDPairsRef, "update", bad)
    else:
        monkeypatch.setattr(pairs, name, bad)
    failures = 0
    for f in PINS:
        try:
            with np.errstate(all="ignore"):
                f()
        except (AssertionError, np.linalg.LinAlgError, ValueError, IndexError, FloatingPointError):
            failures += 1
    assert failures >= 1, f"planted mistake {idx} ({bad.__name__}) slipped through every pin"
