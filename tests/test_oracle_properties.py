"""Property-based pins of the oracles (CPU only; skipped where hypothesis is absent).

Random shapes, ranks and scales instead of fixed cases: without truncation the
incremental oracles must equal the DMD built from its definition (Sec. 2.3) on the whole
snapshot or pair matrices, for every stream the strategy draws, including rank-deficient
ones (repeated or zero columns) and widely scaled ones.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import OnlineDMDPairsRef, OnlineDMDRef  # noqa: E402


def _stream(seed, n, m, rank, scale):
    """n x (m+1) snapshots of rank <= rank, columns scaled by 10^U(-scale, scale)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, rank))
    C = rng.standard_normal((rank, m + 1))
    X = B @ C
    X *= 10.0 ** rng.uniform(-scale, scale, m + 1)[None, :]
    return X


def _definition(Um, Up, tau=1e-10):
    """Rank, projector and full-space operator of the DMD of (Um -> Up) by its definition."""
    Lf, sf, Rt = np.linalg.svd(Um, full_matrices=False)
    keep = int(np.count_nonzero(sf > tau * sf[0]))
    L, S, R = Lf[:, :keep], sf[:keep], Rt[:keep].T
    At = L.T @ Up @ R / S[None, :]
    return keep, S, L @ L.T, L @ At @ L.T


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(8, 60), m=st.integers(2, 14),
       rank=st.integers(1, 14), scale=st.floats(0.0, 2.0))
def test_snapshot_stream_equals_definition(seed, n, m, rank, scale):
    X = _stream(seed, n, m, min(rank, n), scale)
    o = OnlineDMDRef(n, r_max=64)
    for k in range(m + 1):
        o.update(X[:, k])
    keep, S, P, A = _definition(X[:, :-1], X[:, 1:])
    assert o.rank == keep
    np.testing.assert_allclose(o.S, S, rtol=0, atol=1e-11 * S[0])
    assert np.max(np.abs(o.L @ o.L.T - P)) < 1e-9
    Ao = o.L @ o.reduced_operator() @ o.L.T
    # the operator scales like |x_{k+1}| / |x_k|, up to 10^4 here
    assert np.max(np.abs(Ao - A)) < 1e-8 * max(1.0, np.max(np.abs(A)))


@settings(max_examples=40, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(8, 60), m=st.integers(1, 14),
       rank=st.integers(1, 14))
def test_pairs_equal_definition(seed, n, m, rank):
    rng = np.random.default_rng(seed)
    X = _stream(seed, n, m - 1, min(rank, n), 0.0)
    Y = rng.standard_normal((n, m))
    o = OnlineDMDPairsRef(n, r_max=64)
    for k in range(m):
        o.update(X[:, k], Y[:, k])
    keep, S, P, A = _definition(X, Y)
    assert o.rank == keep
    np.testing.assert_allclose(o.S, S, rtol=0, atol=1e-11 * S[0])
    assert np.max(np.abs(o.L @ o.L.T - P)) < 1e-9
    Ao = o.L @ o.reduced_operator() @ o.L.T
    assert np.max(np.abs(Ao - A)) < 1e-8 * max(1.0, np.max(np.abs(A)))
