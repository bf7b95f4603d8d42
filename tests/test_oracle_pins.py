"""Pins of the FP64 oracle against things the paper and the mathematics fix.

Nothing here compares the oracle with itself: the checks are a batch DMD written from
the Sec. 2.3 definitions (brute force on tiny inputs), closed-form eigenvalues of planted
linear streams, exact identities of linear systems, orthonormality and truncation
bounds, and special cases of the credibility check (Sec. 2.2).
"""
import numpy as np
import pytest

from oracle import BatchDMD, OnlineDMDRef
from synth import PlantedModes, WakeField


def match_eigs(a, b):
    """Greedy nearest matching of two eigenvalue sets; returns max relative distance."""
    a = list(np.asarray(a, dtype=complex))
    b = list(np.asarray(b, dtype=complex))
    assert len(a) == len(b)
    worst = 0.0
    for x in sorted(a, key=lambda z: -abs(z)):
        d = [abs(x - y) for y in b]
        i = int(np.argmin(d))
        worst = max(worst, d[i] / max(abs(x), 1e-300))
        b.pop(i)
    return worst


def run_online(X, r_max, tau=1e-10):
    o = OnlineDMDRef(X.shape[0], r_max, tau)
    for k in range(X.shape[1]):
        o.update(X[:, k])
    return o


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("n,m,seed", [(64, 12, 1), (200, 30, 2), (512, 60, 3)])
def test_incremental_equals_batch_without_truncation(n, m, seed):
    """No truncation active (r_max >= m): incremental SVD/DMD = batch SVD/DMD."""
    rng = np.random.default_rng(seed)
    # a linear stream with a moderate spectrum plus full-rank perturbation
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    X = np.empty((n, m + 1))
    X[:, 0] = rng.standard_normal(n)
    for k in range(m):
        X[:, k + 1] = A @ X[:, k] + 0.1 * rng.standard_normal(n)
    o = run_online(X, r_max=m + 5)
    B = BatchDMD(X, r_max=m + 5)
    assert o.rank == B.S.shape[0] == m
    np.testing.assert_allclose(o.S, B.S, rtol=1e-12, atol=0)
    P1 = o.L @ o.L.T
    assert np.max(np.abs(P1 - B.projector())) < 1e-12
    G = o.L.T @ o.L
    assert np.max(np.abs(G - np.eye(o.rank))) < 1e-13 * np.sqrt(o.rank) * 10
    lam, _, _ = o.eig()
    assert match_eigs(lam, B.lam) < 1e-10
    ts = [0, 1, m / 2, m, m + 3.5]
    Xo, Xb = o.predict(ts), B.predict(ts)
    assert np.max(np.abs(Xo - Xb)) / np.max(np.abs(Xb)) < 1e-10


def test_reduced_operator_equals_definition():
    """M S^-1 from the O(r^2) update equals L^T U^+ R S^-1 built from the snapshots."""
    rng = np.random.default_rng(5)
    n, m = 150, 25
    X = rng.standard_normal((n, m + 1))
    o = run_online(X, r_max=40)
    # R from the definition: U^- = L S R^T  =>  R = U^-^T L S^-1
    R = X[:, :-1].T @ o.L / o.S[None, :]
    At_def = o.L.T @ X[:, 1:] @ R / o.S[None, :]
    np.testing.assert_allclose(o.reduced_operator(), At_def, rtol=0, atol=1e-11 * np.abs(At_def).max())
    np.testing.assert_allclose(o.r_first, R[0], atol=1e-12)
    np.testing.assert_allclose(o.r_last, R[-1], atol=1e-12)


# ------------------------------------------------------------------ closed forms
def test_planted_modes_noise_free_recovers_eigenvalues():
    """Rank-6 linear stream (3 conjugate pairs): the DMD eigenvalues are the planted ones."""
    g = PlantedModes(4096, sigma=0.0, seed=0)
    X = g.snapshots(0, 200).T
    o = run_online(X, r_max=10)
    assert o.rank == 6
    lam, _, _ = o.eig()
    assert match_eigs(lam, g.planted_eigenvalues()) < 1e-10


def test_planted_modes_with_noise_close_to_planted():
    """sigma = 1e-8 noise (the 4096-point, 200-snapshot stream): signal eigenvalues within 1e-6."""
    g = PlantedModes(4096, sigma=1e-8, seed=0)
    X = g.snapshots(0, 200).T
    o = run_online(X, r_max=10)
    lam, V, b = o.eig()
    amp = np.abs(b) * np.linalg.norm(o.L @ V, axis=0)
    strong = lam[amp > 1e-3 * amp.max()]
    assert len(strong) == 6
    assert match_eigs(strong, g.planted_eigenvalues()) < 1e-6


def test_linear_system_one_step_identity():
    """x_{k+1} = A x_k with rank(A) <= r: L A~ L^T u^k = u^{k+1} exactly."""
    rng = np.random.default_rng(11)
    n, rk = 300, 5
    Uq, _ = np.linalg.qr(rng.standard_normal((n, rk)))
    core = rng.standard_normal((rk, rk))
    core = core / (1.05 * np.max(np.abs(np.linalg.eigvals(core))))
    A = Uq @ core @ Uq.T
    X = np.empty((n, 40))
    X[:, 0] = Uq @ rng.standard_normal(rk)
    for k in range(39):
        X[:, k + 1] = A @ X[:, k]
    o = run_online(X, r_max=8)
    assert o.rank == rk
    At = o.reduced_operator()
    for k in (3, 17, 38):
        pred = o.L @ (At @ (o.L.T @ X[:, k]))
        assert np.linalg.norm(pred - X[:, k + 1]) <= 1e-11 * np.linalg.norm(X[:, k + 1])


def test_rollout_matches_analytic_stream():
    """Noise-free planted stream: x(t) = generator's closed form for t in and beyond training."""
    g = PlantedModes(1000, mus=(1.0, 0.995), thetas=(0.013, 0.071), sigma=0.0, seed=4)
    X = g.snapshots(0, 60).T
    o = run_online(X, r_max=6)
    for t in (0, 1, 30.5, 59, 200, 1000):
        truth = g.clean(t)
        got = o.predict([t])[:, 0]
        assert np.linalg.norm(got - truth) <= 1e-9 * np.linalg.norm(truth), t
    # x(0) is the projection of u^0 onto span(L)
    x0 = o.predict([0])[:, 0]
    assert np.allclose(x0, o.L @ (o.L.T @ X[:, 0]), atol=1e-12 * np.abs(X).max())
    assert o.predict_imag_max([10.0]) < 1e-10 * np.abs(X).max()


def test_wake_eigen_angles_are_planted_frequencies():
    """Wake field: DMD angles = h omega dt (St = 0.22, Sec. 3), decay rates = exp(-gamma dt).

    The stream is exactly rank 11 but its slow transients separate only at the 1e-8
    level over 400 steps, so the incremental truncation (components below tau are
    dropped every step) perturbs the weakest modes at the truncation level: with a tight
    tau all 11 planted eigenvalues come back; with tau = 1e-10 the shedding harmonics
    (the Strouhal check) still do.
    """
    g = WakeField(nx=64, ny=32, sigma=0.0, seed=0)
    X = g.snapshots(0, 400).T
    planted = g.planted_eigenvalues()
    harmonics = planted[1:7]
    o = run_online(X, r_max=16, tau=1e-13)
    lam, V, b = o.eig()
    amp = np.abs(b) * np.linalg.norm(o.L @ V, axis=0)
    strong = lam[np.argsort(-amp)[:11]]
    assert amp[np.argsort(-amp)[11:]].max(initial=0) < 1e-6 * amp.max()
    assert match_eigs(strong, planted) < 1e-6
    got = strong[np.argmin(np.abs(strong[:, None] - harmonics[None, :]), axis=0)]
    assert np.max(np.abs(np.angle(got) - np.angle(harmonics))) < 1e-8
    o2 = run_online(X, r_max=16, tau=1e-10)
    lam2, V2, b2 = o2.eig()
    got2 = lam2[np.argmin(np.abs(lam2[:, None] - harmonics[None, :]), axis=0)]
    assert np.max(np.abs(got2 - harmonics)) < 1e-5


# ------------------------------------------------------------------ invariants
def test_truncation_bound_and_orthonormality():
    """Truncation active: every ingested snapshot is reconstructed by L L^T within the
    accumulated discarded mass; L stays orthonormal."""
    g = PlantedModes(800, mus=(1.0, 0.99, 0.97, 0.95), thetas=(0.01, 0.05, 0.11, 0.2),
                     sigma=1e-3, seed=9)
    X = g.snapshots(0, 120).T
    o = OnlineDMDRef(800, 10, 1e-10)
    bound_sum = 0.0
    for k in range(X.shape[1]):
        before = o.discarded_sq
        o.update(X[:, k])
        bound_sum += np.sqrt(o.discarded_sq - before)
    assert o.rank == 10
    G = o.L.T @ o.L
    assert np.max(np.abs(G - np.eye(10))) < 1e-12
    proj_err = np.linalg.norm(X[:, :-1] - o.L @ (o.L.T @ X[:, :-1]), axis=0)
    assert np.all(proj_err <= bound_sum * (1 + 1e-9) + 1e-12)
    assert bound_sum > 0  # truncation really was active


def test_rank_cap_keeps_largest():
    """With r_max below the data rank the kept singular values are the largest of K's."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((100, 30))
    o = run_online(X, r_max=4)
    assert o.rank == 4
    assert np.all(np.diff(o.S) <= 0)


def test_zero_leading_snapshot_anchor():
    """u^0 = 0: the basis starts at u^1, u^0's row of R is zero, so b = 0 and x(t) = 0."""
    g = PlantedModes(50, mus=(1.0,), thetas=(0.05,), sigma=0.0, seed=1)
    o = OnlineDMDRef(50, 4)
    o.update(np.zeros(50))
    for k in range(1, 8):
        o.update(g.snapshot(k))
    assert o.rank == 2
    assert np.all(o.r_first == 0)
    assert np.allclose(o.predict([5.0]), 0.0)
    # the operator is still learned from the later pairs
    lam, _, _ = o.eig()
    assert match_eigs(lam, g.planted_eigenvalues()) < 1e-9


def test_repeated_snapshot_adds_no_direction():
    """A snapshot already in span(L) adds no new direction (rho below threshold)."""
    rng = np.random.default_rng(8)
    o = OnlineDMDRef(40, 6)
    a = rng.standard_normal(40)
    for _ in range(5):
        o.update(a)
    assert o.rank == 1
    np.testing.assert_allclose(o.S, [2.0 * np.linalg.norm(a)], rtol=1e-13)  # ||[a a a a]|| = 2||a||
    lam, _, _ = o.eig()
    np.testing.assert_allclose(lam, [1.0], rtol=1e-13)


# ------------------------------------------------------------------ credibility check
def test_check_special_cases():
    """err = ||x(t)-x_fom||/||x_fom||: 0 at the prediction, 1/2 at twice it, 2 at minus it."""
    g = PlantedModes(300, sigma=0.0, seed=2)
    X = g.snapshots(0, 30).T
    o = run_online(X, r_max=8)
    xp = o.predict([31.0])[:, 0]
    err, ok = o.check(31.0, xp, 1e-5)
    assert err < 1e-15 and ok
    err, ok = o.check(31.0, 2 * xp, 1e-5)
    assert abs(err - 0.5) < 1e-14 and not ok
    err, ok = o.check(31.0, -xp, 1e-5)
    assert abs(err - 2.0) < 1e-14 and not ok
    err, ok = o.check(31.0, g.clean(31.0), 1e-5)
    assert err < 1e-10 and ok


def test_integer_horizons_equal_powers_of_the_reduced_operator():
    """Reading A21: for integer t, Phi Lambda^t Phi^+ u0 = L A~^t (S * r_first), the
    identity V Lambda^t V^-1 = A~^t with b = V^-1 (S * r_first).  The oracle's eigen-based
    rollout must equal the plain matrix power, on a stream whose operator has a complex
    pair, a decaying mode and a neutral one."""
    g = PlantedModes(600, mus=(1.0, 0.97, 0.9), thetas=(0.013, 0.071, 0.2), sigma=0.0, seed=5)
    X = g.snapshots(0, 40)
    o = run_online(X.T, r_max=12, tau=1e-12)
    A = o.reduced_operator()
    y = o.S * o.r_first
    for t in (0, 1, 7, 39, 40, 111):
        direct = o.L @ (np.linalg.matrix_power(A, t) @ y)
        via_eig = o.predict([float(t)])[:, 0]
        assert np.linalg.norm(direct - via_eig) <= 1e-9 * np.linalg.norm(via_eig), t
