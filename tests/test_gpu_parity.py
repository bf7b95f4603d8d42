"""Device path vs the FP64 oracle, element by element on identical seeded inputs.

Sizes span several 64-row tiles with a ragged tail; slack values exercise both the
append-only updates and the compaction of the tall basis.  Tolerances (FP64 mode):
eigenvalues 1e-10 relative for modes with amplitude >= 1e-6 of the largest, rollouts
1e-9 relative, singular values 1e-10 of sigma_1.
"""
import numpy as np
import pytest

from oracle import BatchDMD, OnlineDMDRef
from synth import PlantedModes, RandomPlanted, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def match_eigs(a, b):
    a = list(np.asarray(a, dtype=complex))
    b = list(np.asarray(b, dtype=complex))
    worst = 0.0
    for x in sorted(a, key=lambda z: -abs(z)):
        d = [abs(x - y) for y in b]
        i = int(np.argmin(d))
        worst = max(worst, d[i] / max(abs(x), 1e-300))
        b.pop(i)
    return worst


def run_pair(X, r_max, slack=16, tau=1e-10, prec="fp64", refine_every=0):
    import paper_2311_18715_gb300 as pkg

    dev = torch.device("cuda", 0)
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = pkg.OnlineDMD(X.shape[1], r_max, prec=prec, slack=slack, trunc_tol=tau, refine_every=refine_every)
    ref = OnlineDMDRef(X.shape[1], r_max, tau)
    Xd = torch.from_numpy(X).to(dev, dt)
    for k in range(X.shape[0]):
        m.update(Xd[k])
        ref.update(X[k].astype(np.float64) if prec == "fp64" else Xd[k].double().cpu().numpy())
    m.sync()
    m.eigs()  # surfaces any eigensolver status before predictions are compared
    return m, ref


def strong_eigs(lam, amp, frac=1e-6):
    lam = np.asarray(lam)
    amp = np.asarray(amp)
    return lam[amp >= frac * amp.max()]


def assert_horizons(got, want, bar, what=""):
    """Every predicted state against the oracle's, relative to that state's own norm, so that
    one poor horizon cannot hide under larger ones (rows are horizons)."""
    got, want = np.asarray(got), np.asarray(want)
    assert got.shape == want.shape, (got.shape, want.shape)
    for j in range(want.shape[0]):
        e = np.linalg.norm(got[j] - want[j]) / np.linalg.norm(want[j])
        assert e < bar, (what, j, e)


@pytest.mark.parametrize("slack", [0, 4, 16])
def test_planted_modes_4096(slack):
    g = PlantedModes(4096, sigma=1e-8, seed=0)
    X = g.snapshots(0, 200)
    m, ref = run_pair(X, 10, slack=slack)
    assert m.rank == ref.rank == 10
    S = np.array(m.singular_values())
    np.testing.assert_allclose(S, ref.S, rtol=0, atol=1e-10 * ref.S[0])
    lam, amp = m.eigs()
    lam_r, V_r, b_r = ref.eig()
    amp_r = np.abs(b_r) * np.linalg.norm(ref.L @ V_r, axis=0)
    s_dev = strong_eigs(lam, amp)
    s_ref = strong_eigs(lam_r, amp_r)
    assert len(s_dev) == len(s_ref) == 6
    assert match_eigs(s_dev, s_ref) < 1e-10
    ts = [0.0, 1.0, 99.5, 199.0, 200.0, 260.0]
    got = m.predict(ts).cpu().numpy()
    want = ref.predict(ts).T
    assert_horizons(got, want, 1e-9)
    for t in (200.0, 201.0):
        e_dev, _ = m.check(t, torch.from_numpy(g.snapshot(int(t))).cuda())
        e_ref, _ = ref.check(t, g.snapshot(int(t)))
        # |err_dev - err_ref| <= ||x_dev(t) - x_ref(t)|| / ||x_fom|| (triangle inequality),
        # so the rollout tolerance bounds it
        assert abs(e_dev - e_ref) <= 1e-9


@pytest.mark.parametrize("n,slack", [(1000, 0), (1000, 3), (777, 16), (64, 2), (33, 5)])
def test_random_stream_ragged_tiles(n, slack):
    """Random snapshots, truncation active (r_max < m), rows not a multiple of the tile."""
    rng = np.random.default_rng(n + slack)
    X = rng.standard_normal((40, n))
    X[:, : n // 2] *= 3.0
    m, ref = run_pair(X, 8, slack=slack)
    assert m.rank == ref.rank
    S = np.array(m.singular_values())
    np.testing.assert_allclose(S, ref.S, rtol=0, atol=1e-10 * ref.S[0])
    ts = [0.0, 17.0, 39.0, 40.0]
    got = m.predict(ts).cpu().numpy()
    want = ref.predict(ts).T
    assert_horizons(got, want, 1e-9)
    L = m.basis().cpu().numpy().T
    P = L @ L.T
    Pr = ref.L @ ref.L.T
    assert np.max(np.abs(P - Pr)) < 1e-9
    assert np.max(np.abs(L.T @ L - np.eye(L.shape[1]))) < 1e-12


def test_no_truncation_matches_batch_dmd():
    rng = np.random.default_rng(5)
    n, steps = 700, 31
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    X = np.empty((steps, n))
    X[0] = rng.standard_normal(n)
    for k in range(steps - 1):
        X[k + 1] = A @ X[k] + 0.1 * rng.standard_normal(n)
    m, ref = run_pair(X, 32, slack=8)
    B = BatchDMD(X.T, 32)
    assert m.rank == B.S.shape[0] == steps - 1
    np.testing.assert_allclose(m.singular_values(), B.S, rtol=1e-11)
    lam, _ = m.eigs()
    assert match_eigs(lam, B.lam) < 1e-9
    got = m.predict([0.0, 12.0, 30.0]).cpu().numpy()
    want = B.predict([0.0, 12.0, 30.0]).T
    assert_horizons(got, want, 1e-9)


def test_wake_field_small_grid():
    g = WakeField(nx=64, ny=32, sigma=1e-6, seed=0)
    X = g.snapshots(0, 300)
    m, ref = run_pair(X, 16, slack=16)
    assert m.rank == ref.rank
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    got = m.predict([300.0, 320.0]).cpu().numpy()
    want = ref.predict([300.0, 320.0]).T
    assert_horizons(got, want, 1e-9)


def _strong(ref, frac):
    lam, V, b = ref.eig()
    amp = np.abs(b) * np.linalg.norm(ref.L @ V, axis=0)
    return strong_eigs(lam, amp, frac)


def _core_svd_gesvd(K, tau, r_max):
    """The oracle's core SVD step with LAPACK's gesvd driver instead of gesdd (numpy's): the
    same mathematics, another FP64 rounding."""
    import scipy.linalg as sl

    U1, sig, V1t = sl.svd(K, lapack_driver="gesvd")
    keep = int(np.count_nonzero(sig > tau * sig[0])) if sig[0] > 0 else 0
    keep = max(1, min(keep, r_max))
    return U1[:, :keep], sig[:keep], V1t.T[:, :keep], float(np.sum(sig[keep:] ** 2))


def test_wake_full_size_bench_configuration(monkeypatch):
    """The benchmark's workload and launch configuration (512 x 256 x 3 grid, n = 393,216,
    r_max 40, slack 16): many tiles per CTA, every stage of the tall pipelines refilled,
    compactions included.  The oracle runs the same stream at full size.

    Rollouts (every state within 1e-9 relative), check errors (1e-9) and singular values
    (1e-10 of sigma_1) are held to the flat FP64 bars.  The strong eigenvalues are not
    determined to 1e-10 by FP64 arithmetic at this configuration: with r_max below the number
    of noise directions each update chooses among nearly equal noise singular values, and
    the strong eigenvalues move with the directions kept.  The oracle itself, run with
    LAPACK's gesvd driver for the core SVD instead of gesdd (the only change), moves them by
    ~5e-10 (5.35e-10 on an x86 host).  This test computes that spread on the machine it runs
    on and bars the device at max(1e-10, 2 x spread): an FP64 implementation of the method
    is held to the agreement of two FP64 implementations of the oracle.  The noise-subspace
    modes (amplitude ~1e-6 of the largest, noise std 1e-6) are excluded by an amplitude
    threshold of 1e-3 of the largest (reading A12)."""
    import oracle.odmd_ref as odmd_ref

    g = WakeField(512, 256, sigma=1e-6, seed=0)
    X = g.snapshots(0, 120)
    m, ref = run_pair(X, 40, slack=16)
    monkeypatch.setattr(odmd_ref, "core_svd_truncated", _core_svd_gesvd)
    alt = OnlineDMDRef(X.shape[1], 40, 1e-10)
    for k in range(X.shape[0]):
        alt.update(X[k])
    monkeypatch.undo()
    assert m.rank == ref.rank == alt.rank == 40
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    s_ref = _strong(ref, 1e-3)
    spread = match_eigs(_strong(alt, 1e-3), s_ref)
    lam, amp = m.eigs()
    s_dev = strong_eigs(lam, amp, 1e-3)
    assert len(s_dev) == len(s_ref) >= 7
    err = match_eigs(s_dev, s_ref)
    print(f"full-size wake: strong-eigenvalue error {err:.3e}, spread of the two FP64 oracles {spread:.3e}")
    assert err <= max(1e-10, 2 * spread), (err, spread)
    ts = [120.0, 121.0, 135.0, 150.0]
    assert_horizons(m.predict(ts).cpu().numpy(), ref.predict(ts).T, 1e-9)
    x_fom = g.snapshot(125)
    e_dev, _ = m.check(125.0, torch.from_numpy(x_fom).cuda())
    e_ref, _ = ref.check(125.0, x_fom)
    assert abs(e_dev - e_ref) <= 1e-9


def test_many_tiles_per_cta_small_rank():
    """Long stream rows with a small rank: short tiles, many of them per CTA, so the tall
    passes cycle through their stage rings quickly (n ragged against every tile size)."""
    g = RandomPlanted(262147, seed=11)
    X = g.snapshots(0, 40)
    m, ref = run_pair(X, 6, slack=3)
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    got = m.predict([40.0, 41.5]).cpu().numpy()
    want = ref.predict([40.0, 41.5]).T
    assert_horizons(got, want, 1e-9)


def test_edge_cases():
    import paper_2311_18715_gb300 as pkg

    dev = torch.device("cuda", 0)
    # n = 1: rank one at most
    m, ref = run_pair(np.array([[1.0], [2.0], [4.0], [8.0]]), 3, slack=0)
    assert m.rank == 1
    lam, _ = m.eigs()
    np.testing.assert_allclose(lam, [2.0], rtol=1e-14)
    # zero first snapshot: the model starts at u^1, predictions anchored at u^0 = 0
    g = PlantedModes(200, mus=(1.0,), thetas=(0.05,), sigma=0.0, seed=1)
    X = g.snapshots(0, 10)
    X[0] = 0.0
    m, ref = run_pair(X, 4, slack=2)
    assert m.rank == ref.rank == 2
    assert np.max(np.abs(m.predict([5.0]).cpu().numpy())) == 0.0
    # a repeated snapshot adds no direction
    a = np.random.default_rng(2).standard_normal(300)
    m, ref = run_pair(np.stack([a] * 6), 5, slack=1)
    assert m.rank == 1
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=1e-13)
    # state errors
    mm = pkg.OnlineDMD(10, 2)
    with pytest.raises(pkg.OdmdError):
        mm.predict([1.0])
    mm.update(torch.zeros(10, dtype=torch.float64, device=dev))
    with pytest.raises(pkg.OdmdError):
        mm.check(1.0, torch.zeros(10, dtype=torch.float64, device=dev))


def test_clustered_tiny_singular_values():
    """A random planted-mode stream whose noise singular values sit ~1e-10 below the
    largest, packed with relative gaps ~1e-4: offsets between such poles square to 1e-23,
    and a secular-equation step formed in FP32 without rescaling underflowed and stalled.
    The stream is drawn on the device (noise from torch's seeded generator) and handed to
    the oracle as the same bytes."""
    n, r_max = 1637390, 34
    gen = RandomPlanted(n, seed=1010)
    fields = torch.from_numpy(gen.fields).cuda()
    g = torch.Generator(device="cuda")
    X = []
    for k in range(125):
        c = torch.from_numpy(np.asarray(gen.coefficients(k))).cuda()
        g.manual_seed(1_000_003 * (gen.seed + 1) + k)
        X.append(c @ fields + gen.sigma * torch.randn(n, generator=g, device="cuda", dtype=torch.float64))
    X = torch.stack(X).cpu().numpy()
    del fields
    m, ref = run_pair(X, r_max, slack=16)
    assert m.rank == ref.rank
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    got = m.predict([125.0]).cpu().numpy()
    want = ref.predict([125.0]).T
    assert_horizons(got, want, 1e-9)


@pytest.mark.parametrize("stream", ["planted", "wake"])
def test_powers_and_eigen_paths_agree(stream):
    """Integer horizons take their coefficients from powers of the reduced operator, any
    other horizon from the eigen-cache (V Lambda^t b); both are the same quantity (reading
    A21).  A call with only integer horizons takes the first path, the same horizons with
    a fractional one added take the second: both must match each other and the oracle."""
    if stream == "planted":
        X = PlantedModes(4096, sigma=1e-8, seed=0).snapshots(0, 200)
        r_max, ts = 10, [0.0, 1.0, 150.0, 199.0, 200.0, 260.0]
    else:
        X = WakeField(nx=64, ny=32, sigma=1e-6, seed=0).snapshots(0, 300)
        r_max, ts = 16, [0.0, 299.0, 300.0, 301.0, 320.0]
    m, ref = run_pair(X, r_max, slack=4)
    by_powers = m.predict(ts).cpu().numpy()
    by_eigen = m.predict(ts + [0.5]).cpu().numpy()[: len(ts)]
    want = ref.predict(ts).T
    for got in (by_powers, by_eigen):
        for j in range(len(ts)):
            assert np.linalg.norm(got[j] - want[j]) / np.linalg.norm(want[j]) < 1e-9, (stream, ts[j])
    scale = np.linalg.norm(want, axis=1)
    assert np.max(np.linalg.norm(by_powers - by_eigen, axis=1) / scale) < 1e-10


def test_powers_path_resumes_from_earlier_calls():
    """Integer-horizon calls start from the vector A~^t y that the previous call of the same
    model left at its first or last horizon, when that horizon is not after the first one
    asked for; a new snapshot or a refinement makes a new model and the vectors stale.  Every
    call must agree with the oracle and with a call that started from t = 0."""
    X = WakeField(nx=64, ny=32, sigma=1e-6, seed=1).snapshots(0, 301)
    m, ref = run_pair(X[:300], 16, slack=4)
    ts = [float(t) for t in range(300, 350)]
    first = m.predict(ts).cpu().numpy()                   # from t = 0
    want = ref.predict(ts).T
    scale = np.linalg.norm(want, axis=1)
    assert np.max(np.linalg.norm(first - want, axis=1) / scale) < 1e-9
    xs = torch.from_numpy(np.ascontiguousarray(want)).cuda()
    for t in (300.0, 349.0, 360.0, 305.0, 300.0):         # first horizon, last, later, earlier
        j = int(t) - 300
        x_t = xs[j] if j < len(ts) else torch.from_numpy(np.ascontiguousarray(ref.predict([t])[:, 0])).cuda()
        err, _ = m.check(t, x_t)
        assert err < 1e-9, t
    again = m.predict(ts[5:]).cpu().numpy()               # resumes from t = 305 or 300
    assert np.max(np.linalg.norm(again - first[5:], axis=1) / scale[5:]) < 1e-11
    m.update(torch.from_numpy(X[300]).cuda())             # a new model: no reuse
    ref.update(X[300])
    got = m.predict(ts[1:]).cpu().numpy()
    want2 = ref.predict(ts[1:]).T
    assert np.max(np.linalg.norm(got - want2, axis=1) / np.linalg.norm(want2, axis=1)) < 1e-9


def _driven_linear_stream(n, steps, seed):
    """A damped random linear system driven by noise, x_{k+1} = 0.97 A x_k + 0.3 xi_k with
    A Gaussian / sqrt(n): every snapshot adds a direction, so the rank reaches any r_max
    and the truncation and compaction run at every update."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n) * 0.97
    X = np.empty((steps, n))
    X[0] = rng.standard_normal(n)
    for k in range(steps - 1):
        X[k + 1] = A @ X[k] + 0.3 * rng.standard_normal(n)
    return X


@pytest.mark.parametrize("slack", [32, 0])
def test_largest_rank_and_slack(slack):
    """r_max and slack at their limits (64 and 32: 96 basis columns, the widest tiles and
    the largest core and reduced operator), n = 4999 rows (a ragged last tile), 140
    snapshots with more than 64 active directions.  The oracle's own response to a 1e-12
    relative perturbation of the snapshots is 5e-14 of sigma_1 in the singular values,
    3e-12 relative in the predictions and 3e-14 in the projector, far below the bars.
    Predictions take two launches (65 horizons); the refinement runs at its largest size."""
    X = _driven_linear_stream(4999, 140, 11)
    m, ref = run_pair(X, 64, slack=slack, refine_every=1000)  # scratch reserved, refined only on demand
    assert m.rank == ref.rank == 64
    np.testing.assert_allclose(np.array(m.singular_values()), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    L = m.basis().cpu().numpy().T
    assert np.max(np.abs(L @ L.T - ref.L @ ref.L.T)) < 1e-9
    assert np.max(np.abs(L.T @ L - np.eye(64))) < 1e-12
    ts = [float(t) for t in range(0, 130, 2)]
    want = ref.predict(ts).T
    for got in (m.predict(ts).cpu().numpy(), m.predict(ts[:-1] + [128.5]).cpu().numpy()[:-1]):
        assert_horizons(got, want[: got.shape[0]], 1e-9)
    err, _ = m.check(139.0, torch.from_numpy(X[139]).cuda())
    assert abs(err - ref.check(139.0, X[139])[0]) < 1e-9
    m.refine()
    np.testing.assert_allclose(np.array(m.singular_values()), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    L = m.basis().cpu().numpy().T
    assert np.max(np.abs(L.T @ L - np.eye(64))) < 1e-13
    got = m.predict(ts).cpu().numpy()
    assert_horizons(got, want, 1e-9)
