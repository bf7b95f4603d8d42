"""Tall x small products on the tensor cores (split.cu: an exact 7-bit digit split of the
basis and of the small factor, bfloat16 tcgen05.mma into exact FP32 group sums,
double-float epilogue): the multi-horizon rollout and the compaction of the product-form
basis, against the oracle and against the CUDA-core paths.

Rollouts: every predicted state within 1e-9 relative of the oracle's (the FP64
reconstruction tolerance) and within 1e-12 relative of the CUDA-core rollout of the same
model state (a checkpoint of the tensor-core handle loaded into a CUDA-core handle; both
rollouts are exact up to double-float rounding, 2^-48 per element over at most 64 columns).
Horizon counts cover the smallest tensor-core call (8), a full launch (64), a launch split in
two (65: 64 on the tensor cores, 1 on the CUDA cores) and the benchmark's 50; rows are
ragged against the 128-row tile.  Compaction: on a stream whose rank cap equals its planted
rank (every noise direction is dropped again, so rounding differences stay small), a handle that
compacts on the tensor cores and one that compacts on the CUDA cores agree to 1e-12 of
sigma_1 in the singular values and 1e-10 in predictions, and both match the oracle."""
import numpy as np
import pytest

from oracle import OnlineDMDRef
from synth import PlantedModes, RandomPlanted, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(got, want):
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _fed(X, r_max, slack, tensor_cores=True, ref=False):
    import paper_2311_18715_gb300 as pkg

    m = pkg.OnlineDMD(X.shape[1], r_max, slack=slack, tensor_cores=tensor_cores)
    o = OnlineDMDRef(X.shape[1], r_max, 1e-10) if ref else None
    Xd = torch.from_numpy(X).cuda()
    for k in range(X.shape[0]):
        m.update(Xd[k])
        if o is not None:
            o.update(X[k])
    return m, o


def _same_state_cuda_cores(tc):
    import paper_2311_18715_gb300 as pkg

    cc = pkg.OnlineDMD(tc.n, tc.r_max, slack=int(tc.cfg.slack), tensor_cores=False)
    cc.load(tc.save())
    return cc


@pytest.mark.parametrize("case", ["planted", "random_ragged", "wake"])
def test_tensor_core_rollout_against_oracle_and_cuda_cores(case):
    if case == "planted":
        X, r, sl = PlantedModes(4096, sigma=1e-8, seed=0).snapshots(0, 120), 10, 4
    elif case == "random_ragged":
        X, r, sl = RandomPlanted(50001, seed=5).snapshots(0, 70), 24, 8
    else:
        X, r, sl = WakeField(128, 64, sigma=1e-6, seed=2).snapshots(0, 150), 40, 16  # the benchmark's cap
    tc, ref = _fed(X, r, sl, ref=True)
    cc = _same_state_cuda_cores(tc)
    assert tc.rank == ref.rank == cc.rank
    k = X.shape[0]
    for nh in (8, 50, 64, 65):
        ts = [float(k - 3 + h) for h in range(nh)]
        want = ref.predict(ts).T
        got = tc.predict(ts).cpu().numpy()
        base = cc.predict(ts).cpu().numpy()
        assert np.max(_rel(got, want)) < 1e-9, (case, nh, np.max(_rel(got, want)))
        assert np.max(_rel(got, base)) < 1e-12, (case, nh, np.max(_rel(got, base)))


def test_tensor_core_rollout_full_size_benchmark_horizons():
    """The benchmark's configuration and call: n = 393,216 (3072 tiles over the SMs, every
    CTA through many tiles), cap 56, 50 integer horizons, against the CUDA-core rollout of the
    same state."""
    X = WakeField(512, 256, sigma=1e-6, seed=0).snapshots(0, 60)
    tc, _ = _fed(X, 40, 16)
    cc = _same_state_cuda_cores(tc)
    ts = [float(60 + h) for h in range(50)]
    got = tc.predict(ts).cpu().numpy()
    base = cc.predict(ts).cpu().numpy()
    assert np.isfinite(got).all()
    assert np.max(_rel(got, base)) < 1e-12


def test_tensor_core_rollout_forms_the_pending_column():
    """Predictions straight after updates that appended a basis column: the tensor-core
    rollout forms that column from the stored residual, uses it and writes it to the basis.
    Handle a predicts after every update; its twin b has the column written by the separate
    flush pass (save() flushes) and its states come from a CUDA-core handle loaded from it.
    States within 1e-12 of b's and 1e-9 of the oracle's at 8, 50 and 65 horizons (65: the
    second launch, on the CUDA cores, reads the column the first one wrote); afterwards the
    bases agree to 1e-12 (a column left unwritten would not) and both handles go on alike."""
    import paper_2311_18715_gb300 as pkg

    X = WakeField(128, 64, sigma=1e-6, seed=2).snapshots(0, 160)
    n = X.shape[1]
    a = pkg.OnlineDMD(n, 40, slack=16)
    b = pkg.OnlineDMD(n, 40, slack=16)
    o = OnlineDMDRef(n, 40, 1e-10)
    Xd = torch.from_numpy(X).cuda()
    for k in range(X.shape[0]):
        a.update(Xd[k])
        b.update(Xd[k])
        o.update(X[k])
        if k >= 138:
            nh = (8, 50, 65)[k % 3]
            ts = [float(k - 2 + h) for h in range(nh)]
            got = a.predict(ts).cpu().numpy()
            base = _same_state_cuda_cores(b).predict(ts).cpu().numpy()
            want = o.predict(ts).T
            assert np.max(_rel(got, base)) < 1e-12, (k, nh, np.max(_rel(got, base)))
            assert np.max(_rel(got, want)) < 1e-9, (k, nh, np.max(_rel(got, want)))
            La, Lb = a.basis().cpu().numpy(), b.basis().cpu().numpy()
            assert La.shape == Lb.shape
            assert np.max(np.abs(La - Lb)) < 1e-12, (k, np.max(np.abs(La - Lb)))
    assert a.counts() == b.counts()
    Sa, Sb = np.array(a.singular_values()), np.array(b.singular_values())
    assert np.max(np.abs(Sa - Sb)) <= 1e-12 * Sb[0]


@pytest.mark.parametrize("slack,n", [(2, 4096), (5, 100003)])
def test_tensor_core_compaction_against_cuda_cores_and_oracle(slack, n):
    # rank cap = the planted rank: every snapshot's noise (std 1e-8) adds a direction that the
    # truncation drops again, so columns are appended and compacted, with no choice among
    # nearly equal directions
    X = PlantedModes(n, sigma=1e-8, seed=3).snapshots(0, 140)
    tc, ref = _fed(X, 6, slack, ref=True)
    cc, _ = _fed(X, 6, slack, tensor_cores=False)
    assert tc.counts()[1] > 20 and tc.counts() == cc.counts()  # many compactions, the same ones
    S, Sc = np.array(tc.singular_values()), np.array(cc.singular_values())
    assert np.max(np.abs(S - Sc)) <= 1e-12 * Sc[0]
    np.testing.assert_allclose(S, ref.S, rtol=0, atol=1e-10 * ref.S[0])
    ts = [float(h) for h in range(130, 150)]
    got, base, want = tc.predict(ts).cpu().numpy(), cc.predict(ts).cpu().numpy(), ref.predict(ts).T
    assert np.max(_rel(got, base)) < 1e-10
    assert np.max(_rel(got, want)) < 1e-9
    L = tc.basis().cpu().numpy()
    assert np.max(np.abs(L @ L.T - np.eye(L.shape[0]))) < 1e-12


def _fed_prec(X, r_max, slack, prec, tensor_cores):
    import paper_2311_18715_gb300 as pkg

    m = pkg.OnlineDMD(X.shape[1], r_max, prec=prec, slack=slack, tensor_cores=tensor_cores)
    Xd = torch.from_numpy(X).cuda().to(m.dtype)
    for k in range(X.shape[0]):
        m.update(Xd[k])
    return m


@pytest.mark.parametrize("case", ["random_ragged", "wake_cap80"])
def test_tensor_core_rollout_fp32_storage(case):
    """FP32 storage on the tensor cores: one staged plane and up to 96 basis columns (cap 80
    here lies past the double-float path's 64).  The rollout of a model state equals the
    CUDA-core rollout of the same state (a checkpoint loaded into a CUDA-core handle) to
    1e-12 per horizon (both multiply the stored FP32 basis by double-float coefficients), at
    8, 50 and 65 horizons; a prediction straight after an update forms the pending column as
    stored (rounded to FP32) and the basis then matches the flushed one to one FP32 unit."""
    import paper_2311_18715_gb300 as pkg

    if case == "random_ragged":
        X, r, sl = RandomPlanted(50001, seed=5).snapshots(0, 70), 24, 8
    else:
        X, r, sl = WakeField(128, 64, sigma=1e-6, seed=2).snapshots(0, 150), 64, 16
    tc = _fed_prec(X, r, sl, "fp32", True)
    twin = _fed_prec(X, r, sl, "fp32", True)
    cc = pkg.OnlineDMD(tc.n, tc.r_max, prec="fp32", slack=sl, tensor_cores=False)
    cc.load(twin.save())  # the pending column written by the flush
    k = X.shape[0]
    for nh in (8, 50, 65):
        ts = [float(k - 3 + h) for h in range(nh)]
        got = tc.predict(ts).double().cpu().numpy()
        base = cc.predict(ts).double().cpu().numpy()
        assert np.isfinite(got).all()
        assert np.max(_rel(got, base)) < 1e-6, (case, nh, np.max(_rel(got, base)))
    La, Lb = tc.basis().double().cpu().numpy(), cc.basis().double().cpu().numpy()
    assert La.shape == Lb.shape
    assert np.max(np.abs(La - Lb)) <= 2.0 ** -23 * np.max(np.abs(Lb)), np.max(np.abs(La - Lb))
    # with the same stored column, the two rollouts agree to 1e-12 of each horizon's scale
    # before their outputs are rounded to the FP32 of the snapshots: every element within
    # that plus one FP32 unit of itself (the two sums may lie on either side of a rounding
    # boundary)
    tc2 = pkg.OnlineDMD(tc.n, tc.r_max, prec="fp32", slack=sl, tensor_cores=True)
    tc2.load(twin.save())
    ts = [float(k + h) for h in range(50)]
    got, base = tc2.predict(ts).cpu().numpy(), cc.predict(ts).cpu().numpy()
    assert got.dtype == base.dtype == np.float32
    d = np.abs(got.astype(np.float64) - base.astype(np.float64))
    scale = np.max(np.abs(base), axis=1, keepdims=True).astype(np.float64)
    bound = np.spacing(np.abs(base)).astype(np.float64) + 1e-12 * scale
    assert np.all(d <= bound), np.max(d / bound)


def test_tensor_core_compaction_fp32_storage():
    """The FP32 compaction on the tensor cores (the product rounded to FP32 as stored) against
    the CUDA-core one on a stream that compacts often: the same compactions, singular values
    within 1e-6 of sigma_1 of each other and 1e-5 of the oracle's, predictions within 1e-5 of
    each other and of the oracle per horizon."""
    X = PlantedModes(4096, sigma=1e-5, seed=3).snapshots(0, 140)
    tc = _fed_prec(X, 6, 5, "fp32", True)
    cc = _fed_prec(X, 6, 5, "fp32", False)
    ref = OnlineDMDRef(X.shape[1], 6, 1e-10)
    for k in range(X.shape[0]):
        ref.update(X[k].astype(np.float32).astype(np.float64))
    assert tc.counts()[1] > 15 and tc.counts() == cc.counts()
    S, Sc = np.array(tc.singular_values()), np.array(cc.singular_values())
    assert np.max(np.abs(S - Sc)) <= 1e-6 * Sc[0]
    assert np.max(np.abs(S - ref.S)) <= 1e-5 * ref.S[0]
    ts = [float(h) for h in range(130, 150)]
    got, base, want = (tc.predict(ts).double().cpu().numpy(), cc.predict(ts).double().cpu().numpy(),
                       ref.predict(ts).T)
    assert np.max(_rel(got, base)) < 1e-5, np.max(_rel(got, base))
    assert np.max(_rel(got, want)) < 1e-5, np.max(_rel(got, want))


@pytest.mark.parametrize("prec,r,sl", [("fp64", 40, 16), ("fp64", 6, 2), ("fp32", 24, 8)])
def test_pipelined_updates_equal_serial_updates(prec, r, sl):
    """Pipelined updates (an update's core SVD and operator update beside the next update's
    pass over the basis, the default) against updates run one after another
    (ODMD_NO_PIPELINE): bitwise the same singular values, counts, basis and predictions,
    read back at several points of the stream (each read settles the pending update), over
    stretches that compact (slack 2) and that do not, and after a checkpoint round trip."""
    import paper_2311_18715_gb300 as pkg

    X = (WakeField(128, 64, sigma=1e-6, seed=4).snapshots(0, 90) if r == 40 else
         PlantedModes(8192, sigma=1e-6, seed=4).snapshots(0, 90))
    a = pkg.OnlineDMD(X.shape[1], r, prec=prec, slack=sl)
    b = pkg.OnlineDMD(X.shape[1], r, prec=prec, slack=sl, pipeline=False)
    Xd = torch.from_numpy(X).cuda().to(a.dtype)
    for k in range(X.shape[0]):
        a.update(Xd[k])
        b.update(Xd[k])
        if k in (5, 33, 34, 61, 89):
            assert a.singular_values() == b.singular_values(), k
            assert a.counts() == b.counts(), k
            ts = [float(k + h) for h in range(10)]
            assert torch.equal(a.predict(ts), b.predict(ts)), k
            assert torch.equal(a.basis(), b.basis()), k
    assert b.counts()[1] > 0 or sl == 16
    c = pkg.OnlineDMD(X.shape[1], r, prec=prec, slack=sl)
    c.load(a.save())
    for k in range(X.shape[0] - 20, X.shape[0]):
        a.update(Xd[k])
        c.update(Xd[k])
    ts = [float(100 + h) for h in range(50)]
    assert torch.equal(a.predict(ts), c.predict(ts))
