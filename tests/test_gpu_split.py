"""Multi-horizon rollouts on the tensor cores (split.cu: an exact 7-bit digit split of the
basis and the coefficients, bfloat16 tcgen05.mma into exact FP32 group sums, double-float
epilogue) against the oracle and against the CUDA-core path of the same stream.

Bars: every predicted state within 1e-9 relative of the oracle's (the FP64 reconstruction
tolerance), and within 1e-12 relative of the CUDA-core rollout (both paths are exact up to
double-float rounding: 2^-48 relative per element, summed over at most 64 columns).  The
horizon counts cover the smallest tensor-core call (8), a full launch (64), a launch split
in two (65: 64 on the tensor cores, 1 on the CUDA cores) and the benchmark's 50; rows are
ragged against the 128-row tile."""
import numpy as np
import pytest

from oracle import OnlineDMDRef
from synth import PlantedModes, RandomPlanted, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(X, r_max, slack):
    import paper_2311_18715_gb300 as pkg

    tc = pkg.OnlineDMD(X.shape[1], r_max, slack=slack)
    cc = pkg.OnlineDMD(X.shape[1], r_max, slack=slack, tensor_cores=False)
    ref = OnlineDMDRef(X.shape[1], r_max, 1e-10)
    Xd = torch.from_numpy(X).cuda()
    for k in range(X.shape[0]):
        tc.update(Xd[k])
        cc.update(Xd[k])
        ref.update(X[k])
    return tc, cc, ref


def _rel(got, want):
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


@pytest.mark.parametrize("case", ["planted", "random_ragged", "wake"])
def test_tensor_core_rollout_against_oracle_and_cuda_cores(case):
    if case == "planted":
        X, r, sl = PlantedModes(4096, sigma=1e-8, seed=0).snapshots(0, 120), 10, 4
    elif case == "random_ragged":
        X, r, sl = RandomPlanted(50001, seed=5).snapshots(0, 70), 24, 8
    else:
        X, r, sl = WakeField(128, 64, sigma=1e-6, seed=2).snapshots(0, 150), 40, 16  # the benchmark's cap
    tc, cc, ref = _pair(X, r, sl)
    assert tc.rank == ref.rank
    k = X.shape[0]
    for nh in (8, 50, 64, 65):
        ts = [float(k - 3 + h) for h in range(nh)]
        want = ref.predict(ts).T
        got = tc.predict(ts).cpu().numpy()
        base = cc.predict(ts).cpu().numpy()
        assert np.max(_rel(got, want)) < 1e-9, (case, nh, np.max(_rel(got, want)))
        assert np.max(_rel(got, base)) < 1e-12, (case, nh, np.max(_rel(got, base)))
        assert np.max(_rel(base, want)) < 1e-9


def test_tensor_core_rollout_full_size_benchmark_horizons():
    """The benchmark's configuration and call: n = 393,216 (3072 tiles over the SMs, every
    CTA through many tiles), cap 56, 50 integer horizons, against the CUDA-core path."""
    X = WakeField(512, 256, sigma=1e-6, seed=0).snapshots(0, 60)
    import paper_2311_18715_gb300 as pkg

    tc = pkg.OnlineDMD(X.shape[1], 40, slack=16)
    cc = pkg.OnlineDMD(X.shape[1], 40, slack=16, tensor_cores=False)
    Xd = torch.from_numpy(X).cuda()
    for x in Xd:
        tc.update(x)
        cc.update(x)
    ts = [float(60 + h) for h in range(50)]
    got = tc.predict(ts).cpu().numpy()
    base = cc.predict(ts).cpu().numpy()
    assert np.isfinite(got).all()
    assert np.max(_rel(got, base)) < 1e-12
