"""Reduced-precision storage of the tall basis (FP32) against the FP64 oracle.

The oracle runs on the same float32 snapshots (widened to float64).  With the basis held in
FP32 (unit roundoff 2^-24) and compensated arithmetic, the measured errors are: singular
values <= 1e-6 of sigma_1, orthogonality of L within 1e-6, and rollouts within 1e-5 relative
up to 20 steps past the data (the eigenvalues carry ~1e-8 relative error, which t steps of
Lambda^t multiply by t).  The bars below are those figures.
"""
import numpy as np
import pytest

from oracle import OnlineDMDRef
from synth import PlantedModes, RandomPlanted, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_fp32(X, r_max, slack):
    import paper_2311_18715_gb300 as pkg

    dev = torch.device("cuda", 0)
    m = pkg.OnlineDMD(X.shape[1], r_max, prec="fp32", slack=slack, trunc_tol=1e-10)
    ref = OnlineDMDRef(X.shape[1], r_max, 1e-10)
    Xd = torch.from_numpy(X).to(dev, torch.float32)
    for k in range(X.shape[0]):
        m.update(Xd[k])
        ref.update(Xd[k].double().cpu().numpy())
    m.sync()
    return m, ref, Xd


@pytest.mark.parametrize("case", ["planted4096", "wake64x32", "random262147", "wake512x256"])
def test_fp32_storage_against_oracle(case):
    if case == "planted4096":
        # rank cap = the six planted directions: the noise here (std 1e-8) is below FP32
        # resolution, so extra kept directions hold rounding noise whose eigenvalues are
        # set by rounding alone; one slightly outside the unit circle, anchored at u^0 and
        # raised to the 200th power, would decide the rollout (reading A12)
        X, r, sl = PlantedModes(4096, sigma=1e-8, seed=0).snapshots(0, 200), 6, 4
    elif case == "wake64x32":
        X, r, sl = WakeField(64, 32, sigma=1e-6, seed=0).snapshots(0, 300), 16, 16
    elif case == "random262147":
        X, r, sl = RandomPlanted(262147, seed=11).snapshots(0, 40), 6, 3
    else:
        X, r, sl = WakeField(512, 256, sigma=1e-6, seed=0).snapshots(0, 120), 40, 16
    m, ref, Xd = run_fp32(X, r, sl)
    assert m.rank == ref.rank
    S = np.array(m.singular_values())
    assert np.max(np.abs(S - ref.S)) <= 1e-6 * ref.S[0]
    k = X.shape[0]
    ts = [float(k), float(k + 20)]
    got = m.predict(ts).double().cpu().numpy()
    want = ref.predict(ts).T
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5
    L = m.basis().double().cpu().numpy().T
    assert np.max(np.abs(L.T @ L - np.eye(L.shape[1]))) <= 1e-6
    # the credibility check reads float snapshots in this mode
    e_dev, _ = m.check(float(k - 1), Xd[k - 1])
    e_ref, _ = ref.check(float(k - 1), Xd[k - 1].double().cpu().numpy())
    assert abs(e_dev - e_ref) <= 1e-5
