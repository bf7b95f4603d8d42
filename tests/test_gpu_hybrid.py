"""The hybrid FOM/ROM step (odmd_hybrid_step, Sec. 2.1 Fig. 1 with the credibility test of
Sec. 2.2) against the same controller written with the oracle.

At every step the FOM state is given; once a model exists its prediction is taken when its
relative L2 distance to the FOM state is within tol, and the state taken joins the stream.
On a noise-free planted-mode stream the distances are above 1e-3 until the model has the
six modes and below 1e-9 afterwards (accepted predictions feed back, so they creep up from
1e-13), far from tol = 1e-8 on both sides, so both take the same decisions.  With noise the
decisions would sit near the tolerance and a rounding-level difference could flip one.
"""
import numpy as np
import pytest

from oracle import OnlineDMDRef
from synth import PlantedModes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def oracle_hybrid(n, r_max, slack, X, tol):
    ref = OnlineDMDRef(n, r_max, 1e-10)
    taken, accepted, errs = [], [], []
    for k in range(X.shape[0]):
        ok, err = False, np.inf
        if k >= 2 and ref.rank > 0:
            err, ok = ref.check(float(k), X[k], tol)
        s = ref.predict([float(k)])[:, 0] if ok else X[k].copy()
        ref.update(s)
        taken.append(s)
        accepted.append(bool(ok))
        errs.append(err)
    return ref, np.array(taken), accepted, errs


def test_hybrid_step_matches_oracle_controller():
    import paper_2311_18715_gb300 as pkg

    n, r_max, slack, tol = 4096, 6, 4, 1e-8
    X = PlantedModes(n, sigma=0.0, seed=0).snapshots(0, 60)
    ref, taken_ref, acc_ref, err_ref = oracle_hybrid(n, r_max, slack, X, tol)
    m = pkg.OnlineDMD(n, r_max, slack=slack, trunc_tol=1e-10)
    Xd = torch.from_numpy(X).cuda()
    taken, acc, errs = [], [], []
    for k in range(X.shape[0]):
        s, ok, err = m.hybrid_step(Xd[k], tol)
        taken.append(s.cpu().numpy())
        acc.append(ok)
        errs.append(err)
    assert acc == acc_ref
    assert 50 <= sum(acc) < len(acc)  # the ROM takes over once it has the modes
    # an accepted state is the model's own prediction and feeds the next update, so the two
    # streams part at rounding level and the difference grows with the feedback; what the
    # loop guarantees is that every state taken is within tol of the FOM state, so the two
    # sides' states are within 2 tol of each other (and so are the models they build)
    taken = np.array(taken)
    for k in range(len(taken)):
        ref_norm = np.linalg.norm(taken_ref[k])
        assert np.linalg.norm(taken[k] - X[k]) <= tol * np.linalg.norm(X[k]) * (1 + 1e-6)
        assert np.linalg.norm(taken[k] - taken_ref[k]) <= 2 * tol * ref_norm
    for e, er in zip(errs, err_ref):
        assert (np.isinf(e) and np.isinf(er)) or abs(e - er) <= 2 * tol
    np.testing.assert_allclose(m.singular_values(), ref.S, rtol=0, atol=2 * tol * ref.S[0])


def test_hybrid_step_rejects_aliasing_and_takes_fom_before_a_model():
    import paper_2311_18715_gb300 as pkg

    m = pkg.OnlineDMD(64, 4)
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    x = torch.ones(64, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.OdmdError):
        m.hybrid_step(x, out=x)
    for v in (z, z, x):  # zero leading snapshots: no model, the FOM state is taken
        s, ok, err = m.hybrid_step(v)
        assert not ok and np.isinf(err)
        assert torch.equal(s, v)
