"""Device pairs model (FOM-only updates) against the pair oracle, through the C ABI.

Bars as for the snapshot stream: singular values 1e-10 of sigma_1, predictions 1e-9
relative to the state's norm.
"""
import numpy as np
import pytest

from oracle import OnlineDMDPairsRef, hybrid_fom_updates

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair_models(n, r_max, tau=1e-10):
    import paper_2311_18715_gb300 as pkg

    return pkg.OnlineDMDPairs(n, r_max, trunc_tol=tau), OnlineDMDPairsRef(n, r_max, tau)


def _feed(dev, ref, X, Y):
    for i in range(X.shape[1]):
        dev.update(torch.from_numpy(np.ascontiguousarray(X[:, i])).cuda(),
                   torch.from_numpy(np.ascontiguousarray(Y[:, i])).cuda())
        ref.update(X[:, i], Y[:, i])


def _low_rank_map(n, k, seed):
    rng = np.random.default_rng(seed)
    B, _ = np.linalg.qr(rng.standard_normal((n, k)))
    W = rng.standard_normal((k, k)) + 3 * np.eye(k)
    lam = rng.uniform(0.6, 0.99, k) * np.sign(rng.standard_normal(k))
    C = W @ np.diag(lam) @ np.linalg.inv(W)
    return B @ C @ B.T, B


def _compare(dev, ref, u, ts, bar=1e-9):
    s_dev = np.array(dev.singular_values())
    assert len(s_dev) == ref.rank
    np.testing.assert_allclose(s_dev, ref.S, rtol=0, atol=1e-10 * ref.S[0])
    got = dev.predict(torch.from_numpy(np.ascontiguousarray(u)).cuda(), ts).cpu().numpy()
    for j, t in enumerate(ts):
        want = ref.step(u, int(t))
        assert np.linalg.norm(got[j] - want) <= bar * np.linalg.norm(u), (t, np.linalg.norm(got[j] - want))


def test_scattered_pairs_of_a_low_rank_map():
    """Pairs (x_i, A x_i) with x_i drawn at random in A's range, n = 3001 rows."""
    n, k = 3001, 8
    A, B = _low_rank_map(n, k, 1)
    rng = np.random.default_rng(2)
    X = B @ rng.standard_normal((k, k + 4))
    dev, ref = _pair_models(n, 16)
    _feed(dev, ref, X, A @ X)
    assert dev.rank == ref.rank == k and dev.pairs == k + 4
    u = B @ rng.standard_normal(k)
    _compare(dev, ref, u, [0.0, 1.0, 2.0, 5.0, 40.0])
    # and the model is the map itself on its range
    got = dev.predict(torch.from_numpy(u).cuda(), [3.0]).cpu().numpy()[0]
    assert np.linalg.norm(got - np.linalg.matrix_power(A, 3) @ u) <= 1e-9 * np.linalg.norm(u)


@pytest.mark.parametrize("n,r_max,m", [(777, 8, 30), (2000, 64, 90)])
def test_random_pairs_with_truncation(n, r_max, m):
    """Random (x, y) pairs with more directions than r_max: truncation at every update, and
    at r_max 64 the largest core (65 x 65) and rotation."""
    rng = np.random.default_rng(n + r_max)
    X = rng.standard_normal((n, m)) * np.linspace(1.0, 3.0, m)[None, :]
    Y = rng.standard_normal((n, m))
    dev, ref = _pair_models(n, r_max)
    _feed(dev, ref, X, Y)
    assert dev.rank == ref.rank == r_max
    _compare(dev, ref, X[:, -1], [0.0, 1.0, 2.0])


def test_zero_x_is_skipped_and_no_model_is_refused():
    import paper_2311_18715_gb300 as pkg

    n = 500
    dev, ref = _pair_models(n, 4)
    u = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.OdmdError):
        dev.predict(u, [1.0])
    rng = np.random.default_rng(3)
    X = np.zeros((n, 3))
    X[:, 1:] = rng.standard_normal((n, 2))
    Y = rng.standard_normal((n, 3))
    _feed(dev, ref, X, Y)
    assert dev.pairs == 3 and dev.rank == ref.rank == 2
    _compare(dev, ref, X[:, 2], [0.0, 1.0])


def test_hybrid_loop_with_fom_only_updates():
    """The hybrid loop of Fig. 1 in the FOM-only reading, driven from the host with the
    device model (predict one step from the current state; credible when within 1e-6 of
    the FOM, and every fourth step calls the FOM anyway), step for step as the oracle's
    loop: the same FOM steps, states within 1e-9, the same singular values."""
    n, tol, steps = 4096, 1e-6, 80
    Ar, B = _low_rank_map(n, 6, 4)
    A = Ar + 0.3 * (np.eye(n) - B @ B.T)
    rng = np.random.default_rng(5)
    u0 = B @ rng.standard_normal(6) + 1e-3 * rng.standard_normal(n)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def credible(k, prev, pred):
        return k % 4 != 0 and rel(pred, A @ prev) <= tol

    want_states, want_fom, ref = hybrid_fom_updates(lambda k, u: A @ u, credible, u0, steps, 16)
    import paper_2311_18715_gb300 as pkg

    dev = pkg.OnlineDMDPairs(n, 16)
    Ad = torch.from_numpy(A).cuda()
    state = torch.from_numpy(u0).cuda()
    fom_steps = []
    for k in range(1, steps + 1):
        if dev.pairs > 0 and dev.rank > 0:
            pred = dev.predict(state, [1.0])[0].clone()
            if credible(k, state.cpu().numpy(), pred.cpu().numpy()):
                state = pred
                continue
        nxt = Ad @ state
        dev.update(state, nxt)
        fom_steps.append(k)
        state = nxt
        np.testing.assert_allclose(state.cpu().numpy(), want_states[k], rtol=0, atol=1e-9 * np.linalg.norm(u0))
    assert fom_steps == want_fom
    assert np.linalg.norm(state.cpu().numpy() - want_states[-1]) <= 1e-9 * np.linalg.norm(u0)
    np.testing.assert_allclose(np.array(dev.singular_values()), ref.S, rtol=0, atol=1e-10 * ref.S[0])


def test_hybrid_step_residual_through_the_abi():
    """The same loop through odmd_pairs_hybrid_step_residual: the residual of the explicit
    linear FOM u_k = A u_{k-1} is r = b - u with b = A u_{k-1}, so the relative residual is
    the prediction's relative error; every fourth step the callback returns r = b (relative
    residual 1), which sends the step to the FOM.  Step for step as the oracle's loop."""
    n, tol, steps = 4096, 1e-6, 80
    Ar, B = _low_rank_map(n, 6, 4)
    A = Ar + 0.3 * (np.eye(n) - B @ B.T)
    rng = np.random.default_rng(5)
    u0 = B @ rng.standard_normal(6) + 1e-3 * rng.standard_normal(n)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    want_states, want_fom, ref = hybrid_fom_updates(
        lambda k, u: A @ u, lambda k, prev, pred: k % 4 != 0 and rel(pred, A @ prev) <= tol, u0, steps, 16)
    import paper_2311_18715_gb300 as pkg

    dev = pkg.OnlineDMDPairs(n, 16)
    Ad = torch.from_numpy(A).cuda()
    state = torch.from_numpy(u0).cuda().clone()
    nxt, r, b = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))

    def residual(k):
        b.copy_(Ad @ state)
        if k % 4 == 0:
            r.copy_(b)
        else:
            torch.sub(b, nxt, out=r)

    def fom(k):
        nxt.copy_(Ad @ nxt)

    fom_steps = []
    for k in range(1, steps + 1):
        acc, _ = dev.hybrid_step_residual(residual, fom, k, state, nxt, r, b, tol)
        if not acc:
            fom_steps.append(k)
    assert fom_steps == want_fom
    assert np.linalg.norm(state.cpu().numpy() - want_states[-1]) <= 1e-9 * np.linalg.norm(u0)
    np.testing.assert_allclose(np.array(dev.singular_values()), ref.S, rtol=0, atol=1e-10 * ref.S[0])
