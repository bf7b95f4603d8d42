"""Many instances in one call: odmd_update_batch / odmd_predict_batch on instances of
different sizes and ranks, each on its own stream (so their kernels overlap on the GPU),
against the same instances driven one call at a time.  The kernels reduce in a fixed
order, so the two must agree bitwise; one instance is also checked against the oracle."""
import numpy as np
import pytest

from oracle import OnlineDMDRef
from synth import RandomPlanted

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(3000, 6), (70001, 12), (262147, 20), (1000, 8), (40000, 64)]


def test_batch_calls_equal_single_calls():
    import paper_2311_18715_gb300 as pkg

    steps = 30
    data = [torch.from_numpy(RandomPlanted(n, seed=i).snapshots(0, steps)).cuda()
            for i, (n, _) in enumerate(SHAPES)]
    torch.cuda.synchronize()
    batch = [pkg.OnlineDMD(n, r, slack=4, stream=torch.cuda.Stream()) for n, r in SHAPES]
    single = [pkg.OnlineDMD(n, r, slack=4) for n, r in SHAPES]
    # a small instance created last: the kernels' shared-memory limits are per process, so
    # creating it must not shrink what the larger instances above need
    tiny = pkg.OnlineDMD(100, 2, slack=0)
    for k in range(steps):
        pkg.update_batch(batch, [d[k] for d in data])
        for m, d in zip(single, data):
            m.update(d[k])
    ts = [[float(steps), steps + 2.5], [0.0], [float(steps + 10)], [1.0, 2.0, 3.0], [float(steps)]]
    got = pkg.predict_batch(batch, ts)
    torch.cuda.synchronize()
    for m, s, t, g in zip(batch, single, ts, got):
        assert m.rank == s.rank
        assert np.array_equal(np.array(m.singular_values()), np.array(s.singular_values()))
        assert torch.equal(g, s.predict(t))
    tiny.close()
    ref = OnlineDMDRef(SHAPES[2][0], SHAPES[2][1], 1e-10)
    for k in range(steps):
        ref.update(data[2][k].cpu().numpy())
    np.testing.assert_allclose(batch[2].singular_values(), ref.S, rtol=0, atol=1e-10 * ref.S[0])
    want = ref.predict(ts[2]).T
    assert np.linalg.norm(got[2].cpu().numpy() - want) / np.linalg.norm(want) < 1e-9


def test_batch_rejects_repeated_handles():
    import paper_2311_18715_gb300 as pkg

    m = pkg.OnlineDMD(100, 4)
    x = torch.ones(100, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.OdmdError):
        pkg.update_batch([m, m], [x, x])
