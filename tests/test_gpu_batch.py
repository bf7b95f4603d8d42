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


def test_batch_groups_by_storage_format():
    """One call over FP32-storage and FP64-accuracy instances: the library runs each group of
    like instances as one multi-instance launch per step (FP32 groups compact on the CUDA
    cores, FP64 ones on the tensor cores), and every instance still equals the same instance
    updated on its own, bitwise, through several compactions."""
    import paper_2311_18715_gb300 as pkg

    shapes = [(5000, 6, "fp32"), (20011, 10, "fp64"), (65537, 8, "fp32"), (3001, 12, "fp64"), (9000, 4, "fp32")]
    steps = 24
    gens = [RandomPlanted(n, seed=40 + i) for i, (n, _, _) in enumerate(shapes)]
    data64 = [torch.from_numpy(g.snapshots(0, steps)).cuda() for g in gens]
    data = [d.float() if p == "fp32" else d for d, (_, _, p) in zip(data64, shapes)]
    torch.cuda.synchronize()
    batch = [pkg.OnlineDMD(n, r, prec=p, slack=2, stream=torch.cuda.Stream()) for n, r, p in shapes]
    single = [pkg.OnlineDMD(n, r, prec=p, slack=2) for n, r, p in shapes]
    for k in range(steps):
        pkg.update_batch(batch, [d[k] for d in data])
        for m, d in zip(single, data):
            m.update(d[k])
    torch.cuda.synchronize()
    # the tuner has timed every split on the first calls of each group and kept one
    fp32 = [m for m, (_, _, p) in zip(batch, shapes) if p == "fp32"]
    fp64 = [m for m, (_, _, p) in zip(batch, shapes) if p == "fp64"]
    assert pkg.batch_split(fp32) in (1,)
    assert pkg.batch_split(fp64) in (1,)
    assert pkg.batch_split(batch) == -1  # never one group
    for m, s in zip(batch, single):
        assert m.rank == s.rank
        assert m.counts()[1] == s.counts()[1] >= 3  # (snapshots, compactions)
        assert np.array_equal(np.array(m.singular_values()), np.array(s.singular_values()))
        t = [float(steps), float(steps + 7)]
        assert torch.equal(m.predict(t), s.predict(t))


def test_batch_tuner_splits_are_bitwise_equal():
    """A group of eight instances: the tuner times S = 1, 2 and 4 sub-batches (two calls each)
    and keeps one; every split gives the instances exactly the results of their own updates."""
    import paper_2311_18715_gb300 as pkg

    shapes = [(4000 + 1013 * i, 4 + (i % 3), "fp64") for i in range(8)]
    steps = 14
    data = [torch.from_numpy(RandomPlanted(n, seed=70 + i).snapshots(0, steps)).cuda()
            for i, (n, _, _) in enumerate(shapes)]
    torch.cuda.synchronize()
    batch = [pkg.OnlineDMD(n, r, slack=3, stream=torch.cuda.Stream()) for n, r, _ in shapes]
    single = [pkg.OnlineDMD(n, r, slack=3) for n, r, _ in shapes]
    for k in range(steps):
        pkg.update_batch(batch, [d[k] for d in data])
        for m, d in zip(single, data):
            m.update(d[k])
        if k == 3:
            assert pkg.batch_split(batch) == 0  # still timing (six calls from the second on)
    torch.cuda.synchronize()
    assert pkg.batch_split(batch) in (1, 2, 4)
    for m, s in zip(batch, single):
        assert np.array_equal(np.array(m.singular_values()), np.array(s.singular_values()))
        t = [float(steps), float(steps + 3)]
        assert torch.equal(m.predict(t), s.predict(t))
