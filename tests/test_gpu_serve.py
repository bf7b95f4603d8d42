"""Serving: requests of different sizes admitted by footprint under a memory budget that
holds only a few at a time, their updates batched as they arrive; each request's answers
must be the same as when it runs alone (the kernels reduce in a fixed order, so they are
bitwise equal; the bar is 1e-12 relative)."""
import numpy as np
import pytest

from synth import RandomPlanted

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _source(n, seed, record=None):
    """Snapshot k of a random planted-mode stream, drawn on the device; with `record`, a host
    copy of every snapshot drawn is kept there (the oracle then reads the same bytes)."""
    gen = RandomPlanted(n, seed=seed)
    fields = torch.from_numpy(gen.fields).cuda()

    def draw(k, out):
        c = torch.from_numpy(np.asarray(gen.coefficients(k), dtype=np.float64)).cuda()
        out.copy_(c @ fields)
        if record is not None:
            record[k] = out.cpu().numpy().copy()

    return draw, fields.numel() * 8


def _trace():
    import paper_2311_18715_gb300.serve as S

    rng = np.random.default_rng(4)
    reqs = []
    for i in range(8):
        n = int(rng.integers(2000, 40000))
        src, nb = _source(n, 50 + i)
        reqs.append(S.Request(rid=i, arrival=0.002 * i, n=n, r_max=int(rng.integers(4, 13)),
                              snapshots=int(rng.integers(20, 60)), horizons=[1.0, 7.5, 30.0],
                              source=src, source_bytes=nb, keep=True))
    return reqs


def test_serving_results_equal_alone_and_in_the_mix():
    import paper_2311_18715_gb300.serve as S

    reqs = _trace()
    # a budget that holds about three of these requests at once: the rest wait in line
    need = sorted(S.Server()._need(r) for r in reqs)
    server = S.Server(hbm_budget=need[-1] + need[-2] + need[-3])
    mixed = {r.rid: r for r in server.run(reqs)}
    assert sorted(mixed) == [r.rid for r in reqs]
    assert max(r.admitted for r in mixed.values()) > min(r.finished for r in mixed.values())  # queued
    for q in reqs:
        alone = S.Server().run([S.Request(**{**q.__dict__, "arrival": 0.0})])[0]
        a, b = mixed[q.rid].predictions.numpy(), alone.predictions.numpy()
        assert mixed[q.rid].updates == q.snapshots
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_serving_refuses_a_request_larger_than_the_budget():
    import paper_2311_18715_gb300.serve as S

    reqs = _trace()[:1]
    with pytest.raises(ValueError):
        S.Server(hbm_budget=1 << 20).run(reqs)


def test_served_answers_match_the_oracle():
    """Every answer of a served mix, per horizon, against the oracle fed the snapshots the
    request streamed (1e-9 relative, the FP64 reconstruction tolerance)."""
    import paper_2311_18715_gb300.serve as S
    from oracle import OnlineDMDRef

    rng = np.random.default_rng(9)
    reqs, recs = [], []
    for i in range(5):
        n = int(rng.integers(3000, 30000))
        rec = {}
        src, nb = _source(n, 80 + i, rec)
        recs.append(rec)
        reqs.append(S.Request(rid=i, arrival=0.001 * i, n=n, r_max=int(rng.integers(4, 13)),
                              snapshots=int(rng.integers(30, 70)), horizons=[1.0, 12.0, 40.0],
                              source=src, source_bytes=nb, keep=True))
    need = sorted(S.Server()._need(r) for r in reqs)
    res = {r.rid: r for r in S.Server(hbm_budget=need[-1] + need[-2]).run(reqs)}
    for q, rec in zip(reqs, recs):
        ref = OnlineDMDRef(q.n, q.r_max, 1e-10)
        for k in range(q.snapshots):
            ref.update(rec[k])
        ts = [float(q.snapshots - 1 + h) for h in q.horizons]
        want = ref.predict(ts).T
        got = res[q.rid].predictions.numpy()
        err = np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)
        assert np.max(err) < 1e-9, (q.rid, err)
