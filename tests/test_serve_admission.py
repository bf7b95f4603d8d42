"""Host logic of the serving loop (paper_2311_18715_gb300/serve.py) on the CPU, with the
models, the batched calls and the CUDA streams replaced by fakes: admission in arrival
order by exact footprint, never past the memory budget or the active-session cap; a
request's memory returns as soon as its answers are read, so a waiting request is admitted
while others still run; every request streams all its snapshots and gets one answer per
horizon."""
import contextlib

import pytest
import torch

import paper_2311_18715_gb300.serve as serve


class _FakeModel:
    live = []
    created = []

    def __init__(self, n, r_max, prec="fp64", slack=16, device=None, stream=None):
        self.n, self.r_max, self.prec, self.slack = n, r_max, prec, slack
        self.stream = stream
        self.updates = 0
        self.closed = False
        _FakeModel.live.append(self)
        _FakeModel.created.append(self)

    def sync(self):
        pass

    def close(self):
        self.closed = True
        _FakeModel.live.remove(self)


def _install(monkeypatch, per_elem=100):
    _FakeModel.live, _FakeModel.created = [], []
    log = {"rounds": []}

    def update_batch(models, xs):
        assert len(models) == len(xs)
        for m, x in zip(models, xs):
            assert x.numel() == m.n
            m.updates += 1
        log["rounds"].append([id(m) for m in models])

    def predict_batch(models, ts):
        return [torch.zeros(len(t), m.n) for m, t in zip(models, ts)]

    monkeypatch.setattr(serve, "OnlineDMD", _FakeModel)
    monkeypatch.setattr(serve, "update_batch", update_batch)
    monkeypatch.setattr(serve, "predict_batch", predict_batch)
    monkeypatch.setattr(serve, "footprint", lambda n, r, prec="fp64", slack=16: per_elem * n)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    return log


def _req(rid, n, snaps, horizons=(1.0, 2.0), arrival=0.0):
    return serve.Request(rid=rid, arrival=arrival, n=n, r_max=8, snapshots=snaps, horizons=list(horizons),
                         source=lambda k, buf: buf.fill_(float(k)), keep=True)


def test_admission_by_footprint_in_arrival_order(monkeypatch):
    log = _install(monkeypatch)
    need = serve.Server(device=torch.device("cpu"))._need(_req(0, 1000, 1))
    assert need == 100 * 1000 + 8 * 1000  # footprint + the snapshot buffer (FP64)
    # room for two of the four at a time
    srv = serve.Server(device=torch.device("cpu"), hbm_budget=2 * need + need // 2)
    snaps = [5, 3, 4, 2]
    reqs = [_req(i, 1000, s) for i, s in enumerate(snaps)]  # all waiting at the start
    res = srv.run(reqs)
    for rnd in log["rounds"]:
        assert len(rnd) <= 2
    assert [m.n for m in _FakeModel.created] == [1000] * 4
    assert [r.rid for r in sorted(res, key=lambda r: r.admitted)] == [0, 1, 2, 3]  # arrival order
    by = {r.rid: r for r in res}
    for i, s in enumerate(snaps):
        assert by[i].updates == s
        assert by[i].predictions.shape == (2, 1000)
    # request 2 waits for the first to finish (request 1, 3 snapshots), then runs beside 0
    assert by[2].admitted >= by[1].finished
    assert by[2].admitted < by[0].finished
    assert all(m.closed for m in _FakeModel.created) and not _FakeModel.live


def test_never_past_budget_or_active_cap(monkeypatch):
    log = _install(monkeypatch)
    sizes = [3000, 1000, 2000, 1000, 4000, 1000, 1000, 2500]
    reqs = [_req(i, n, 2 + i % 3) for i, n in enumerate(sizes)]
    probe = serve.Server(device=torch.device("cpu"))
    budget = probe._need(_req(0, 5000, 1))
    srv = serve.Server(device=torch.device("cpu"), hbm_budget=budget, max_active=3)
    seen = []
    real_update = serve.update_batch

    def update_batch(models, xs):
        used = sum(probe._need(_req(0, m.n, 1)) for m in _FakeModel.live)
        seen.append((len(_FakeModel.live), used))
        real_update(models, xs)

    monkeypatch.setattr(serve, "update_batch", update_batch)
    res = srv.run(reqs)
    assert len(res) == len(reqs)
    assert max(a for a, _ in seen) <= 3
    assert max(u for _, u in seen) <= budget
    assert max(a for a, _ in seen) >= 2  # requests did overlap
    assert {r.rid: r.updates for r in res} == {i: 2 + i % 3 for i in range(len(reqs))}


def test_request_larger_than_budget_is_refused(monkeypatch):
    _install(monkeypatch)
    srv = serve.Server(device=torch.device("cpu"), hbm_budget=10_000)
    with pytest.raises(ValueError, match="more device memory than the budget"):
        srv.run([_req(0, 1000, 2)])
