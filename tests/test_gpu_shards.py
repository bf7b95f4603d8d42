"""Row shards on one GPU (odmd_set_row_shards): the passes that end in a reduction run as G
launches over contiguous ranges of the row blocks, and one more launch adds the per-block
partials in block order -- the exchange of a run on G GPUs.  Every result must be bitwise
that of the unsharded handle on the same stream: singular values, eigenvalues, predictions
and check errors, for G = 2, 3, 4, through truncation and compaction of the tall basis."""
import numpy as np
import pytest

from synth import PlantedModes, RandomPlanted, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stream(case):
    if case == "planted":
        return PlantedModes(4096, sigma=1e-8, seed=0).snapshots(0, 90), 10, 4
    if case == "wake":
        return WakeField(64, 32, sigma=1e-6, seed=0).snapshots(0, 120), 16, 16
    return RandomPlanted(5001, seed=3).snapshots(0, 60), 8, 0  # ragged last tile, rotation every update


def _run(X, r, slack, shards, prec="fp64"):
    import paper_2311_18715_gb300 as pkg

    dt = torch.float64 if prec == "fp64" else torch.float32
    m = pkg.OnlineDMD(X.shape[1], r, prec=prec, slack=slack)
    m.set_row_shards(shards)
    Xd = torch.from_numpy(X).cuda().to(dt)
    for k in range(X.shape[0]):
        m.update(Xd[k])
    m.sync()
    k = X.shape[0]
    ts = [0.0, float(k - 1), float(k), float(k + 7)]
    out = {"S": np.array(m.singular_values()), "pred": m.predict(ts).cpu().numpy(),
           "frac": m.predict([k + 0.5]).cpu().numpy(), "check": m.check(float(k - 1), Xd[k - 1])[0],
           "eig": np.asarray(m.eigs()[0]), "counts": m.counts(), "rows": m.row_blocks()}
    m.close()
    return out


@pytest.mark.parametrize("case", ["planted", "wake", "ragged"])
def test_sharded_runs_are_bitwise_the_unsharded_one(case):
    from paper_2311_18715_gb300 import shards as sh

    X, r, slack = _stream(case)
    base = _run(X, r, slack, 1)
    rows = base["rows"]
    assert rows == sh.row_blocks(X.shape[1], len(rows) - 1)
    for G in (2, 3, 4):
        got = _run(X, r, slack, G)
        for key in ("S", "pred", "frac", "eig"):
            assert got[key].tobytes() == base[key].tobytes(), (case, G, key)
        assert got["check"] == base["check"] and got["counts"] == base["counts"], (case, G)


def test_fp32_storage_and_bad_shard_counts():
    import paper_2311_18715_gb300 as pkg

    X, r, slack = _stream("wake")
    base = _run(X, r, slack, 1, prec="fp32")
    got = _run(X, r, slack, 3, prec="fp32")
    assert got["S"].tobytes() == base["S"].tobytes() and got["pred"].tobytes() == base["pred"].tobytes()
    m = pkg.OnlineDMD(X.shape[1], r)
    nblocks = len(m.row_blocks()) - 1
    for bad in (0, -1, nblocks + 1):
        with pytest.raises(pkg.OdmdError):
            m.set_row_shards(bad)
    m.set_row_shards(nblocks)  # one block per shard is allowed
    m.close()
