"""odmd_update_host: snapshots read from host memory (pinned or pageable, any row stride)
give bit for bit the model that device-resident snapshots give."""
import numpy as np
import pytest

from synth import PlantedModes, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,pinned", [("fp64", True), ("fp64", False), ("fp32", True)])
def test_host_ingest_equals_device_ingest(prec, pinned):
    import paper_2311_18715_gb300 as pkg

    X = PlantedModes(3000, sigma=1e-8, seed=2).snapshots(0, 70)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xh = torch.from_numpy(X).to(dt)
    if pinned:
        Xh = Xh.pin_memory()
    a = pkg.OnlineDMD(3000, 8, prec=prec, slack=4)
    b = pkg.OnlineDMD(3000, 8, prec=prec, slack=4)
    Xd = Xh.cuda()
    for k in range(70):
        a.update(Xd[k])
    b.update_host(Xh[:25])
    b.update_host(Xh[25:])
    b.sync()
    a.sync()
    np.testing.assert_array_equal(np.array(a.singular_values()), np.array(b.singular_values()))
    ts = [69.0, 80.0]
    np.testing.assert_array_equal(a.predict(ts).cpu().numpy(), b.predict(ts).cpu().numpy())
    assert a.counts() == b.counts()


def test_host_ingest_strided_rows():
    import paper_2311_18715_gb300 as pkg

    X = WakeField(48, 24, sigma=1e-6, seed=1).snapshots(0, 40)
    n = X.shape[1]
    wide = np.zeros((40, n + 37))
    wide[:, :n] = X
    Xh = torch.from_numpy(wide)[:, :n]          # rows n + 37 elements apart
    a = pkg.OnlineDMD(n, 12, slack=6)
    b = pkg.OnlineDMD(n, 12, slack=6)
    for k in range(40):
        a.update(torch.from_numpy(X[k]).cuda())
    b.update_host(Xh)
    b.sync()
    np.testing.assert_array_equal(np.array(a.singular_values()), np.array(b.singular_values()))
    with pytest.raises(ValueError):
        b.update_host(torch.from_numpy(X).cuda())   # a device tensor is refused
