"""Checkpoint / resume (odmd_checkpoint_size, odmd_save, odmd_load).

A model saved after some snapshots and loaded into a fresh handle of the same
configuration must continue exactly as the original: the same singular values, basis,
predictions and check errors, bit for bit, through pending appends and compactions.
Foreign, truncated, corrupted or mismatched checkpoints are refused."""
import numpy as np
import pytest

from synth import PlantedModes, WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _model(n, r_max, prec="fp64", slack=4, refine_every=0):
    import paper_2311_18715_gb300 as pkg

    return pkg.OnlineDMD(n, r_max, prec=prec, slack=slack, refine_every=refine_every)


def _state(m, ts, x_fom):
    m.sync()
    return (np.array(m.singular_values()), m.basis().cpu().numpy(), m.predict(ts).cpu().numpy(),
            m.check(ts[0], x_fom)[0], m.counts())


@pytest.mark.parametrize("prec,split", [("fp64", 60), ("fp64", 61), ("fp32", 37)])
def test_resume_continues_bit_for_bit(prec, split):
    g = PlantedModes(4096, sigma=1e-8, seed=0)
    X = g.snapshots(0, 121)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = torch.from_numpy(X).cuda().to(dt)
    a = _model(4096, 10, prec)
    for k in range(split):
        a.update(Xd[k])
    ck = a.save()
    b = _model(4096, 10, prec, refine_every=0)
    b.load(ck)
    assert b.counts()[0] == split and b.rank == a.rank
    for m in (a, b):
        for k in range(split, 120):
            m.update(Xd[k])
    ts = [120.0, 133.5, 160.0]
    sa, sb = _state(a, ts, Xd[120]), _state(b, ts, Xd[120])
    for u, v in zip(sa, sb):
        np.testing.assert_array_equal(u, v)


def test_resume_then_refine_and_wake_rollout():
    # the double-float wake at a size with many tiles per CTA; the resumed handle reserves
    # refinement scratch the saved one did not (the checkpoint does not depend on it)
    g = WakeField(128, 64, sigma=1e-6, seed=3)
    X = torch.from_numpy(g.snapshots(0, 90)).cuda()
    a = _model(X.shape[1], 24, slack=8)
    for k in range(45):
        a.update(X[k])
    ck = a.save()
    b = _model(X.shape[1], 24, slack=8, refine_every=1000)
    b.load(ck)
    for m in (a, b):
        for k in range(45, 89):
            m.update(X[k])
    np.testing.assert_array_equal(np.array(a.singular_values()), np.array(b.singular_values()))
    ts = [float(t) for t in range(89, 139)]
    np.testing.assert_array_equal(a.predict(ts).cpu().numpy(), b.predict(ts).cpu().numpy())
    b.refine()
    np.testing.assert_allclose(np.array(b.singular_values()), np.array(a.singular_values()), rtol=0,
                               atol=1e-12 * a.singular_values()[0])


def test_load_refuses_bad_checkpoints():
    import paper_2311_18715_gb300 as pkg

    X = torch.from_numpy(PlantedModes(500, seed=1).snapshots(0, 12)).cuda()
    a = _model(500, 6)
    for k in range(12):
        a.update(X[k])
    ck = a.save()
    with pytest.raises(pkg.OdmdError):
        _model(500, 7).load(ck)              # different r_max
    with pytest.raises(pkg.OdmdError):
        _model(501, 6).load(ck)              # different n
    with pytest.raises(pkg.OdmdError):
        _model(500, 6, slack=5).load(ck)     # different slack
    with pytest.raises(pkg.OdmdError):
        _model(500, 6).load(ck[:-8])         # truncated
    bad = bytearray(ck)
    bad[len(bad) // 2] ^= 0x40
    with pytest.raises(pkg.OdmdError):
        _model(500, 6).load(bytes(bad))      # corrupted payload
    bad = bytearray(ck)
    bad[0] ^= 1
    with pytest.raises(pkg.OdmdError):
        _model(500, 6).load(bytes(bad))      # not a checkpoint
    b = _model(500, 6)
    b.load(ck)                                # the original loads
    assert b.rank == a.rank


def _fnv1a_words(h, data):
    """FNV-1a over 8-byte little-endian words, then the tail bytes (the checkpoint's checksum)."""
    mask = (1 << 64) - 1
    n8 = len(data) // 8 * 8
    for w in np.frombuffer(data[:n8], dtype="<u8").tolist():
        h = ((h ^ w) * 1099511628211) & mask
    for b in data[n8:]:
        h = ((h ^ b) * 1099511628211) & mask
    return h


# header layout: magic 8, version u32, header_bytes u32, n i64, r_max/prec/slack/cap/ldg/ctl_bytes
# i32, nsnap i64, cur_h i32, curc_h i32, region u64[6], checksum u64
_HDR, _NSNAP, _CUR, _CURC, _SUM = 120, 48, 56, 60, 112


def _reseal(buf):
    """Recompute the checksum of a checkpoint whose header was edited (header with a zero
    checksum field, then every region), so that only the range checks can refuse it."""
    b = bytearray(buf)
    b[_SUM:_SUM + 8] = bytes(8)
    h = _fnv1a_words(1469598103934665603, bytes(b[:_HDR]))
    h = _fnv1a_words(h, bytes(b[_HDR:]))
    b[_SUM:_SUM + 8] = int(h).to_bytes(8, "little")
    return bytes(b)


def test_load_refuses_out_of_range_header_scalars():
    """Buffer indices outside {0, 1} and a negative snapshot count are refused even when the
    checksum matches; an edited header without a matching checksum is refused too."""
    import struct

    import paper_2311_18715_gb300 as pkg

    X = torch.from_numpy(PlantedModes(500, seed=1).snapshots(0, 9)).cuda()
    a = _model(500, 6)
    for k in range(9):
        a.update(X[k])
    ck = a.save()
    assert _reseal(ck) == ck  # the test's checksum is the library's
    for off, fmt, val in [(_CUR, "<i", 2), (_CURC, "<i", -1), (_NSNAP, "<q", -5), (_CUR, "<i", 1 - struct.unpack_from("<i", ck, _CUR)[0])]:
        bad = bytearray(ck)
        struct.pack_into(fmt, bad, off, val)
        with pytest.raises(pkg.OdmdError):
            _model(500, 6).load(bytes(bad))            # checksum no longer matches
        with pytest.raises(pkg.OdmdError):
            _model(500, 6).load(_reseal(bytes(bad)))   # range or control-block check
    b = _model(500, 6)
    b.load(ck)
    assert b.rank == a.rank
