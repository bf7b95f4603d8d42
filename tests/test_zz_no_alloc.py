"""odmd_check_noalloc: the credibility check for callers that must not allocate.

Some callers cannot allocate device memory (a callback inside a host solver's time loop
whose memory is owned by the solver's pool allocator, a process under a hard device-memory
cap).  odmd_check_noalloc serves them with a fixed scratch array inside the library.  This
test calls it through the C ABI on a prediction written by odmd_predict and compares it with
odmd_check on the same model, time and FOM snapshot, for two calls in a row (the second
call reuses the scratch the first one left behind), at two sizes.  It sits in a file of its
own that is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from synth import PlantedModes, RandomPlanted

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-9  # absolute, on relative errors: the tolerance of the check parity tests


def _model_and_fom(gen, n, m, r_max):
    import paper_2311_18715_gb300 as pkg

    dev = torch.device("cuda", 0)
    X = torch.from_numpy(gen.snapshots(0, m + 1)).to(dev)
    model = pkg.OnlineDMD(n, r_max, slack=4)
    for k in range(m):
        model.update(X[k])
    return model, X[m].contiguous()


def _noalloc(pred, fom, tol):
    import paper_2311_18715_gb300 as pkg

    lib = pkg.load_library()
    err = C.c_double(-1.0)
    ok = C.c_int32(-1)
    st = lib.odmd_check_noalloc(C.c_void_p(pred.data_ptr()), C.c_void_p(fom.data_ptr()), pred.numel(),
                                tol, C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(err),
                                C.byref(ok))
    assert st == 0, lib.odmd_last_error(None)
    return err.value, ok.value


@pytest.mark.parametrize("n, m", [(4096, 60), (1000, 40)])
def test_noalloc_check_matches_odmd_check_twice(n, m):
    gen = PlantedModes(n, sigma=1e-8, seed=0) if n == 4096 else RandomPlanted(n, seed=3)
    model, fom = _model_and_fom(gen, n, m, 10)
    for t, tol in ((float(m), 1e-5), (float(m) + 0.5, 1e-12)):
        pred = model.predict([t])[0].contiguous()
        want, want_pass = model.check(t, fom, tol)
        torch.cuda.synchronize()
        got = [_noalloc(pred, fom, tol) for _ in range(2)]
        for err, ok in got:
            assert abs(err - want) <= TOL, (err, want)
            assert bool(ok) == want_pass
        assert got[0] == got[1]  # the reduction order is fixed: two calls agree bitwise
    model.close()


def test_noalloc_check_special_cases_and_limit():
    import paper_2311_18715_gb300 as pkg

    dev = torch.device("cuda", 0)
    z = torch.zeros(777, dtype=torch.float64, device=dev)
    y = torch.ones(777, dtype=torch.float64, device=dev)
    assert pkg.check_noalloc(z, z) == (0.0, True)
    err, ok = pkg.check_noalloc(y, z)
    assert err == float("inf") and not ok
    err, ok = pkg.check_noalloc(2 * y, y, tol=1.5)
    assert err == pytest.approx(1.0, abs=1e-15) and ok
    # sizes beyond the fixed scratch are refused before anything runs
    lib = pkg.load_library()
    st = lib.odmd_check_noalloc(C.c_void_p(y.data_ptr()), C.c_void_p(y.data_ptr()), 33554432 + 1, 0.0,
                                None, None, None)
    assert st == 1 and b"exceeds the limit" in lib.odmd_last_error(None)
