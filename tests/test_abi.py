"""The C ABI library loads and exports every entry point include/odmd.h declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:odmd_status|const char\*)\s+(odmd_\w+)\s*\(", text, re.M))
    return names


def test_header_declares_the_path_calls():
    names = declared_functions()
    for required in ("odmd_create", "odmd_update", "odmd_predict", "odmd_check", "odmd_destroy",
                     "odmd_footprint"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    import paper_2311_18715_gb300 as pkg

    pkg.build()
    lib = pkg.load_library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.EXPORTED) >= declared_functions()


def test_footprint_and_argument_checks_on_host():
    import ctypes as C

    import paper_2311_18715_gb300 as pkg
    from paper_2311_18715_gb300._lib import OdmdConfig

    pkg.build()
    lib = pkg.load_library()
    cfg = OdmdConfig()
    assert lib.odmd_config_default(C.byref(cfg), 393216, 40) == 0
    nb = C.c_size_t()
    assert lib.odmd_footprint(C.byref(cfg), C.byref(nb)) == 0
    # two float planes of N x ceil8(r_max+slack) dominate; then six n-element buffers of 8
    # bytes (two snapshot slots, the check input, the stored residual, two host-staging slots)
    plane = 393216 * 60 * 4  # row stride: 56 columns rounded up to an odd number of 16-byte chunks
    assert 2 * plane < nb.value < 2 * plane + 6 * 393216 * 8 + (8 << 20)
    bad = OdmdConfig()
    lib.odmd_config_default(C.byref(bad), 100, 65)
    assert lib.odmd_footprint(C.byref(bad), C.byref(nb)) == 1  # ODMD_ERR_ARG
    assert b"r_max" in lib.odmd_last_error(None)
    lib.odmd_config_default(C.byref(bad), 100, 8)
    bad.trunc_tol = 1e-16
    assert lib.odmd_footprint(C.byref(bad), C.byref(nb)) == 1
    lib.odmd_config_default(C.byref(bad), 100, 8)
    bad.prec = 2  # ODMD_BF16: refused, with the reason
    assert lib.odmd_footprint(C.byref(bad), C.byref(nb)) == 1
    assert b"BF16" in lib.odmd_last_error(None)
    assert lib.odmd_update(None, None) == 1
    # checkpoint entry points refuse a NULL handle before touching the device
    assert lib.odmd_checkpoint_size(None, None) == 1
    assert lib.odmd_save(None, None, 0) == 1
    assert lib.odmd_load(None, None, 0) == 1


def test_plain_c_client_compiles_links_and_runs():
    """include/odmd.h is strict C99 (-pedantic -Werror) and a C program linked against
    libodmd.so gets answers from its host-side entry points without a GPU."""
    import shutil
    import subprocess
    import tempfile

    import paper_2311_18715_gb300 as pkg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pkg.build()
    libdir = os.path.dirname(pkg.load_library()._name)
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "abi_host")
        cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
               os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", libdir, "-lodmd", "-Wl,-rpath," + libdir,
               "-o", exe]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
        run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert run.returncode == 0 and run.stdout.strip() == "ok", run.stderr


def test_library_exports_nothing_the_header_does_not_declare():
    """Every odmd_* function symbol libodmd.so defines is declared in include/odmd.h (and the
    other way round), so nothing undocumented is part of the ABI."""
    import shutil
    import subprocess

    import paper_2311_18715_gb300 as pkg

    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("no nm")
    pkg.build()
    path = pkg.load_library()._name
    out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {parts[2] for parts in (l.split() for l in out.splitlines())
                if len(parts) == 3 and parts[1] == "T" and parts[2].startswith("odmd_")}
    assert exported == declared_functions()


def test_header_compiles_as_cplusplus():
    import shutil
    import subprocess
    import tempfile

    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "h.cc")
        with open(src, "w") as f:
            f.write('#include "odmd.h"\nint main() { odmd_config c; return odmd_config_default(&c, 10, 2); }\n')
        res = subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                              "-I", os.path.join(ROOT, "include"), src], capture_output=True, text=True)
        assert res.returncode == 0, res.stderr
