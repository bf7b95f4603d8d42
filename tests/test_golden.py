"""What the paper prints (tests/golden/paper_values.txt) against what this repository
assumes: the library's default credibility tolerance is the paper's epsilon_DMD, and the
synthetic wake sheds at the paper's Strouhal number."""
import ctypes as C

import numpy as np

from synth import WakeField


def test_default_tolerance_is_the_papers(paper_values):
    import paper_2311_18715_gb300 as pkg
    from paper_2311_18715_gb300._lib import OdmdConfig

    pkg.build()
    lib = pkg.load_library()
    cfg = OdmdConfig()
    assert lib.odmd_config_default(C.byref(cfg), 1000, 8) == 0
    assert cfg.check_tol == paper_values["eps_dmd"]


def test_synthetic_wake_sheds_at_the_papers_strouhal(paper_values):
    g = WakeField(nx=64, ny=32, sigma=0.0)
    st = paper_values["strouhal"]
    # per-step rotation of the fundamental: 2 pi St dt (D = U = 1)
    lam = g.planted_eigenvalues()[1]
    assert abs(np.angle(lam) - 2 * np.pi * st * g.dt) < 1e-15
    # and a sampled time series at the paper's probe point shows it
    i = int(np.argmin(np.abs(np.linspace(0, 25, g.nx) - paper_values["probe_x_over_D"])))
    j = int(np.argmin(np.abs(np.linspace(-2.05, 2.05, g.ny) - paper_values["probe_y_over_D"])))
    probe = g.nx * g.ny + j * g.nx + i          # u_y of grid point (i, j)
    ks = np.arange(0, 40000, 20)
    series = np.array([g.clean(int(k))[probe] for k in ks])
    f = np.fft.rfftfreq(len(series), d=20 * g.dt)
    spec = np.abs(np.fft.rfft(series - series.mean()))
    assert abs(f[np.argmax(spec)] - st) <= f[1]   # within one bin of the discrete spectrum
