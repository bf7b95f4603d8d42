"""Spectrum and probe checks on the device model.

The synthetic cylinder wake sheds at Strouhal number St = 0.22 (Sec. 3 of the paper):
its shedding harmonics have per-step eigenvalues exp(+-i 2 pi St h dt), h = 1, 2, 3.
The frequencies the device's DMD recovers from its eigen-angles, f = |arg lambda| /
(2 pi dt), must be those harmonics; and a probe-point time series of the device's
rollout beyond the training window must follow the generator's own field."""
import numpy as np
import pytest

from synth import WakeField

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _wake_model(g, count, r_max=16, tau=1e-13):
    import paper_2311_18715_gb300 as pkg

    X = torch.from_numpy(g.snapshots(0, count)).cuda()
    m = pkg.OnlineDMD(X.shape[1], r_max, trunc_tol=tau, slack=16)
    for k in range(count):
        m.update(X[k])
    m.sync()
    return m


def test_strouhal_from_device_eigen_angles():
    g = WakeField(nx=64, ny=32, sigma=0.0, seed=0)
    m = _wake_model(g, 400)
    lam, amp = m.eigs()
    lam = np.asarray(lam)
    harmonics = g.planted_eigenvalues()[1:4]   # exp(+i omega_h dt), h = 1..3
    got = lam[np.argmin(np.abs(lam[:, None] - harmonics[None, :]), axis=0)]
    f = np.abs(np.angle(got)) / (2.0 * np.pi * g.dt)
    # the oracle pins the angles to 1e-8 at this tau (test_oracle_pins); 1e-8 / (2 pi dt) = 3e-7
    np.testing.assert_allclose(f, 0.22 * np.arange(1, 4), rtol=0, atol=1e-6)
    assert np.max(np.abs(got - harmonics)) < 1e-6
    # the harmonics are among the modes that carry the field (amplitude of each >= 1e-3 of
    # the largest), not noise-level modes that happen to lie nearby
    amp = np.asarray(amp)
    idx = np.argmin(np.abs(lam[:, None] - harmonics[None, :]), axis=0)
    assert np.all(amp[idx] >= 1e-3 * amp.max())


def test_probe_time_series_against_the_field():
    # train on 400 steps, roll out 200 more, follow the strongest-varying point of the field
    g = WakeField(nx=64, ny=32, sigma=0.0, seed=0)
    m = _wake_model(g, 400)
    ts = np.arange(400, 600, 4, dtype=np.float64)
    truth = np.stack([g.snapshot(int(t)) for t in ts])
    probe = int(np.argmax(truth.std(axis=0)))
    series = np.concatenate([m.predict([float(t) for t in ts[i:i + 25]]).cpu().numpy()[:, probe]
                             for i in range(0, len(ts), 25)])
    # eigenvalues within 1e-6 of the planted ones, carried over up to 200 steps, on a signal
    # of order 1: a relative error of a few 1e-5 is the expected size; the bar is 1e-4
    err = np.linalg.norm(series - truth[:, probe]) / np.linalg.norm(truth[:, probe])
    assert err < 1e-4, err


def test_probe_spectrum_gives_the_papers_strouhal(paper_values):
    """The paper's own verification (Sec. 3): the temporal spectrum of u_y at (10D, 0, 0)
    gives St = 0.22 'within the precision of the discrete values of frequency'.  Here the
    series is the device model's rollout, sampled every 10 steps over 2,000 samples (100
    time units: a frequency bin of 0.01).  The stream is the noise-free wake: trained on
    noisy snapshots, the model also holds noise-level modes whose eigenvalues can lie just
    outside the unit circle, and over a 20,000-step extrapolation those grow until they
    dominate the series (measured: the peak moved one bin, to 0.23)."""
    g = WakeField(nx=64, ny=32, sigma=0.0, seed=0)
    m = _wake_model(g, 400)
    i = int(np.argmin(np.abs(np.linspace(0, 25, g.nx) - paper_values["probe_x_over_D"])))
    j = int(np.argmin(np.abs(np.linspace(-2.05, 2.05, g.ny) - paper_values["probe_y_over_D"])))
    probe = g.nx * g.ny + j * g.nx + i
    ts = [float(t) for t in range(400, 400 + 20000, 10)]
    series = np.concatenate([m.predict(ts[a:a + 64]).cpu().numpy()[:, probe] for a in range(0, len(ts), 64)])
    f = np.fft.rfftfreq(len(series), d=10 * g.dt)
    spec = np.abs(np.fft.rfft(series - series.mean()))
    st = f[np.argmax(spec)]
    assert abs(st - paper_values["strouhal"]) < 0.5 * f[1], st   # the bin of 0.22 itself
