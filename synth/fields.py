"""Synthetic snapshot generators (inputs only; no DMD arithmetic).

The paper's own workload is an MFEM incompressible Navier-Stokes run of the flow past a
cylinder at Re=100 (Section 3): it cannot be reproduced here (no solver, no mesh), so
these seeded fields stand in for it, with shapes and scales taken from that section:
Strouhal number 0.22, a domain of 25D x 4.1D, a step of 0.005 convective time units
(10^4 steps over t* from 50 to 100).

Every generator is *separable*: a snapshot is a fixed set of spatial fields combined
with scalar time coefficients, plus white noise drawn from a per-step seed
(``numpy.random.default_rng([seed, stream, k])``), so any step k can be drawn on its
own and in any order, on any machine, with the same bytes.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def _noise(seed: int, stream: int, k: int, n: int) -> np.ndarray:
    """Standard-normal vector for step k; independent of the order steps are drawn in."""
    return np.random.default_rng([int(seed), int(stream), int(k)]).standard_normal(n)


class _Separable:
    """x_k = sum_f fields[f] * coeff_f(k) + sigma * xi_k."""

    n: int
    sigma: float
    seed: int
    stream: int
    fields: np.ndarray  # (F, n) float64

    def coefficients(self, k: float) -> np.ndarray:  # pragma: no cover - abstract
        raise NotImplementedError

    def clean(self, k: float) -> np.ndarray:
        """Noise-free snapshot at (possibly fractional) step k."""
        return self.coefficients(k) @ self.fields

    def snapshot(self, k: int) -> np.ndarray:
        x = self.clean(k)
        if self.sigma > 0.0:
            x = x + self.sigma * _noise(self.seed, self.stream, k, self.n)
        return x

    def snapshots(self, k0: int, count: int) -> np.ndarray:
        """(count, n) array of steps k0 .. k0+count-1 (row k is snapshot k0+k)."""
        out = np.empty((count, self.n), dtype=np.float64)
        for i in range(count):
            out[i] = self.snapshot(k0 + i)
        return out


class PlantedModes(_Separable):
    """Sum of complex-conjugate mode pairs with planted eigenvalues, plus white noise.

    x_k = sum_j 2 Re(phi_j lambda_j^k) + sigma xi_k, with phi_j = (g_j + i h_j)/sqrt(2),
    g_j, h_j ~ N(0, I_n) and lambda_j = mu_j exp(2 pi i theta_j).  All spatial modes
    are drawn first from ``default_rng(seed)``; the noise of step k comes from its own
    per-step seed.  With sigma = 0 the stream is exactly linear of rank 2P.
    """

    def __init__(self, n: int, mus: Sequence[float] = (1.0, 0.999, 0.99),
                 thetas: Sequence[float] = (0.02, 0.04, 0.06), sigma: float = 1e-8,
                 seed: int = 0, amplitudes: Sequence[float] | None = None):
        if len(mus) != len(thetas):
            raise ValueError("mus and thetas must have equal length")
        self.n = int(n)
        self.mus = np.asarray(mus, dtype=np.float64)
        self.thetas = np.asarray(thetas, dtype=np.float64)
        self.sigma = float(sigma)
        self.seed = int(seed)
        self.stream = 1
        P = len(self.mus)
        amp = np.ones(P) if amplitudes is None else np.asarray(amplitudes, dtype=np.float64)
        rng = np.random.default_rng(self.seed)
        g = rng.standard_normal((P, self.n))
        h = rng.standard_normal((P, self.n))
        # fields: rows [g_1..g_P, h_1..h_P] scaled by 2/sqrt(2) * amplitude
        scale = (2.0 / math.sqrt(2.0)) * amp[:, None]
        self.fields = np.concatenate([g * scale, h * scale], axis=0)

    def coefficients(self, k: float) -> np.ndarray:
        ang = 2.0 * np.pi * self.thetas * k
        rad = self.mus ** k
        # 2 Re((g + i h) mu^k e^{i k a}) / sqrt(2) = sqrt(2) mu^k (g cos - h sin)
        return np.concatenate([rad * np.cos(ang), -rad * np.sin(ang)])

    def planted_eigenvalues(self) -> np.ndarray:
        """The 2P eigenvalues the stream is built from (mu e^{+-2 pi i theta})."""
        lam = self.mus * np.exp(2j * np.pi * self.thetas)
        return np.concatenate([lam, lam.conj()])


def wake_grid_shape(n: int) -> tuple[int, int]:
    """Grid (nx, ny) with nx = 2 ny and 3 nx ny = n (u, v, p stacked)."""
    cells = n // 3
    ny = int(round(math.sqrt(cells / 2)))
    if 3 * 2 * ny * ny != n:
        raise ValueError(f"n={n} is not 3 * 2 ny^2")
    return 2 * ny, ny


class WakeField(_Separable):
    """Cylinder-wake-shaped field on an nx x ny grid, fields (u, v, p) stacked.

    Domain x in [0, 25], y in [-2.05, 2.05] (units of D, Section 3).  Index of grid
    point (i, j) within a field is j * nx + i; the state is [u; v; p], n = 3 nx ny.

    * mean flow: u = 1 - 0.5 g(y) behind the cylinder (x > 5), else 1;
    * shedding, harmonics h = 1..3: omega_h = 2 pi St h with St = 0.22, wavenumber
      k_h = omega_h / 0.85 (convection at 0.85 U), envelope g(y) s(x) with
      g(y) = exp(-(y/w)^2), s(x) = 1 - exp(-(x-5)/2) for x > 5 else 0:
      u += A_u sin(k x - omega t) g s,  v += A_v cos(k x - omega t) g s,
      p += A_p sin(k x - omega t + pi/4) g s;
    * four decaying transients: seeded N(0,1) shapes times 0.1 exp(-gamma t);
    * white noise of standard deviation ``sigma`` per step.

    Time is t = k dt.  Written in separable form: sin(kx - wt) = sin(kx) cos(wt) -
    cos(kx) sin(wt), so each snapshot is a combination of 11 fixed fields.
    """

    def __init__(self, nx: int = 512, ny: int = 256, dt: float = 0.005, sigma: float = 1e-6,
                 seed: int = 0, strouhal: float = 0.22, convect: float = 0.85, width: float = 1.0,
                 amp_u: Sequence[float] = (0.3, 0.1, 0.03), amp_v: Sequence[float] = (0.5, 0.15, 0.05),
                 amp_p: Sequence[float] = (0.2, 0.06, 0.02),
                 gammas: Sequence[float] = (0.5, 1.0, 2.0, 4.0), transient_amp: float = 0.1):
        self.nx, self.ny = int(nx), int(ny)
        self.n = 3 * self.nx * self.ny
        self.dt = float(dt)
        self.sigma = float(sigma)
        self.seed = int(seed)
        self.stream = 2
        self.omegas = 2.0 * np.pi * strouhal * np.arange(1, 4)
        self.gammas = np.asarray(gammas, dtype=np.float64)
        x = np.linspace(0.0, 25.0, self.nx)
        y = np.linspace(-2.05, 2.05, self.ny)
        X, Y = np.meshgrid(x, y)  # (ny, nx): index j * nx + i
        X = X.ravel()
        Y = Y.ravel()
        g = np.exp(-(Y / width) ** 2)
        behind = X > 5.0
        s = np.where(behind, 1.0 - np.exp(-(np.where(behind, X, 5.0) - 5.0) / 2.0), 0.0)
        env = g * s
        cells = self.nx * self.ny
        zeros = np.zeros(cells)
        fields = []
        mean_u = np.where(behind, 1.0 - 0.5 * g, 1.0)
        fields.append(np.concatenate([mean_u, zeros, zeros]))
        for h in range(3):
            kx = (self.omegas[h] / convect) * X
            # coefficient of cos(w t) and of sin(w t)
            cu, su = amp_u[h] * np.sin(kx) * env, -amp_u[h] * np.cos(kx) * env
            cv, sv = amp_v[h] * np.cos(kx) * env, amp_v[h] * np.sin(kx) * env
            cp, sp = (amp_p[h] * np.sin(kx + np.pi / 4) * env,
                      -amp_p[h] * np.cos(kx + np.pi / 4) * env)
            fields.append(np.concatenate([cu, cv, cp]))
            fields.append(np.concatenate([su, sv, sp]))
        rng = np.random.default_rng(self.seed)
        for _ in range(len(self.gammas)):
            fields.append(transient_amp * rng.standard_normal(self.n))
        self.fields = np.asarray(fields)

    def coefficients(self, k: float) -> np.ndarray:
        t = k * self.dt
        c = [1.0]
        for w in self.omegas:
            c.append(math.cos(w * t))
            c.append(math.sin(w * t))
        c.extend(np.exp(-self.gammas * t))
        return np.asarray(c)

    def planted_eigenvalues(self) -> np.ndarray:
        """Per-step eigenvalues of the noise-free stream (11 of them)."""
        rot = np.exp(1j * self.omegas * self.dt)
        return np.concatenate([[1.0 + 0j], rot, rot.conj(), np.exp(-self.gammas * self.dt) + 0j])


class RandomPlanted(PlantedModes):
    """A planted-mode stream with randomly drawn parameters (batched and serving loads).

    P ~ U{p_lo..p_hi} pairs, |lambda| ~ U[0.98, 1], theta ~ U[0.005, 0.2], drawn from
    ``default_rng([seed, 7])`` before the modes are drawn from ``default_rng(seed)``.
    """

    def __init__(self, n: int, seed: int, sigma: float = 1e-8, p_lo: int = 2, p_hi: int = 8):
        prm = np.random.default_rng([int(seed), 7])
        P = int(prm.integers(p_lo, p_hi + 1))
        mus = prm.uniform(0.98, 1.0, P)
        thetas = prm.uniform(0.005, 0.2, P)
        super().__init__(n, mus=mus, thetas=thetas, sigma=sigma, seed=seed)
