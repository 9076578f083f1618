"""Seeded synthetic inputs shaped like the paper's workloads (arXiv:2507.04115, Sec. 7).

This module holds no arithmetic of the method itself: it only draws driving fields E(t) and
per-instance grid parameters.  Both the CUDA path and the CPU oracle take their inputs from
here.  The paper's own fields come from CUPRAD runs that are not available; focused
Gaussian-beam samples stand in for them (Sec. 2 describes the beam the pipeline propagates).

Units are atomic units unless stated.  A sin^2 pulse of n cycles is
    E(t) = E0 sin^2(pi t / Tp) cos(w (t - Tp/2) + phi)  for 0 <= t <= Tp,  0 afterwards,
with Tp = n 2 pi / w; the carrier-envelope phase phi is referenced to the envelope centre.
The field time axis starts at t = 0 (Sec. 4.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

AU_INTENSITY_W_CM2 = 3.50944758e16      # intensity of a 1 a.u. field amplitude
AU_LENGTH_M = 5.29177210903e-11
ARGON_GROUND_ENERGY = -0.579            # target E_g for the soft-core argon model (Sec. 7.5)


def omega_from_wavelength_nm(lam_nm: float) -> float:
    """Photon energy (a.u.) of a wavelength in nm: 45.5634 / lambda[nm]."""
    return 45.56335 / lam_nm


def field_from_intensity(i_w_cm2):
    return np.sqrt(np.asarray(i_w_cm2, dtype=np.float64) / AU_INTENSITY_W_CM2)


def pulse_steps(n_cycles: float, omega: float, dt: float) -> int:
    """Number of time steps Nt covering the pulse, floor(Tp / dt)."""
    return int(math.floor(n_cycles * 2.0 * math.pi / omega / dt + 1e-9))


def sin2_pulse(n_steps, dt, E0, omega, n_cycles, phi=0.0):
    """Samples E_n = E(n dt), n = 0..n_steps, of one sin^2 pulse (float64)."""
    t = np.arange(n_steps + 1, dtype=np.float64) * dt
    Tp = n_cycles * 2.0 * np.pi / omega
    env = np.where(t <= Tp, np.sin(np.pi * t / Tp) ** 2, 0.0)
    return E0 * env * np.cos(omega * (t - 0.5 * Tp) + phi)


def sin2_pulse_batch(n_steps, dt, E0, omega, n_cycles, phi, out=None, xp=np):
    """Rows E_i(n dt), n = 0..n_steps, for per-instance amplitude E0[i], phase phi[i] and scalar
    omega / n_cycles.  ``xp`` is numpy or torch (then ``out`` may be a device tensor)."""
    if xp is np:
        t = np.arange(n_steps + 1, dtype=np.float64) * dt
        Tp = n_cycles * 2.0 * np.pi / omega
        env = np.where(t <= Tp, np.sin(np.pi * t / Tp) ** 2, 0.0)
        res = np.asarray(E0)[:, None] * env[None, :] * np.cos(omega * (t[None, :] - 0.5 * Tp) + np.asarray(phi)[:, None])
        if out is not None:
            out[...] = res
            return out
        return res
    import torch
    dev = out.device if out is not None else "cpu"
    t = torch.arange(n_steps + 1, dtype=torch.float64, device=dev) * dt
    Tp = n_cycles * 2.0 * math.pi / omega
    env = torch.where(t <= Tp, torch.sin(math.pi * t / Tp) ** 2, torch.zeros_like(t))
    e0 = torch.as_tensor(np.asarray(E0), dtype=torch.float64, device=dev)
    ph = torch.as_tensor(np.asarray(phi), dtype=torch.float64, device=dev)
    res = e0[:, None] * env[None, :] * torch.cos(omega * (t[None, :] - 0.5 * Tp) + ph[:, None])
    if out is not None:
        out.copy_(res)
        return out
    return res


@dataclass
class Workload:
    """A batch of independent TDSE instances with uniform or per-instance parameters."""
    name: str
    N: np.ndarray            # int32 [n]
    dx: np.ndarray           # float64 [n]
    n_steps: np.ndarray      # int64 [n]  (Nt per instance)
    E0: np.ndarray           # float64 [n]
    omega: np.ndarray        # float64 [n]
    n_cycles: np.ndarray     # float64 [n]
    phi: np.ndarray          # float64 [n]
    dt: float
    target_energy: float = ARGON_GROUND_ENERGY
    charge: float = 1.0
    mask_width: float = 20.0
    mask_exponent: float = 0.125
    extra: dict = field(default_factory=dict)

    @property
    def n_inst(self) -> int:
        return int(self.N.size)

    def field_rows(self, idx=None):
        """Host float64 field rows for the instances ``idx`` (list of arrays, each Nt_i + 1 long)."""
        idx = range(self.n_inst) if idx is None else idx
        return [sin2_pulse(int(self.n_steps[i]), self.dt, self.E0[i], self.omega[i], self.n_cycles[i], self.phi[i])
                for i in idx]

    def point_steps(self) -> float:
        return float(np.sum(self.N.astype(np.float64) * self.n_steps.astype(np.float64)))


def _uniform(name, n, N, dx, n_steps, E0, omega, n_cycles, phi, dt, **kw):
    return Workload(name=name, N=np.full(n, N, np.int32), dx=np.full(n, dx), n_steps=np.full(n, n_steps, np.int64),
                    E0=np.asarray(E0, np.float64) * np.ones(n), omega=np.full(n, omega),
                    n_cycles=np.full(n, float(n_cycles)), phi=np.asarray(phi, np.float64) * np.ones(n), dt=dt, **kw)


def single_atom() -> Workload:
    """One argon-like atom: N = 2000, dx = 0.2 (x in [-200, 200]), 800 nm (w = 0.057), 4-cycle sin^2,
    E0 = 0.0534 (1e14 W/cm^2), CEP 0, dt = 0.05, cos^(1/8) mask on the outer 20 a.u."""
    w, dt = 0.057, 0.05
    return _uniform("single N=2000 dx=0.2 800nm 4cyc 1e14 dt=0.05", 1, 2000, 0.2, pulse_steps(4, w, dt),
                    0.0534, w, 4, 0.0, dt)


def gaussian_beam_volume(n_r=64, n_z=128, lam_nm=800.0, n_cycles=10, N=4096, dx=0.15, dt=0.02,
                         w0_m=50e-6, zR_m=5e-3, i0_w_cm2=2e14, noise=0.02, seed=1, name=None) -> Workload:
    """Macroscopic volume of a focused Gaussian beam: r in [0, w0] (n_r points), z in [-zR, zR] (n_z).
    I(r,z) = I0 (w0/w)^2 exp(-2 r^2/w^2), w = w0 sqrt(1 + (z/zR)^2); phase -atan(z/zR) + k r^2 / (2 R(z)),
    R = z (1 + (zR/z)^2); amplitude times U(1 - noise, 1 + noise) per instance.  Instance i = ir * n_z + iz."""
    rng = np.random.default_rng(seed)
    w = omega_from_wavelength_nm(lam_nm)
    r = np.linspace(0.0, w0_m, n_r)
    z = np.linspace(-zR_m, zR_m, n_z)
    R, Zc = np.meshgrid(r, z, indexing="ij")
    wz = w0_m * np.sqrt(1.0 + (Zc / zR_m) ** 2)
    inten = i0_w_cm2 * (w0_m / wz) ** 2 * np.exp(-2.0 * R ** 2 / wz ** 2)
    k = 2.0 * np.pi / (lam_nm * 1e-9)
    with np.errstate(divide="ignore", invalid="ignore"):
        curv = np.where(Zc == 0.0, 0.0, k * R ** 2 / (2.0 * Zc * (1.0 + (zR_m / np.where(Zc == 0.0, 1.0, Zc)) ** 2)))
    phi = -np.arctan(Zc / zR_m) + curv
    amp = field_from_intensity(inten).ravel() * rng.uniform(1.0 - noise, 1.0 + noise, n_r * n_z)
    n = n_r * n_z
    nm = name or ("volume %dx%d N=%d dx=%g %gnm %dcyc dt=%g" % (n_r, n_z, N, dx, lam_nm, n_cycles, dt))
    wl = _uniform(nm, n, N, dx, pulse_steps(n_cycles, w, dt), amp, w, n_cycles, phi.ravel(), dt)
    wl.extra.update(dict(n_r=n_r, n_z=n_z, lam_nm=lam_nm, w0_m=w0_m, zR_m=zR_m))
    return wl


def volume_batch() -> Workload:
    """8192 = 64 r x 128 z instances, N = 4096, dx = 0.15, dt = 0.02, 800 nm 10-cycle pulse, on-axis
    intensity 1-2e14 W/cm^2 with Gouy and curvature phases, +-2 % seeded amplitude noise (seed 1)."""
    return gaussian_beam_volume()


def adjoint_batch() -> Workload:
    """1024 = 16 r x 64 z instances as the volume batch but N = 2048 and 6 cycles."""
    return gaussian_beam_volume(n_r=16, n_z=64, n_cycles=6, N=2048, seed=3,
                                name="adjoint volume 16x64 N=2048 dx=0.15 800nm 6cyc dt=0.02")


def large_volume() -> Workload:
    """131072 = 256 r x 512 z, N = 4096, dx = 0.15, 1800 nm 8-cycle pulse, peak 1e14 W/cm^2 (seed 4)."""
    return gaussian_beam_volume(n_r=256, n_z=512, lam_nm=1800.0, n_cycles=8, i0_w_cm2=1e14, seed=4,
                                name="large volume 256x512 N=4096 dx=0.15 1800nm 8cyc dt=0.02")


def uneven_batch(n=16384, seed=2, dt=0.02) -> Workload:
    """Uneven batch: N ~ U{1024, 2048, 4096, 8192}, dx ~ U{0.15, 0.2}, cycles ~ U{4..16},
    wavelength ~ U{800, 1030, 1800} nm, intensity log-uniform in [5e13, 3e14] W/cm^2, CEP 0."""
    rng = np.random.default_rng(seed)
    N = rng.choice(np.array([1024, 2048, 4096, 8192], np.int32), n)
    dx = rng.choice(np.array([0.15, 0.2]), n)
    ncyc = rng.integers(4, 17, n).astype(np.float64)
    lam = rng.choice(np.array([800.0, 1030.0, 1800.0]), n)
    inten = np.exp(rng.uniform(np.log(5e13), np.log(3e14), n))
    w = np.array([omega_from_wavelength_nm(l) for l in lam])
    steps = np.array([pulse_steps(c, ww, dt) for c, ww in zip(ncyc, w)], np.int64)
    return Workload(name="uneven %d" % n, N=N, dx=dx, n_steps=steps, E0=field_from_intensity(inten), omega=w,
                    n_cycles=ncyc, phi=np.zeros(n), dt=dt)


def subsample(n_inst: int, k: int, seed: int) -> np.ndarray:
    """k distinct instance indices drawn with a fixed seed (sorted)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_inst, size=min(k, n_inst), replace=False))
