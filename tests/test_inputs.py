"""The seeded synthetic input recipes (no GPU): unit conversions against the physical constants,
the sin^2 pulse's defining properties, agreement of the numpy and torch generators, and the
shapes of the workloads the benchmark and the tests run."""
import math

import numpy as np
import pytest

from paper_2507_04115_gb300 import inputs

# CODATA 2018
HARTREE_EV = 27.211386245988
HC_EV_NM = 1239.8419843320026
EPS0 = 8.8541878128e-12
C_LIGHT = 299792458.0
E_AU_V_M = 5.14220674763e11


def test_unit_conversions_match_physical_constants():
    for lam in (800.0, 1030.0, 1800.0):
        assert abs(inputs.omega_from_wavelength_nm(lam) - HC_EV_NM / lam / HARTREE_EV) < 1e-5 * HC_EV_NM / lam / HARTREE_EV
    i_au_w_cm2 = 0.5 * EPS0 * C_LIGHT * E_AU_V_M ** 2 * 1e-4   # cycle-averaged intensity of a 1 a.u. amplitude
    assert abs(inputs.AU_INTENSITY_W_CM2 - i_au_w_cm2) < 1e-6 * i_au_w_cm2
    assert abs(float(inputs.field_from_intensity(1e14)) - 0.0534) < 1e-4


def test_sin2_pulse_defining_properties():
    w, ncyc = 0.057, 4
    Tp = ncyc * 2 * math.pi / w
    dt = Tp / 4000          # Tp/2 falls on a sample
    n = 4400
    for phi in (0.0, 0.7, math.pi):
        E = inputs.sin2_pulse(n, dt, 0.05, w, ncyc, phi)
        assert E.shape == (n + 1,)
        assert E[0] == 0.0
        assert np.all(E[4001:] == 0.0)                              # zero after the pulse
        assert abs(E[2000] - 0.05 * math.cos(phi)) < 1e-15          # CEP referenced to the centre
        assert np.max(np.abs(E)) <= 0.05 + 1e-15
    assert inputs.pulse_steps(ncyc, w, dt) == 4000


def test_batch_generators_agree_with_single_rows():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    E0 = rng.uniform(0.02, 0.08, 5)
    phi = rng.uniform(-3, 3, 5)
    rows = inputs.sin2_pulse_batch(700, 0.05, E0, 0.057, 2.0, phi)
    for i in range(5):
        assert np.array_equal(rows[i], inputs.sin2_pulse(700, 0.05, E0[i], 0.057, 2.0, phi[i]))
    out = torch.empty((5, 701), dtype=torch.float64)
    inputs.sin2_pulse_batch(700, 0.05, E0, 0.057, 2.0, phi, out=out, xp=torch)
    assert np.max(np.abs(out.numpy() - rows)) < 1e-15


def test_gaussian_beam_focus_and_gouy_phase():
    wl = inputs.gaussian_beam_volume(n_r=4, n_z=5, noise=0.0, i0_w_cm2=2e14)
    assert wl.n_inst == 20
    # instance ir * n_z + iz; z runs from -zR to zR, so iz = 2 is the focus
    assert abs(wl.E0[2] - float(inputs.field_from_intensity(2e14))) < 1e-15
    # on axis the phase is the Gouy phase -atan(z / zR): +pi/4 at z = -zR, -pi/4 at z = zR
    assert abs(wl.phi[0] - math.pi / 4) < 1e-15 and abs(wl.phi[4] + math.pi / 4) < 1e-15
    # on axis at z = +-zR the intensity is halved
    assert abs(wl.E0[0] ** 2 / wl.E0[2] ** 2 - 0.5) < 1e-12


def test_workload_shapes():
    v = inputs.volume_batch()
    assert v.n_inst == 8192 and set(v.N.tolist()) == {4096} and v.dx[0] == 0.15 and v.dt == 0.02
    assert int(v.n_steps[0]) == 55159 and v.point_steps() == 8192 * 4096 * 55159
    a = inputs.adjoint_batch()
    assert a.n_inst == 1024 and set(a.N.tolist()) == {2048}
    s = inputs.single_atom()
    assert s.n_inst == 1 and int(s.N[0]) == 2000 and int(s.n_steps[0]) == 8818
    u = inputs.uneven_batch()
    assert u.n_inst == 16384
    assert len(set(zip(u.N.tolist(), u.dx.tolist()))) == 8
    assert u.n_steps.min() > 0 and u.n_steps.max() <= inputs.pulse_steps(16, inputs.omega_from_wavelength_nm(1800.0), 0.02)
    big = inputs.large_volume()
    assert big.n_inst == 131072


def test_subsample_is_deterministic_sorted_and_distinct():
    a = inputs.subsample(1000, 16, 7)
    assert np.array_equal(a, inputs.subsample(1000, 16, 7))
    assert np.all(np.diff(a) > 0) and a[0] >= 0 and a[-1] < 1000
    assert np.array_equal(inputs.subsample(5, 16, 1), np.arange(5))
