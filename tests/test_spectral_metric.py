"""The spectral-error metric of the stated bounds (no GPU): planted errors on synthetic spectra are
reported exactly, harmonics below the window are left out of the worst-harmonic number and shown by
the wider-window diagnostic."""
import numpy as np

from paper_2507_04115_gb300.spectral_metrics import (HARMONIC_DECADES, harmonic_cutoff, harmonic_errors_by_decades,
                                                      spectral_errors)


def _spectrum(L, dt, omega0, powers):
    """Bins of an L-sample DFT with power p_h in the bin nearest to each odd harmonic h."""
    S = np.zeros(L // 2 + 1)
    for h, p in powers.items():
        k = int(round(h * omega0 * L * dt / (2 * np.pi)))
        S[k] = p
    return S


def test_planted_harmonic_errors():
    L, dt, w = 8192, 0.05, 0.057
    q_cut = 15.2
    ref = {1: 1.0, 3: 1e-2, 5: 1e-3, 7: 1e-5, 9: 1e-7, 11: 1e-9, 13: 1e-3, 15: 1e-4}
    S_ref = _spectrum(L, dt, w, ref)
    got = dict(ref)
    got[5] *= 1.02       # 2 % on a harmonic inside the 4-decade window
    got[9] *= 1.5        # 50 % on one 7 decades down: outside the stated window
    S = _spectrum(L, dt, w, got)
    l2, worst = spectral_errors(S, S_ref, w, dt, L, q_cut)
    assert HARMONIC_DECADES == 4.0
    assert abs(worst - 0.02) < 1e-12
    by = harmonic_errors_by_decades(S, S_ref, w, dt, L, q_cut)
    assert abs(by["4"] - 0.02) < 1e-12 and abs(by["8"] - 0.5) < 1e-12 and by["2"] == 0.0
    exact = np.linalg.norm(S - S_ref) / np.linalg.norm(S_ref)
    assert abs(l2 - exact) < 1e-15
    # bins above 1.5 q_cut do not count in the L2 number
    S2 = S.copy()
    S2[-1] = 10.0
    assert spectral_errors(S2, S_ref, w, dt, L, q_cut)[0] == l2


def test_cutoff_law():
    # 800 nm at 1e14 W/cm^2 (E0 = 0.0534, omega = 0.057): U_p = 0.2194, q_cut = (0.579 + 3.17 U_p)/omega
    up = 0.0534 ** 2 / (4 * 0.057 ** 2)
    assert abs(harmonic_cutoff(0.0534, 0.057) - (0.579 + 3.17 * up) / 0.057) < 1e-12
    assert 22.0 < harmonic_cutoff(0.0534, 0.057) < 22.6
