"""The spectral-error metric behind the stated accuracy bounds (reading Err of the design notes), used
by the benchmark and the tests to compare a spectrum S with a reference S_ref of the same instance:

  (i)  relative L2 of S over the bins with q <= 1.5 q_cut;
  (ii) max over the odd harmonics h <= q_cut of |S_h - S_h^ref| / S_h^ref, S_h the power summed over
       the bins with h - 1/2 < q <= h + 1/2, over the harmonics whose reference power lies within
       HARMONIC_DECADES decades of the strongest odd harmonic.  The window is what the path can
       resolve: the MIXED solve (float wavefunction and float back substitution) leaves an error
       floor under the spectrum, so harmonics far below the strongest one (a weak, long-wavelength
       field: 7-8 decades between the fundamental and the plateau) carry relative errors of order
       one however well the strong ones agree; harmonic_errors_by_decades reports the error over
       wider windows as a diagnostic;

with q = omega / omega0 and q_cut = (I_p + 3.17 U_p) / omega0, U_p = E0^2 / (4 omega0^2) (Sec. 7.1's
cutoff law, I_p = 0.579 a.u.).  Pure bookkeeping: no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

HARMONIC_DECADES = 4.0
# stated bounds (relative L2, worst odd harmonic within HARMONIC_DECADES decades of the strongest)
# of each precision against the FP64 oracle
FP64_BOUND = (1e-6, 1e-6)
MIXED_BOUND = (3e-3, 3e-1)


def harmonic_cutoff(E0, omega, ip=0.579):
    up = E0 ** 2 / (4 * omega ** 2)
    return (ip + 3.17 * up) / omega


def harmonic_powers(S, S_ref, omega0, dt, L, q_cut):
    """[(h, power of S, power of S_ref)] over the odd harmonics h <= q_cut, the power summed over the
    bins with h - 1/2 < q <= h + 1/2."""
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    q = np.arange(S.size) * 2 * np.pi / (L * dt) / omega0
    out = []
    for h in range(1, int(q_cut) + 1, 2):
        win = (q > h - 0.5) & (q <= h + 0.5)
        if win.any():
            out.append((h, float(S[win].sum()), float(S_ref[win].sum())))
    return out


def _worst_within(rows, decades):
    rows = [(a, b) for _, a, b in rows if b > 0]
    if not rows:
        return 0.0
    floor = max(b for _, b in rows) * 10.0 ** (-decades)
    errs = [abs(a - b) / b for a, b in rows if b >= floor]
    return max(errs) if errs else 0.0


def harmonic_errors_by_decades(S, S_ref, omega0, dt, L, q_cut, decades=(2, 4, 6, 8)):
    """{D: worst relative error over the odd harmonics h <= q_cut whose reference power lies within
    D decades of the strongest of them} (a diagnostic of how the error grows toward the weakest
    harmonics)."""
    rows = harmonic_powers(S, S_ref, omega0, dt, L, q_cut)
    return {str(D): _worst_within(rows, D) for D in decades}


def spectral_errors(S, S_ref, omega0, dt, L, q_cut):
    """(relative L2 over q <= 1.5 q_cut, worst relative error over the odd harmonics within
    HARMONIC_DECADES decades of the strongest) of S against S_ref; bins k of an L-sample DFT."""
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    k = np.arange(S.size)
    q = k * 2 * np.pi / (L * dt) / omega0
    sel = q <= 1.5 * q_cut
    l2 = float(np.linalg.norm(S[sel] - S_ref[sel]) / np.linalg.norm(S_ref[sel]))
    return l2, _worst_within(harmonic_powers(S, S_ref, omega0, dt, L, q_cut), HARMONIC_DECADES)
