"""The spectral-error metric behind the stated accuracy bounds (reading Err of the design notes), used
by the benchmark and the tests to compare a spectrum S with a reference S_ref of the same instance:

  (i)  relative L2 of S over the bins with q <= 1.5 q_cut;
  (ii) max over the odd harmonics h <= q_cut of |S_h - S_h^ref| / S_h^ref, S_h the power summed over
       the bins with h - 1/2 < q <= h + 1/2, over the harmonics whose reference power lies within
       HARMONIC_DECADES decades of the strongest odd harmonic (a harmonic with no power left, e.g.
       beyond the cutoff of a box too small for the electron's excursion, has no meaningful
       relative error);

with q = omega / omega0 and q_cut = (I_p + 3.17 U_p) / omega0, U_p = E0^2 / (4 omega0^2) (Sec. 7.1's
cutoff law, I_p = 0.579 a.u.).  Pure bookkeeping: no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

HARMONIC_DECADES = 8.0
# stated bounds (relative L2, worst odd harmonic) of each precision against the FP64 oracle
FP64_BOUND = (1e-6, 1e-6)
MIXED_BOUND = (3e-3, 3e-2)


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


def plateau_errors_by_decades(S, S_ref, omega0, dt, L, q_cut, decades=(2, 4, 6, 8)):
    """{D: worst relative error over the plateau harmonics 3 <= h <= q_cut whose reference power lies
    within D decades of the strongest of them} (a diagnostic of how the error grows toward the
    weakest harmonics)."""
    rows = [(h, a, b) for h, a, b in harmonic_powers(S, S_ref, omega0, dt, L, q_cut) if h >= 3 and b > 0]
    out = {}
    if not rows:
        return out
    top = max(b for _, _, b in rows)
    for D in decades:
        errs = [abs(a - b) / b for _, a, b in rows if b >= top * 10.0 ** (-D)]
        out[str(D)] = max(errs) if errs else 0.0
    return out


def spectral_errors(S, S_ref, omega0, dt, L, q_cut):
    """(relative L2 over q <= 1.5 q_cut, worst relative error over the odd harmonics within
    HARMONIC_DECADES decades of the strongest) of S against S_ref; bins k of an L-sample DFT."""
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    k = np.arange(S.size)
    q = k * 2 * np.pi / (L * dt) / omega0
    sel = q <= 1.5 * q_cut
    l2 = float(np.linalg.norm(S[sel] - S_ref[sel]) / np.linalg.norm(S_ref[sel]))
    pairs = []
    for h in range(1, int(q_cut) + 1, 2):
        win = (q > h - 0.5) & (q <= h + 0.5)
        if win.any():
            pairs.append((S[win].sum(), S_ref[win].sum()))
    worst = 0.0
    if pairs:
        floor = max(b for _, b in pairs) * 10.0 ** (-HARMONIC_DECADES)
        for a, b in pairs:
            if b >= floor and b > 0:
                worst = max(worst, abs(a - b) / b)
    return l2, worst
