"""The spectral-error metric of the stated bounds (reading Err): two numbers against the FP64
oracle's spectrum S_ref of the same instance,
  (i)  relative L2 of S over the bins with q <= 1.5 q_cut,
  (ii) max over the odd harmonics h <= q_cut of |S_h - S_h^ref| / S_h^ref, S_h the power summed
       over the bins with h - 1/2 < q <= h + 1/2,
with q = omega / omega0 and q_cut = (I_p + 3.17 U_p) / omega0, U_p = E0^2 / (4 omega0^2) (Sec. 7.1's
cutoff law, I_p = 0.579 a.u.)."""
import numpy as np

# Stated bounds of the two precisions (the same pair is quoted in the design notes and the benchmark)
FP64_BOUND = (1e-6, 1e-6)
MIXED_BOUND = (1e-3, 3e-2)


def harmonic_cutoff(E0, omega, ip=0.579):
    up = E0 ** 2 / (4 * omega ** 2)
    return (ip + 3.17 * up) / omega


def spectral_errors(S, S_ref, omega0, dt, L, q_cut):
    k = np.arange(S.size)
    q = k * 2 * np.pi / (L * dt) / omega0
    sel = q <= 1.5 * q_cut
    l2 = float(np.linalg.norm(S[sel] - S_ref[sel]) / np.linalg.norm(S_ref[sel]))
    worst = 0.0
    for h in range(1, int(q_cut) + 1, 2):
        win = (q > h - 0.5) & (q <= h + 0.5)
        if win.any():
            a, b = S[win].sum(), S_ref[win].sum()
            worst = max(worst, abs(a - b) / b)
    return l2, worst


def oracle_job(args):
    """One oracle propagation (spawned worker): (psi0, E, dx, dt, a, mask) -> (psi, d, acc)."""
    import oracle
    psi0, E, dx, dt, a, mask = args
    return oracle.propagate(psi0, E, dx, dt, a, mask_values=mask)


def oracle_pool_map(jobs, workers=None):
    """Oracle propagations in spawned processes (spawn: safe after the parent touched CUDA)."""
    import multiprocessing as mp
    import os
    workers = workers or min(len(jobs), os.cpu_count() or 1)
    if workers <= 1:
        return [oracle_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(processes=workers) as pool:
        return pool.map(oracle_job, jobs, chunksize=1)


def oracle_adjoint_job(args):
    """One oracle adjoint (spawned worker): (psi0, E, dx, dt, a, gd, ga, mask) -> dL/dE."""
    import oracle
    psi0, E, dx, dt, a, gd, ga, mask = args
    return oracle.adjoint(psi0, E, dx, dt, a, gd, ga, mask_values=mask)


def start_pool(fn, jobs, workers=None):
    """map_async of fn over jobs in a spawned pool started now (the caller may use the GPU meanwhile);
    returns (pool, async result)."""
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    pool = mp.get_context("spawn").Pool(processes=workers)
    return pool, pool.map_async(fn, jobs, chunksize=1)
