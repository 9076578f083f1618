"""Test helpers for the spectral comparisons: the metric and the stated bounds (from the package's
spectral_metrics) and the oracle propagations in spawned worker processes."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2507_04115_gb300.spectral_metrics import (FP64_BOUND, MIXED_BOUND, harmonic_cutoff,  # noqa: E402,F401
                                                    spectral_errors)


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
