"""The C-ABI library builds, loads and exports every entry point of include/tdse.h; host-side
argument validation rejects bad calls before any CUDA work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_04115_gb300 import build, tdse
    build.build()
    return tdse.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tdse_[a-z_0-9]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_2507_04115_gb300 import tdse
    declared = _declared()
    assert declared, "no entry points found in include/"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(tdse.EXPORTS) | (declared - set(tdse.EXPORTS))
    assert set(tdse.EXPORTS) <= declared


def test_create_rejects_bad_arguments_without_gpu(lib):
    from paper_2507_04115_gb300 import tdse
    good = [(256, 0.2, 1.2, 1.0)]
    bad_cases = [
        dict(inst=[(8, 0.2, 1.2, 1.0)]),                 # N too small
        dict(inst=[(256, -0.2, 1.2, 1.0)]),              # dx <= 0
        dict(inst=[(256, 0.2, 0.0, 1.0)]),               # softening <= 0
        dict(dt=0.0),                                    # dt == 0
        dict(n_steps=[-1]),                              # negative steps
        dict(row_offsets=[5, 2]),                        # decreasing offsets
        dict(precision=7),                               # unknown precision
    ]
    for case in bad_cases:
        kw = dict(inst=good, n_steps=[10], row_offsets=[0, 11], dt=0.05)
        kw.update(case)
        with pytest.raises(tdse.TDSEError) as ei:
            tdse.tdse_batch_create(kw["inst"], kw["n_steps"], kw["row_offsets"], kw["dt"],
                                   precision=kw.get("precision", tdse.TDSE_FP64))
        assert ei.value.status == tdse.TDSE_ERR_ARG, case
        assert tdse.tdse_last_error()


def test_null_handles_are_rejected(lib):
    from paper_2507_04115_gb300 import tdse
    assert lib.tdse_propagate(None, None, None, None, 0, 0, 1, None) == tdse.TDSE_ERR_ARG
    assert lib.tdse_ground_state(None, 0.1, 10, 1e-12, None, None, None) == tdse.TDSE_ERR_ARG
    assert lib.tdse_get_psi(None, 0, None, None) == tdse.TDSE_ERR_ARG
    info = tdse.tdse_plan_info()
    assert lib.tdse_plan(None, ctypes.byref(info)) == tdse.TDSE_ERR_ARG
    offs = np.array([0, 4], dtype=np.int64)
    assert lib.tdse_spectrum(None, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1, 0.1, 0, 2, None,
                             None) == tdse.TDSE_ERR_ARG
    n = ctypes.c_int32(-1)
    assert lib.tdse_autotune(None, None, None, None, 0, 0, 4, 1, None, 0, ctypes.byref(n), None) == tdse.TDSE_ERR_ARG
    assert n.value == -1
    assert lib.tdse_energy_distribution(None, None, 4, 0.05, None, None) == tdse.TDSE_ERR_ARG
    assert lib.tdse_set_wait_limit(None, 10) == tdse.TDSE_ERR_ARG
    assert lib.tdse_set_adjoint_gamma_tape(None, 1) == tdse.TDSE_ERR_ARG
    assert lib.tdse_populations(None, 1.0, None, None) == tdse.TDSE_ERR_ARG
    assert lib.tdse_resample_field(None, 1, 8, 0.1, 0.01, 10, 10, None, 0, None) == tdse.TDSE_ERR_ARG
    lib.tdse_batch_destroy(None)


def test_package_import_does_not_load_library():
    import importlib
    import paper_2507_04115_gb300
    importlib.reload(paper_2507_04115_gb300)
    from paper_2507_04115_gb300 import inputs
    assert inputs.pulse_steps(4, 0.057, 0.05) == 8818


def test_layout_cost_model_on_the_host(lib):
    """tdse_model_layout runs the planner's cost model without a GPU: the workloads' batches get the
    layouts the GPU path uses (32 instances per warp when the groups fill the SMs, lanes per instance
    otherwise), and bad arguments are refused."""
    from paper_2507_04115_gb300 import inputs, tdse
    assert tdse.model_layout([4096] * 8192, 0.15, 1.19, 0.02) == 1          # volume batch: 256 groups
    assert tdse.model_layout([2048] * 1024, 0.15, 1.19, 0.02) == 4          # adjoint batch: 32 -> 128 groups
    assert tdse.model_layout([2000], 0.2, 1.19, 0.05) == 32                  # single atom
    assert tdse.model_layout([2000], 0.2, 1.19, 0.05, scheme=tdse.TDSE_NUMEROV_SPLIT) > 1
    wl = inputs.uneven_batch()
    assert tdse.model_layout(wl.N, wl.dx, 1.19, wl.dt) == 1                  # 16384 instances in 8 classes
    # fewer SMs: the same small batch needs fewer lanes to fill them
    assert tdse.model_layout([2048] * 1024, 0.15, 1.19, 0.02, sm_count=32) == 1
    # a class whose sweeps cannot be truncated (dt / (4 dx^2) >= 0.85) keeps 32-wide groups
    assert tdse.model_layout([512], 0.05, 1.19, 0.01) == 1
    with pytest.raises(tdse.TDSEError):
        tdse.model_layout([8], 0.2, 1.19, 0.05)
    with pytest.raises(tdse.TDSEError):
        tdse.model_layout([512], 0.2, 1.19, 0.05, sm_count=0)


def test_far_field_entry_points_reject_bad_grids_without_gpu(lib):
    """tdse_dipole_spectrum and tdse_hankel validate on the host before any CUDA call."""
    from paper_2507_04115_gb300 import tdse
    dp = ctypes.POINTER(ctypes.c_double)
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first

    def arr(v):
        a = np.ascontiguousarray(v, dtype=np.float64)
        return a, a.ctypes.data_as(dp)

    rho, prho = arr([0.0, 1e-5, 2e-5])
    z, pz = arr([-1e-3, 0.0, 1e-3])
    k, pk = arr([1e8])
    ro, pro = arr([0.0, 1e-3])
    good = dict(rho=prho, nr=3, z=pz, nz=3, k=pk, nk=1, zo=0.5, ro=pro, no=2)
    bad = [dict(nr=0), dict(z=arr([0.0, -1e-3, 1e-3])[1]), dict(zo=1e-3), dict(k=arr([-1.0])[1]),
           dict(ro=arr([0.0, -1.0])[1]), dict(rho=arr([-1e-6, 1e-5, 2e-5])[1]), dict(nr=4096)]
    keep = [rho, z, k, ro]
    for case in bad:
        kw = dict(good)
        kw.update(case)
        rc = lib.tdse_hankel(fake, kw["rho"], kw["nr"], kw["z"], kw["nz"], kw["k"], kw["nk"], kw["zo"], kw["ro"],
                             kw["no"], fake, 0, None)
        assert rc == tdse.TDSE_ERR_ARG, case
    offs = np.array([0, 10, 5], dtype=np.int64)       # decreasing
    om, pom = arr([0.1])
    rc = lib.tdse_dipole_spectrum(fake, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 2, 0.02, pom, 1, None,
                                  fake, None)
    assert rc == tdse.TDSE_ERR_ARG
    offs = np.array([0, 10], dtype=np.int64)
    rc = lib.tdse_dipole_spectrum(fake, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1, -0.02, pom, 1, None,
                                  fake, None)
    assert rc == tdse.TDSE_ERR_ARG
    del keep
