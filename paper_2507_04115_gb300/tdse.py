"""Thin ctypes binding of libtdse.so (C ABI in include/tdse.h).

Argument marshalling only: every numerical step runs in the library's CUDA kernels.  Device
buffers are torch tensors (float64, contiguous, on the batch's device); host arrays are numpy.
There is no CPU fallback: ``load()`` raises if the library is missing or cannot be opened.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

TDSE_OK, TDSE_ERR_ARG, TDSE_ERR_CUDA, TDSE_ERR_NONFINITE, TDSE_ERR_TIMEOUT, TDSE_ERR_NOMEM, TDSE_ERR_STATE = range(7)
TDSE_FP64, TDSE_MIXED = 0, 1
TDSE_FULL_CN, TDSE_NUMEROV_SPLIT = 0, 1

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtdse.so")
_lib = None

#: C-ABI entry points declared in include/tdse.h
EXPORTS = ("tdse_batch_create", "tdse_batch_destroy", "tdse_ground_state", "tdse_propagate", "tdse_get_psi",
           "tdse_set_psi", "tdse_check", "tdse_spectrum", "tdse_plan", "tdse_set_launch", "tdse_propagate_static",
           "tdse_probe_pipes", "tdse_copy_state", "tdse_adjoint", "tdse_autotune", "tdse_set_layout", "tdse_energy_distribution", "tdse_set_wait_limit", "tdse_resample_field", "tdse_model_layout",
           "tdse_populations", "tdse_ionisation", "tdse_dipole_spectrum", "tdse_hankel",
           "tdse_propagate_checkpointed", "tdse_adjoint_checkpointed", "tdse_set_adjoint_gamma_tape",
           "tdse_last_error")


class tdse_instance(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("dx", ctypes.c_double), ("softening", ctypes.c_double),
                ("charge", ctypes.c_double)]


class tdse_absorber(ctypes.Structure):
    _fields_ = [("width", ctypes.c_double), ("exponent", ctypes.c_double)]


class tdse_plan_info(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int64), ("segments", ctypes.c_int32), ("halo", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("ctas", ctypes.c_int32), ("slice_steps", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_int64), ("psi_bytes", ctypes.c_int64),
                ("lanes_per_instance", ctypes.c_int32), ("longest_share", ctypes.c_double)]


class tdse_pipe_rates(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp64_warp_instr_per_s", ctypes.c_double),
                ("fp64_one_lane_warp_instr_per_s", ctypes.c_double),
                ("fp64_tflops_warps_per_sm", ctypes.c_double * 3), ("fp32_fma_tflops", ctypes.c_double),
                ("cvt_pairs_per_s", ctypes.c_double), ("sm_count", ctypes.c_int32), ("sm_clock_mhz", ctypes.c_double),
                ("rcp_f64_approx_fma_slots", ctypes.c_double), ("rcp_seed_fma_slots", ctypes.c_double),
                ("dadd_fma_slots", ctypes.c_double), ("dmul_fma_slots", ctypes.c_double),
                ("add_as_fma_slots", ctypes.c_double), ("mul_as_fma_slots", ctypes.c_double),
                ("fma_repeat_slots", ctypes.c_double)]


class tdse_tune_trial(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("slice_steps", ctypes.c_int32),
                ("ctas", ctypes.c_int32), ("ms", ctypes.c_float)]


class TDSEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("tdse status %d: %s" % (status, msg))
        self.status = status


_vp, _dp, _i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)


def load(path: str | None = None):
    """Open libtdse.so and declare the C signatures.  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libtdse.so is not built (expected at %s): run __graft_entry__.build()" % p)
    L = ctypes.CDLL(p)
    L.tdse_batch_create.argtypes = [ctypes.POINTER(tdse_instance), ctypes.c_int64, ctypes.c_double, _i64p, _i64p,
                                    ctypes.POINTER(tdse_absorber), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(_vp)]
    L.tdse_batch_destroy.argtypes = [_vp]
    L.tdse_batch_destroy.restype = None
    L.tdse_ground_state.argtypes = [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_double, _dp, _i64p, _vp]
    L.tdse_propagate.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp]
    L.tdse_get_psi.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
    L.tdse_set_psi.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
    L.tdse_check.argtypes = [_vp, _i64p, _vp]
    L.tdse_spectrum.argtypes = [_vp, _i64p, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _vp, _vp]
    L.tdse_plan.argtypes = [_vp, ctypes.POINTER(tdse_plan_info)]
    L.tdse_set_launch.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.tdse_propagate_static.argtypes = [ctypes.POINTER(tdse_instance), ctypes.c_int64, ctypes.c_double,
                                        ctypes.POINTER(tdse_absorber), ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                                        _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp]
    L.tdse_probe_pipes.argtypes = [ctypes.c_int, ctypes.POINTER(tdse_pipe_rates)]
    L.tdse_copy_state.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
    L.tdse_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp]
    L.tdse_propagate_checkpointed.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.c_int32, _vp]
    L.tdse_adjoint_checkpointed.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.tdse_autotune.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                ctypes.POINTER(tdse_tune_trial), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _vp]
    L.tdse_set_layout.argtypes = [_vp, ctypes.c_int32]
    L.tdse_set_wait_limit.argtypes = [_vp, ctypes.c_int64]
    L.tdse_set_adjoint_gamma_tape.argtypes = [_vp, ctypes.c_int32]
    L.tdse_model_layout.argtypes = [ctypes.POINTER(tdse_instance), ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.tdse_resample_field.argtypes = [_vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_int, _vp]
    L.tdse_energy_distribution.argtypes = [_vp, _dp, ctypes.c_int32, ctypes.c_double, _vp, _vp]
    L.tdse_populations.argtypes = [_vp, ctypes.c_double, _vp, _vp]
    L.tdse_ionisation.argtypes = [_vp, _dp, ctypes.c_int32, ctypes.c_double, _vp, _vp, _vp]
    L.tdse_dipole_spectrum.argtypes = [_vp, _i64p, ctypes.c_int64, ctypes.c_double, _dp, ctypes.c_int32, _vp, _vp, _vp]
    L.tdse_hankel.argtypes = [_vp, _dp, ctypes.c_int32, _dp, ctypes.c_int32, _dp, ctypes.c_int32, ctypes.c_double,
                              _dp, ctypes.c_int32, _vp, ctypes.c_int, _vp]
    L.tdse_last_error.argtypes = []
    L.tdse_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("tdse_batch_destroy", "tdse_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != TDSE_OK:
        raise TDSEError(rc, load().tdse_last_error().decode())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------------- C-ABI mirrors

def tdse_batch_create(inst, n_steps, row_offsets, dt, absorber=(20.0, 0.125), precision=TDSE_FP64,
                      scheme=TDSE_FULL_CN, device=0):
    """inst: sequence of (N, dx, softening, charge); returns the opaque handle."""
    L = load()
    n = len(inst)
    arr = (tdse_instance * n)(*[tdse_instance(int(a), float(b), float(c), float(d)) for a, b, c, d in inst])
    ns = np.ascontiguousarray(n_steps, dtype=np.int64)
    ro = np.ascontiguousarray(row_offsets, dtype=np.int64)
    if ns.size != n or ro.size != n + 1:
        raise ValueError("n_steps needs n entries and row_offsets n + 1")
    ab = None if absorber is None else ctypes.byref(tdse_absorber(float(absorber[0]), float(absorber[1])))
    h = _vp()
    _check(L.tdse_batch_create(arr, n, float(dt), ns.ctypes.data_as(_i64p), ro.ctypes.data_as(_i64p), ab,
                               int(precision), int(scheme), int(device), ctypes.byref(h)))
    return h


def tdse_batch_destroy(h):
    load().tdse_batch_destroy(h)


def tdse_last_error():
    return load().tdse_last_error().decode()


class Batch:
    """A batch of independent TDSE instances living on one GPU (see include/tdse.h)."""

    def __init__(self, N, dx, softening, n_steps, dt, charge=1.0, row_offsets=None, absorber=(20.0, 0.125),
                 precision=TDSE_FP64, scheme=TDSE_FULL_CN, device=0, lanes_per_instance=0):
        N = np.atleast_1d(np.asarray(N, dtype=np.int64))
        n = N.size
        dx = np.broadcast_to(np.asarray(dx, dtype=np.float64), (n,))
        a = np.broadcast_to(np.asarray(softening, dtype=np.float64), (n,))
        Z = np.broadcast_to(np.asarray(charge, dtype=np.float64), (n,))
        self.n_steps = np.broadcast_to(np.asarray(n_steps, dtype=np.int64), (n,)).copy()
        if row_offsets is None:
            row_offsets = np.concatenate([[0], np.cumsum(self.n_steps + 1)])
        self.row_offsets = np.ascontiguousarray(row_offsets, dtype=np.int64)
        self.N = N
        self.dx = np.array(dx)
        self.softening = np.array(a)
        self.charge = np.array(Z)
        self.precision = int(precision)
        self.scheme = int(scheme)
        self.lanes_per_instance = 0          # 0 = the planner's cost model (see set_layout)
        self.dt = float(dt)
        self.device = int(device)
        self.n_inst = n
        self._h = tdse_batch_create(list(zip(N, dx, a, Z)), self.n_steps, self.row_offsets, dt, absorber, precision,
                                    scheme, device)
        if lanes_per_instance:
            self.set_layout(lanes_per_instance)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            tdse_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def ground_state(self, dtau=0.1, max_iter=20000, tol=1e-13, stream=None):
        e = np.zeros(self.n_inst)
        it = np.zeros(self.n_inst, dtype=np.int64)
        _check(load().tdse_ground_state(self._h, float(dtau), int(max_iter), float(tol), e.ctypes.data_as(_dp),
                                        it.ctypes.data_as(_i64p), _stream_ptr(stream)))
        return e, it

    def propagate(self, E, d, a, step_begin=0, step_end=None, sample_base=0, stream=None):
        """Device tensors E, d, a laid out by row_offsets (see tdse_propagate).  CPU tensors are
        copied to the device before and the outputs back after the call (end-to-end use)."""
        import torch
        if step_end is None:
            step_end = int(self.n_steps.max())
        host = not E.is_cuda
        if host:
            dev = torch.device("cuda", self.device)
            Ed = E.to(dev, non_blocking=True)
            dd = torch.empty(d.shape, dtype=torch.float64, device=dev)
            ad = torch.empty(a.shape, dtype=torch.float64, device=dev)
        else:
            Ed, dd, ad = E, d, a
        _check(load().tdse_propagate(self._h, _dev_ptr(Ed, "E"), _dev_ptr(dd, "d"), _dev_ptr(ad, "a"),
                                     int(sample_base), int(step_begin), int(step_end), _stream_ptr(stream)))
        if host:
            d.copy_(dd, non_blocking=True)
            a.copy_(ad, non_blocking=True)

    def get_psi(self, inst, stream=None):
        import torch
        out = torch.empty(2 * int(self.N[inst]), dtype=torch.float64, device=torch.device("cuda", self.device))
        _check(load().tdse_get_psi(self._h, int(inst), _dev_ptr(out, "psi"), _stream_ptr(stream)))
        return torch.view_as_complex(out.view(-1, 2))

    def set_psi(self, inst, psi, stream=None):
        import torch
        t = torch.view_as_real(psi.to(torch.complex128).contiguous()).reshape(-1).contiguous()
        if t.numel() != 2 * int(self.N[inst]):
            raise ValueError("psi must have N complex entries")
        _check(load().tdse_set_psi(self._h, int(inst), _dev_ptr(t, "psi"), _stream_ptr(stream)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def check(self, stream=None):
        bad = ctypes.c_int64(-1)
        rc = load().tdse_check(self._h, ctypes.byref(bad), _stream_ptr(stream))
        if rc == TDSE_ERR_NONFINITE:
            return int(bad.value)
        _check(rc)
        return -1

    def plan(self):
        info = tdse_plan_info()
        _check(load().tdse_plan(self._h, ctypes.byref(info)))
        return dict(n_groups=info.n_groups, segments=info.segments, halo=info.halo,
                    warps_per_cta=info.warps_per_cta, ctas=info.ctas, slice_steps=info.slice_steps,
                    scratch_bytes=info.scratch_bytes, psi_bytes=info.psi_bytes,
                    lanes_per_instance=info.lanes_per_instance, longest_share=info.longest_share)

    def energy_distribution(self, E_grid, epsilon, out=None, stream=None):
        """P[i, k]: energy distribution of instance i's current state at E_grid[k] with resolution
        epsilon (see tdse_energy_distribution); returns a float64 device tensor n_inst x len(E_grid)."""
        import torch
        Eg = np.ascontiguousarray(E_grid, dtype=np.float64)
        if out is None:
            out = torch.empty((self.n_inst, Eg.size), dtype=torch.float64, device=torch.device("cuda", self.device))
        _check(load().tdse_energy_distribution(self._h, Eg.ctypes.data_as(_dp), int(Eg.size), float(epsilon),
                                               _dev_ptr(out, "P"), _stream_ptr(stream)))
        return out

    def ionisation(self, E_nodes, epsilon, out=None, P_out=None, stream=None):
        """Ionisation probability of every instance's current state: the trapezoid integral of the
        energy distribution over the ascending nodes E_nodes (see tdse_ionisation); a float64 device
        tensor of n_inst values.  P_out (n_inst x len(E_nodes)) optionally receives the distribution."""
        import torch
        En = np.ascontiguousarray(E_nodes, dtype=np.float64)
        if out is None:
            out = torch.empty(self.n_inst, dtype=torch.float64, device=torch.device("cuda", self.device))
        Pp = None if P_out is None else _dev_ptr(P_out, "P_out")
        _check(load().tdse_ionisation(self._h, En.ctypes.data_as(_dp), int(En.size), float(epsilon), Pp,
                                      _dev_ptr(out, "out"), _stream_ptr(stream)))
        return out

    def populations(self, r_core, out=None, stream=None):
        """[i, 0]: ground-state population of instance i's current state, [i, 1]: its probability
        within |x| < r_core (see tdse_populations); a float64 device tensor n_inst x 2."""
        import torch
        if out is None:
            out = torch.empty((self.n_inst, 2), dtype=torch.float64, device=torch.device("cuda", self.device))
        _check(load().tdse_populations(self._h, float(r_core), _dev_ptr(out, "out"), _stream_ptr(stream)))
        return out

    def set_wait_limit(self, polls=1 << 22):
        """Bound of the MIXED bulk-copy waits in polls (see tdse_set_wait_limit; 0 = give up at once)."""
        _check(load().tdse_set_wait_limit(self._h, int(polls)))

    def set_adjoint_gamma_tape(self, enable=True):
        """Use the adjoint's gamma tape when it fits (see tdse_set_adjoint_gamma_tape)."""
        _check(load().tdse_set_adjoint_gamma_tape(self._h, 1 if enable else 0))

    def set_layout(self, lanes_per_instance=0):
        """Lanes per instance of the layout (see tdse_set_layout; 0 = cost model).  Discards the state."""
        _check(load().tdse_set_layout(self._h, int(lanes_per_instance)))
        self.lanes_per_instance = int(lanes_per_instance)

    def save_state(self, stream=None):
        """Device copy of every wavefunction (opaque layout; see tdse_copy_state)."""
        import torch
        buf = torch.empty(self.plan()["psi_bytes"] // 8, dtype=torch.float64, device=torch.device("cuda", self.device))
        _check(load().tdse_copy_state(self._h, _dev_ptr(buf, "state"), 0, _stream_ptr(stream)))
        return buf

    def load_state(self, buf, stream=None):
        _check(load().tdse_copy_state(self._h, _dev_ptr(buf, "state"), 1, _stream_ptr(stream)))

    def adjoint(self, E, gd, ga, gE=None, ckpt_every=256, stream=None):
        """dL/dE for loss gradients gd = dL/dd, ga = dL/da (device tensors in the row layout,
        sample_base 0), from the batch's current state as psi^0 (see tdse_adjoint)."""
        import torch
        if gE is None:
            gE = torch.zeros_like(E)
        _check(load().tdse_adjoint(self._h, _dev_ptr(E, "E"), _dev_ptr(gd, "gd"), _dev_ptr(ga, "ga"),
                                   _dev_ptr(gE, "gE"), int(ckpt_every), _stream_ptr(stream)))
        return gE

    def propagate_checkpointed(self, E, d, a, ckpt_every=256, step_begin=0, step_end=None, sample_base=0,
                               stream=None):
        """tdse_propagate that also records the adjoint's checkpoints (see tdse_propagate_checkpointed)."""
        if step_end is None:
            step_end = int(self.n_steps.max())
        _check(load().tdse_propagate_checkpointed(self._h, _dev_ptr(E, "E"), _dev_ptr(d, "d"), _dev_ptr(a, "a"),
                                                  int(sample_base), int(step_begin), int(step_end), int(ckpt_every),
                                                  _stream_ptr(stream)))

    def adjoint_checkpointed(self, E, gd, ga, gE=None, stream=None):
        """dL/dE from the last complete checkpointed propagation (see tdse_adjoint_checkpointed)."""
        import torch
        if gE is None:
            gE = torch.zeros_like(E)
        _check(load().tdse_adjoint_checkpointed(self._h, _dev_ptr(E, "E"), _dev_ptr(gd, "gd"), _dev_ptr(ga, "ga"),
                                                _dev_ptr(gE, "gE"), _stream_ptr(stream)))
        return gE

    def autotune(self, E, d, a, step_begin=0, step_end=None, sample_base=0, repeats=1, stream=None):
        """Time candidate launch shapes on steps [step_begin, step_end) of the field rows E (d and a
        rows there are overwritten) and keep the fastest (see tdse_autotune).  The batch's state is
        unchanged.  Returns the trials as dicts, in the order run."""
        if step_end is None:
            step_end = int(self.n_steps.max())
        cap = 64
        trials = (tdse_tune_trial * cap)()
        n = ctypes.c_int32(0)
        _check(load().tdse_autotune(self._h, _dev_ptr(E, "E"), _dev_ptr(d, "d"), _dev_ptr(a, "a"), int(sample_base),
                                    int(step_begin), int(step_end), int(repeats), trials, cap, ctypes.byref(n),
                                    _stream_ptr(stream)))
        return [dict(warps_per_cta=t.warps_per_cta, ctas_per_sm=t.ctas_per_sm, slice_steps=t.slice_steps,
                     ctas=t.ctas, ms=float(t.ms)) for t in trials[: min(n.value, cap)]]

    def set_launch(self, warps_per_cta=0, ctas_per_sm=0, slice_steps=0, max_ctas=0):
        """Override the persistent grid (see tdse_set_launch); 0 keeps a default."""
        _check(load().tdse_set_launch(self._h, int(warps_per_cta), int(ctas_per_sm), int(slice_steps),
                                      int(max_ctas)))


def spectrum(a, offsets, dt, k_begin, k_end, out=None, stream=None):
    """S[r, k - k_begin] = dt^2 |DFT of row r at bin k|^2 (see tdse_spectrum); a is a device tensor."""
    import torch
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    n_rows = offs.size - 1
    if out is None:
        out = torch.empty((n_rows, k_end - k_begin), dtype=torch.float64, device=a.device)
    _check(load().tdse_spectrum(_dev_ptr(a, "a"), offs.ctypes.data_as(_i64p), n_rows, float(dt), int(k_begin),
                                int(k_end), _dev_ptr(out, "S"), _stream_ptr(stream)))
    return out


def dipole_spectrum(a, offsets, dt, omegas, weight=None, out=None, stream=None):
    """out[r, w] = weight_r dt/sqrt(2 pi) sum_n a_r,n exp(i omegas[w] n dt) (see tdse_dipole_spectrum);
    a is a float64 device tensor holding the rows at offsets; returns a complex128 device tensor."""
    import torch
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    n_rows = offs.size - 1
    if out is None:
        out = torch.empty((n_rows, om.size), dtype=torch.complex128, device=a.device)
    if out.dtype != torch.complex128 or not out.is_contiguous() or out.numel() < n_rows * om.size:
        raise ValueError("out must be a contiguous complex128 tensor of n_rows x len(omegas)")
    wp = None
    if weight is not None:
        wp = _dev_ptr(weight, "weight")
        if weight.numel() < n_rows:
            raise ValueError("weight needs one value per row")
    with torch.cuda.device(a.device):
        _check(load().tdse_dipole_spectrum(_dev_ptr(a, "a"), offs.ctypes.data_as(_i64p), n_rows, float(dt),
                                           om.ctypes.data_as(_dp), int(om.size), wp,
                                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def hankel(S, rho_src, z_src, k, z_obs, rho_obs, out=None, stream=None):
    """Far field E[w, o] of a homogeneous medium (see tdse_hankel).  S: complex128 device tensor
    (n_rho, n_z, n_omega); grids are host arrays (SI units); returns a complex128 device tensor
    (n_omega, n_obs)."""
    import torch
    rs = np.ascontiguousarray(np.atleast_1d(rho_src), dtype=np.float64)
    zs = np.ascontiguousarray(np.atleast_1d(z_src), dtype=np.float64)
    kk = np.ascontiguousarray(np.atleast_1d(k), dtype=np.float64)
    ro = np.ascontiguousarray(np.atleast_1d(rho_obs), dtype=np.float64)
    if S.dtype != torch.complex128 or not S.is_cuda or not S.is_contiguous() or tuple(S.shape) != (rs.size, zs.size, kk.size):
        raise ValueError("S must be a contiguous complex128 CUDA tensor of shape (n_rho, n_z, n_omega)")
    if out is None:
        out = torch.empty((kk.size, ro.size), dtype=torch.complex128, device=S.device)
    if out.dtype != torch.complex128 or not out.is_contiguous() or out.numel() < kk.size * ro.size or out.device != S.device:
        raise ValueError("out must be a contiguous complex128 tensor of n_omega x n_obs on S's device")
    with torch.cuda.device(S.device):
        _check(load().tdse_hankel(ctypes.c_void_p(S.data_ptr()), rs.ctypes.data_as(_dp), int(rs.size),
                                  zs.ctypes.data_as(_dp), int(zs.size), kk.ctypes.data_as(_dp), int(kk.size),
                                  float(z_obs), ro.ctypes.data_as(_dp), int(ro.size), ctypes.c_void_p(out.data_ptr()),
                                  int(S.device.index or 0), _stream_ptr(stream)))
    return out


def model_layout(N, dx, softening, dt, charge=1.0, precision=TDSE_FP64, scheme=TDSE_FULL_CN, sm_count=152):
    """Lanes per instance the cost model picks for such a batch (see tdse_model_layout); no GPU needed."""
    N = np.atleast_1d(np.asarray(N, dtype=np.int64))
    n = N.size
    dx = np.broadcast_to(np.asarray(dx, dtype=np.float64), (n,))
    a = np.broadcast_to(np.asarray(softening, dtype=np.float64), (n,))
    Z = np.broadcast_to(np.asarray(charge, dtype=np.float64), (n,))
    arr = (tdse_instance * n)(*[tdse_instance(int(N[i]), float(dx[i]), float(a[i]), float(Z[i])) for i in range(n)])
    out = ctypes.c_int32(0)
    _check(load().tdse_model_layout(arr, n, float(dt), int(precision), int(scheme), int(sm_count), ctypes.byref(out)))
    return int(out.value)


def resample_field(coarse, dt_coarse, dt_fine, n_fine, out=None, out_stride=None, stream=None):
    """Zero-padded DFT interpolation of coarse field rows (see tdse_resample_field).  coarse: float64
    CUDA tensor (n_rows, M); returns (n_rows, out_stride) with the first n_fine columns written."""
    import torch
    n_rows, M = coarse.shape
    stride = int(out_stride or n_fine)
    if out is None:
        out = torch.zeros((n_rows, stride), dtype=torch.float64, device=coarse.device)
    _check(load().tdse_resample_field(_dev_ptr(coarse.contiguous(), "coarse"), int(n_rows), int(M), float(dt_coarse),
                                      float(dt_fine), int(n_fine), stride, _dev_ptr(out, "out"),
                                      int(coarse.device.index or 0), _stream_ptr(stream)))
    return out


def tdse_propagate_static(inst, n_inst, dt, n_steps, row_stride, psi, E, d, a, step_begin, step_end, sample_base=0,
                          absorber=(20.0, 0.125), stream=None):
    """Allocation-free propagation (see include/tdse.h).  inst = (N, dx, softening, charge); psi is a
    float64 device tensor holding the lane-interleaved wavefunctions, 2 * 32 * ceil(n_inst/32) * N values."""
    import torch
    ab = None if absorber is None else ctypes.byref(tdse_absorber(float(absorber[0]), float(absorber[1])))
    ins = tdse_instance(int(inst[0]), float(inst[1]), float(inst[2]), float(inst[3]))
    for name, t in (("psi", psi), ("E", E), ("d", d), ("a", a)):
        _dev_ptr(t, name)
        if t.device != psi.device:
            raise ValueError("%s is on %s, psi on %s: every buffer must be on one device" % (name, t.device, psi.device))
    need_psi = 2 * 32 * ((int(n_inst) + 31) // 32) * int(inst[0])
    if psi.numel() < need_psi:
        raise ValueError("psi holds %d doubles, the lane-interleaved layout needs %d" % (psi.numel(), need_psi))
    need_row = int(n_inst) * int(row_stride)
    for name, t in (("E", E), ("d", d), ("a", a)):
        if t.numel() < need_row:
            raise ValueError("%s holds %d doubles, n_inst * row_stride = %d" % (name, t.numel(), need_row))
    # the entry point launches on the current device: make it the buffers' device
    with torch.cuda.device(psi.device):
        _check(load().tdse_propagate_static(ctypes.byref(ins), int(n_inst), float(dt), ab, int(n_steps),
                                            int(row_stride), _dev_ptr(psi, "psi"), _dev_ptr(E, "E"), _dev_ptr(d, "d"),
                                            _dev_ptr(a, "a"), int(sample_base), int(step_begin), int(step_end),
                                            _stream_ptr(stream)))


def tdse_probe_pipes(device=0):
    """Measured FP64/FP32 pipe rates of the device (see include/tdse.h) as a dict."""
    r = tdse_pipe_rates()
    _check(load().tdse_probe_pipes(int(device), ctypes.byref(r)))
    return dict(fp64_fma_tflops=r.fp64_fma_tflops, fp64_warp_instr_per_s=r.fp64_warp_instr_per_s,
                fp64_one_lane_warp_instr_per_s=r.fp64_one_lane_warp_instr_per_s,
                fp64_tflops_warps_per_sm=list(r.fp64_tflops_warps_per_sm), fp32_fma_tflops=r.fp32_fma_tflops,
                cvt_pairs_per_s=r.cvt_pairs_per_s, sm_count=r.sm_count, sm_clock_mhz=r.sm_clock_mhz,
                rcp_f64_approx_fma_slots=r.rcp_f64_approx_fma_slots, rcp_seed_fma_slots=r.rcp_seed_fma_slots,
                dadd_fma_slots=r.dadd_fma_slots, dmul_fma_slots=r.dmul_fma_slots,
                add_as_fma_slots=r.add_as_fma_slots, mul_as_fma_slots=r.mul_as_fma_slots,
                fma_repeat_slots=r.fma_repeat_slots)


def _make_autograd():
    import torch

    class TDSEPropagate(torch.autograd.Function):
        """(d, a) = propagate(E) for an FP64 FULL_CN batch, differentiable with respect to the field
        samples E through the library's adjoint kernel.  The batch must hold the initial state; the
        forward pass records the adjoint's checkpoints (so the backward pass recomputes only from them)
        and the initial state is restored afterwards.  The recording belongs to the batch: run each
        forward's backward before the next forward on the same batch."""

        @staticmethod
        def forward(ctx, E, batch, ckpt_every):
            E = E.contiguous()
            psi0 = batch.save_state()
            d = torch.zeros_like(E)
            a = torch.zeros_like(E)
            batch.propagate_checkpointed(E, d, a, ckpt_every)
            batch.load_state(psi0)
            ctx.batch = batch
            ctx.ckpt_every = ckpt_every
            ctx.save_for_backward(E)
            return d, a

        @staticmethod
        def backward(ctx, gd, ga):
            (E,) = ctx.saved_tensors
            gd = torch.zeros_like(E) if gd is None else gd.contiguous()
            ga = torch.zeros_like(E) if ga is None else ga.contiguous()
            gE = ctx.batch.adjoint_checkpointed(E, gd, ga)
            return gE, None, None

    return TDSEPropagate


_autograd_fn = None


def tdse_propagate_autograd(E, batch, ckpt_every=256):
    """Differentiable propagation: returns (d, a); gradients flow to E (see TDSEPropagate)."""
    global _autograd_fn
    if _autograd_fn is None:
        _autograd_fn = _make_autograd()
    return _autograd_fn.apply(E, batch, ckpt_every)
