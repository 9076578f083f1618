"""tdse_propagate_static: the allocation-free entry point for callers that cannot call cudaMalloc
(for instance code inside a host application that hands out all device memory from its own pool).

It must give the same results as the allocating path (tdse_batch_create + tdse_propagate) on the
same inputs, call after call: the static scratch keeps the previous call's contents, so the second
call checks that everything that has to start from zero is cleared.  This file is collected last;
it must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-9   # the parity tolerance of the FP64 path (see test_gpu_parity.py)


def _rel(x, ref, floor=1e-6):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(ref))) / max(np.max(np.abs(ref)), floor))


def _env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_04115_gb300 import build, inputs, tdse
    build.build()
    tdse.load()
    return inputs, tdse


def _compare(tdse, inputs, n, N, dx, a, dt, nt, absorber, calls, gs_iters=1500):
    """Propagate the same initial states through tdse_propagate and tdse_propagate_static over the
    given consecutive step ranges; compare d, a after every call and psi at the end."""
    dev = torch.device("cuda", 0)
    inst = (N, dx, a, 1.0)
    rows = [inputs.sin2_pulse(nt, dt, 0.04 + 0.001 * i, 0.057, 1.0, 0.1 * i) for i in range(n)]
    stride = nt + 1
    E = torch.from_numpy(np.concatenate(rows)).to(dev)

    b = tdse.Batch([N] * n, dx, a, [nt] * n, dt, absorber=absorber, lanes_per_instance=1)
    b.ground_state(max_iter=gs_iters, tol=0.0)
    # the same initial states in the lane-interleaved layout of the static entry point
    groups = (n + 31) // 32
    psi = torch.zeros((groups, N, 32, 2), dtype=torch.float64, device=dev)
    for i in range(n):
        psi[i // 32, :, i % 32, :] = torch.view_as_real(b.get_psi(i))
    psi = psi.reshape(-1).contiguous()

    d_ref, a_ref = torch.zeros_like(E), torch.zeros_like(E)
    d_st, a_st = torch.zeros_like(E), torch.zeros_like(E)
    for (s0, s1) in calls:
        b.propagate(E, d_ref, a_ref, s0, s1)
        tdse.tdse_propagate_static(inst, n, dt, nt, stride, psi, E, d_st, a_st, s0, s1, absorber=absorber)
        torch.cuda.synchronize()
        hi = s1 + 1
        for i in range(n):
            sl = slice(i * stride, i * stride + hi)
            assert _rel(d_st[sl].cpu().numpy(), d_ref[sl].cpu().numpy()) < RTOL, (s0, i)
            assert _rel(a_st[sl].cpu().numpy(), a_ref[sl].cpu().numpy()) < RTOL, (s0, i)
    psi_st = psi.view(groups, N, 32, 2)
    for i in sorted({0, min(31, n - 1), min(32, n - 1), n - 1}):
        ref = torch.view_as_real(b.get_psi(i))
        assert float((psi_st[i // 32, :, i % 32, :] - ref).abs().max()) < 1e-12
    b.close()


def test_static_entry_point_matches_allocating_path_on_consecutive_calls():
    inputs, tdse = _env()
    dev = torch.device("cuda", 0)
    # 45 instances: the second group is ragged; two calls in a row
    _compare(tdse, inputs, 45, 512, 0.2, 1.19, 0.05, 300, (20.0, 0.125), [(0, 140), (140, 300)])
    # no absorber: the plateau is the whole grid and no point is masked
    _compare(tdse, inputs, 40, 384, 0.2, 1.19, 0.05, 120, None, [(0, 60), (60, 120)])
    # N = 16384: the solver rows of one CTA take 17 MB, so only 3 CTAs fit the 64 MiB array and the
    # 4 groups share them (the static grid is smaller than both the group count and the SM count)
    _compare(tdse, inputs, 128, 16384, 0.2, 1.19, 0.05, 16, (20.0, 0.125), [(0, 8), (8, 16)], gs_iters=100)

    # sizes whose scratch does not fit the static array are refused by the library with a clear
    # error, before anything is launched (the raw C call: the binding would refuse the short
    # buffers itself)
    import ctypes
    L = tdse.load()
    small = torch.zeros(64, dtype=torch.float64, device=dev)
    p = ctypes.c_void_p(small.data_ptr())
    ins = tdse.tdse_instance(1 << 20, 0.1, 1.2, 1.0)
    rc = L.tdse_propagate_static(ctypes.byref(ins), 32, 0.05, None, 1, 2, p, p, p, p, 0, 0, 1,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tdse.TDSE_ERR_ARG
    assert "static scratch" in tdse.tdse_last_error()
    # the binding checks buffer sizes against the layout before the call
    with pytest.raises(ValueError):
        tdse.tdse_propagate_static((512, 0.2, 1.19, 1.0), 32, 0.05, 4, 5, small, small, small, small, 0, 4)
