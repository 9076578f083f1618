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


def test_static_entry_point_matches_allocating_path_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_04115_gb300 import build, inputs, tdse
    build.build()
    tdse.load()
    dev = torch.device("cuda", 0)
    n, N, dx, a, dt, nt = 45, 512, 0.2, 1.19, 0.05, 300      # 45: the second group is ragged
    inst = (N, dx, a, 1.0)
    rows = [inputs.sin2_pulse(nt, dt, 0.04 + 0.001 * i, 0.057, 1.0, 0.1 * i) for i in range(n)]
    stride = nt + 1
    E = torch.from_numpy(np.concatenate(rows)).to(dev)

    b = tdse.Batch([N] * n, dx, a, [nt] * n, dt, absorber=(20.0, 0.125))
    b.ground_state(max_iter=1500, tol=0.0)
    # the same initial states in the lane-interleaved layout of the static entry point
    groups = (n + 31) // 32
    psi = torch.zeros((groups, N, 32, 2), dtype=torch.float64, device=dev)
    for i in range(n):
        psi[i // 32, :, i % 32, :] = torch.view_as_real(b.get_psi(i))
    psi = psi.reshape(-1).contiguous()

    d_ref, a_ref = torch.zeros_like(E), torch.zeros_like(E)
    d_st, a_st = torch.zeros_like(E), torch.zeros_like(E)
    for (s0, s1) in [(0, 140), (140, nt)]:          # two calls in a row
        b.propagate(E, d_ref, a_ref, s0, s1)
        tdse.tdse_propagate_static(inst, n, dt, nt, stride, psi, E, d_st, a_st, s0, s1)
        torch.cuda.synchronize()
        hi = s1 + 1
        for i in range(n):
            sl = slice(i * stride, i * stride + hi)
            assert _rel(d_st[sl].cpu().numpy(), d_ref[sl].cpu().numpy()) < RTOL, (s0, i)
            assert _rel(a_st[sl].cpu().numpy(), a_ref[sl].cpu().numpy()) < RTOL, (s0, i)
    psi_st = psi.view(groups, N, 32, 2)
    for i in (0, 31, 32, n - 1):
        ref = torch.view_as_real(b.get_psi(i))
        assert float((psi_st[i // 32, :, i % 32, :] - ref).abs().max()) < 1e-12
    b.close()

    # sizes whose scratch does not fit the static array are refused with a clear error
    with pytest.raises(tdse.TDSEError) as ei:
        big = torch.zeros(64, dtype=torch.float64, device=dev)
        tdse.tdse_propagate_static((1 << 20, 0.1, 1.2, 1.0), 32, dt, 1, 2, big, big, big, big, 0, 1)
    assert ei.value.status == tdse.TDSE_ERR_ARG
    assert "static scratch" in tdse.tdse_last_error()
