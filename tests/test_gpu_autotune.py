"""The launch-shape autotuner (tdse_autotune): it leaves the batch's state as it found it, keeps the
fastest shape it timed, and the propagation under that shape still matches the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_SERIES = 1e-9
GS_KW = dict(dtau=0.1, max_iter=1500, tol=0.0)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_04115_gb300 import build, tdse
    build.build()
    tdse.load()
    import oracle
    oracle.build()
    return tdse, oracle


def _rel(x, ref, floor=1e-4):   # floor: see test_gpu_parity._rel
    return float(np.max(np.abs(np.asarray(x) - np.asarray(ref))) / max(np.max(np.abs(ref)), floor))


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_restores_state_and_keeps_fastest(env, precision):
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    rng = np.random.default_rng(17)
    n = 70   # three groups of 32 lanes, the last one partly empty
    N = rng.choice(np.array([512, 1024]), n)
    dx, soft, dt = 0.2, 1.2, 0.05
    nt = rng.integers(150, 260, n)
    w = inputs.omega_from_wavelength_nm(800.0)
    rows = [inputs.sin2_pulse(int(nt[i]), dt, rng.uniform(0.03, 0.07), w, 0.75, 0.0) for i in range(n)]
    offs = np.concatenate([[0], np.cumsum(nt + 1)])
    E = np.zeros(int(offs[-1]))
    for i, r in enumerate(rows):
        E[offs[i]: offs[i] + r.size] = r
    dev = torch.device("cuda", 0)
    Et = torch.from_numpy(E).to(dev)
    b = tdse.Batch(N, dx, soft, nt, dt, row_offsets=offs, absorber=(10.0, 0.125), precision=precision)
    b.ground_state(**GS_KW)
    before = b.save_state().clone()
    d = torch.zeros_like(Et)
    acc = torch.zeros_like(Et)
    trials = b.autotune(Et, d, acc, 0, 64, repeats=2)
    torch.cuda.synchronize()
    assert len(trials) >= 2
    assert all(t["ms"] > 0 for t in trials)
    # the state is the one before the call, bit for bit
    assert torch.equal(b.save_state(), before)
    # the kept shape is the fastest trial
    best = min(trials, key=lambda t: t["ms"])
    p = b.plan()
    assert (p["warps_per_cta"], p["ctas"], p["slice_steps"]) == (best["warps_per_cta"], best["ctas"], best["slice_steps"])
    # and the propagation under it matches the oracle
    d.zero_()
    acc.zero_()
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    assert b.check() == -1
    dh, ah = d.cpu().numpy(), acc.cpu().numpy()
    tol = RTOL_SERIES if precision == 0 else 2e-3
    for i in inputs.subsample(n, 6, 3):
        psi0, _, _ = oracle.ground_state(int(N[i]), dx, soft, **GS_KW)
        m = oracle.mask(int(N[i]), dx, 10.0, 0.125)
        _, d_o, a_o = oracle.propagate(psi0, rows[i], dx, dt, soft, mask_values=m)
        sl = slice(offs[i], offs[i + 1])
        assert _rel(dh[sl], d_o) < tol, i
        assert _rel(ah[sl], a_o) < tol, i
    b.close()


def test_autotune_rejects_bad_arguments(env):
    tdse, _ = env
    b = tdse.Batch([256], 0.2, 1.2, [10], 0.05)
    b.ground_state(dtau=0.1, max_iter=10, tol=0.0)
    E = torch.zeros(11, dtype=torch.float64, device="cuda")
    with pytest.raises(tdse.TDSEError):
        b.autotune(E, torch.zeros_like(E), torch.zeros_like(E), 5, 5)   # empty range
    with pytest.raises(tdse.TDSEError):
        b.autotune(E, torch.zeros_like(E), torch.zeros_like(E), 0, 5, repeats=0)
    b.close()
