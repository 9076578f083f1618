"""Populations of the instance states (tdse_populations, Sec. 7.5) against the FP64 oracle: the
oracle is handed the GPU's own wavefunctions (tdse_get_psi) and its own ground state, so the
comparison covers the reductions.  Both schemes, both precisions, ragged multi-class batches,
32-wide and lane-split layouts; the ground state itself, r_core limits and the state check.  The
third class's box (+-80 a.u.) is wider than the ground state's support, so the kernel reads only
part of its rows there (the tail it skips is below 1e-17) while the oracle sums every point."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GS_KW = dict(dtau=0.1, max_iter=800, tol=0.0)


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


# (scheme, precision, lanes per instance, instances): the kernel gives each group a cluster of up
# to 8 CTAs sized to fill the SMs; 180 one-instance groups take clusters of fewer than 8
@pytest.mark.parametrize("scheme,precision,lanes,n", [(0, 0, 0, 45), (0, 0, 8, 45), (1, 0, 1, 45), (0, 1, 0, 45),
                                                      (1, 1, 4, 45), (0, 0, 32, 180)])
def test_populations_match_oracle(env, scheme, precision, lanes, n):
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    rng = np.random.default_rng(73)
    # three classes, ragged groups
    classes = [(300, 0.2, 1.2), (420, 0.15, 1.3), (1600, 0.1, 1.25)]
    cls = rng.integers(0, 3, n)
    N = np.array([classes[c][0] for c in cls])
    dx = np.array([classes[c][1] for c in cls])
    soft = np.array([classes[c][2] for c in cls])
    dt = 0.05
    nt = rng.integers(100, 300, n)
    rows = [inputs.sin2_pulse(int(k), dt, rng.uniform(0.05, 0.15), 0.057, 1.0, rng.uniform(0, 6)) for k in nt]
    offs = np.concatenate([[0], np.cumsum(nt + 1)])
    E = np.zeros(int(offs[-1]))
    for i, r in enumerate(rows):
        E[offs[i]: offs[i] + r.size] = r
    dev = torch.device("cuda", 0)
    Et = torch.from_numpy(E).to(dev)
    b = tdse.Batch(N, dx, soft, nt, dt, row_offsets=offs, absorber=(10.0, 0.125), precision=precision,
                   scheme=scheme, lanes_per_instance=lanes)
    b.ground_state(**GS_KW)
    psi0 = {c: oracle.ground_state(classes[c][0], classes[c][1], classes[c][2], scheme=scheme, **GS_KW)[0]
            for c in range(len(classes))}
    # right after the ground state: population 1, near-core probability of psi0
    pop = b.populations(3.0).cpu().numpy()
    tol1 = 1e-12 if precision == 0 else 1e-6
    for i in range(n):
        assert abs(pop[i, 0] - 1.0) < tol1, i
        ref = oracle.populations(psi0[cls[i]], psi0[cls[i]], dx[i], soft[i], 3.0)
        assert abs(pop[i, 1] - ref[1]) < tol1, i
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    for r_core in (2.5, 0.0, float("inf")):
        pop = b.populations(r_core).cpu().numpy()
        for i in range(n):
            psi = b.get_psi(i).cpu().numpy()
            ref = oracle.populations(psi, psi0[cls[i]], dx[i], soft[i], r_core)
            assert abs(pop[i, 0] - ref[0]) < 1e-10, (i, r_core)
            assert abs(pop[i, 1] - ref[1]) < 1e-12, (i, r_core)
            if r_core == 0.0:
                assert pop[i, 1] == 0.0
    # the field moved population out of the ground state, and the mask took some norm
    assert np.min(pop[:, 0]) < 1.0 - 1e-4
    b.close()


def test_populations_need_a_ground_state(env):
    tdse, _ = env
    b = tdse.Batch([256], 0.2, 1.2, [10], 0.05)
    b.set_psi(0, torch.full((256,), 0.1, dtype=torch.complex128, device="cuda"))
    with pytest.raises(tdse.TDSEError):
        b.populations(1.0)
    b.ground_state(dtau=0.1, max_iter=10, tol=0.0)
    with pytest.raises(tdse.TDSEError):
        b.populations(-1.0)
    with pytest.raises(tdse.TDSEError):
        b.populations(float("nan"))
    b.populations(1.0)
    b.set_layout(8)   # discards the state
    with pytest.raises(tdse.TDSEError):
        b.populations(1.0)
    b.close()


@pytest.mark.parametrize("n", [250, 1300])
def test_populations_many_groups(env, n):
    """One-instance groups: 250 give clusters of 5 CTAs (the volume benchmark's shape, 256 groups),
    1300 exceed the grid target so every cluster is a single CTA; sampled instances against the
    oracle."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    rng = np.random.default_rng(29)
    N, dx, a, dt = 160, 0.25, 1.2, 0.05
    nt = 120
    E = np.concatenate([inputs.sin2_pulse(nt, dt, rng.uniform(0.05, 0.2), 0.057, 1.0, rng.uniform(0, 6))
                        for _ in range(n)])
    Et = torch.from_numpy(E).to("cuda")
    b = tdse.Batch([N] * n, dx, a, [nt] * n, dt, absorber=(8.0, 0.125), lanes_per_instance=32)
    b.ground_state(**GS_KW)
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    pop = b.populations(1.5).cpu().numpy()
    psi0 = oracle.ground_state(N, dx, a, **GS_KW)[0]
    for i in [0, 1, n - 1] + list(rng.integers(0, n, 20)):
        ref = oracle.populations(b.get_psi(int(i)).cpu().numpy(), psi0, dx, a, 1.5)
        assert abs(pop[i, 0] - ref[0]) < 1e-10, i
        assert abs(pop[i, 1] - ref[1]) < 1e-12, i
    b.close()


def test_populations_mixed_subnormal_and_zero_states(env):
    """MIXED states stored as float: entries that are float subnormals, signed zeros and normals
    (the kernel widens them to double with integer operations) give the oracle's sums over the
    same stored values."""
    tdse, oracle = env
    N, dx, a = 256, 0.2, 1.2
    b = tdse.Batch([N] * 3, dx, a, [10] * 3, 0.05, precision=1)
    b.ground_state(**GS_KW)
    psi0 = oracle.ground_state(N, dx, a, **GS_KW)[0]
    rng = np.random.default_rng(5)
    scales = [1e-40, 2e-39, 0.05]   # subnormal, subnormal near the normal range, normal
    for i, sc in enumerate(scales):
        v = sc * (rng.uniform(-1, 1, N) + 1j * rng.uniform(-1, 1, N))
        v[::7] = 0.0
        v[3::11] = -0.0
        b.set_psi(i, torch.from_numpy(v).to("cuda"))
    pop = b.populations(4.0).cpu().numpy()
    for i in range(3):
        psi = b.get_psi(i).cpu().numpy()
        ref = oracle.populations(psi, psi0, dx, a, 4.0)
        assert ref[0] > 0 and ref[1] > 0
        assert abs(pop[i, 0] - ref[0]) <= 1e-9 * ref[0], i
        assert abs(pop[i, 1] - ref[1]) <= 1e-12 * ref[1], i
    b.close()
