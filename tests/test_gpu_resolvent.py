"""Energy distribution of the instance states (tdse_energy_distribution, Sec. 6.1) against the FP64
oracle: the oracle is handed the GPU's own wavefunctions (tdse_get_psi), so the comparison covers
the resolvent solves alone.  Both schemes, both precisions (the solves run in FP64), ragged
multi-class batches, 32-wide and lane-split layouts."""
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


@pytest.mark.parametrize("scheme,precision,lanes", [(0, 0, 1), (0, 0, 8), (1, 0, 1), (0, 1, 1)])
def test_energy_distribution_matches_oracle(env, scheme, precision, lanes):
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    rng = np.random.default_rng(61)
    n = 37
    classes = [(300, 0.2, 1.2), (420, 0.15, 1.3)]
    cls = rng.integers(0, 2, n)
    N = np.array([classes[c][0] for c in cls])
    dx = np.array([classes[c][1] for c in cls])
    soft = np.array([classes[c][2] for c in cls])
    dt = 0.05
    nt = rng.integers(100, 260, n)
    rows = [inputs.sin2_pulse(int(k), dt, rng.uniform(0.05, 0.12), 0.057, 1.0, rng.uniform(0, 6)) for k in nt]
    offs = np.concatenate([[0], np.cumsum(nt + 1)])
    E = np.zeros(int(offs[-1]))
    for i, r in enumerate(rows):
        E[offs[i]: offs[i] + r.size] = r
    dev = torch.device("cuda", 0)
    Et = torch.from_numpy(E).to(dev)
    b = tdse.Batch(N, dx, soft, nt, dt, row_offsets=offs, absorber=(10.0, 0.125), precision=precision,
                   scheme=scheme, lanes_per_instance=lanes)
    b.ground_state(**GS_KW)
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    E_grid = np.concatenate([np.linspace(-0.9, 1.5, 61), [-0.579, 0.0, 0.3]])
    eps = 0.03
    P = b.energy_distribution(E_grid, eps).cpu().numpy()
    assert P.shape == (n, E_grid.size)
    for i in range(n):
        psi = b.get_psi(i).cpu().numpy()
        ref = oracle.energy_distribution(psi, E_grid, dx[i], soft[i], eps, scheme=scheme)
        assert np.max(np.abs(P[i] - ref)) < 1e-9 * np.max(ref), i
    b.close()


def test_energy_distribution_of_ground_state_peaks_at_its_energy(env):
    """Right after the ground state the distribution is a Lorentzian at the ground energy: its peak
    value is 1/(pi eps) (norm 1) and half of it at E_g +- eps."""
    tdse, _ = env
    N, dx, a, eps = 600, 0.2, 1.19, 0.02
    b = tdse.Batch([N] * 3, dx, a, [1] * 3, 0.05)
    e, _ = b.ground_state(dtau=0.1, max_iter=20000, tol=1e-13)
    Eg = float(e[0])
    P = b.energy_distribution([Eg, Eg - eps, Eg + eps], eps).cpu().numpy()
    for i in range(3):
        assert abs(P[i, 0] * np.pi * eps - 1.0) < 1e-6
        assert abs(P[i, 1] * np.pi * eps - 0.5) < 1e-6
        assert abs(P[i, 2] * np.pi * eps - 0.5) < 1e-6
    b.close()


@pytest.mark.parametrize("scheme,precision", [(0, 0), (1, 0), (0, 1)])
def test_ionisation_matches_oracle(env, scheme, precision):
    """Ionisation probability (Sec. 6.1: the energy integral of P over the continuum) of propagated
    states against the oracle's trapezoid over the same nodes, given the GPU's own wavefunctions;
    the distribution written beside it equals tdse_energy_distribution's.  Right after the ground
    state every instance gives the bound state's Lorentzian tail above the threshold,
    (atan(eps/|E_g|) - atan(eps/(E_max - E_g)))/pi."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    rng = np.random.default_rng(67)
    n, N, dx, a, dt = 35, 400, 0.2, 1.19, 0.05
    nt = rng.integers(150, 300, n)
    rows = [inputs.sin2_pulse(int(k), dt, rng.uniform(0.06, 0.12), 0.057, 1.0, rng.uniform(0, 6)) for k in nt]
    offs = np.concatenate([[0], np.cumsum(nt + 1)])
    E = np.zeros(int(offs[-1]))
    for i, r in enumerate(rows):
        E[offs[i]: offs[i] + r.size] = r
    dev = torch.device("cuda", 0)
    Et = torch.from_numpy(E).to(dev)
    b = tdse.Batch([N] * n, dx, a, nt, dt, row_offsets=offs, absorber=(10.0, 0.125), precision=precision,
                   scheme=scheme)
    eps = 0.03
    nodes = np.linspace(0.0, 2.5, 401)
    e, _ = b.ground_state(**GS_KW)
    ion0 = b.ionisation(nodes, eps).cpu().numpy()
    Eg = float(e[0])
    tail = (np.arctan(eps / abs(Eg)) - np.arctan(eps / (2.5 - Eg))) / np.pi
    assert np.max(np.abs(ion0 - tail)) < 2e-3 * tail      # trapezoid error at h = eps / 4.8
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    P = torch.empty((n, nodes.size), dtype=torch.float64, device=dev)
    ion = b.ionisation(nodes, eps, P_out=P).cpu().numpy()
    P2 = b.energy_distribution(nodes, eps).cpu().numpy()
    assert np.array_equal(P.cpu().numpy(), P2)
    for i in range(n):
        psi = b.get_psi(i).cpu().numpy()
        ref = oracle.ionisation(psi, nodes, dx, a, eps, scheme=scheme)
        assert abs(ion[i] - ref) < 1e-10 * max(ref, 1e-3), (i, ion[i], ref)
    with pytest.raises(tdse.TDSEError):
        b.ionisation([0.0, 1.0, 0.5], eps)                  # nodes must ascend
    b.close()
