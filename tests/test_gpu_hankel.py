"""The output side of the path on the GPU against the FP64 oracle: the macroscopic source spectrum
(tdse_dipole_spectrum, the paper's Fourier convention) and the far field of a homogeneous medium
(tdse_hankel, Eq. "Hankel long homogeneous" of Sec. 3.2 by direct grid integration, Sec. 4.3).

Tolerance.  Both sides sum the same FP64 terms in different orders; the far field is a coherent
sum whose terms cancel (the field at a point can be far below the sum of magnitudes), so the bound
is relative to each frequency's largest |E|: 1e-10 there, three orders above the rounding of the
sums.  The source spectrum is compared at 1e-12 of its largest value."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_dipole_spectrum_matches_oracle(env):
    """Ragged rows (including an empty one and one shorter than a tile), weights, frequencies at
    and off the DFT bins, negative and zero frequencies."""
    tdse, oracle = env
    rng = np.random.default_rng(71)
    lens = [0, 1, 300, 513, 4097, 20000]
    offs = np.concatenate([[0], np.cumsum(lens)])
    a = rng.standard_normal(int(offs[-1]))
    dt = 0.02
    om = np.concatenate([[0.0, -0.3], np.linspace(0.05, 2.0, 200)])
    wt = rng.uniform(0.5, 2.0, len(lens))
    dev = torch.device("cuda", 0)
    out = tdse.dipole_spectrum(torch.from_numpy(a).to(dev), offs, dt, om, weight=torch.from_numpy(wt).to(dev))
    got = out.cpu().numpy()
    for r, L in enumerate(lens):
        ref = oracle.dipole_spectrum(a[offs[r]: offs[r + 1]], dt, om, weight=wt[r])
        assert np.max(np.abs(got[r] - ref)) <= 1e-12 * max(np.max(np.abs(ref)), 1e-300), r
    out2 = tdse.dipole_spectrum(torch.from_numpy(a).to(dev), offs, dt, om)
    assert np.allclose(out2.cpu().numpy() * wt[:, None], got, rtol=1e-14, atol=0)


def _check(E, ref):
    for w in range(ref.shape[0]):
        scale = np.max(np.abs(ref[w]))
        assert np.max(np.abs(E[w] - ref[w])) <= 1e-10 * scale, w


@pytest.mark.parametrize("n_rho,n_z,n_obs", [(40, 24, 150), (64, 128, 128), (1500, 3, 33), (7, 1, 260)])
def test_hankel_matches_oracle(env, n_rho, n_z, n_obs):
    """Random complex sources on non-uniform grids: several z' tiles (64 x 128), a tile holding a
    single plane (1500 radii), the thin medium (one plane), observation counts that leave a ragged
    CTA, rho' starting at 0 and above 0."""
    tdse, oracle = env
    rng = np.random.default_rng(73 + n_rho)
    lam = np.array([40e-9, 52e-9, 61e-9])
    k = 2 * np.pi / lam
    rho = np.sort(rng.uniform(0.0, 8e-5, n_rho))
    rho[0] = 0.0 if n_rho % 2 == 0 else rho[0]
    z = np.sort(rng.uniform(-5e-3, 5e-3, n_z))
    ro = np.linspace(0.0, 2.5e-3, n_obs)
    S = (rng.standard_normal((n_rho, n_z, k.size)) + 1j * rng.standard_normal((n_rho, n_z, k.size)))
    S *= np.exp(-(rho / 4e-5) ** 2)[:, None, None]
    dev = torch.device("cuda", 0)
    E = tdse.hankel(torch.from_numpy(S).to(dev), rho, z, k, 0.6, ro).cpu().numpy()
    _check(E, oracle.hankel_far_field(S, rho, z, k, 0.6, ro))


def test_far_field_of_a_propagated_volume(env):
    """End to end on the GPU: a small Gaussian-beam volume (4 radii x 6 planes) propagated through
    the pulse, its a(t) transformed at harmonic frequencies with a density weight, and the far field
    of that source; the oracle recomputes the transform and the integral from the GPU's own a(t)."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    wl = inputs.gaussian_beam_volume(n_r=4, n_z=6, n_cycles=2, N=600, dx=0.2, dt=0.05, seed=5)
    n, N, dx, dt = wl.n_inst, int(wl.N[0]), float(wl.dx[0]), wl.dt
    Nt = int(wl.n_steps[0])
    a_soft = oracle.fit_softening(wl.target_energy, N, dx)
    rows = np.concatenate(wl.field_rows())
    dev = torch.device("cuda", 0)
    Et = torch.from_numpy(rows).to(dev)
    b = tdse.Batch(wl.N, dx, a_soft, wl.n_steps, dt, absorber=(wl.mask_width, wl.mask_exponent))
    b.ground_state(dtau=0.1, max_iter=800, tol=0.0)
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    b.close()
    offs = np.arange(n + 1) * (Nt + 1)
    omega0 = float(wl.omega[0])
    om = omega0 * np.array([3.0, 5.0, 7.0, 9.0])
    rho = np.linspace(0.0, wl.extra["w0_m"], wl.extra["n_r"])
    z = np.linspace(-wl.extra["zR_m"], wl.extra["zR_m"], wl.extra["n_z"])
    dens = np.linspace(0.8, 1.2, n)
    S = tdse.dipole_spectrum(acc, offs, dt, om, weight=torch.from_numpy(dens).to(dev))
    t_au_s, c = 2.4188843265857e-17, 299792458.0
    k = om / t_au_s / c
    ro = np.linspace(0.0, 4e-3, 50)
    E = tdse.hankel(S.view(wl.extra["n_r"], wl.extra["n_z"], om.size), rho, z, k, 0.5, ro).cpu().numpy()
    ah = acc.cpu().numpy()
    S_ref = np.array([oracle.dipole_spectrum(ah[offs[i]: offs[i + 1]], dt, om, weight=dens[i]) for i in range(n)])
    assert np.max(np.abs(S.cpu().numpy() - S_ref)) <= 1e-12 * np.max(np.abs(S_ref))
    _check(E, oracle.hankel_far_field(S_ref.reshape(wl.extra["n_r"], wl.extra["n_z"], om.size), rho, z, k, 0.5, ro))
