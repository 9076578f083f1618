"""Complete propagations at the configurations' own sizes and lengths, asserted against the FP64
oracle with the stated spectral bounds (spectral_metrics: relative L2 over q <= 1.5 q_cut and the
worst odd harmonic within four decades of the strongest; FP64_BOUND and MIXED_BOUND).

Each test runs a seeded subsample of a configuration's instances through the whole pulse in a batch
of its own, with the launch layout the full batch uses (32 instances per warp, the same warps per
CTA), so every instance goes through exactly the arithmetic it gets inside the full batch
(test_gpu_parity.py::test_batch_position_invariance: an instance's results do not depend on its
slot or neighbours).  The oracle runs the same instances in spawned processes, one per core."""
import numpy as np
import pytest

from spectral_metrics import FP64_BOUND, MIXED_BOUND, harmonic_cutoff, oracle_pool_map, spectral_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _gpu_run(tdse, wl, idx, soft, precision, warps, rows):
    """Propagate instances idx of workload wl (whole pulse) in one batch with 32-wide groups."""
    dev = torch.device("cuda", 0)
    nt = wl.n_steps[idx]
    offs = np.concatenate([[0], np.cumsum(nt + 1)])
    Et = torch.from_numpy(np.concatenate(rows)).to(dev)
    b = tdse.Batch(wl.N[idx], wl.dx[idx], soft, nt, wl.dt, row_offsets=offs,
                   absorber=(wl.mask_width, wl.mask_exponent), precision=precision, lanes_per_instance=1)
    b.set_launch(warps_per_cta=warps)
    b.ground_state(**GS_KW)
    d, acc = torch.zeros_like(Et), torch.zeros_like(Et)
    b.propagate(Et, d, acc)
    torch.cuda.synchronize()
    assert b.check() == -1
    b.close()
    return offs, acc


def _spectral_check(tdse, oracle, wl, idx, accs_ref, acc, offs, bound):
    worst = (0.0, 0.0)
    for j, i in enumerate(idx):
        L = int(offs[j + 1] - offs[j])
        omega = float(wl.omega[i])
        S = tdse.spectrum(acc[int(offs[j]): int(offs[j + 1])], [0, L], wl.dt, 0, L).cpu().numpy()[0]
        S_ref = oracle.spectrum(accs_ref[j], wl.dt)
        l2, h = spectral_errors(S, S_ref, omega, wl.dt, L, harmonic_cutoff(float(wl.E0[i]), omega))
        assert l2 <= bound[0] and h <= bound[1], (int(i), l2, h, bound)
        worst = (max(worst[0], l2), max(worst[1], h))
    return worst


def _oracle_refs(oracle, wl, idx, soft, rows):
    jobs = []
    for j, i in enumerate(idx):
        N, dx = int(wl.N[i]), float(wl.dx[i])
        psi0, _, _ = oracle.ground_state(N, dx, soft[j], **GS_KW)
        jobs.append((psi0, rows[j], dx, wl.dt, soft[j], oracle.mask(N, dx, wl.mask_width, wl.mask_exponent)))
    return [r[2] for r in oracle_pool_map(jobs)]


def test_volume_batch_full_length_spectra_fp64_and_mixed(env):
    """The 8192 x 4096 volume batch's configuration (55159 steps, 800 nm, 10 cycles): four instances
    of the benchmark's oracle sample, FP64 with the benchmark's 12-warp layout and MIXED with its
    12-warp layout, whole pulse, both spectral numbers within the stated bound of each precision."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    wl = inputs.volume_batch()
    idx = inputs.subsample(wl.n_inst, 16, 101)[:4]
    a = oracle.fit_softening(wl.target_energy, int(wl.N[0]), float(wl.dx[0]))
    soft = np.full(idx.size, a)
    rows = wl.field_rows(idx)
    refs = _oracle_refs(oracle, wl, idx, soft, rows)
    for precision, bound in ((tdse.TDSE_FP64, FP64_BOUND), (tdse.TDSE_MIXED, MIXED_BOUND)):
        offs, acc = _gpu_run(tdse, wl, idx, soft, precision, 12, rows)
        got = _spectral_check(tdse, oracle, wl, idx, refs, acc, offs, bound)
        print("volume full length, precision %d: rel L2 %.3g, worst odd harmonic %.3g" % (precision, *got))


def test_adjoint_batch_full_length_gradient(env):
    """The adjoint configuration at its own size: 1024 instances (16 r x 64 z), N = 2048, 6 cycles,
    33096 steps, checkpoints every 256 steps; loss = sum over every instance of dt^2 |DFT(a)|^2 over
    the harmonics 21-31.  dL/dE of four sampled instances (seed 103) against the oracle's exact
    discrete adjoint over the whole pulse (1e-9 of the largest component), and the gradient of the
    first of them against central differences of the forward kernel on 32 random field samples
    (step 1e-4 E0: the O(h^2) and rounding errors of the differences are ~1e-7 relative, so the
    bound is 1e-5 of the larger of |dL/dE_k| and 1 % of the instance's largest component)."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    from spectral_metrics import oracle_adjoint_job, start_pool
    wl = inputs.adjoint_batch()
    n, N, dx, dt = wl.n_inst, int(wl.N[0]), float(wl.dx[0]), wl.dt
    Nt = int(wl.n_steps[0])
    L = Nt + 1
    a = oracle.fit_softening(wl.target_energy, N, dx)
    dev = torch.device("cuda", 0)
    q = np.fft.fftfreq(L, dt) * 2 * np.pi / float(wl.omega[0])
    win = torch.from_numpy(((np.abs(q) >= 21) & (np.abs(q) <= 31)).astype(np.float64)).to(dev)

    E = torch.empty((n, L), dtype=torch.float64, device=dev)
    inputs.sin2_pulse_batch(Nt, dt, wl.E0, float(wl.omega[0]), float(wl.n_cycles[0]), wl.phi, out=E, xp=torch)
    b = tdse.Batch([N] * n, dx, a, [Nt] * n, dt, absorber=(wl.mask_width, wl.mask_exponent))
    b.ground_state(**GS_KW)
    psi0 = b.save_state()
    d, acc = torch.zeros_like(E), torch.zeros_like(E)
    b.propagate(E.view(-1), d.view(-1), acc.view(-1))
    A = torch.fft.fft(acc, dim=1)
    ga = (2 * dt * dt * L * torch.fft.ifft(A * win[None, :], dim=1).real).contiguous()
    b.load_state(psi0)
    gE = b.adjoint(E.view(-1), torch.zeros_like(E).view(-1), ga.view(-1), ckpt_every=256).view(n, L)
    torch.cuda.synchronize()
    b.close()

    sample = inputs.subsample(n, 4, 103)
    psi_o, _, _ = oracle.ground_state(N, dx, a, **GS_KW)
    m = oracle.mask(N, dx, wl.mask_width, wl.mask_exponent)
    Eh, gah = E.cpu().numpy(), ga.cpu().numpy()
    pool, res = start_pool(oracle_adjoint_job, [(psi_o, Eh[i], dx, dt, a, np.zeros(L), gah[i], m) for i in sample])

    # central differences of the forward kernel for the first sampled instance
    i0 = int(sample[0])
    rng = np.random.default_rng(103)
    ks = np.sort(rng.choice(L, 32, replace=False))
    h = 1e-4 * float(np.max(np.abs(Eh[i0])))
    rows = np.repeat(Eh[i0][None, :], 2 * ks.size, axis=0)
    for j, k in enumerate(ks):
        rows[2 * j, k] += h
        rows[2 * j + 1, k] -= h
    Ef = torch.from_numpy(rows).to(dev)
    bf = tdse.Batch([N] * rows.shape[0], dx, a, [Nt] * rows.shape[0], dt, absorber=(wl.mask_width, wl.mask_exponent))
    bf.ground_state(**GS_KW)
    df, af = torch.zeros_like(Ef), torch.zeros_like(Ef)
    bf.propagate(Ef.view(-1), df.view(-1), af.view(-1))
    Lf = ((torch.abs(torch.fft.fft(af, dim=1)) ** 2 * win[None, :]).sum(dim=1) * dt * dt).cpu().numpy()
    bf.close()
    g0 = gE[i0].cpu().numpy()
    gmax = float(np.max(np.abs(g0)))
    for j, k in enumerate(ks):
        fd = (Lf[2 * j] - Lf[2 * j + 1]) / (2 * h)
        assert abs(fd - g0[k]) <= 1e-5 * max(abs(g0[k]), 0.01 * gmax), (int(k), fd, g0[k])

    refs = res.get()
    pool.close()
    pool.join()
    gEh = gE.cpu().numpy()
    for j, i in enumerate(sample):
        err = float(np.max(np.abs(gEh[i] - refs[j])) / np.max(np.abs(refs[j])))
        assert err < 1e-9, (int(i), err)


def test_uneven_batch_full_length_spectra(env):
    """The uneven batch's configuration (N 1024..8192, two dx, 4-16 cycles at 800/1030/1800 nm,
    up to 198575 steps): six instances of its oracle sample (seed 102), whole pulses, FP64 and MIXED,
    both spectral numbers within each precision's stated bound."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    wl = inputs.uneven_batch()
    idx = inputs.subsample(wl.n_inst, 64, 102)[:6]
    soft_of = {}
    for i in idx:
        c = (int(wl.N[i]), float(wl.dx[i]))
        if c not in soft_of:
            soft_of[c] = oracle.fit_softening(wl.target_energy, c[0], c[1])
    soft = np.array([soft_of[(int(wl.N[i]), float(wl.dx[i]))] for i in idx])
    rows = wl.field_rows(idx)
    refs = _oracle_refs(oracle, wl, idx, soft, rows)
    for precision, bound in ((tdse.TDSE_FP64, FP64_BOUND), (tdse.TDSE_MIXED, MIXED_BOUND)):
        offs, acc = _gpu_run(tdse, wl, idx, soft, precision, 12, rows)
        got = _spectral_check(tdse, oracle, wl, idx, refs, acc, offs, bound)
        print("uneven full length, precision %d: rel L2 %.3g, worst odd harmonic %.3g" % (precision, *got))


def test_large_volume_full_length_mixed_spectra(env):
    """The large volume's configuration in MIXED (1800 nm, 8 cycles, 99288 steps, N = 4096): four
    instances of its oracle sample (seed 104), whole pulse, within the MIXED bound."""
    tdse, oracle = env
    from paper_2507_04115_gb300 import inputs
    wl = inputs.large_volume()
    idx = inputs.subsample(wl.n_inst, 32, 104)[:4]
    a = oracle.fit_softening(wl.target_energy, int(wl.N[0]), float(wl.dx[0]))
    soft = np.full(idx.size, a)
    rows = wl.field_rows(idx)
    refs = _oracle_refs(oracle, wl, idx, soft, rows)
    offs, acc = _gpu_run(tdse, wl, idx, soft, tdse.TDSE_MIXED, 12, rows)
    got = _spectral_check(tdse, oracle, wl, idx, refs, acc, offs, MIXED_BOUND)
    print("large volume full length, MIXED: rel L2 %.3g, worst odd harmonic %.3g" % got)
