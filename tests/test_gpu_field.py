"""Field ingestion (tdse_resample_field, Sec. 4.2) against the oracle's zero-padded DFT interpolant:
odd and even numbers of coarse samples, fine steps that do and do not divide the coarse step,
outputs past the coarse window (periodic), and rows written into a batch-style strided layout."""
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
    return tdse, oracle


@pytest.mark.parametrize("M,dt_c,dt_f,n_fine", [(300, 0.8, 0.02, 12000), (301, 0.8, 0.03, 9000), (64, 1.0, 0.37, 400),
                                                (2, 1.0, 0.1, 25), (4096, 0.25, 0.02, 60000)])
def test_resample_matches_oracle(env, M, dt_c, dt_f, n_fine):
    tdse, oracle = env
    rng = np.random.default_rng(M)
    n_rows = 5
    t = np.arange(M) * dt_c
    coarse = np.stack([np.sin(0.05 * t + rng.uniform(0, 6)) * np.exp(-((t - t.mean()) / (0.3 * t[-1] + 1)) ** 2)
                       + 0.01 * rng.standard_normal(M) for _ in range(n_rows)])
    stride = n_fine + 7
    out = tdse.resample_field(torch.from_numpy(coarse).to("cuda"), dt_c, dt_f, n_fine, out_stride=stride)
    got = out.cpu().numpy()
    for r in range(n_rows):
        ref = oracle.resample_field(coarse[r], dt_c, dt_f, n_fine)
        assert np.max(np.abs(got[r, :n_fine] - ref)) < 1e-12 * max(1.0, np.max(np.abs(coarse[r])))
        assert np.all(got[r, n_fine:] == 0.0)   # the stride padding is left alone
