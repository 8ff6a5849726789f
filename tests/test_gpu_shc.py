"""SHC (Eqs. 20-23) on the GPU through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, series_rel_err, spectrum_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(N, T, nc, K, seed, device_inputs=True, drive=0.0):
    from paper_2102_03691_gb300.mhc import SpectralHeatCurrent
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed)
    tr = synth.Trajectory(mass, drive_g=drive, seed=seed)
    v, W = tr.next_block(T)
    s = SpectralHeatCurrent(N, nc, k_max=K, dt_ps=0.002, T_K=300.0, V_A3=N * 20.02,
                            F_e=(1e-4, 0.0, 0.0))
    for t0 in range(0, T, K):
        a, b = np.ascontiguousarray(v[t0:t0 + K]), np.ascontiguousarray(W[t0:t0 + K])
        if device_inputs:
            a, b = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        s.push(a, b)
    return s, v, W


@pytest.mark.parametrize("N,T,nc,K", [(10, 50, 20, 16), (6, 400, 300, 100), (37, 260, 256, 64)])
def test_shc_corr_and_kappa_match_oracle(N, T, nc, K):
    need_gpu()
    s, v, W = run(N, T, nc, K, seed=600 + N, drive=1e-3)
    Kg, cnt = s.read_corr()
    Ko, cnto = oracle.shc_corr(v, W, nc)
    np.testing.assert_array_equal(cnt, cnto)
    assert np.all(series_rel_err(Kg.T, Ko.T) <= REL_TOL)
    f = np.linspace(0.0, 60.0, 97)
    for window in (0, 1):
        kg = s.read_kappa(f, window)
        ko = oracle.shc_kappa(Ko, cnto, 0.002, 300.0, N * 20.02, 1e-4, f, window)
        assert np.all(spectrum_rel_err(kg.T, ko.T) <= REL_TOL)
    s.close()


def test_shc_lag_zero_is_total_current_and_host_equals_device():
    need_gpu()
    N, T, nc, K = 20, 64, 16, 32
    s1, v, W = run(N, T, nc, K, seed=610, device_inputs=True)
    s2, _, _ = run(N, T, nc, K, seed=610, device_inputs=False)
    K1, _ = s1.read_corr()
    K2, _ = s2.read_corr()
    np.testing.assert_array_equal(K1, K2)
    J = np.einsum("tiab,tib->ta", W.astype(np.float64).reshape(T, N, 3, 3), v.astype(np.float64))
    np.testing.assert_allclose(K1.reshape(3, 3, nc)[:, :, 0].sum(axis=1), J.sum(axis=0),
                               rtol=1e-6, atol=1e-6 * np.abs(J).sum(axis=0).max())
    s1.close()
    s2.close()


def test_shc_si_n8000_full_size():
    # the paper's SHC setting on the Si-8000 shape: 250 lags (500 fs at 2 fs), K = 256,
    # two blocks (512 samples, the ring wraps); every lag checked against the oracle
    need_gpu()
    N, nc, K, T = 8000, 250, 256, 512
    s, v, W = run(N, T, nc, K, seed=20210211)
    Kg, cnt = s.read_corr()
    Ko, cnto = oracle.shc_corr(v, W, nc)
    assert np.all(series_rel_err(Kg.T, Ko.T) <= REL_TOL)
    s.close()
