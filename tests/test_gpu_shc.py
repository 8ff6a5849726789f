"""SHC (Eqs. 20-23) on the GPU through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, check_shc_corr, spectrum_rel_err
from tests.test_gpu_parity import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(N, T, nc, K, seed, device_inputs=True, drive=0.0, precision="fp16x3", blocks=None):
    from paper_2102_03691_gb300.mhc import SpectralHeatCurrent
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed)
    tr = synth.Trajectory(mass, drive_g=drive, seed=seed)
    v, W = tr.next_block(T)
    s = SpectralHeatCurrent(N, nc, k_max=K, dt_ps=0.002, T_K=300.0, V_A3=N * 20.02,
                            F_e=(1e-4, 0.0, 0.0), precision=precision)
    starts = list(range(0, T, K)) if blocks is None else blocks
    for t0, t1 in zip(starts, starts[1:] + [T]):
        a, b = np.ascontiguousarray(v[t0:t1]), np.ascontiguousarray(W[t0:t1])
        if device_inputs:
            a, b = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        s.push(a, b)
    return s, v, W


@pytest.mark.parametrize("N,T,nc,K", [(10, 50, 20, 16), (6, 400, 300, 100), (37, 260, 256, 64)])
def test_shc_corr_and_kappa_match_oracle(N, T, nc, K):
    need_gpu()
    s, v, W = run(N, T, nc, K, seed=600 + N, drive=1e-3)
    Kg, cnt = s.read_corr()
    _, Ko, cnto = check_shc_corr(Kg, v, W, nc, REL_TOL, f"SHC N={N}")
    np.testing.assert_array_equal(cnt, cnto)
    f = np.linspace(0.0, 60.0, 97)
    for window in (0, 1):
        kg = s.read_kappa(f, window)
        ko = oracle.shc_kappa(Ko, cnto, 0.002, 300.0, N * 20.02, 1e-4, f, window)
        assert np.all(spectrum_rel_err(kg.T, ko.T) <= REL_TOL)
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16x3"])
def test_shc_precisions_ragged_blocks(precision):
    # 150 atoms (two 128-atom chunks, the second ragged), 140 lags over blocks of uneven
    # length (37, 100, 5, 128, 30: the tau tiles start off the block boundaries and the
    # last step tile of each block is ragged), so the virial ring wraps
    need_gpu()
    starts = [0, 37, 137, 142, 270]
    s, v, W = run(150, 300, 140, 128, seed=620, drive=1e-3, precision=precision, blocks=starts)
    Kg, cnt = s.read_corr()
    _, Ko, cnto = check_shc_corr(Kg, v, W, 140, TOL[precision], f"SHC ragged {precision}")
    np.testing.assert_array_equal(cnt, cnto)
    s.close()


@pytest.mark.parametrize("N", [12000, 17000, 33000])
def test_shc_large_systems_pack_paths(N):
    # N = 12000 packs by bulk copies with 2048 atoms per CTA (clusters of 6); N = 17000 with 8
    # atoms per thread in registers (clusters of 5); N = 33000 is past what a cluster of 8
    # holds and takes the two-pass one-CTA-per-step kernel
    need_gpu()
    s, v, W = run(N, 24, 8, 12, seed=640 + N % 7)
    Kg, cnt = s.read_corr()
    check_shc_corr(Kg, v, W, 8, REL_TOL, f"SHC N={N}")
    s.close()


def test_shc_tensor_path_is_deterministic_and_profiled():
    need_gpu()
    s1, v, W = run(300, 200, 64, 100, seed=630)
    s2, _, _ = run(300, 200, 64, 100, seed=630)
    K1, _ = s1.read_corr()
    K2, _ = s2.read_corr()
    np.testing.assert_array_equal(K1, K2)
    s1.set_profile(True)
    a, b = torch.from_numpy(v[:100]).cuda(), torch.from_numpy(W[:100]).cuda()
    s1.push(a, b)
    s1.push(a, b)
    ms, n = s1.kernel_time()
    assert n == 2 and ms > 0
    s1.close()
    s2.close()


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
    check_shc_corr(Kg, v, W, nc, REL_TOL, "SHC Si-8000")
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_shc_host_inputs_back_to_back_reuse_one_buffer(precision):
    # host blocks are read before each push returns; one pinned buffer refilled after every
    # push (no sync in between) gives bitwise the device-input result
    need_gpu()
    from paper_2102_03691_gb300.mhc import SpectralHeatCurrent
    N, T, nc, K = 96, 160, 24, 32
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=650)
    v, W = synth.Trajectory(mass, seed=650).next_block(T)
    out = []
    for host in (True, False):
        s = SpectralHeatCurrent(N, nc, k_max=K, dt_ps=0.002, T_K=300.0, V_A3=N * 20.02,
                                F_e=(1e-4, 0.0, 0.0), precision=precision)
        bv = torch.empty((K, N, 3), dtype=torch.float32).pin_memory()
        bw = torch.empty((K, N, 9), dtype=torch.float32).pin_memory()
        for t0 in range(0, T, K):
            if host:
                bv.copy_(torch.from_numpy(v[t0:t0 + K]))
                bw.copy_(torch.from_numpy(W[t0:t0 + K]))
                s.push(bv, bw)
            else:
                s.push(torch.from_numpy(v[t0:t0 + K]).cuda(), torch.from_numpy(W[t0:t0 + K]).cuda())
        out.append(s.read_corr()[0])
        s.close()
    np.testing.assert_array_equal(out[0], out[1])
