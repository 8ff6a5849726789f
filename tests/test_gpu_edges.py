"""Degenerate and extreme cases through the C ABI against the FP64 oracle: one atom, one-step
pushes, every mode excluded, a single bin, one lag, more lags than steps, and the same for the
direction split and the spectral heat current."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, ModalRef, check, stage_corr_check
from tests.test_gpu_parity import TOL, make_case, need_gpu, oracle_ref, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_one_atom_one_step_pushes(precision):
    # N = 1 (three modes), K = 1 per push, 2 bins, 3 lags over 5 steps.  (BF16x3 is left out:
    # its ~16-bit operand pairs give errors that only average down over many atoms.)
    need_gpu()
    c = make_case(N=1, M=3, T=5, B=2, seed=901)
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, precision, K=1, L=3)
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-12)
    o.check_current(Jb, TOL[precision], f"one atom {precision}")
    C, cnt = h.read_corr()
    np.testing.assert_array_equal(cnt, [5, 4, 3])
    o.check_corr(C, 3, TOL[precision], f"one atom corr {precision}")
    h.close()


def test_every_mode_excluded_gives_zeros():
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    c = make_case(N=20, M=60, T=8, B=3, seed=902)
    h = ModalHeatCurrent(precision="fp16x3", k_max=8, n_lags=4)
    h.set_modes(c["E"], c["mass"], c["f"])
    h.set_bin_ids(np.full(60, -1, np.int32), 3)
    assert h.info()["n_modes_kept"] == 0
    h.push(c["v"], c["W"])
    assert np.all(h.read_binned_current() == 0)
    o = oracle.modal_current(c["E"], c["mass"], c["v"], c["W"], np.full(60, -1, np.int32), 3)
    np.testing.assert_allclose(h.read_total_current(), o["J"], rtol=1e-12, atol=1e-12)
    C, _ = h.read_corr()
    assert np.all(C == 0)
    mean, kap = h.read_hnema()
    assert np.all(mean == 0) and np.all(kap == 0)
    h.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_single_bin_single_lag_and_lags_beyond_the_run(precision):
    need_gpu()
    c = make_case(N=30, M=90, T=12, B=1, seed=903)
    o = oracle_ref(c)
    # one lag
    h, Jb, _ = run_gpu(c, precision, K=5, L=1)
    o.check_current(Jb, TOL[precision], f"single bin {precision}")
    C, cnt = h.read_corr()
    _, cnt0 = o.check_corr(C, 1, TOL[precision], f"one lag {precision}")
    np.testing.assert_array_equal(cnt, cnt0)
    h.close()
    # 20 lags over 12 steps: lags 12..19 have no origins and stay zero
    h, Jb, _ = run_gpu(c, precision, K=5, L=20)
    C, cnt = h.read_corr()
    _, cnt0 = o.check_corr(C, 20, TOL[precision], f"lags beyond the run {precision}")
    np.testing.assert_array_equal(cnt, cnt0)
    assert np.all(C[..., 12:] == 0) and np.all(cnt[12:] == 0)
    kt, kw = h.read_kappa_gk(0.0, 0.19)
    assert np.all(np.isfinite(kt)) and np.all(np.isfinite(kw))
    o.check_kappa(kt, None, 20, 0.01, 300.0, 1.0, 0.0, 0.19, TOL[precision],
                  f"kappa beyond the run {precision}")
    # the window average alone (weighted sum over the lags, lag 0 and empty lags included)
    for lo, hi in ((0.0, 0.19), (0.0, 0.0), (0.05, 0.14), (0.3, 0.5)):
        kw2 = h.read_kappa_window(lo, hi)
        _, kw1 = h.read_kappa_gk(lo, hi)
        np.testing.assert_allclose(kw2, kw1, rtol=1e-10, atol=1e-11 * max(np.abs(kw1).max(), 1e-300))
    assert np.all(h.read_kappa_window(0.3, 0.5) == 0)   # no lag in the window
    h.close()


def test_direction_split_one_atom():
    need_gpu()
    c = make_case(N=1, M=3, T=4, B=1, seed=904)
    od = oracle_ref(c, direction=True)
    h, Jb, _ = run_gpu(c, "fp16x3", K=2, direction=True)
    od.check_current(Jb, REL_TOL, "direction split, one atom")
    h.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_shc_one_atom_and_lags_beyond_the_run(precision):
    # one atom, 10 lags over 6 samples pushed one at a time
    need_gpu()
    from paper_2102_03691_gb300.mhc import SpectralHeatCurrent
    mass = synth.masses(1, 28.085)
    v, W = synth.Trajectory(mass, seed=905).next_block(6)
    s = SpectralHeatCurrent(1, 10, k_max=1, dt_ps=0.002, T_K=300.0, V_A3=20.02,
                            F_e=(1e-4, 0.0, 0.0), precision=precision)
    for t in range(6):
        s.push(torch.from_numpy(v[t:t + 1]).cuda(), torch.from_numpy(W[t:t + 1]).cuda())
    K, cnt = s.read_corr()
    Ko, cnto = oracle.shc_corr(v, W, 10)
    np.testing.assert_array_equal(cnt, cnto)
    assert np.all(K[:, 6:] == 0)
    check(K, Ko, oracle.shc_corr(np.abs(v), np.abs(W), 10)[0], None, REL_TOL,
          f"SHC one atom {precision}")
    s.close()


@pytest.mark.parametrize("N", [9000, 9001])
def test_pack_paths_large_system(N):
    # N = 9000 is packed by clusters of 5 CTAs of 2048 atoms (bulk copies), N = 9001 (not a
    # multiple of 4) by the one-CTA-per-step kernel; 300 kept modes, 8 steps, 4 bins
    need_gpu()
    from tests.test_gpu_parity import make_case
    c = make_case(N=N, M=300, T=8, B=4, seed=906)
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, "fp16x3", K=8, L=3)
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-9 * np.abs(o.J).max())
    o.check_current(Jb, REL_TOL, f"pack path N={N}")
    h.close()


@pytest.mark.parametrize("direction", [False, True])
def test_largest_block_with_lag_correlation(direction):
    # K = 1024 (the largest block): the lag correlation runs 32 step warps a CTA and needs more
    # than 48 KB of shared memory; 2200 steps end in a ragged block of 152; 7 bins (row groups
    # of 4 bins end ragged), 70 lags (the last lag CTA half full)
    need_gpu()
    L, K, T, B = 70, 1024, 2200, 7
    c = make_case(N=40, M=120, T=T, B=B, seed=905, drive=2e-3)
    h, Jb, J = run_gpu(c, "fp16x3", K=K, L=L, direction=direction)
    o = oracle_ref(c, direction=direction)
    o.check_current(Jb, REL_TOL, f"K=1024 currents direction={direction}")
    C, cnt = h.read_corr()
    _, cnt0 = o.check_corr(C, L, REL_TOL, f"K=1024 Eq. 17 sums direction={direction}")
    np.testing.assert_array_equal(cnt, cnt0)
    # the lag stage alone, fed with the library's own binned currents
    stage_corr_check(C, o.rows(Jb), J, L, REL_TOL, "K=1024 lag stage")
    h.close()


def test_green_kubo_read_out_beyond_1024_lags():
    # L = 1100 lags: more than 8 lags a thread of the read-out (the path that recomputes C(l)
    # instead of keeping it in registers); 1300 steps in ragged blocks of 256; kappa(tau) at
    # every lag and the window average against the oracle
    need_gpu()
    L, K, T, B = 1100, 256, 1300, 3
    dt, TK, V = 0.01, 300.0, 16 * 20.02
    c = make_case(N=16, M=48, T=T, B=B, seed=906, drive=2e-3)
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, "fp16x3", K=K, L=L, dt_ps=dt, T_K=TK, V_A3=V)
    kt, kw = h.read_kappa_gk(8.0, 10.5)
    _, n = o.check_kappa(kt, kw, L, dt, TK, V, 8.0, 10.5, REL_TOL, "1100 lags kappa")
    assert n == 251
    # the window average alone (one weighted sum a row) against the oracle
    kw2 = h.read_kappa_window(8.0, 10.5)
    o.check_kappa(kt, kw2, L, dt, TK, V, 8.0, 10.5, REL_TOL, "1100 lags kappa window alone")
    np.testing.assert_allclose(kw2, kw, rtol=1e-10, atol=1e-11 * np.abs(kw).max())
    # the Green-Kubo stage alone: the oracle's integral of the library's own Eq. 17 sums
    C, cnt = h.read_corr()
    okt = oracle.gk_kappa(C, cnt, dt, TK, V)
    skt = oracle.gk_kappa(np.abs(C), cnt, dt, TK, V)
    check(kt, okt, skt, None, 1e-11, "1100 lags Green-Kubo stage")
    h.close()


def test_fp32_fma_measurement():
    # the FP32 comparison path's peak: a plausible FMA throughput (152 SMs x 128 lanes x 2 flops
    # at 1-2.1 GHz is 39-82 TFLOP/s), and the C ABI rejects a null output
    need_gpu()
    import ctypes
    from paper_2102_03691_gb300 import mhc
    t = mhc.measure_fp32_fma(0)
    assert 20.0 < t < 200.0, t
    assert mhc.load().mhc_measure_fp32_fma(0, None, None) == 1
