"""GPU parity of the bin-bin cross-correlations (MHC_FLAG_XCORR) against the FP64 oracle:
X_{bb'}^{mu nu}(l) = sum over origins of J_b^mu(t) J_{b'}^nu(t - l), the mode-mode correlations
of GKMA at bin resolution."""
import numpy as np
import pytest

import oracle
from tests.parity import REL_TOL, check
from tests.test_gpu_parity import TOL, make_case, need_gpu, oracle_ref, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_xcorr_small_ragged_blocks(precision):
    # 48 atoms, all 144 modes in 6 bins, 70 steps in blocks of 16 (the last ragged), 12 lags
    need_gpu()
    L, K, T, B = 12, 16, 70, 6
    c = make_case(N=48, M=144, T=T, B=B, seed=801, drive=2e-3)
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, precision, K=K, L=L, xcorr=True)
    X, cnt = h.read_xcorr()
    assert X.shape == (B, B, 3, 3, L)
    np.testing.assert_array_equal(cnt, np.maximum(T - np.arange(L), 0))
    o.check_xcorr(X, L, TOL[precision], f"xcorr {precision}")
    # every mode binned: the second bin summed out gives the Eq. 17 sums of the same run
    # (each side within its bound of the oracle)
    C, _ = h.read_corr()
    _, _, SC, SCd = o.corr(L, full=True)
    _, SX, SXd = o.xcorr(L, full=True)
    check(X.sum(axis=1), C, SX.sum(axis=1) + SC, SXd.sum(axis=1) + SCd, TOL[precision],
          "xcorr sum rule")
    h.close()


def test_xcorr_kappa_and_state_roundtrip():
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    L, K, T, B = 10, 8, 48, 4
    dt, TK, V = 0.01, 300.0, 32 * 20.02
    c = make_case(N=32, M=96, T=T, B=B, seed=802, drive=2e-3)
    o = oracle_ref(c)
    Xo, SX, SXd = o.xcorr(L, full=True)
    cnt = np.maximum(T - np.arange(L), 0).astype(np.int64)

    def fresh():
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, dt_ps=dt, T_K=TK, V_A3=V,
                             xcorr=True)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, c["f_hi"], B)
        return h
    a = fresh()
    for t0 in range(0, T, K):
        a.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    kt, kw = a.read_kappa_xcorr(0.03, 0.09)
    okt = oracle.gk_kappa(Xo.reshape(B * B, 3, 3, L), cnt, dt, TK, V)
    skt = oracle.gk_kappa(SX.reshape(B * B, 3, 3, L), cnt, dt, TK, V)
    sdt = oracle.gk_kappa(SXd.reshape(B * B, 3, 3, L), cnt, dt, TK, V)
    okw, n = oracle.kappa_window(okt, dt, 0.03, 0.09)
    skw, _ = oracle.kappa_window(skt, dt, 0.03, 0.09)
    sdw, _ = oracle.kappa_window(sdt, dt, 0.03, 0.09)
    assert n == 7
    check(kt.reshape(okt.shape), okt, skt, sdt, REL_TOL, "kappa_xcorr(tau)")
    check(kw.reshape(okw.shape), okw, skw, sdw, REL_TOL, "kappa_xcorr window")
    _, kw_only = a.read_kappa_xcorr(0.03, 0.09, with_tau=False)   # one weighted sum a row
    check(kw_only.reshape(okw.shape), okw, skw, sdw, REL_TOL, "kappa_xcorr window alone")
    Xa, _ = a.read_xcorr()
    b = fresh()
    for t0 in range(0, 24, K):
        b.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    blob = b.get_state()
    b.close()
    b2 = fresh()
    b2.set_state(blob)
    for t0 in range(24, T, K):
        b2.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    Xb, _ = b2.read_xcorr()
    np.testing.assert_array_equal(Xa, Xb)


def test_xcorr_with_direction_split():
    # rows = (direction of motion, bin): X over 3B rows against the oracle's J_b^{ab}
    need_gpu()
    L, K, T, B = 6, 16, 40, 3
    c = make_case(N=40, M=120, T=T, B=B, seed=803)
    od = oracle_ref(c, direction=True)
    h, Jb, J = run_gpu(c, "fp16x3", K=K, L=L, xcorr=True, direction=True)
    X, _ = h.read_xcorr()
    assert X.shape == (3, B, 3, B, 3, 3, L)
    od.check_xcorr(X, L, REL_TOL, "xcorr direction")
    h.close()


def test_xcorr_in_grouped_pushes_equals_single_handles():
    need_gpu()
    from paper_2102_03691_gb300 import synth
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent, ModalHeatCurrentGroup
    sizes, K, L, B = [80, 120], 16, 8, 5
    systems = []
    for j, N in enumerate(sizes):
        E = synth.eigvecs(3 * N, 3 * N, 810 + j)
        f = synth.frequencies(3 * N, 0.0, 52.0, 810 + j)
        mass = synth.masses(N, 12.011)
        blocks = [synth.Trajectory(mass, seed=810 + j).next_block(3 * K)]
        systems.append((E, f, mass, blocks[0]))

    def handles():
        hs = []
        for E, f, mass, _ in systems:
            h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, xcorr=True, split_d=1)
            h.set_modes(E, mass, f)
            h.set_bins_uniform(0.0, 52.0, B)
            hs.append(h)
        return hs
    solo, grouped = handles(), handles()
    grp = ModalHeatCurrentGroup(grouped)
    for step in range(3):
        sl = slice(step * K, (step + 1) * K)
        for h, (_, _, _, (v, W)) in zip(solo, systems):
            h.push(v[sl], W[sl])
        grp.push([s[3][0][sl] for s in systems], [s[3][1][sl] for s in systems])
    for hs, hg in zip(solo, grouped):
        np.testing.assert_array_equal(hs.read_xcorr()[0], hg.read_xcorr()[0])
    grp.close()


@pytest.mark.parametrize("B,direction", [(70, False), (40, True)])
def test_xcorr_several_row_and_column_tiles(B, direction):
    # 3B = 210 rows (two column tiles of 192 and a ragged one of 18; two row tiles of 128) and,
    # with the direction split, 9B = 360 rows (two column tiles, three row tiles); ragged blocks
    need_gpu()
    L, K, T = 20, 64, 150
    c = make_case(N=100, M=300, T=T, B=B, seed=804, drive=2e-3)
    o = oracle_ref(c, direction=direction)
    h, Jb, J = run_gpu(c, "fp16x3", K=K, L=L, xcorr=True, direction=direction)
    X, cnt = h.read_xcorr()
    np.testing.assert_array_equal(cnt, np.maximum(T - np.arange(L), 0))
    n = 3 * o.rows(o.Jb).shape[1]   # rows (bin row, component) of the contraction
    o.check_xcorr(X, L, REL_TOL, f"xcorr {n} rows")
    # the tensor-core stage alone, fed with the library's own binned currents
    rows = o.rows(Jb)
    check(X.reshape(-1), oracle.gkma_xcorr(rows, L).reshape(-1),
          oracle.gkma_xcorr(np.abs(rows), L).reshape(-1), None, REL_TOL, f"xcorr {n} rows stage")
    h.close()
