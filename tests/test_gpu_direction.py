"""GPU parity of the direction-resolved split (MHC_FLAG_DIRECTION) against the FP64 oracle.

J_n^{ab} = Xdot_n sum_i m_i^{-1/2} W_i^{ab} e^b_{i,n}: the current along a carried by the
atoms' motion along b (Sec. II.A), per mode and binned.  The library stores the d axis
direction-major and parks the finished bracket sums of the first two directions in a
per-CTA device scratch, so these cases span several direction segments, promotion chunks,
mode tiles and ragged column tiles, on every tile configuration.
"""
import numpy as np
import pytest

import oracle
from tests.parity import REL_TOL, ModalRef, check
from tests.test_gpu_parity import TOL, make_case, need_gpu, oracle_ref, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16x3", "fp16x3"]


def oracle_dir(c):
    return oracle_ref(c, direction=True)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_direction_split_ragged(precision):
    # N = 50 (one 128-column segment per direction, mostly padding), M = 130 of 150 modes
    # (two mode tiles, ragged), K = 23 (ragged column tiles), modes above 13 THz excluded
    need_gpu()
    c = make_case(N=50, M=130, T=46, B=5, seed=201, f_hi=16.0)
    c["bins"] = oracle.bins_uniform(c["f"], 0.0, 13.0, 5)
    c["f_hi"] = 13.0
    assert (c["bins"] < 0).sum() > 0
    o = oracle_dir(c)
    h, Jb, J = run_gpu(c, precision, K=23, direction=True)
    assert Jb.shape == (46, 3, 5, 3)
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-12)
    o.check_current(Jb, TOL[precision], f"direction ragged {precision}")
    h.close()


TILES = {1: (256, False), 2: (256, False), 3: (128, False), 4: (128, False),
         5: (256, True), 6: (256, True), 7: (128, True), 8: (128, True)}


@pytest.mark.parametrize("tile_config", [1, 2, 3, 4, 5, 6, 7, 8, 0])
def test_direction_split_multi_segment(tile_config):
    # N = 300: three segments of 384 columns (three promotion chunks each); all 900 modes
    # (eight mode tiles); K = 150 steps = 600 columns (five column tiles, the last ragged)
    need_gpu()
    c = make_case(N=300, M=900, T=300, B=8, seed=202)
    o = oracle_dir(c)
    h, Jb, J = run_gpu(c, "fp16x3", K=150, tile_config=tile_config, direction=True)
    o.check_current(Jb, REL_TOL, f"direction multi-segment cfg{tile_config}")
    # completeness per direction (all 3N modes): the bins of direction b add up to
    # J^{ab} = sum_i W_i^{ab} v_i^b, within the sum of the bins' bounds
    check(Jb.sum(axis=2), o.Jd, o.S.sum(axis=2), o.Sd.sum(axis=2), REL_TOL,
          "completeness per direction")
    info = h.info()
    if tile_config:
        assert (info["tile_n"], info["tile_pair"]) == TILES[tile_config]
    h.close()


def test_direction_split_is_bitwise_across_its_tiles():
    need_gpu()
    c = make_case(N=120, M=360, T=64, B=6, seed=203)
    _, a, _ = run_gpu(c, "fp16x3", K=64, tile_config=3, direction=True)
    for cfg in (1, 2, 4, 5, 6, 7, 8):
        _, b, _ = run_gpu(c, "fp16x3", K=64, tile_config=cfg, direction=True)
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_direction_split_adds_up_to_the_plain_path(precision):
    need_gpu()
    c = make_case(N=96, M=288, T=48, B=6, seed=204)
    _, Jd, _ = run_gpu(c, precision, K=48, direction=True)
    _, Jp, _ = run_gpu(c, precision, K=48)
    o = oracle_dir(c)
    o.check_current(Jd, TOL[precision], f"direction split {precision}")
    # the split summed over b against the plain path: each within its bound of the oracle
    check(Jd.sum(axis=1), Jp, 2 * o.S.sum(axis=1), 2 * o.Sd.sum(axis=1), TOL[precision],
          f"direction sum vs plain {precision}")


def test_direction_split_gkma_hnema_and_state():
    need_gpu()
    L, K, T, B = 12, 16, 64, 4
    c = make_case(N=64, M=192, T=T, B=B, seed=205, drive=2e-3)
    o = oracle_dir(c)
    dt, TK, V = 0.01, 300.0, 64 * 20.02
    kw_ = dict(dt_ps=dt, T_K=TK, V_A3=V, direction=True)
    h, Jb, J = run_gpu(c, "fp16x3", K=K, L=L, **kw_)
    C, cnt = h.read_corr()
    assert C.shape == (3, B, 3, 3, L)
    _, cnt0 = o.check_corr(C, L, REL_TOL, "direction corr")
    np.testing.assert_array_equal(cnt, cnt0)
    kt, kw = h.read_kappa_gk(0.05, 0.11)
    o.check_kappa(kt, kw, L, dt, TK, V, 0.05, 0.11, REL_TOL, "direction kappa")
    mean, kap = h.read_hnema()
    assert mean.shape == (3, B, 3)
    o.check_hnema(mean, kap, TK, V, [1e-5, 0, 0], REL_TOL, "direction HNEMA")

    # resume from a state blob: bitwise the uninterrupted run
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent

    def fresh():
        g = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, **kw_)
        g.set_modes(c["E"], c["mass"], c["f"])
        g.set_bins_uniform(0.0, c["f_hi"], B)
        return g
    a = fresh()
    for t0 in range(0, 32, K):
        a.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    blob = a.get_state()
    a.close()
    b = fresh()
    b.set_state(blob)
    for t0 in range(32, T, K):
        b.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    Cb, _ = b.read_corr()
    np.testing.assert_array_equal(C, Cb)
    # a blob of the split does not load into a handle without it
    p = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, dt_ps=dt, T_K=TK, V_A3=V)
    p.set_modes(c["E"], c["mass"], c["f"])
    p.set_bins_uniform(0.0, c["f_hi"], 3 * B)
    from paper_2102_03691_gb300.mhc import MhcError
    with pytest.raises(MhcError):
        p.set_state(blob)


def test_direction_split_not_in_groups():
    need_gpu()
    from paper_2102_03691_gb300.mhc import MhcError, ModalHeatCurrent, ModalHeatCurrentGroup
    c = make_case(N=16, M=48, T=4, B=2, seed=206)
    h = ModalHeatCurrent(precision="fp16x3", k_max=4, direction=True)
    h.set_modes(c["E"], c["mass"], c["f"])
    h.set_bins_uniform(0.0, c["f_hi"], 2)
    with pytest.raises(MhcError):
        ModalHeatCurrentGroup([h])
    h.close()


@pytest.fixture(scope="module")
def case_n2000():
    return make_case(N=2000, M=6000, T=256, B=16, seed=207)


@pytest.mark.parametrize("tile_config", [1, 5])
def test_direction_split_several_tiles_per_cta(case_n2000, tile_config):
    # N = 2000, all 6000 modes, K = 256: 188 one-SM or 96 CTA-pair tiles of 256 columns, more
    # than the CTAs (pairs) resident at once, so CTAs reuse their parking scratch across tiles
    need_gpu()
    c = case_n2000
    h, Jb, J = run_gpu(c, "fp16x3", K=256, tile_config=tile_config, direction=True)
    steps = [0, 101, 255]
    o = ModalRef(c["E"], c["mass"], c["v"][steps], c["W"][steps], c["bins"], c["B"],
                 direction=True)
    o.check_current(Jb[steps], REL_TOL, f"direction N=2000 cfg{tile_config}")
    h.close()
    _, Jb3, _ = run_gpu(c, "fp16x3", K=256, tile_config=3, direction=True)
    np.testing.assert_array_equal(Jb, Jb3)
