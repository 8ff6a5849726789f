"""The d-axis split of the tensor-core projection and the autotuner's choices of split count
and block length, through the C ABI against the FP64 oracle.

A split cuts the reduction of Eqs. 13 and 16 over the 3N degrees of freedom into ranges of
whole 128-element promotion chunks; each (mode tile, column tile, range) runs as its own unit
and a finish kernel adds the ranges in a fixed order before the Eq. 16 product and the bin
sums.  The balanced split (split_d = -1) cuts the chunks of all tiles, tile after tile, into
one range of equal length per CTA (pair); a tile that a range boundary cuts is finished the
same way, the others by the projection kernel itself.  The results differ from the unsplit
kernel only in the order of FP32 additions."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.parity import REL_TOL, TOL, check
from tests.test_gpu_parity import make_case, need_gpu, oracle_ref, run_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case_n400():
    # D = 1200 (19 k-blocks of 64, 38 of 32: the last split is ragged), all 1200 modes,
    # 6 bins, 130 steps in blocks of 65 (ragged column tiles)
    c = make_case(N=400, M=1200, T=130, B=6, seed=1101, drive=2e-3)
    c["ref"] = oracle_ref(c)
    return c


@pytest.mark.parametrize("tile_config", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("split_d", [2, 3, 4, -1])
def test_split_matches_oracle_on_every_tile(case_n400, tile_config, split_d):
    # split_d = -1 on this case: 10 chunks a tile, 10-30 tiles on 76 CTA pairs or 152 CTAs, so
    # every tile is cut into ~5-9 segments (more than the finish kernel stages at once)
    need_gpu()
    c = case_n400
    L = 9
    h, Jb, J = run_gpu(c, "fp16x3", K=65, L=L, tile_config=tile_config, split_d=split_d)
    info = h.info()
    assert info["tile_split"] == split_d
    c["ref"].check_current(Jb, REL_TOL, f"split {split_d} tile {tile_config}")
    C, _ = h.read_corr()
    c["ref"].check_corr(C, L, REL_TOL, f"split {split_d} tile {tile_config} corr")
    h.close()
    # against the unsplit kernel: within the bound of each side
    _, Jb1, _ = run_gpu(c, "fp16x3", K=65, L=L, tile_config=tile_config, split_d=1)
    check(Jb, Jb1, 2 * c["ref"].S, 2 * c["ref"].Sd, REL_TOL, "split vs unsplit")


@pytest.fixture(scope="module")
def case_n1000():
    # D = 3000 (24 chunks a tile), 3000 modes, one block of 1024 steps: 192 CTA-pair tiles
    # (4608 chunks, ~61 a pair) or 768 one-SM tiles of 128 columns (~121 chunks a CTA), so the
    # balanced split leaves most tiles whole and cuts the rest in two or three
    c = make_case(N=1000, M=3000, T=1024, B=12, seed=1102, drive=1e-3)
    c["ref"] = oracle_ref(c)
    return c


@pytest.mark.parametrize("tile_config", [4, 5])
def test_balanced_split_mixes_whole_and_cut_tiles(case_n1000, tile_config):
    need_gpu()
    c = case_n1000
    h, Jb, _ = run_gpu(c, "fp16x3", K=1024, tile_config=tile_config, split_d=-1)
    assert h.info()["tile_split"] == -1
    c["ref"].check_current(Jb, REL_TOL, f"balanced split, tile {tile_config}")
    h.close()
    _, Jb1, _ = run_gpu(c, "fp16x3", K=1024, tile_config=tile_config, split_d=1)
    check(Jb, Jb1, 2 * c["ref"].S, 2 * c["ref"].Sd, REL_TOL, "balanced vs unsplit")


@pytest.mark.parametrize("split_d", [3, -1])
@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_split_graph_replay_and_repeat_are_bitwise(case_n400, precision, split_d):
    need_gpu()
    from paper_2102_03691_gb300.mhc import FLAG_NO_GRAPH
    c = case_n400
    outs = []
    for flags in (FLAG_NO_GRAPH, 0, 0):
        h, Jb, _ = run_gpu(c, precision, K=65, L=5, tile_config=5, split_d=split_d, flags=flags)
        C, _ = h.read_corr()
        outs.append((Jb, C, h.info()["graph_replays"]))
        h.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
    assert outs[0][2] == 0 and outs[1][2] == 2    # a fixed tile: every push replays a graph
    c["ref"].check_current(outs[0][0], TOL[precision], f"split graph {precision}")


def test_autotuner_may_split_small_problems(case_n400):
    # 1200 modes and K = 65: 5 CTA-pair tiles on ~76 resident pairs, so the autotuner tries
    # d-axis splits; whatever it picks matches the oracle, and a second handle of the same
    # shape reuses the choice (bitwise the same results)
    need_gpu()
    c = case_n400
    h1, Jb1, _ = run_gpu(c, "fp16x3", K=65)
    h2, Jb2, _ = run_gpu(c, "fp16x3", K=65)
    i1, i2 = h1.info(), h2.info()
    assert (i1["tile_n"], i1["tile_k"], i1["tile_pair"], i1["tile_split"]) == \
        (i2["tile_n"], i2["tile_k"], i2["tile_pair"], i2["tile_split"])
    np.testing.assert_array_equal(Jb1, Jb2)
    c["ref"].check_current(Jb1, REL_TOL, f"autotuned split {i1['tile_split']}")
    print("autotuned:", {k: i1[k] for k in ("tile_n", "tile_k", "tile_pair", "stages", "tile_split")})
    h1.close()
    h2.close()


def test_autotune_k_leaves_the_accumulators_alone(case_n400):
    need_gpu()
    from paper_2102_03691_gb300.mhc import MhcError, ModalHeatCurrent
    c = case_n400
    K, L = 65, 6

    def fresh():
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, c["f_hi"], c["B"])
        return h
    a = fresh()
    a.push(c["v"][:K], c["W"][:K])
    best, rate = a.autotune_k([16, 32, 65])
    assert best in (16, 32, 65) and rate > 0
    with pytest.raises(MhcError):
        a.read_total_current()        # the last block's operands were overwritten
    a.push(c["v"][K:2 * K], c["W"][K:2 * K])
    b = fresh()
    for t0 in (0, K):
        b.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    np.testing.assert_array_equal(a.read_binned_current(), b.read_binned_current())
    np.testing.assert_array_equal(a.read_corr()[0], b.read_corr()[0])
    np.testing.assert_array_equal(a.read_hnema()[0], b.read_hnema()[0])
    a.close()
    b.close()


_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_2102_03691_gb300 import synth
from paper_2102_03691_gb300.mhc import ModalHeatCurrent
N, M, K = 200, 600, 40
E = synth.eigvecs(3 * N, M, 1201)
mass = synth.masses(N, 28.085)
v, W = synth.Trajectory(mass, seed=1201).next_block(K)
h = ModalHeatCurrent(precision="fp16x3", k_max=K)
h.set_modes(E, mass, synth.frequencies(M, 0.0, 16.0, 1201))
h.set_bins_uniform(0.0, 16.0, 4)
h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
i = h.info()
print("CFG", i["tile_n"], i["tile_k"], i["tile_pair"], i["stages"], i["tile_split"])
h.close()
"""


def test_tune_cache_file_is_reused_by_a_new_process(tmp_path):
    need_gpu()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    script = tmp_path / "child.py"
    script.write_text(_CHILD)
    env = dict(os.environ, MHC_TUNE_CACHE=str(cache))
    cfgs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        cfgs.append([ln for ln in r.stdout.splitlines() if ln.startswith("CFG")][0])
    lines = cache.read_text().splitlines()
    assert len(lines) == 1, lines          # the second process found the entry
    assert cfgs[0] == cfgs[1]
    # line: sm prec dir K split_req D_ld M_eff bn bk stages pair split device
    cfg = cfgs[0].split()
    assert lines[0].split()[7:12] == [cfg[1], cfg[2], cfg[4], cfg[3], cfg[5]]
