"""Grouped launch (mhc_group_*): several systems of uneven size in one persistent
tensor-core launch must give bitwise the results of pushing each system on its own,
and match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import ModalRef
from tests.test_gpu_parity import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def system(N, seed, E=None):
    D = 3 * N
    if E is None:
        E = synth.eigvecs(D, D, seed)
    f = synth.frequencies(D, 0.0, 52.0, seed)
    mass = synth.masses(N, 12.011)
    tr = synth.Trajectory(mass, seed=seed)
    return dict(N=N, E=E, f=f, mass=mass, tr=tr)


def handle(s, K, L, precision="fp16x3", B=52):
    # unsplit d axis, as in the grouped launch, so that solo pushes are bitwise comparable
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    h = ModalHeatCurrent(precision=precision, k_max=K, n_lags=L, split_d=1)
    h.set_modes(s["E"], s["mass"], s["f"])
    h.set_bins_uniform(0.0, 52.0, B)
    return h


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
def test_group_equals_individual_pushes_and_oracle(precision):
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrentGroup
    sizes = [120, 200, 360, 80]          # 40 atoms per CNT cell x {3, 5, 9, 2}
    K, L, B = 40, 10, 52
    systems = [system(N, 300 + j) for j, N in enumerate(sizes)]
    blocks = [[s["tr"].next_block(K) for _ in range(2)] for s in systems]
    solo = [handle(s, K, L, precision) for s in systems]
    grouped = [handle(s, K, L, precision) for s in systems]
    grp = ModalHeatCurrentGroup(grouped)
    for step in range(2):
        for h, bl in zip(solo, blocks):
            h.push(*bl[step])
        grp.push([bl[step][0] for bl in blocks], [bl[step][1] for bl in blocks])
        for hs, hg in zip(solo, grouped):
            np.testing.assert_array_equal(hs.read_binned_current(), hg.read_binned_current())
            np.testing.assert_array_equal(hs.read_total_current(), hg.read_total_current())
    grp.close()
    tol = TOL[precision]
    for s, bl, hg in zip(systems, blocks, grouped):
        Cg, _ = hg.read_corr()
        v = np.concatenate([b[0] for b in bl])
        W = np.concatenate([b[1] for b in bl])
        bins = oracle.bins_uniform(s["f"], 0.0, 52.0, B)
        o = ModalRef(s["E"], s["mass"], v, W, bins, B)
        o.check_current(hg.read_binned_current(), tol, f"group N={s['N']} {precision}",
                        steps=slice(K, 2 * K))
        o.check_corr(Cg, L, tol, f"group N={s['N']} corr {precision}")


def test_cnt_batch_16_systems_full_size():
    # The uneven CNT (10,10) batch: 16 systems, N = 40 u with u in [12, 100], all 3N modes,
    # 52 bins of 1 THz.  One grouped block of K = 64 steps; the oracle recomputes every step
    # of every system (all modes) from the same inputs.
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrentGroup
    sizes = synth.cnt_group_sizes()
    assert len(sizes) == 16 and min(sizes) >= 480 and max(sizes) <= 4000
    K, B = 64, 52
    systems, handles, blocks = [], [], []
    for j, N in enumerate(sizes):
        Ed = synth.eigvecs_device(3 * N, 3 * N, 20210208 + j)
        s = system(N, 20210208 + j, E=Ed)
        h = handle(s, K, 0)
        s["E"] = Ed.double().cpu().numpy()
        del Ed
        systems.append(s)
        handles.append(h)
        blocks.append(s["tr"].next_block(K))
    grp = ModalHeatCurrentGroup(handles)
    grp.push([b[0] for b in blocks], [b[1] for b in blocks])
    for s, h, (v, W) in zip(systems, handles, blocks):
        Jb = h.read_binned_current()
        bins = oracle.bins_uniform(s["f"], 0.0, 52.0, B)
        # the whole block of every system: the projections as FP64 matrix products
        o = ModalRef(s["E"], s["mass"], v, W, bins, B, mm=True)
        o.check_current(Jb, TOL["fp16x3"], f"CNT batch N={s['N']}")
    grp.close()


def test_group_graph_replay_matches_direct():
    # group pushes after the first replay one captured CUDA graph covering every system
    need_gpu()
    from paper_2102_03691_gb300.mhc import FLAG_NO_GRAPH, ModalHeatCurrentGroup
    sizes = [160, 80, 240]
    K, L = 32, 8
    systems = [system(N, 500 + j) for j, N in enumerate(sizes)]
    blocks = [[s["tr"].next_block(K) for _ in range(4)] for s in systems]
    results = []
    for flags in (FLAG_NO_GRAPH, 0):
        hs = [handle(s, K, L) for s in systems]
        hs[0].set_flags(flags)
        grp = ModalHeatCurrentGroup(hs)
        out = []
        for step in range(4):
            grp.push([bl[step][0] for bl in blocks], [bl[step][1] for bl in blocks])
            out.append([h.read_binned_current().copy() for h in hs])
        kap_all = grp.read_hnema()
        kap_one = np.concatenate([h.read_hnema()[1].ravel() for h in hs])
        np.testing.assert_array_equal(kap_all, kap_one)
        results.append((out, [h.read_corr()[0] for h in hs], hs[0].info()["graph_replays"]))
        grp.close()
    for a, b in zip(results[0][0], results[1][0]):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    for x, y in zip(results[0][1], results[1][1]):
        np.testing.assert_array_equal(x, y)
    assert results[0][2] == 0 and results[1][2] == 3


def test_group_host_inputs_back_to_back():
    # host inputs of every system are uploaded before the group push returns (staging
    # overlaps the previous push); the caller's buffers are refilled right after each push.
    # Asynchronous host inputs: two pinned buffers a system, each refilled as soon as the
    # push after the one that used it has returned
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrentGroup
    sizes = [120, 80, 200]
    K, L, T = 16, 6, 5
    systems = [system(N, 700 + j) for j, N in enumerate(sizes)]
    blocks = [[s["tr"].next_block(K) for _ in range(T)] for s in systems]
    res = []
    for mode in ("host", "device", "async"):
        hs = [handle(s, K, L) for s in systems]
        grp = ModalHeatCurrentGroup(hs)
        bufs = [(np.empty_like(bl[0][0]), np.empty_like(bl[0][1])) for bl in blocks]
        pinned = [[(torch.empty(bl[0][0].shape).pin_memory(), torch.empty(bl[0][1].shape).pin_memory())
                   for _ in range(2)] for bl in blocks]
        for step in range(T):
            if mode == "host":
                for (bv, bw), bl in zip(bufs, blocks):
                    bv[:], bw[:] = bl[step]
                grp.push([b[0] for b in bufs], [b[1] for b in bufs])
            elif mode == "async":
                cur = [p[step % 2] for p in pinned]
                for (bv, bw), bl in zip(cur, blocks):
                    bv.copy_(torch.from_numpy(bl[step][0]))
                    bw.copy_(torch.from_numpy(bl[step][1]))
                grp.push([b[0] for b in cur], [b[1] for b in cur], async_inputs=True)
            else:
                grp.push([torch.from_numpy(bl[step][0]).cuda() for bl in blocks],
                         [torch.from_numpy(bl[step][1]).cuda() for bl in blocks])
        for h in hs:
            h.sync()
        res.append(([h.read_corr()[0] for h in hs], grp.read_hnema()))
        grp.close()
    for r in res[1:]:
        for x, y in zip(res[0][0], r[0]):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(res[0][1], r[1])


@pytest.mark.parametrize("sizes", [[1100, 40, 200], [81, 120, 50]])
def test_group_pack_clusters_and_fallback(sizes):
    # [1100, 40, 200]: one pack launch for all systems in clusters of two CTAs (the 40- and
    # 200-atom systems leave their second rank without atoms); [81, 120, 50]: a system with
    # N % 4 != 0 sends the group back to one pack per system.  Both bitwise the solo pushes.
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrentGroup
    K, L = 24, 6
    systems = [system(N, 900 + j) for j, N in enumerate(sizes)]
    blocks = [[s["tr"].next_block(K) for _ in range(2)] for s in systems]
    solo = [handle(s, K, L) for s in systems]
    grouped = [handle(s, K, L) for s in systems]
    grp = ModalHeatCurrentGroup(grouped)
    for step in range(2):
        for h, bl in zip(solo, blocks):
            h.push(*bl[step])
        grp.push([bl[step][0] for bl in blocks], [bl[step][1] for bl in blocks])
        for hs, hg in zip(solo, grouped):
            np.testing.assert_array_equal(hs.read_binned_current(), hg.read_binned_current())
            np.testing.assert_array_equal(hs.read_total_current(), hg.read_total_current())
    for hs, hg in zip(solo, grouped):
        np.testing.assert_array_equal(hs.read_corr()[0], hg.read_corr()[0])
        np.testing.assert_array_equal(hs.read_hnema()[0], hg.read_hnema()[0])
    grp.close()


def test_group_pack_large_system_uses_wide_ctas():
    # a 9000-atom system (120 modes of a thin basis) sends the whole group to 512-thread pack
    # CTAs (clusters of 5 for it, of 1 for the 200-atom system): bitwise the solo pushes
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrentGroup
    K, L = 16, 4
    big = system(9000, 950, E=synth.eigvecs(27000, 120, 950))
    big["f"] = synth.frequencies(120, 0.0, 52.0, 950)
    systems = [big, system(200, 951)]
    blocks = [[s["tr"].next_block(K) for _ in range(2)] for s in systems]
    solo = [handle(s, K, L) for s in systems]
    grouped = [handle(s, K, L) for s in systems]
    grp = ModalHeatCurrentGroup(grouped)
    for step in range(2):
        for h, bl in zip(solo, blocks):
            h.push(*bl[step])
        grp.push([bl[step][0] for bl in blocks], [bl[step][1] for bl in blocks])
        for hs, hg in zip(solo, grouped):
            np.testing.assert_array_equal(hs.read_binned_current(), hg.read_binned_current())
            np.testing.assert_array_equal(hs.read_total_current(), hg.read_total_current())
    grp.close()


def test_group_autotune_k_leaves_the_accumulators_alone():
    # mhc_group_autotune_k times grouped packs and projections on synthetic blocks: the
    # members' sums afterwards are bitwise those of a group that never ran it
    need_gpu()
    from paper_2102_03691_gb300.mhc import MhcError, ModalHeatCurrentGroup
    sizes, L = [120, 80, 200], 6
    systems = [system(N, 1400 + j) for j, N in enumerate(sizes)]
    blocks = [[s["tr"].next_block(16) for _ in range(2)] for s in systems]
    out = []
    for tune in (True, False):
        hs = [handle(s, 32, L) for s in systems]
        grp = ModalHeatCurrentGroup(hs)
        if tune:
            hs[0].push(*blocks[0][0])            # one solo push first: its reads then fail
            best, rate = grp.autotune_k([8, 16, 32])
            assert best in (8, 16, 32) and rate > 0
            with pytest.raises(MhcError):
                hs[0].read_total_current()
            hs[0].reset()
        for step in range(2):
            grp.push([bl[step][0] for bl in blocks], [bl[step][1] for bl in blocks])
        out.append(([h.read_corr()[0] for h in hs], [h.read_hnema()[0] for h in hs],
                    [h.read_binned_current() for h in hs]))
        grp.close()
    for a, b in zip(out[0], out[1]):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
