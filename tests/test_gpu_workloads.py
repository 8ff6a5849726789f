"""Parity at the workloads' full sizes, in the launch configuration bench.py times
(autotuned tile, graph replay after the first push).

The oracle cannot run whole blocks at these sizes in test time, so it recomputes
sampled steps (all modes) from the same inputs; the lag correlation and the HNEMA
averages are checked through properties that hold at any size (the Eq. 18 sum rule
over bins, since these workloads keep all 3N modes), using the total current, which
is itself checked against the oracle to 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def setup(name, n_blocks, direction=False):
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    w = synth.WORKLOADS[name]
    N, M, K, L, B = w["N"], w["M"], w["K"], w["L"], w["B"]
    Ed = synth.eigvecs_device(3 * N, M, w["seed"])
    f = synth.frequencies(M, *w["f"], w["seed"])
    mass = synth.masses(N, w["mass"])
    V = N * w["V_per_atom"]
    drive = synth.drive_coupling(w["kappa_drive"], w["T_K"], V, w["Fe"][0], mass) \
        if w.get("kappa_drive") else 0.0
    tr = synth.Trajectory(mass, drive_g=drive, seed=w["seed"])
    h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, dt_ps=w["dt_ps"], T_K=w["T_K"],
                         V_A3=V, F_e=w["Fe"], direction=direction)
    h.set_modes(Ed, mass, f)
    h.set_bins_uniform(w["f"][0], w["f"][1], B)
    blocks, Jb, J = [], [], []
    for _ in range(n_blocks):
        v, W = tr.next_block(K)
        h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
        Jb.append(h.read_binned_current().copy())
        J.append(h.read_total_current().copy())
        blocks.append((v, W))
    E = Ed.double().cpu().numpy()
    del Ed
    bins = oracle.bins_uniform(f, w["f"][0], w["f"][1], B)
    return dict(w=w, h=h, E=E, mass=mass, bins=bins, blocks=blocks, Jb=np.concatenate(Jb),
                J=np.concatenate(J), V=V)


def check_sampled_steps(s, steps):
    K = s["w"]["K"]
    scale = np.abs(s["Jb"]).max(axis=0)
    for t in steps:
        v, W = s["blocks"][t // K]
        o = oracle.modal_current(s["E"], s["mass"], v[t % K:t % K + 1], W[t % K:t % K + 1],
                                 s["bins"], s["w"]["B"])
        np.testing.assert_allclose(s["J"][t], o["J"][0], rtol=1e-12, atol=1e-9)
        err = np.abs(s["Jb"][t] - o["Jb"][0]) / np.where(scale > 0, scale, 1.0)
        assert np.all(err <= REL_TOL), (t, float(err.max()))
        assert np.all(s["Jb"][t][scale == 0] == 0)


def hcacf_sum_rule(s):
    # Eq. 18: with every mode binned, sum_b C_b(l) equals the total-current correlation
    C, cnt = s["h"].read_corr()
    J = s["J"]
    T = J.shape[0]
    L = C.shape[-1]
    assert np.array_equal(cnt, np.maximum(T - np.arange(L), 0))
    ref = np.stack([[[(J[l:, m] * J[:T - l, n]).sum() for l in range(L)] for n in range(3)]
                    for m in range(3)])
    tot = C.sum(axis=0)
    scale = np.abs(ref).max(axis=-1, keepdims=True)
    assert np.all(np.abs(tot - ref) / scale <= REL_TOL)


def test_gkma_si_n8000_full_size():
    need_gpu()
    s = setup("gkma_si_n8000", n_blocks=2)        # 512 steps > 500 lags: the ring wraps
    assert s["h"].info()["graph_replays"] == 1
    check_sampled_steps(s, [0, 255, 256, 511])
    hcacf_sum_rule(s)
    s["h"].close()


def test_gkma_si_n8000_direction_split_full_size():
    # the direction-resolved split at the Si-8000 sizes (24000 modes, 64 bins, 500 lags):
    # sampled steps against the oracle's J_n^{ab}; per-direction completeness over the bins
    need_gpu()
    s = setup("gkma_si_n8000", n_blocks=2, direction=True)
    K, B = s["w"]["K"], s["w"]["B"]
    assert s["Jb"].shape == (2 * K, 3, B, 3)
    scale = np.abs(s["Jb"]).max(axis=0)
    for t in [0, 255, 256, 511]:
        v, W = s["blocks"][t // K]
        o = oracle.modal_current_dir(s["E"], s["mass"], v[t % K:t % K + 1], W[t % K:t % K + 1],
                                     s["bins"], B)
        np.testing.assert_allclose(s["J"][t], o["Jd"][0].sum(axis=0), rtol=1e-12, atol=1e-9)
        err = np.abs(s["Jb"][t] - o["Jbd"][0]) / np.where(scale > 0, scale, 1.0)
        assert np.all(err <= REL_TOL), (t, float(err.max()))
        # all 3N modes kept: the bins of direction b add up to J^{ab}, within the bins' bounds
        tot = s["Jb"][t].sum(axis=1)
        assert np.all(np.abs(tot - o["Jd"][0]) <= REL_TOL * scale.sum(axis=1))
    C, cnt = s["h"].read_corr()
    assert C.shape == (3, B, 3, 3, s["w"]["L"])
    # Eq. 18 over bins and directions
    J = s["J"]
    T, L = J.shape[0], C.shape[-1]
    ref = np.stack([[[(J[l:, m] * J[:T - l, n]).sum() for l in range(L)] for n in range(3)]
                    for m in range(3)])
    tot = C.sum(axis=(0, 1))
    assert np.all(np.abs(tot - ref) / np.abs(ref).max(axis=-1, keepdims=True) <= REL_TOL)
    s["h"].close()


def test_hnema_graphene_n4096_full_size():
    need_gpu()
    s = setup("hnema_graphene_n4096", n_blocks=2)
    check_sampled_steps(s, [0, 200])
    mean, kap = s["h"].read_hnema()
    # Eq. 18 applied to Eq. 19: the bins' mean currents add up to the mean total current
    np.testing.assert_allclose(mean.sum(axis=0), s["J"].mean(axis=0), rtol=REL_TOL,
                               atol=REL_TOL * np.abs(s["J"]).mean())
    assert np.all(np.isfinite(kap))
    s["h"].close()


def test_mode_subset_n20000_m6000_full_size():
    need_gpu()
    s = setup("subset_si_n20000_m6000", n_blocks=1)
    check_sampled_steps(s, [0, 511])
    s["h"].close()
