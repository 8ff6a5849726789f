"""Parity at the workloads' full sizes, in the launch configuration bench.py times
(autotuned tile, graph replay after the first push).

Every step of every pushed block is recomputed by the oracle with the projections of
Eqs. 13 and 16 written as FP64 matrix products (oracle.modal_current_mm), and every binned
current, Eq. 17 sum, kappa(tau) value, kappa window and HNEMA mean is compared element by
element with the conditioned metric of tests/parity.py.  The lag correlation and the
Green-Kubo integral are also checked as stages on their own, fed with the library's own
binned currents (the oracle's Eq. 17 sums and integral of those inputs).
"""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, ModalRef, check, stage_corr_check

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
    vs, Ws, Jb, J = [], [], [], []
    for _ in range(n_blocks):
        v, W = tr.next_block(K)
        h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
        Jb.append(h.read_binned_current().copy())
        J.append(h.read_total_current().copy())
        vs.append(v)
        Ws.append(W)
    E = Ed.double().cpu().numpy()          # the float32 basis the library was given
    del Ed
    bins = oracle.bins_uniform(f, w["f"][0], w["f"][1], B)
    v, W = np.concatenate(vs), np.concatenate(Ws)
    ref = ModalRef(E, mass, v, W, bins, B, direction=direction, mm=True)
    del E
    return dict(w=w, h=h, ref=ref, Jb=np.concatenate(Jb), J=np.concatenate(J), V=V)


def check_run(s, name):
    w, h, o = s["w"], s["h"], s["ref"]
    np.testing.assert_allclose(s["J"], o.J, rtol=1e-12, atol=1e-9)
    assert not np.any(o.small)               # every bin takes the per-bin metric of sum |J_n|
    o.check_current(s["Jb"], REL_TOL, f"{name} binned currents")
    mean, kap = h.read_hnema()
    o.check_hnema(mean, kap, w["T_K"], s["V"], w["Fe"], REL_TOL, f"{name} HNEMA")
    L = w["L"]
    if not L:
        return
    C, cnt = h.read_corr()
    T = s["J"].shape[0]
    assert np.array_equal(cnt, np.maximum(T - np.arange(L), 0))
    o.check_corr(C, L, REL_TOL, f"{name} Eq. 17 sums")
    stage_corr_check(C, o.rows(s["Jb"]), s["J"], L, REL_TOL, f"{name} lag stage")
    tau_hi = (L - 1) * w["dt_ps"]
    tau_lo = 0.8 * tau_hi
    kt, kw = h.read_kappa_gk(tau_lo, tau_hi)
    o.check_kappa(kt, kw, L, w["dt_ps"], w["T_K"], s["V"], tau_lo, tau_hi, REL_TOL,
                  f"{name} kappa")
    # the Green-Kubo stage alone: the oracle's integral of the library's own Eq. 17 sums
    Cr = C.reshape(-1, 3, 3, L)
    okt = oracle.gk_kappa(Cr, cnt, w["dt_ps"], w["T_K"], s["V"])
    skt = oracle.gk_kappa(np.abs(Cr), cnt, w["dt_ps"], w["T_K"], s["V"])
    check(kt.reshape(okt.shape), okt, skt, None, 1e-11, f"{name} Green-Kubo stage")
    if w["M"] != 3 * w["N"]:
        return
    # Eq. 18: with every mode binned, the bins' Eq. 17 sums add up to the total-current
    # correlation of the library's own total current
    J = s["J"]
    ref = np.stack([[[(J[l:, m] * J[:T - l, n]).sum() for l in range(L)] for n in range(3)]
                    for m in range(3)])
    _, _, SC, SCd = o.corr(L, full=True)
    rows = C.reshape(-1, 3, 3, L)
    check(rows.sum(axis=0), ref, SC.sum(axis=0), SCd.sum(axis=0), REL_TOL,
          f"{name} Eq. 18 sum rule")


def test_gkma_si_n8000_full_size():
    need_gpu()
    s = setup("gkma_si_n8000", n_blocks=2)        # 512 steps > 500 lags: the ring wraps
    assert s["h"].info()["graph_replays"] == 1
    check_run(s, "Si-8000")
    s["h"].close()


def test_gkma_si_n8000_direction_split_full_size():
    # the direction-resolved split at the Si-8000 sizes (24000 modes, 64 bins, 500 lags)
    need_gpu()
    s = setup("gkma_si_n8000", n_blocks=2, direction=True)
    K, B = s["w"]["K"], s["w"]["B"]
    assert s["Jb"].shape == (2 * K, 3, B, 3)
    check_run(s, "Si-8000 direction")
    # all 3N modes kept: the bins of direction b add up to J^{ab}, within the bins' bounds
    o = s["ref"]
    check(s["Jb"].sum(axis=2).sum(axis=1), o.J, o.S.sum(axis=(1, 2)), o.Sd.sum(axis=(1, 2)), REL_TOL,
          "Si-8000 direction completeness")
    s["h"].close()


def test_hnema_graphene_n4096_full_size():
    need_gpu()
    s = setup("hnema_graphene_n4096", n_blocks=2)
    check_run(s, "graphene-4096")
    s["h"].close()


def test_mode_subset_n20000_m6000_full_size():
    need_gpu()
    s = setup("subset_si_n20000_m6000", n_blocks=1)
    check_run(s, "subset 20000/6000")
    s["h"].close()
