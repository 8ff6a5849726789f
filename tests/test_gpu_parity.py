"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Each case feeds the same seeded inputs to libmhc.so and to oracle/ and compares
element by element with the conditioned metric of tests/parity.py (1e-5 relative on
every binned current, Eq. 17 sum and kappa bin, against the scale of the sum it is made of).
"""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, TOL, ModalRef, check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16x3", "fp16x3"]


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make_case(N, M, T, B, seed, f_hi=16.0, iso=True, drive=0.0, rho=0.8):
    D = 3 * N
    E = synth.eigvecs(D, M, seed)
    f = synth.frequencies(M, 0.0, f_hi, seed)
    mass = (synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed) if iso
            else synth.masses(N, 28.085))
    tr = synth.Trajectory(mass, rho_v=rho, rho_W=rho, drive_g=drive, seed=seed)
    v, W = tr.next_block(T)
    bins = oracle.bins_uniform(f, 0.0, f_hi, B)
    return dict(E=E, f=f, mass=mass, v=v, W=W, bins=bins, B=B, f_hi=f_hi)


def run_gpu(c, precision, K, L=0, device_inputs=True, layout="dof", e_dtype=np.float64,
            bin_ids=False, **kw):
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    T = c["v"].shape[0]
    h = ModalHeatCurrent(precision=precision, k_max=K, n_lags=L, **kw)
    E = c["E"].astype(e_dtype)
    if layout == "mode":
        E = np.ascontiguousarray(E.T)
    h.set_modes(E, c["mass"], c["f"], layout=layout)
    if bin_ids:
        h.set_bin_ids(c["bins"], c["B"])
    else:
        h.set_bins_uniform(0.0, c["f_hi"], c["B"])
    Jb, J = [], []
    for t0 in range(0, T, K):
        v = c["v"][t0:t0 + K]
        W = c["W"][t0:t0 + K]
        if device_inputs:
            v = torch.from_numpy(np.ascontiguousarray(v)).cuda()
            W = torch.from_numpy(np.ascontiguousarray(W)).cuda()
        h.push(v, W)
        Jb.append(h.read_binned_current().copy())
        J.append(h.read_total_current().copy())
    return h, np.concatenate(Jb), np.concatenate(J)


def oracle_ref(c, direction=False):
    """FP64 oracle outputs of case c with the scales of the conditioned metric."""
    return ModalRef(c["E"], c["mass"], c["v"], c["W"], c["bins"], c["B"], direction=direction)


# ----------------------------------------------------------------------------- small
@pytest.mark.parametrize("precision", PRECISIONS)
def test_tiny_system_all_paths(precision):
    need_gpu()
    c = make_case(N=8, M=24, T=6, B=4, seed=101)
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, precision, K=6)
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-12)
    o.check_current(Jb, TOL[precision], f"tiny {precision}")
    h.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_ragged_tiles_subset_and_exclusions(precision):
    # M = 200 kept of D = 300 (two 128-mode tiles, ragged), K = 37 steps (ragged
    # column tiles), frequencies beyond f_max excluded, 7 bins.
    need_gpu()
    N, M = 100, 200
    c = make_case(N=N, M=M, T=80, B=7, seed=102, f_hi=18.0)
    c["bins"] = oracle.bins_uniform(c["f"], 0.0, 14.0, 7)   # f > 14 THz excluded
    c["f_hi"] = 14.0
    assert (c["bins"] < 0).sum() > 0
    o = oracle_ref(c)
    h, Jb, J = run_gpu(c, precision, K=37)
    o.check_current(Jb, TOL[precision], f"ragged {precision}")
    info = h.info()
    assert info["n_modes_kept"] == int((c["bins"] >= 0).sum())
    h.close()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_layouts_dtypes_and_memory_spaces_agree_bitwise(precision):
    need_gpu()
    c = make_case(N=40, M=120, T=20, B=5, seed=103)
    _, a, Ja = run_gpu(c, precision, K=10, device_inputs=True, layout="dof")
    _, b, Jbb = run_gpu(c, precision, K=10, device_inputs=False, layout="mode")
    _, d, _ = run_gpu(c, precision, K=10, bin_ids=True)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, d)
    np.testing.assert_array_equal(Ja, Jbb)
    # float32 eigenvectors: same values up to the rounding of E itself
    _, e, _ = run_gpu(c, precision, K=10, e_dtype=np.float32)
    oracle_ref(c).check_current(e, TOL[precision], f"float32 E {precision}")


def test_graph_replay_matches_direct_launches():
    # pushes after the first of each K replay a captured CUDA graph; device inputs from
    # two buffers and host inputs through the staging copy, GKMA on
    need_gpu()
    from paper_2102_03691_gb300.mhc import FLAG_NO_GRAPH, ModalHeatCurrent
    c = make_case(N=64, M=192, T=96, B=6, seed=108)
    K, L = 16, 20
    outs = []
    for flags in (FLAG_NO_GRAPH, 0):
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L, flags=flags)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, 16.0, 6)
        bufs = [(torch.from_numpy(np.ascontiguousarray(c["v"][t0:t0 + K])).cuda(),
                 torch.from_numpy(np.ascontiguousarray(c["W"][t0:t0 + K])).cuda()) for t0 in (0, K)]
        Jb = []
        for i, t0 in enumerate(range(0, 96, K)):
            if i % 3 == 2:   # host input
                v, W = np.ascontiguousarray(c["v"][t0:t0 + K]), np.ascontiguousarray(c["W"][t0:t0 + K])
            else:
                v, W = bufs[i % 3]
                v.copy_(torch.from_numpy(np.ascontiguousarray(c["v"][t0:t0 + K])))
                W.copy_(torch.from_numpy(np.ascontiguousarray(c["W"][t0:t0 + K])))
            h.push(v, W)
            Jb.append(h.read_binned_current().copy())
        C, cnt = h.read_corr()
        outs.append((np.concatenate(Jb), C, h.info()["graph_replays"]))
        h.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == 0 and outs[1][2] == 5
    o = oracle_ref(c)
    o.check_current(outs[1][0], REL_TOL, "graph replay")
    o.check_corr(outs[1][1], L)


def test_async_host_inputs_match_synchronous_pushes():
    # MHC_MEM_HOST_ASYNC: the push returns before its upload; the caller refills a buffer as
    # soon as the push after the one that used it has returned (two pinned buffers), and mixes
    # in device and synchronous host pushes: bitwise the results of synchronous host pushes
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    c = make_case(N=64, M=192, T=128, B=6, seed=109)
    K, L = 16, 20
    outs = []
    for mode in ("sync", "async"):
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, 16.0, 6)
        pinned = [(torch.empty((K, 64, 3)).pin_memory(), torch.empty((K, 64, 9)).pin_memory())
                  for _ in range(2)]
        for i, t0 in enumerate(range(0, 128, K)):   # no reads in between: they would wait
            v = np.ascontiguousarray(c["v"][t0:t0 + K])
            W = np.ascontiguousarray(c["W"][t0:t0 + K])
            if mode == "sync":
                h.push(v, W)
            elif i == 3:
                h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
            elif i == 5:
                h.push(v, W)
            else:
                bv, bw = pinned[i % 2]
                bv.copy_(torch.from_numpy(v))
                bw.copy_(torch.from_numpy(W))
                h.push(bv, bw, async_inputs=True)
        h.sync()
        C, cnt = h.read_corr()
        outs.append((h.read_binned_current().copy(), C, *h.read_hnema()))
        h.close()
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    oracle_ref(c).check_corr(outs[1][1], L)


def test_deterministic_repeat():
    need_gpu()
    c = make_case(N=64, M=192, T=32, B=6, seed=104)
    _, a, _ = run_gpu(c, "bf16x3", K=16)
    _, b, _ = run_gpu(c, "bf16x3", K=16)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_identity_basis_direction_decomposition(precision):
    # E = I: each mode is one Cartesian dof, J_{3i+b}^a = W_i^{ab} v_i^b; with one
    # bin per velocity direction b the bins give the direction split of Sec. II.A.
    need_gpu()
    N = 50
    c = make_case(N=N, M=3 * N, T=8, B=3, seed=105)
    c["E"] = np.eye(3 * N)
    c["bins"] = (np.arange(3 * N) % 3).astype(np.int32)
    o = oracle_ref(c)
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    h = ModalHeatCurrent(precision=precision, k_max=8)
    h.set_modes(c["E"], c["mass"], None)
    h.set_bin_ids(c["bins"], 3)
    h.push(c["v"], c["W"])
    Jb = h.read_binned_current()
    expect = np.einsum("tiab,tib->tba", c["W"].astype(np.float64).reshape(8, N, 3, 3),
                       c["v"].astype(np.float64))
    np.testing.assert_allclose(o.Jb, expect, rtol=1e-12, atol=1e-10)
    o.check_current(Jb, REL_TOL, f"identity basis {precision}")


# ----------------------------------------------------------------------------- GKMA / HNEMA
@pytest.mark.parametrize("precision", PRECISIONS)
def test_gkma_and_hnema_small(precision):
    need_gpu()
    L, K, T = 12, 16, 70
    c = make_case(N=48, M=144, T=T, B=6, seed=106, drive=2e-3)
    o = oracle_ref(c)
    dt, TK, V = 0.01, 300.0, 48 * 20.02
    h, Jb, J = run_gpu(c, precision, K=K, L=L, dt_ps=dt, T_K=TK, V_A3=V)
    tol = TOL[precision]
    o.check_current(Jb, tol, f"Jb {precision}")
    C, cnt = h.read_corr()
    _, ocnt = o.check_corr(C, L, tol, f"corr {precision}")
    np.testing.assert_array_equal(cnt, ocnt)
    kt, kw = h.read_kappa_gk(0.05, 0.11)
    _, n = o.check_kappa(kt, kw, L, dt, TK, V, 0.05, 0.11, tol, f"kappa_gk {precision}")
    assert n == 7
    mean, kap = h.read_hnema()
    o.check_hnema(mean, kap, TK, V, [1e-5, 0, 0], tol, f"HNEMA {precision}")


@pytest.mark.parametrize("pinned", [False, True])
def test_host_inputs_back_to_back_reuse_one_buffer(pinned):
    # Host inputs go through two staging buffers on a copy stream; the call returns only once
    # it has read the caller's memory, so one host buffer can be refilled right after each push
    # while earlier pushes are still running.  Bitwise equal to device inputs.
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    K, T = 8, 64
    c = make_case(N=64, M=192, T=T, B=4, seed=108)

    def run(host):
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=6)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, c["f_hi"], 4)
        if pinned:
            bv = torch.empty((K, 64, 3), dtype=torch.float32).pin_memory()
            bw = torch.empty((K, 64, 9), dtype=torch.float32).pin_memory()
        else:
            bv, bw = np.empty((K, 64, 3), np.float32), np.empty((K, 64, 9), np.float32)
        for t0 in range(0, T, K):
            if host:
                bv[:] = torch.from_numpy(c["v"][t0:t0 + K]) if pinned else c["v"][t0:t0 + K]
                bw[:] = torch.from_numpy(c["W"][t0:t0 + K]) if pinned else c["W"][t0:t0 + K]
                h.push(bv, bw)
            else:
                h.push(torch.from_numpy(c["v"][t0:t0 + K]).cuda(), torch.from_numpy(c["W"][t0:t0 + K]).cuda())
        C, _ = h.read_corr()
        m, _ = h.read_hnema()
        h.close()
        return C, m
    Ca, ma = run(True)
    Cb, mb = run(False)
    np.testing.assert_array_equal(Ca, Cb)
    np.testing.assert_array_equal(ma, mb)


def test_state_roundtrip_is_bitwise():
    need_gpu()
    L, K = 10, 8
    c = make_case(N=32, M=96, T=40, B=4, seed=107)
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent

    def fresh():
        h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L)
        h.set_modes(c["E"], c["mass"], c["f"])
        h.set_bins_uniform(0.0, 16.0, 4)
        return h
    a = fresh()
    for t0 in range(0, 40, K):
        a.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    Ca, _ = a.read_corr()
    ma, _ = a.read_hnema()
    b = fresh()
    for t0 in range(0, 24, K):
        b.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    blob = b.get_state()
    b.close()
    b2 = fresh()
    b2.set_state(blob)
    for t0 in range(24, 40, K):
        b2.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
    Cb, _ = b2.read_corr()
    mb, _ = b2.read_hnema()
    np.testing.assert_array_equal(Ca, Cb)
    np.testing.assert_array_equal(ma, mb)


# ----------------------------------------------------------------------------- workload sizes
@pytest.mark.parametrize("precision", PRECISIONS)
def test_gkma_si_n512_full_run(precision):
    # The N = 512 Si-like GKMA workload at full size: 1536 modes, 1000 steps,
    # 100 frequency bins, 200 lags, every output compared with the oracle.
    need_gpu()
    w = synth.WORKLOADS["gkma_si_n512"]
    c = make_case(N=w["N"], M=w["M"], T=w["T_s"], B=w["B"], seed=w["seed"], iso=False)
    L = w["L"]
    o = oracle_ref(c)
    V = w["N"] * w["V_per_atom"]
    h, Jb, J = run_gpu(c, precision, K=w["K"], L=L, dt_ps=w["dt_ps"], T_K=w["T_K"], V_A3=V)
    tol = TOL[precision]
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-9)
    o.check_current(Jb, tol, f"N512 Jb {precision}")
    C, cnt = h.read_corr()
    o.check_corr(C, L, tol, f"N512 corr {precision}")
    tau_lo, tau_hi = 0.8 * (L - 1) * w["dt_ps"], (L - 1) * w["dt_ps"]
    kt, kw = h.read_kappa_gk(tau_lo, tau_hi)
    o.check_kappa(kt, kw, L, w["dt_ps"], w["T_K"], V, tau_lo, tau_hi, tol,
                  f"N512 kappa {precision}")
    mean, kap = h.read_hnema()
    o.check_hnema(mean, kap, w["T_K"], V, w["Fe"], tol, f"N512 HNEMA {precision}")


def test_orthonormality_check_fp64_on_gpu():
    # max |E^T E - I| in FP64 on the GPU: ~1e-15 for a QR basis; perturbing one entry by d
    # changes row/column n of E^T E by d*E[r,m] (m != n) and the diagonal by 2 d E[r,n] + d^2
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    N = 40
    D = 3 * N
    E = synth.eigvecs(D, D, 109)
    mass = synth.masses(N, 28.085)
    for probe in (0, 17):        # full check, and 17 probe modes
        h = ModalHeatCurrent(precision="fp16x3", k_max=4, ortho_probe=probe)
        h.set_modes(E, mass, None)
        assert h.check_orthonormality(1e-12) < 1e-13
        h.close()
    r, n, d = 5, 0, 1e-3          # mode 0 is probe 0 in both settings
    E2 = E.copy()
    E2[r, n] += d
    expect = max(np.abs(d * np.delete(E[r], n)).max(), abs(2 * d * E[r, n] + d * d))
    h = ModalHeatCurrent(precision="fp16x3", k_max=4, ortho_probe=0)
    with pytest.warns(UserWarning):
        h.set_modes(E2, mass, None)
    assert abs(h.check_orthonormality(1e-6) - expect) < 1e-13
    h.close()


def test_unbinned_per_mode_currents_and_correlations():
    # one bin per mode (B = M): the binned output is the per-mode current J_n (Eq. 16) and
    # the GKMA sums become per-mode correlations with the total current (Eq. 17)
    need_gpu()
    N, K, L = 64, 32, 6
    c = make_case(N=N, M=3 * N, T=2 * K, B=1, seed=110)
    M = 3 * N
    ids = np.arange(M, dtype=np.int32)
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=L)
    h.set_modes(c["E"], c["mass"], c["f"])
    h.set_bin_ids(ids, M)
    Jb = []
    for t0 in (0, K):
        h.push(c["v"][t0:t0 + K], c["W"][t0:t0 + K])
        Jb.append(h.read_binned_current().copy())
    Jb = np.concatenate(Jb)
    o = oracle.modal_current(c["E"], c["mass"], c["v"], c["W"], ids, M, want_modes=True)
    np.testing.assert_allclose(o["Jb"], o["Jn"], rtol=0, atol=0)
    # one mode per bin: judged against the condition number of Eq. 16 (tests/parity.py)
    ref = ModalRef(c["E"], c["mass"], c["v"], c["W"], ids, M)
    assert np.all(ref.small)
    ref.check_current(Jb, REL_TOL, "per-mode currents")
    C, _ = h.read_corr()
    ref.check_corr(C, L, REL_TOL, "per-mode Eq. 17 sums")
    h.close()


def test_polarization_resolved_bins():
    # in-plane / out-of-plane decomposition (Sec. III.A.ii): modes classified by the weight
    # of their eigenvector on z; bin id = frequency bin + B * class.  The two classes add up
    # to the frequency-only binning and each matches the oracle.
    need_gpu()
    N, K, B = 60, 24, 10
    c = make_case(N=N, M=3 * N, T=K, B=B, seed=111, f_hi=50.0)
    M = 3 * N
    zfrac = (c["E"].reshape(N, 3, M)[:, 2, :] ** 2).sum(axis=0)
    cls = (zfrac >= 1.0 / 3.0).astype(np.int32)
    fb = oracle.bins_uniform(c["f"], 0.0, 50.0, B)
    ids = np.where(fb >= 0, fb + B * cls, -1).astype(np.int32)
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    h = ModalHeatCurrent(precision="fp16x3", k_max=K)
    h.set_modes(c["E"], c["mass"], c["f"])
    h.set_bin_ids(ids, 2 * B)
    h.push(c["v"], c["W"])
    J2 = h.read_binned_current()
    o2 = ModalRef(c["E"], c["mass"], c["v"], c["W"], ids, 2 * B)
    o2.check_current(J2, REL_TOL, "polarization classes")
    h.set_bins_uniform(0.0, 50.0, B)
    h.push(c["v"], c["W"])
    J1 = h.read_binned_current()
    o1 = ModalRef(c["E"], c["mass"], c["v"], c["W"], fb, B)
    o1.check_current(J1, REL_TOL, "frequency bins")
    # the two classes add up to the frequency binning, within the bound of either side
    check(J2[:, :B] + J2[:, B:], J1, o2.S[:, :B] + o2.S[:, B:] + o1.S,
          o2.Sd[:, :B] + o2.Sd[:, B:] + o1.Sd, REL_TOL,
          "classes add up")
    h.close()
