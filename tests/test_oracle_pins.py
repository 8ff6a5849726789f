"""Pins for the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a hand-derived
worked example (tests/golden), a closed form, an invariant of the method
(Parseval for Eq. 13-14, completeness for Eq. 15/18, the direction
decomposition of Sec. II.A), an independent algorithm (FFT correlation), an
independent restatement (oracle/brute.py, per-atom vectors in scalar
Python), or independent constants (scipy.constants).  The last tests plant
mistakes in copies of the oracle source and check that the pins catch them.
"""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2102_03691_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def golden(name):
    with open(GOLDEN) as f:
        for ex in json.load(f)["examples"]:
            if ex["name"] == name:
                return ex
    raise KeyError(name)


def tiny_system(N, M=None, T=4, seed=1, iso=True):
    D = 3 * N
    M = D if M is None else M
    E = synth.eigvecs(D, M, seed)
    mass = (synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed) if iso
            else synth.masses(N, 28.085))
    tr = synth.Trajectory(mass, rho_v=0.5, rho_W=0.5, seed=seed)
    v, W = tr.next_block(T)
    return E, mass, v, W


# ---------------------------------------------------------------- golden
def test_golden_one_atom_identity_basis():
    ex = golden("one_atom_identity_basis")
    E = np.array(ex["E_dof_major"], float)
    r = oracle.modal_current(E, ex["mass"], np.array(ex["v"], np.float32),
                             np.array(ex["W"], np.float32), [0, 0, 0], 1, want_modes=True)
    np.testing.assert_allclose(r["xdot"], ex["xdot"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jn"], ex["Jn"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["J"], ex["J"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jb"][0, 0], ex["J"][0], rtol=0, atol=1e-12)


def test_golden_two_atoms_mixed_basis():
    ex = golden("two_atoms_mixed_basis_two_steps")
    E = np.array(ex["E_dof_major"], float)
    bins = oracle.bins_uniform(ex["freq_THz"], ex["bins"]["f_min"], ex["bins"]["f_max"],
                               ex["bins"]["B"])
    assert bins.tolist() == ex["bins"]["bin_of_mode"]
    v = np.array(ex["v"], np.float32)
    W = np.array(ex["W"], np.float32)
    r = oracle.modal_current(E, ex["mass"], v, W, bins, 2, want_modes=True)
    np.testing.assert_allclose(r["xdot"], ex["xdot"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jn"], ex["Jn"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["J"], ex["J"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jb"], ex["Jb"], rtol=0, atol=1e-12)
    assert abs(np.sum(r["xdot"][0] ** 2) - ex["parseval_step0"]) < 1e-12
    C, cnt = oracle.gkma_corr(r["Jb"], r["J"], 2)
    assert cnt.tolist() == [2, 1]
    np.testing.assert_allclose(C[0, 0, 0] / cnt, ex["C_bin0_xx"], rtol=1e-15)
    np.testing.assert_allclose(C[1, 2, 1] / cnt, ex["C_bin1_zy"], rtol=1e-15)
    kap = oracle.gk_kappa(C, cnt, 0.01, 300.0, 1000.0)
    c = oracle_conv_factor(300.0, 1000.0)
    assert kap[0, 0, 0, 0] == 0.0
    np.testing.assert_allclose(kap[0, 0, 0, 1] / c, ex["int_bin0_xx_lag1"], rtol=1e-12)
    mean, _ = oracle.hnema(r["Jb"], 300.0, 1000.0, [1e-5, 0, 0])
    np.testing.assert_allclose(mean, ex["meanJb"], rtol=0, atol=1e-12)


def oracle_conv_factor(T_K, V_A3):
    """1/(k_B T^2 V) in W/(m K) per (eV A/ps)^2 ps, from scipy's CODATA constants."""
    sc = pytest.importorskip("scipy.constants")
    kB_eV = sc.k / sc.e
    wmk = sc.e / (1e-12 * 1e-10)       # 1 eV/(ps A K) -> W/(m K)
    return wmk / (kB_eV * T_K * T_K * V_A3)


# ---------------------------------------------------------------- binning
def test_bins_edges_and_exclusions():
    f = np.array([0.0, 0.25, 0.2499999999, 15.75, 16.0, 16.0000001, -1e-9, np.nan, np.inf, 8.0])
    b = oracle.bins_uniform(f, 0.0, 16.0, 64)
    # half-open bins of 0.25 THz (Sec. III.A.iii); last bin closed; outside -> -1
    assert b.tolist() == [0, 1, 0, 63, 63, -1, -1, -1, -1, 32]


def test_bins_counts_match_histogram():
    f = synth.frequencies(5000, 0.0, 16.0, seed=3)
    b = oracle.bins_uniform(f, 0.0, 16.0, 64)
    hist, _ = np.histogram(f, bins=64, range=(0.0, 16.0))
    assert np.array_equal(np.bincount(b, minlength=64), hist)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("N,M,T,L", [(1, 3, 3, 2), (2, 6, 5, 3), (3, 7, 6, 4), (5, 15, 4, 3)])
def test_oracle_matches_scalar_brute_force(N, M, T, L):
    E, mass, v, W = tiny_system(N, M, T, seed=10 + N)
    B = 3
    f = synth.frequencies(M, 0.0, 3.0, seed=N)
    bins = oracle.bins_uniform(f, 0.0, 3.0, B)
    r = oracle.modal_current(E, mass, v, W, bins, B, want_modes=True)
    ref = brute.run(E, mass, v, W, bins, B, L=L)
    np.testing.assert_allclose(r["xdot"], ref["xdot"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["Jn"], ref["Jn"], rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(r["J"], ref["J"], rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(r["Jb"], ref["Jb"], rtol=1e-12, atol=1e-11)
    C, cnt = oracle.gkma_corr(r["Jb"], r["J"], L)
    np.testing.assert_allclose(C / cnt, ref["C"], rtol=1e-12, atol=1e-10)
    mean, _ = oracle.hnema(r["Jb"], 300.0, 100.0, [1e-5, 0, 0])
    np.testing.assert_allclose(mean, ref["meanJb"], rtol=1e-12, atol=1e-11)


# ---------------------------------------------------------------- invariants
def test_parseval_and_inverse_transform():
    # Eq. 13 with a square orthonormal basis preserves sum_i m_i |v_i|^2, and
    # Eq. 14 inverts it.
    N = 20
    E, mass, v, W = tiny_system(N, T=3, seed=5)
    r = oracle.modal_current(E, mass, v, W, np.zeros(3 * N, np.int32), 1, want_modes=True)
    for t in range(3):
        lhs = np.sum(r["xdot"][t] ** 2)
        rhs = np.sum(mass[:, None] * v[t].astype(np.float64) ** 2)
        assert abs(lhs - rhs) <= 1e-12 * rhs
        v_back = (E @ r["xdot"][t]).reshape(N, 3) / np.sqrt(mass)[:, None]
        np.testing.assert_allclose(v_back, v[t], rtol=0, atol=1e-10)


def test_completeness_all_modes():
    # Eq. 15 / Eq. 18: with all 3N modes the modal currents sum to J (Eq. 10).
    N = 16
    E, mass, v, W = tiny_system(N, T=4, seed=6)
    ref_J = np.einsum("tiab,tib->ta", W.astype(np.float64).reshape(4, N, 3, 3),
                      v.astype(np.float64))
    r = oracle.modal_current(E, mass, v, W, np.zeros(3 * N, np.int32), 1, want_modes=True)
    np.testing.assert_allclose(r["J"], ref_J, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(r["Jn"].sum(axis=1), ref_J, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(r["Jb"][:, 0, :], ref_J, rtol=1e-10, atol=1e-9)


def test_identity_basis_direction_decomposition():
    # E = I: mode 3i+b carries J^a = W_i^{ab} v_i^b (Sec. II.A direction split).
    N = 7
    _, mass, v, W = tiny_system(N, T=2, seed=8)
    E = np.eye(3 * N)
    r = oracle.modal_current(E, mass, v, W, np.zeros(3 * N, np.int32), 1, want_modes=True)
    Wm = W.astype(np.float64).reshape(2, N, 3, 3)
    expect = np.einsum("tiab,tib->tiba", Wm, v.astype(np.float64)).reshape(2, 3 * N, 3)
    np.testing.assert_allclose(r["Jn"], expect, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- direction split (Sec. II.A)
def test_golden_direction_split_rotated_basis():
    ex = golden("one_atom_rotated_basis_direction_split")
    r = oracle.modal_current_dir(np.array(ex["E_dof_major"], float), ex["mass"],
                                 np.array(ex["v"], np.float32), np.array(ex["W"], np.float32),
                                 [0, 0, 0], 1, want_modes=True)
    np.testing.assert_allclose(r["Jnd"], ex["Jnd"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jd"], ex["Jd"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jbd"][:, :, 0, :], np.array(ex["Jnd"]).sum(axis=1), atol=1e-12)


def test_golden_direction_split_two_atoms():
    ex = golden("two_atoms_mixed_basis_two_steps")
    r = oracle.modal_current_dir(np.array(ex["E_dof_major"], float), ex["mass"],
                                 np.array(ex["v"], np.float32), np.array(ex["W"], np.float32),
                                 ex["bins"]["bin_of_mode"], ex["bins"]["B"])
    np.testing.assert_allclose(r["Jbd"], ex["Jbd"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["Jd"], ex["Jd"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,M,T", [(1, 3, 2), (2, 5, 3), (4, 12, 2)])
def test_direction_split_matches_scalar_brute_force(N, M, T):
    E, mass, v, W = tiny_system(N, M, T=T, seed=30 + N)
    bins = np.arange(M) % 2
    r = oracle.modal_current_dir(E, mass, v, W, bins, 2)
    ref = np.array(brute.run_dir(E, mass, v, W, bins, 2))
    np.testing.assert_allclose(r["Jbd"], ref, rtol=1e-12, atol=1e-12)


def test_direction_split_completeness_per_direction():
    # With all 3N orthonormal modes, sum_n e^b_{i,n} e^b'_{j,n} = delta_ij delta_bb', so the
    # modes of each direction b add up to J^{ab} = sum_i W_i^{ab} v_i^b.
    N = 12
    E, mass, v, W = tiny_system(N, T=3, seed=41)
    ref = np.einsum("tiab,tib->tba", W.astype(np.float64).reshape(3, N, 3, 3), v.astype(np.float64))
    r = oracle.modal_current_dir(E, mass, v, W, np.zeros(3 * N, np.int32), 1, want_modes=True)
    np.testing.assert_allclose(r["Jd"], ref, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(r["Jnd"].sum(axis=1), ref, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(r["Jbd"][:, :, 0, :], ref, rtol=1e-10, atol=1e-9)


def test_direction_split_adds_up_to_eq16():
    N = 5
    E, mass, v, W = tiny_system(N, 11, T=3, seed=43)
    bins = np.array([0, 1, 2] * 4)[:11]
    rd = oracle.modal_current_dir(E, mass, v, W, bins, 3, want_modes=True)
    r = oracle.modal_current(E, mass, v, W, bins, 3, want_modes=True)
    np.testing.assert_allclose(rd["Jnd"].sum(axis=2), r["Jn"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rd["Jbd"].sum(axis=1), r["Jb"], rtol=1e-12, atol=1e-12)


def test_direction_split_planar_modes():
    # A basis of in-plane (x, y only) and out-of-plane (z only) modes, as for flat graphene:
    # in-plane modes carry nothing along beta = z, out-of-plane modes nothing along x, y.
    N = 6
    rng = np.random.default_rng(44)
    Qxy, _ = np.linalg.qr(rng.standard_normal((2 * N, 2 * N)))
    Qz, _ = np.linalg.qr(rng.standard_normal((N, N)))
    E = np.zeros((3 * N, 3 * N))
    xy = np.array([3 * i + b for i in range(N) for b in (0, 1)])
    z = np.array([3 * i + 2 for i in range(N)])
    E[np.ix_(xy, np.arange(2 * N))] = Qxy
    E[np.ix_(z, np.arange(2 * N, 3 * N))] = Qz
    _, mass, v, W = tiny_system(N, T=2, seed=44)
    r = oracle.modal_current_dir(E, mass, v, W, np.zeros(3 * N, np.int32), 1, want_modes=True)
    assert np.all(r["Jnd"][:, :2 * N, 2, :] == 0)
    assert np.all(r["Jnd"][:, 2 * N:, :2, :] == 0)
    assert np.abs(r["Jnd"][:, :2 * N, :2, :]).max() > 0


def test_mode_permutation_and_sign_flips():
    N = 6
    E, mass, v, W = tiny_system(N, T=2, seed=9)
    rng = np.random.default_rng(0)
    perm = rng.permutation(3 * N)
    signs = rng.choice([-1.0, 1.0], size=3 * N)
    z = np.zeros(3 * N, np.int32)
    a = oracle.modal_current(E, mass, v, W, z, 1, want_modes=True)
    b = oracle.modal_current(E[:, perm] * signs, mass, v, W, z, 1, want_modes=True)
    np.testing.assert_allclose(b["xdot"], a["xdot"][:, perm] * signs, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(b["Jn"], a["Jn"][:, perm], rtol=1e-12, atol=1e-12)


def test_scaling_laws():
    N = 5
    E, mass, v, W = tiny_system(N, 11, T=2, seed=12)
    bins = np.arange(11, dtype=np.int32) % 3
    a = oracle.modal_current(E, mass, v, W, bins, 3, want_modes=True)
    v2 = (v * np.float32(2.0)).astype(np.float32)        # exact in float32
    b = oracle.modal_current(E, mass, v2, W, bins, 3, want_modes=True)
    np.testing.assert_allclose(b["Jb"], 2 * a["Jb"], rtol=1e-13, atol=1e-12)
    W4 = (W * np.float32(4.0)).astype(np.float32)
    c = oracle.modal_current(E, mass, v, W4, bins, 3, want_modes=True)
    np.testing.assert_allclose(c["Jn"], 4 * a["Jn"], rtol=1e-13, atol=1e-12)
    d = oracle.modal_current(E, mass * 9.0, v, W, bins, 3, want_modes=True)
    np.testing.assert_allclose(d["Jn"], a["Jn"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(d["xdot"], 3 * a["xdot"], rtol=1e-13, atol=1e-12)


def test_excluded_modes_do_not_contribute():
    N = 4
    E, mass, v, W = tiny_system(N, T=2, seed=13)
    bins = np.array([0, -1, 1, 1, -1, 0, 0, 1, -1, 1, 0, 0], np.int32)
    r = oracle.modal_current(E, mass, v, W, bins, 2, want_modes=True)
    for b in range(2):
        np.testing.assert_allclose(r["Jb"][:, b], r["Jn"][:, bins == b].sum(axis=1),
                                   rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- GKMA / HNEMA
def test_constant_input_correlation_closed_form():
    # v and W fixed for all t: C_b(l) = J_b J for every lag, and the trapezoid
    # integral is linear in tau: kappa(l) = c dt l J_b J.
    N = 4
    E, mass, v, W = tiny_system(N, T=1, seed=14)
    T, L = 12, 5
    vv = np.repeat(v, T, axis=0)
    WW = np.repeat(W, T, axis=0)
    bins = np.arange(3 * N, dtype=np.int32) % 2
    r = oracle.modal_current(E, mass, vv, WW, bins, 2)
    C, cnt = oracle.gkma_corr(r["Jb"], r["J"], L)
    prod = np.einsum("bm,n->bmn", r["Jb"][0], r["J"][0])
    for l in range(L):
        np.testing.assert_allclose(C[..., l] / cnt[l], prod, rtol=1e-13, atol=1e-12)
    dt, TK, V = 0.01, 300.0, 500.0
    kap = oracle.gk_kappa(C, cnt, dt, TK, V)
    c = oracle_conv_factor(TK, V)
    for l in range(L):
        np.testing.assert_allclose(kap[..., l], c * dt * l * prod, rtol=1e-9, atol=1e-12)
    kw, n = oracle.kappa_window(kap, dt, 0.02, 0.04)
    assert n == 3
    np.testing.assert_allclose(kw, c * dt * 3 * prod, rtol=1e-9, atol=1e-12)
    mean, kh = oracle.hnema(r["Jb"], TK, V, [0.0, 2e-5, 0.0])
    np.testing.assert_allclose(mean, r["Jb"][0], rtol=1e-13)
    sc = pytest.importorskip("scipy.constants")
    wmk = sc.e / (1e-12 * 1e-10)
    np.testing.assert_allclose(kh, r["Jb"][0] / (TK * V * 2e-5) * wmk, rtol=1e-9)


def test_correlation_matches_fft_and_hcacf():
    # Direct O(T L) sums vs an FFT cross-correlation (different algorithm), and
    # the Eq. 18 sum rule: with all modes binned, sum_b C_b(l) is the total
    # heat-current autocorrelation.
    N = 6
    E, mass, v, W = tiny_system(N, T=40, seed=15)
    B, L = 4, 9
    bins = np.arange(3 * N, dtype=np.int32) % B
    r = oracle.modal_current(E, mass, v, W, bins, B)
    C, cnt = oracle.gkma_corr(r["Jb"], r["J"], L)
    T = r["J"].shape[0]
    nfft = 2 * T
    for b in range(B):
        for mu in range(3):
            for nu in range(3):
                fa = np.fft.rfft(r["Jb"][:, b, mu], nfft)
                fb = np.fft.rfft(r["J"][:, nu], nfft)
                cc = np.fft.irfft(fa * np.conj(fb), nfft)[:L]   # sum_t a(t) b(t-l)
                np.testing.assert_allclose(C[b, mu, nu], cc, rtol=1e-9, atol=1e-8)
    hcacf = np.array([[[np.sum(r["J"][l:, m] * r["J"][:T - l, n]) for l in range(L)]
                       for n in range(3)] for m in range(3)])
    np.testing.assert_allclose(C.sum(axis=0), hcacf, rtol=1e-9, atol=1e-8)


# ---------------------------------------------------------------- bin-bin cross-correlation
def test_xcorr_golden_two_atoms():
    # hand example: bins 0, 1 of the two-atom case, lag 0 and 1 (values from the golden Jb;
    # step 1 is twice step 0 here, so the lag direction is pinned by the FFT test below)
    ex = golden("two_atoms_mixed_basis_two_steps")
    Jb = np.array(ex["Jb"], float)          # [2][2][3]
    X = oracle.gkma_xcorr(Jb, 2)
    # bin0 x with bin1 z: lag 0 = 10*4.5 + 20*9, lag 1 = Jb[1][0][x] * Jb[0][1][z] = 20 * 4.5
    np.testing.assert_allclose(X[0, 1, 0, 2], [10 * 4.5 + 20 * 9, 20 * 4.5], rtol=0, atol=1e-12)
    # bin1 y with bin0 y: lag 0 = 0.5*2.5 + 1*5, lag 1 = 1 * 2.5
    np.testing.assert_allclose(X[1, 0, 1, 1], [0.5 * 2.5 + 1 * 5, 1 * 2.5], rtol=0, atol=1e-12)


def test_xcorr_sums_to_eq17_with_every_mode_binned():
    # all 3N modes binned: sum over the second bin is the total current (Eq. 15), so the
    # cross-correlations add up to the Eq. 17 sums
    N, T, L, B = 6, 40, 7, 4
    E, mass, v, W = tiny_system(N, T=T, seed=52)
    bins = np.arange(3 * N) % B
    r = oracle.modal_current(E, mass, v, W, bins, B)
    X = oracle.gkma_xcorr(r["Jb"], L)
    C, _ = oracle.gkma_corr(r["Jb"], r["J"], L)
    np.testing.assert_allclose(X.sum(axis=1), C, rtol=1e-10, atol=1e-10 * np.abs(C).max())


def test_xcorr_matches_fft_and_lag0_symmetry():
    rng = np.random.default_rng(53)
    T, B, L = 64, 3, 9
    Jb = rng.standard_normal((T, B, 3))
    X = oracle.gkma_xcorr(Jb, L)
    n = 2 * T
    F = np.fft.rfft(Jb, n=n, axis=0)                                  # [f][B][3]
    # sum_t x(t) y(t - l) = irfft(X(f) conj(Y(f)))[l]
    full = np.fft.irfft(F[:, :, None, :, None] * np.conj(F[:, None, :, None, :]), n=n, axis=0)
    ref = np.moveaxis(full[:L], 0, -1)                                 # [B][B][3][3][L]
    np.testing.assert_allclose(X, ref, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(X[:, :, :, :, 0], np.transpose(X[:, :, :, :, 0], (1, 0, 3, 2)),
                               rtol=1e-13, atol=1e-13)


def test_impulse_correlation():
    # A single nonzero modal-current sample at t0 gives one term per lag.
    T, B, L, t0 = 10, 2, 4, 6
    Jb = np.zeros((T, B, 3))
    Jb[t0, 1, 2] = 3.0
    J = np.arange(T * 3, dtype=float).reshape(T, 3) + 1.0
    C, cnt = oracle.gkma_corr(Jb, J, L)
    for l in range(L):
        np.testing.assert_allclose(C[1, 2, :, l], 3.0 * J[t0 - l], rtol=1e-15)
    assert np.all(C[0] == 0) and np.all(C[1, :2] == 0)


def test_hnema_sum_rule():
    # Eq. 18 applied to Eq. 19: sum_b <J_b> = <J> with all modes kept.
    N = 8
    E, mass, v, W = tiny_system(N, T=6, seed=16)
    bins = np.arange(3 * N, dtype=np.int32) % 5
    r = oracle.modal_current(E, mass, v, W, bins, 5)
    mean, _ = oracle.hnema(r["Jb"], 300.0, 100.0, [1e-5, 0, 0])
    np.testing.assert_allclose(mean.sum(axis=0), r["J"].mean(axis=0), rtol=1e-10, atol=1e-9)


def test_orthonormality_residual():
    E = synth.eigvecs(60, 60, seed=2)
    assert oracle.orthonormality(E) < 1e-13
    # perturbing one entry by d changes row/column 7 of E^T E by d*E[3,m]
    # (m != 7) and the diagonal by 2 d E[3,7] + d^2
    d = 1e-3
    E2 = E.copy()
    E2[3, 7] += d
    off = np.abs(d * np.delete(E[3], 7)).max()
    diag = abs(2 * d * E[3, 7] + d * d)
    assert abs(oracle.orthonormality(E2) - max(off, diag)) < 1e-13


def test_drive_coupling_gives_target_mean_current():
    # The drive option of the input generator shifts <J^x> to kappa T V F_e.
    N = 64
    mass = synth.masses(N, 12.011)
    TK, V, Fe, kap = 300.0, N * 8.77, 1e-5, 3000.0
    g = synth.drive_coupling(kap, TK, V, Fe, mass)
    tr = synth.Trajectory(mass, rho_v=0.0, rho_W=0.0, drive_g=g, seed=3)
    v, W = tr.next_block(4000)
    Jx = np.einsum("tib,tib->t", W[:, :, 0:3].astype(np.float64), v.astype(np.float64))
    target = kap / synth.WMK_PER_EV_PS_A_K * TK * V * Fe
    se = Jx.std() / np.sqrt(len(Jx))
    assert abs(Jx.mean() - target) < 5 * se


# ---------------------------------------------------------------- planted mistakes
MUTATIONS = {
    "W_transposed": ("we += (double)Wt[i * 9 + 3 * a + b] * e[3 * i + b];",
                     "we += (double)Wt[i * 9 + 3 * b + a] * e[3 * i + b];"),
    "mass_weight_dropped": ("x += sqm[i] * ev;", "x += ev;"),
    "inverse_mass_as_mass": ("y[a] += isqm[i] * we;", "y[a] += sqm[i] * we;"),
    "lag_on_total_current": ("s += Jb[(t * B + b) * 3 + mu] * J[(t - l) * 3 + nu];",
                             "s += Jb[((t - l) * B + b) * 3 + mu] * J[t * 3 + nu];"),
    "trapezoid_half_dropped": ("acc += 0.5 * (prev + C) * dt_ps;", "acc += (prev + C) * dt_ps;"),
    "last_bin_open": ("if (b >= B) b = B - 1;", "if (b >= B) b = -1;"),
    "shc_lag_on_velocity": ("s += (double)W[((t - l) * N + i) * 9 + 3 * a + b] *\n                             (double)v[(t * N + i) * 3 + b];",
                            "s += (double)W[(t * N + i) * 9 + 3 * a + b] *\n                             (double)v[((t - l) * N + i) * 3 + b];"),
    "dir_wrong_eigvec_component": ("y += (double)Wt[i * 9 + 3 * a + b] * e[3 * i + b] / sqrt(mass[i]);",
                                   "y += (double)Wt[i * 9 + 3 * a + b] * e[3 * i + a] / sqrt(mass[i]);"),
    "dir_bin_layout_swapped": ("jb[((int64_t)b * B + bn) * 3 + a] += jn[n * 9 + 3 * b + a];",
                               "jb[((int64_t)b * B + bn) * 3 + a] += jn[n * 9 + 3 * a + b];"),
    "xcorr_lag_on_second_bin": ("s += Jb[(t * B + b) * 3 + mu] * Jb[((t - l) * B + b2) * 3 + nu];",
                                "s += Jb[((t - l) * B + b) * 3 + mu] * Jb[(t * B + b2) * 3 + nu];"),
    "shc_trapezoid_dropped": ("const double trap = (l == 0 || l == nc - 1) ? 0.5 : 1.0;",
                              "const double trap = 1.0;"),
}


def _compile_mutant(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mhc_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", str(p), "-o",
                    str(so), "-lm"], check=True)
    return ctypes.CDLL(str(so))


def _pins_pass(L):
    """Run a subset of the pins above against library handle L; True if all pass."""
    real = oracle.lib()
    for fn in ("orc_bins_uniform", "orc_modal_current", "orc_gkma_corr", "orc_gk_kappa",
               "orc_hnema", "orc_kappa_window", "orc_orthonormality", "orc_shc_corr",
               "orc_shc_kappa", "orc_modal_current_dir", "orc_gkma_xcorr"):
        getattr(L, fn).argtypes = getattr(real, fn).argtypes
        getattr(L, fn).restype = getattr(real, fn).restype
    checks = [test_golden_one_atom_identity_basis, test_golden_two_atoms_mixed_basis,
              test_bins_edges_and_exclusions, test_parseval_and_inverse_transform,
              test_identity_basis_direction_decomposition,
              test_constant_input_correlation_closed_form,
              lambda: test_oracle_matches_scalar_brute_force(3, 7, 6, 4),
              lambda: test_shc_matches_scalar_brute_force(3, 7, 4),
              test_shc_spectrum_constant_input_closed_form,
              test_golden_direction_split_rotated_basis, test_golden_direction_split_two_atoms,
              test_xcorr_golden_two_atoms, test_xcorr_matches_fft_and_lag0_symmetry]
    oracle._lib = L
    try:
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        oracle._lib = real


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    oracle.lib()
    assert _pins_pass(oracle.lib()), "pins must pass on the unmodified oracle"
    assert not _pins_pass(_compile_mutant(tmp_path, name)), f"mutation {name} not detected"


# ---------------------------------------------------------------- SHC (Eq. 20-23)
def test_shc_lag_zero_is_total_heat_current():
    # Eq. 21 reduces to the heat current of Eq. 10 at t = 0 (Sec. II.C)
    N, T = 9, 12
    _, mass, v, W = tiny_system(N, T=T, seed=31)
    K, cnt = oracle.shc_corr(v, W, 5)
    J = np.einsum("tiab,tib->ta", W.astype(np.float64).reshape(T, N, 3, 3), v.astype(np.float64))
    np.testing.assert_allclose(K.reshape(3, 3, 5)[:, :, 0].sum(axis=1), J.sum(axis=0),
                               rtol=1e-12, atol=1e-11)
    assert cnt.tolist() == [12, 11, 10, 9, 8]


@pytest.mark.parametrize("N,T,nc", [(1, 4, 3), (3, 7, 4), (4, 9, 9)])
def test_shc_matches_scalar_brute_force(N, T, nc):
    _, mass, v, W = tiny_system(N, T=T, seed=40 + N)
    K, cnt = oracle.shc_corr(v, W, nc)
    ref = np.array(brute.shc(v, W, nc))
    np.testing.assert_allclose(K / np.maximum(cnt, 1), ref, rtol=1e-12, atol=1e-10)


def test_shc_correlation_matches_fft():
    # direct lag sums vs FFT cross-correlation per atom and tensor pair
    N, T, nc = 5, 64, 20
    _, mass, v, W = tiny_system(N, T=T, seed=33)
    K, _ = oracle.shc_corr(v, W, nc)
    Wd = W.astype(np.float64).reshape(T, N, 3, 3)
    vd = v.astype(np.float64)
    ref = np.zeros((3, 3, nc))
    nfft = 2 * T
    for a in range(3):
        for b in range(3):
            fv = np.fft.rfft(vd[:, :, b], nfft, axis=0)
            fw = np.fft.rfft(Wd[:, :, a, b], nfft, axis=0)
            ref[a, b] = np.fft.irfft(fv * np.conj(fw), nfft, axis=0)[:nc].sum(axis=1)
    np.testing.assert_allclose(K.reshape(3, 3, nc), ref, rtol=1e-9, atol=1e-8)


def test_shc_spectrum_constant_input_closed_form():
    # K(l) = K constant: the trapezoid cosine sum has the closed form
    #   sum_{l=0}^{m} c_l cos(l th) = sin(m th) cot(th/2) / 2  (c_0 = c_m = 1/2, else 1),
    # so Ktilde = dt K sin(m th) cot(th/2) with th = omega dt, and 2 m dt K at omega = 0.
    nc, dt, TK, V, Fe = 30, 0.002, 300.0, 1000.0, 1e-4
    m = nc - 1
    Kc = np.tile(np.linspace(-2.0, 3.0, 9)[:, None], (1, nc)) * 7.0
    cnt = np.full(nc, 7, dtype=np.int64)
    f = np.array([0.0, 1.3, 17.0, 101.0])
    kap = oracle.shc_kappa(Kc, cnt, dt, TK, V, Fe, f, window=0)
    sc = pytest.importorskip("scipy.constants")
    wmk = sc.e / (1e-12 * 1e-10)
    Kv = Kc[:, 0] / 7.0
    th = 2 * np.pi * f * dt
    with np.errstate(divide="ignore", invalid="ignore"):
        kt = np.where(th > 0, dt * np.sin(m * th) / np.tan(th / 2), 2 * m * dt)
    expect = 2 * np.outer(Kv, kt) / (V * TK * Fe) * wmk
    np.testing.assert_allclose(kap, expect, rtol=1e-9, atol=1e-9 * np.abs(expect).max())


def test_shc_spectrum_sum_rule():
    # integral of kappa(f) over [0, 1/(2 dt)] recovers K(0)/(V T F_e) (discrete Fourier
    # inversion of the even cosine series), for any K and either window
    nc, dt, TK, V, Fe = 40, 0.002, 300.0, 500.0, 2e-4
    rng = np.random.default_rng(5)
    Ks = rng.standard_normal((9, nc)) * 50.0
    cnt = np.full(nc, 1, dtype=np.int64)
    f = np.linspace(0.0, 1.0 / (2 * dt), 20001)
    sc = pytest.importorskip("scipy.constants")
    wmk = sc.e / (1e-12 * 1e-10)
    for window in (0, 1):
        kap = oracle.shc_kappa(Ks, cnt, dt, TK, V, Fe, f, window=window)
        total = np.trapezoid(kap, f, axis=1)
        np.testing.assert_allclose(total, Ks[:, 0] / (V * TK * Fe) * wmk, rtol=1e-6,
                                   atol=1e-9 * np.abs(Ks[:, 0]).max() / (V * TK * Fe) * wmk)
