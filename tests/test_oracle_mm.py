"""Pins of oracle.modal_current_mm (Eqs. 13 and 16 as FP64 matrix products, for full-size
systems) and of the conditioned parity metric built on it (tests/parity.py).  CPU only.

modal_current_mm is held to the plain loops of mhc_oracle.c (themselves pinned by hand
examples, brute force and invariants in test_oracle_pins.py) and to the invariants the
method fixes; the metric is held to closed forms of its scales and to planted errors."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import MIN_MODES, ModalRef, check


def case(N, M, T, B, seed, f_cut=16.0):
    E = synth.eigvecs(3 * N, M, seed)
    f = synth.frequencies(M, 0.0, 16.0, seed)
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed)
    v, W = synth.Trajectory(mass, drive_g=1e-3, seed=seed).next_block(T)
    bins = oracle.bins_uniform(f, 0.0, f_cut, B)
    return E, mass, v, W, bins


@pytest.mark.parametrize("N,M,T,B,cut,chunk", [(7, 21, 5, 3, 16.0, 2), (30, 70, 9, 6, 12.0, 4),
                                               (40, 120, 3, 1, 16.0, 256)])
def test_mm_equals_the_loops(N, M, T, B, cut, chunk):
    E, mass, v, W, bins = case(N, M, T, B, 31 + N, cut)
    a = oracle.modal_current(E, mass, v, W, bins, B, want_modes=True)
    b = oracle.modal_current_mm(E, mass, v, W, bins, B, parts=True, steps_per_product=chunk)
    scale = np.abs(a["Jn"]).max()
    np.testing.assert_allclose(b["Jb"], a["Jb"], rtol=0, atol=1e-12 * scale * M)
    np.testing.assert_allclose(b["J"], a["J"], rtol=1e-13, atol=1e-12 * np.abs(a["J"]).max())
    np.testing.assert_allclose(b["xdot"], a["xdot"], rtol=0, atol=1e-12 * np.abs(a["xdot"]).max())
    np.testing.assert_allclose(b["xdot"][:, :, None] * b["y"], a["Jn"], rtol=0, atol=1e-12 * scale)


def test_mm_direction_equals_the_loops():
    E, mass, v, W, bins = case(25, 60, 6, 4, 77, 13.0)
    a = oracle.modal_current_dir(E, mass, v, W, bins, 4, want_modes=True)
    b = oracle.modal_current_mm(E, mass, v, W, bins, 4, parts=True, direction=True)
    scale = np.abs(a["Jnd"]).max()
    np.testing.assert_allclose(b["Jb"], a["Jbd"], rtol=0, atol=1e-12 * scale * 60)
    np.testing.assert_allclose(b["xdot"][:, :, None, None] * b["y"], a["Jnd"], rtol=0,
                               atol=1e-12 * scale)
    np.testing.assert_allclose(b["J"], a["Jd"].sum(axis=1), rtol=1e-13,
                               atol=1e-12 * np.abs(b["J"]).max())


def test_mm_completeness_and_parseval():
    # every mode of a square orthonormal basis kept: sum_b J_b = J (Eq. 15) and
    # sum_n Xdot_n^2 = sum_i m_i |v_i|^2 (Eqs. 13-14)
    N = 20
    E, mass, v, W, _ = case(N, 3 * N, 4, 5, 91)
    bins = (np.arange(3 * N) % 5).astype(np.int32)
    r = oracle.modal_current_mm(E, mass, v, W, bins, 5, parts=True)
    np.testing.assert_allclose(r["Jb"].sum(axis=1), r["J"], rtol=1e-11, atol=1e-11)
    ke = (mass[None, :, None] * v.astype(np.float64) ** 2).sum(axis=(1, 2))
    np.testing.assert_allclose((r["xdot"] ** 2).sum(axis=1), ke, rtol=1e-12)


def test_mm_of_absolute_values_is_the_sum_of_absolute_terms():
    # on |E|, |v|, |W| the projections are the sums of the absolute values of their terms
    N, M = 6, 10
    E, mass, v, W, bins = case(N, M, 2, 2, 5)
    a = oracle.modal_current_mm(np.abs(E), mass, np.abs(v), np.abs(W), bins, 2, parts=True)
    sqm = np.sqrt(mass)
    for t in range(2):
        for n in range(M):
            A = sum(abs(sqm[i] * E[3 * i + b, n] * float(v[t, i, b]))
                    for i in range(N) for b in range(3))
            assert abs(a["xdot"][t, n] - A) <= 1e-12 * A
            for al in range(3):
                Bs = sum(abs(float(W[t, i, 3 * al + b]) * E[3 * i + b, n] / sqm[i])
                         for i in range(N) for b in range(3))
                assert abs(a["y"][t, n, al] - Bs) <= 1e-12 * Bs


def test_identity_basis_dot_scale_is_twice_the_mode_current():
    # E = I: Xdot_{3i+b} = sqrt(m_i) v_i^b and y^a = W_i^{ab} / sqrt(m_i) are single terms,
    # so the first-order condition A|y| + |x|B of a one-mode bin is exactly 2 |J_n|
    N = 5
    D = 3 * N
    mass = synth.masses(N, 28.085)
    v, W = synth.Trajectory(mass, seed=3).next_block(3)
    ids = np.arange(D, dtype=np.int32)
    ref = ModalRef(np.eye(D), mass, v, W, ids, D)
    assert np.all(ref.small)
    np.testing.assert_allclose(ref.S, 2 * np.abs(ref.Jb), rtol=1e-14)


def test_bin_scale_is_the_sum_of_mode_magnitudes():
    E, mass, v, W, bins = case(30, 90, 4, 3, 17)
    ref = ModalRef(E, mass, v, W, bins, 3)
    assert np.all(np.bincount(bins[bins >= 0]) >= MIN_MODES)
    Jn = oracle.modal_current(E, mass, v, W, bins, 3, want_modes=True)["Jn"]
    for b in range(3):
        np.testing.assert_allclose(ref.S[:, b], np.abs(Jn[:, bins == b]).sum(axis=1), rtol=1e-14)
    # the Eq. 17 scale is the correlation of S with |J|, which bounds |C| term by term
    C, cnt, SC = ref.corr(4)
    assert np.all(np.abs(C) <= SC * (1 + 1e-12))


def test_check_catches_planted_errors():
    o = np.array([[1.0, -2.0, 0.0], [0.5, 0.05, 0.0]])
    S = np.array([[4.0, 4.0, 0.0], [4.0, 4.0, 0.0]])
    live = S > 0
    check(o + 3e-6 * live, o, S)                        # 7.5e-7 of S, at most 6e-6 of |o|
    g = o.copy()
    g[1, 1] += 3.9e-5                                   # 9.75e-6 of S; |o| < 0.1 S: no
    check(g, o, S)                                      # pointwise check, 7.8e-4 of |o| is fine
    g = o.copy()
    g[1, 1] += 5e-5                                     # 1.25e-5 of S
    with pytest.raises(AssertionError):
        check(g, o, S)
    g = o.copy()
    g[0, 2] = 1e-300                                    # an empty bin must stay exactly zero
    with pytest.raises(AssertionError):
        check(g, o, S)
    g = o.copy()
    g[0, 1] += 3.9e-5                                   # 9.75e-6 of S but 1.95e-5 of |o|,
    with pytest.raises(AssertionError):                 # and |o| >= 0.1 S (condition <= 10)
        check(g, o, S)
    check(g, o, S, pointwise=False)                     # without the pointwise check: passes
    check(g, o, S, S_wc=10 * S)                         # condition number 20: passes
