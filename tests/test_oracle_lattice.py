"""Pins of the lattice-dynamics oracle (oracle.lattice_modes: Gamma-point eigenmodes of the
mass-weighted force constants, Sec. II.B), CPU only: a hand-solved one-atom case, the closed
form of two atoms joined by a spring, the library eigenvalues of random symmetric matrices,
residual and orthonormality, the acoustic sum rule of a spring lattice, and planted mistakes."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth

A2_PS2_PER_EV_AMU = 9648.533212331
TWO_PI = 2.0 * np.pi


def freq_of(w2):
    return np.sign(w2) * np.sqrt(np.abs(w2) * A2_PS2_PER_EV_AMU) / TWO_PI


def projector(E, cols):
    Q = E[:, cols]
    return Q @ Q.T


def test_one_atom_hand_solved():
    # Dyn = Phi / m with Phi = [[2, 1, 0], [1, 2, 0], [0, 0, 3]], m = 2: eigenvalues 1/2, 3/2, 3/2;
    # e_0 = (1, -1, 0)/sqrt(2) (sign: first largest component positive), and the eigenspace of
    # 3/2 is span{(1, 1, 0)/sqrt(2), (0, 0, 1)}
    Phi = np.array([[2.0, 1.0, 0.0], [1.0, 2.0, 0.0], [0.0, 0.0, 3.0]])
    w2, f, E, sweeps = oracle.lattice_modes(Phi, np.array([2.0]))
    assert sweeps >= 0
    np.testing.assert_allclose(w2, [0.5, 1.5, 1.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(f, freq_of(np.array([0.5, 1.5, 1.5])), rtol=1e-15)
    np.testing.assert_allclose(E[:, 0], np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0), atol=1e-15)
    P = np.outer([1, 1, 0], [1, 1, 0]) / 2.0 + np.outer([0, 0, 1], [0, 0, 1])
    np.testing.assert_allclose(projector(E, [1, 2]), P, atol=1e-15)


@pytest.mark.parametrize("m1,m2,k", [(28.0, 28.0, 10.0), (12.011, 28.085, 4.5)])
def test_two_atoms_joined_by_a_spring(m1, m2, k):
    # Phi = [[k I, -k I], [-k I, k I]]: w^2 = 0 (three translations, eigenvectors proportional
    # to (sqrt(m1) u, sqrt(m2) u)) and w^2 = k (1/m1 + 1/m2) (three, (sqrt(m2) u, -sqrt(m1) u))
    Phi = np.block([[k * np.eye(3), -k * np.eye(3)], [-k * np.eye(3), k * np.eye(3)]])
    w2, f, E, _ = oracle.lattice_modes(Phi, np.array([m1, m2]))
    wopt = k * (1.0 / m1 + 1.0 / m2)
    np.testing.assert_allclose(w2[:3], 0.0, atol=1e-14 * wopt)
    np.testing.assert_allclose(w2[3:], wopt, rtol=1e-14)
    np.testing.assert_allclose(f[3:], freq_of(np.array([wopt] * 3)), rtol=1e-14)
    a = np.array([np.sqrt(m1), np.sqrt(m2)]) / np.sqrt(m1 + m2)
    b = np.array([np.sqrt(m2), -np.sqrt(m1)]) / np.sqrt(m1 + m2)
    np.testing.assert_allclose(projector(E, [0, 1, 2]), np.kron(np.outer(a, a), np.eye(3)), atol=1e-14)
    np.testing.assert_allclose(projector(E, [3, 4, 5]), np.kron(np.outer(b, b), np.eye(3)), atol=1e-14)


@pytest.mark.parametrize("N,seed", [(5, 1), (17, 2), (40, 3)])
def test_random_symmetric_against_library_eigenvalues(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3 * N, 3 * N))
    Phi = A + A.T
    mass = rng.uniform(1.0, 60.0, N)
    w2, f, E, sweeps = oracle.lattice_modes(Phi, mass)
    assert 0 <= sweeps <= 20
    sq = np.repeat(np.sqrt(mass), 3)
    Dyn = Phi / np.outer(sq, sq)
    nrm = np.abs(Dyn).max()
    np.testing.assert_allclose(w2, np.linalg.eigvalsh(Dyn), rtol=0, atol=1e-12 * nrm)
    assert np.abs(Dyn @ E - E * w2).max() <= 1e-12 * nrm                # residual
    assert np.abs(E.T @ E - np.eye(3 * N)).max() <= 1e-13               # orthonormality
    big = np.abs(E).argmax(axis=0)                                      # sign convention
    assert np.all(E[big, np.arange(3 * N)] > 0)
    np.testing.assert_allclose(f, freq_of(w2), rtol=1e-15)


def test_spring_lattice_acoustic_sum_rule():
    # a periodic spring network: exactly three zero modes, spanned by the mass-weighted uniform
    # translations sqrt(m_i) u; all other w^2 positive
    dims = (3, 3, 2)
    N = 18
    Phi = synth.force_constants(dims, 7)
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=7)
    w2, f, E, _ = oracle.lattice_modes(Phi, mass)
    scale = w2.max()
    assert np.all(np.abs(w2[:3]) <= 1e-13 * scale) and np.all(w2[3:] > 1e-6 * scale)
    T = np.zeros((3 * N, 3))
    for a in range(3):
        T[a::3, a] = np.sqrt(mass)
    T /= np.linalg.norm(T, axis=0)
    np.testing.assert_allclose(projector(E, [0, 1, 2]), T @ T.T, atol=1e-12)


# ---------------------------------------------------------------- planted mistakes
MUTATIONS = {
    "mass_weight_without_sqrt": ("A[r * D + c] = Phi[r * D + c] / sqrt(mass[r / 3] * mass[c / 3]);",
                                 "A[r * D + c] = Phi[r * D + c] / (mass[r / 3] * mass[c / 3]);"),
    "rotation_sign_flipped": ("A[k * D + p] = c * akp - s * akq;", "A[k * D + p] = c * akp + s * akq;"),
    "eigvec_rows_instead_of_columns": ("const double vkp = V[k * D + p], vkq = V[k * D + q];",
                                       "const double vkp = V[p * D + k], vkq = V[q * D + k];"),
    "frequency_without_unit": ("const double w = sqrt(fabs(lam) * 9648.533212331);",
                               "const double w = sqrt(fabs(lam));"),
}


def _mutant(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "mhc_oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-ffp-contract=off", str(p), "-o", str(so),
                    "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    L.orc_lattice_modes.argtypes = oracle.lib().orc_lattice_modes.argtypes
    L.orc_lattice_modes.restype = oracle.lib().orc_lattice_modes.restype
    return L


def _pins_pass(L):
    real = oracle.lib()
    oracle._lib = L
    try:
        for c in (test_one_atom_hand_solved, lambda: test_two_atoms_joined_by_a_spring(12.011, 28.085, 4.5),
                  lambda: test_random_symmetric_against_library_eigenvalues(5, 1)):
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
    assert _pins_pass(oracle.lib())
    assert not _pins_pass(_mutant(tmp_path, name)), f"mutation {name} not detected"
