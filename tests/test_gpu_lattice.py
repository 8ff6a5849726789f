"""Gamma-point lattice dynamics on the GPU (mhc_lattice_modes, Sec. II.B) against the FP64
oracle (cyclic Jacobi), and the basis it produces fed straight into mhc_set_modes.

Eigenvalues are unique and compared element by element; eigenvectors are unique only up to
sign (fixed by a convention that ties can flip) and, inside a degenerate eigenspace, up to a
rotation, so they are compared through the projector onto each cluster of equal eigenvalues.
At the 512-atom size the oracle is too slow for a test: there the GPU result is checked by its
residual, orthonormality, the library eigenvalues and the acoustic sum rule."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, ModalRef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dyn(Phi, mass):
    sq = np.repeat(np.sqrt(mass), 3)
    return Phi / np.outer(sq, sq)


def clusters(w2, rel_gap=1e-8):
    """Index groups of (numerically) equal eigenvalues."""
    scale = max(np.abs(w2).max(), 1e-300)
    groups, cur = [], [0]
    for n in range(1, len(w2)):
        if w2[n] - w2[n - 1] <= rel_gap * scale:
            cur.append(n)
        else:
            groups.append(cur)
            cur = [n]
    groups.append(cur)
    return groups


def compare_modes(w2g, fg, Eg, w2o, fo, Eo, tol_w=1e-12, tol_e=1e-9):
    scale = np.abs(w2o).max()
    np.testing.assert_allclose(w2g, w2o, rtol=0, atol=tol_w * scale)
    np.testing.assert_allclose(fg, fo, rtol=1e-10, atol=1e-4)   # zero modes: noise
    for g in clusters(w2o):
        Pg = Eg[:, g] @ Eg[:, g].T
        Po = Eo[:, g] @ Eo[:, g].T
        assert np.abs(Pg - Po).max() <= tol_e, (g, np.abs(Pg - Po).max())


@pytest.mark.parametrize("case", ["lattice_4x4x4", "lattice_6x6x6", "random_40", "odd_5x5x1"])
def test_lattice_modes_match_the_oracle(case):
    need_gpu()
    from paper_2102_03691_gb300.mhc import lattice_modes
    if case.startswith("random"):
        rng = np.random.default_rng(1301)
        N = 40
        A = rng.standard_normal((3 * N, 3 * N))
        Phi = A + A.T
        mass = rng.uniform(1.0, 60.0, N)
    else:
        dims = {"lattice_4x4x4": (4, 4, 4), "lattice_6x6x6": (6, 6, 6), "odd_5x5x1": (5, 5, 1)}[case]
        N = dims[0] * dims[1] * dims[2]      # 5x5x1: 25 atoms, 3N = 75 is odd
        Phi = synth.force_constants(dims, 1302)
        mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=1302)
    w2o, fo, Eo, so = oracle.lattice_modes(Phi, mass)
    assert so >= 0
    for where in ("host", "device"):
        P = Phi if where == "host" else torch.from_numpy(Phi).cuda()
        E_out = None if where == "host" else torch.empty((3 * N, 3 * N), dtype=torch.float64,
                                                         device="cuda")
        w2g, fg, Eg, sg = lattice_modes(P, mass, E_out=E_out)
        Eg = Eg if where == "host" else Eg.cpu().numpy()
        assert sg > 0
        compare_modes(w2g, fg, Eg, w2o, fo, Eo)
        Dm = dyn(Phi, mass)
        assert np.abs(Dm @ Eg - Eg * w2g).max() <= 1e-11 * np.abs(w2o).max()
        assert np.abs(Eg.T @ Eg - np.eye(3 * N)).max() <= 1e-12
        big = np.abs(Eg).argmax(axis=0)
        assert np.all(Eg[big, np.arange(3 * N)] > 0)


def test_lattice_modes_512_atoms_full_size():
    # the N = 512 Si-like workload's basis from an 8 x 8 x 8 spring lattice: 1536 modes
    need_gpu()
    from paper_2102_03691_gb300.mhc import lattice_modes
    N = 512
    Phi = synth.force_constants((8, 8, 8), 1303)
    mass = synth.masses(N, 28.085)
    w2g, fg, Eg, sg = lattice_modes(Phi, mass)
    print(f"512 atoms: {sg} sweeps, f in [{fg[3]:.3f}, {fg[-1]:.3f}] THz")
    Dm = dyn(Phi, mass)
    scale = np.abs(w2g).max()
    np.testing.assert_allclose(w2g, np.linalg.eigvalsh(Dm), rtol=0, atol=1e-11 * scale)
    assert np.abs(Dm @ Eg - Eg * w2g).max() <= 1e-11 * scale
    assert np.abs(Eg.T @ Eg - np.eye(3 * N)).max() <= 1e-12
    assert np.all(np.abs(w2g[:3]) <= 1e-12 * scale) and w2g[3] > 1e-6 * scale   # sum rule


def test_force_constants_to_binned_currents_on_the_gpu():
    # Phi -> lattice modes (GPU) -> mhc_set_modes from device memory -> pushes (FP16x3); the
    # binned currents against the oracle run on the oracle's own lattice modes (binned
    # currents depend only on each bin's eigenspace, so the comparison is basis-independent)
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    dims, K, B = (4, 4, 4), 32, 6
    N = 64
    Phi = synth.force_constants(dims, 1304)
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=1304)
    v, W = synth.Trajectory(mass, seed=1304).next_block(2 * K)
    h = ModalHeatCurrent(precision="fp16x3", k_max=K, n_lags=4)
    fg = h.set_modes_from_force_constants(Phi, mass)
    w2o, fo, Eo, _ = oracle.lattice_modes(Phi, mass)
    f_lo, f_hi = -0.5, float(fo.max()) + 0.5
    h.set_bins_uniform(f_lo, f_hi, B)
    Jb = []
    for t0 in (0, K):
        h.push(torch.from_numpy(v[t0:t0 + K]).cuda(), torch.from_numpy(W[t0:t0 + K]).cuda())
        Jb.append(h.read_binned_current().copy())
    bins = oracle.bins_uniform(fo, f_lo, f_hi, B)
    assert np.array_equal(bins, oracle.bins_uniform(fg, f_lo, f_hi, B))
    ref = ModalRef(Eo, mass, v, W, bins, B)
    ref.check_current(np.concatenate(Jb), REL_TOL, "lattice basis, binned currents")
    C, _ = h.read_corr()
    ref.check_corr(C, 4, REL_TOL, "lattice basis, Eq. 17 sums")
    h.close()
