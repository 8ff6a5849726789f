"""Seeded synthetic inputs for the modal heat-current path.

This module only *generates inputs*: eigenvector matrices, mode frequencies,
atomic masses and streams of per-atom velocities v_i(t) and per-atom virials
W_i(t).  It holds none of the method's arithmetic (no projection, no product,
no binning, no correlation), so the CUDA path and the CPU oracle can both be
fed from it without sharing any computation.

Stand-ins for the paper's workloads (Sec. III.A: CNT (10,10), graphene and
natural Si at 300 K; Sec. III.C.ii: Si-8000 performance test):

* E: the real Gamma-point eigenvector matrix, dof-major E[3i+b, n] = e^b_{i,n}
  (Eq. 13, 14).  Lattice dynamics needs a potential and a relaxed structure,
  neither of which exists here, so E is the Q factor of a seeded Gaussian
  matrix (Haar-distributed orthonormal columns); columns are sign-fixed by
  sign(R_nn).  A mode subset (M < 3N) is the thin QR of a 3N x M Gaussian.
* frequencies: i.i.d. uniform draws on the stated THz range.
* v_i(t): Maxwell-Boltzmann components at temperature T,
  sigma_v^2 = k_B T / m_i (converted to A^2/ps^2), with AR(1) time
  correlation rho so that the heat-current autocorrelation decays over a few
  samples as in a real MD trajectory.
* W_i(t): nine independent N(0, sigma_W^2) components (eV), AR(1) in time,
  full non-symmetric 3x3 (Sec. II.A: the per-atom virial of Eq. 8 is not
  symmetric).
* drive: optional stand-in for the HNEMD driving force (Eq. 12).  A small
  coupling g adds g * v_i^b to W_i^{xb}, which gives the x heat current a
  positive mean <J^x> = g * sum_i <|v_i|^2>, as a driven system would have.
  g is chosen from a target kappa via <J^x> = kappa T V F_e (Eq. 19 summed
  over modes).

Units: v in A/ps, W in eV, m in amu, J in eV*A/ps, V in A^3, T in K.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KB_EV_PER_K = 8.617333262145179e-5    # Boltzmann constant, eV/K (SI exact ratio)
A2_PS2_PER_EV_AMU = 9648.533212331     # 1 eV/amu expressed in A^2/ps^2
WMK_PER_EV_PS_A_K = 1602.176634        # 1 eV/(ps*A*K) in W/(m*K)

SI_ISOTOPES = ((27.9769265, 0.922), (28.9764947, 0.047), (29.9737702, 0.031))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def eigvecs(D: int, M: int, seed: int) -> np.ndarray:
    """Seeded real orthonormal D x M matrix (dof-major), float64.

    Q of the (thin when M < D) QR of a standard Gaussian D x M matrix, with
    column n multiplied by sign(R_nn) so the draw is Haar-distributed and
    reproducible.
    """
    if M > D:
        raise ValueError("M modes cannot exceed 3N degrees of freedom")
    G = _rng(seed).standard_normal((D, M))
    Q, R = np.linalg.qr(G, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return np.ascontiguousarray(Q * s[None, :])


def eigvecs_device(D: int, M: int, seed: int, device="cuda"):
    """The recipe of eigvecs() computed with torch on a GPU (float32 QR), for bases
    too large to factorise on the host in reasonable time.  Returns a float32
    [D][M] CUDA tensor with orthonormal columns (to float32 rounding)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn(D, M, generator=g, device=device, dtype=torch.float32)
    Q, R = torch.linalg.qr(G, mode="reduced")
    del G
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    del R
    return (Q * s[None, :]).contiguous()


def force_constants(dims: tuple, seed: int, k_long=(6.0, 12.0), k_trans=(0.5, 2.0)) -> np.ndarray:
    """Seeded harmonic force constants Phi [3N][3N] (eV/A^2) of a periodic simple-cubic
    spring network with dims = (n1, n2, n3) cells of one atom (N = n1 n2 n3), the stand-in for
    the lattice dynamics of a relaxed structure (Sec. II.B; no potential exists here).  Each
    nearest-neighbour bond i-j along unit vector u gets a seeded stiffness tensor
    K = k_L u u^T + k_T (I - u u^T) (k_L, k_T uniform on the given ranges), and
    Phi_ij = -K (i != j), Phi_ii = sum_j K: symmetric, positive semi-definite, with the three
    uniform translations as its zero modes (acoustic sum rule)."""
    n1, n2, n3 = dims
    N = n1 * n2 * n3
    rng = _rng(seed + 6700417)
    Phi = np.zeros((3 * N, 3 * N))

    def idx(a, b, c):
        return ((a % n1) * n2 + (b % n2)) * n3 + (c % n3)
    for a in range(n1):
        for b in range(n2):
            for c in range(n3):
                i = idx(a, b, c)
                for ax, j in ((0, idx(a + 1, b, c)), (1, idx(a, b + 1, c)), (2, idx(a, b, c + 1))):
                    kl = rng.uniform(*k_long)
                    kt = rng.uniform(*k_trans)
                    if j == i:
                        continue
                    u = np.zeros(3)
                    u[ax] = 1.0
                    K = kl * np.outer(u, u) + kt * (np.eye(3) - np.outer(u, u))
                    Phi[3 * i:3 * i + 3, 3 * j:3 * j + 3] -= K
                    Phi[3 * j:3 * j + 3, 3 * i:3 * i + 3] -= K
                    Phi[3 * i:3 * i + 3, 3 * i:3 * i + 3] += K
                    Phi[3 * j:3 * j + 3, 3 * j:3 * j + 3] += K
    return Phi


def frequencies(M: int, f_lo: float, f_hi: float, seed: int) -> np.ndarray:
    """i.i.d. uniform mode frequencies on [f_lo, f_hi) THz, float64."""
    return _rng(seed + 7919).uniform(f_lo, f_hi, size=M)


def masses(N: int, m: float | None = None, seed: int = 0,
           isotopes: tuple = ()) -> np.ndarray:
    """Per-atom masses (amu).  Either one mass for all atoms or a seeded draw
    from an isotope table of (mass, abundance) pairs (natural Si: Sec. III.A.iii).
    """
    if isotopes:
        ms = np.array([a for a, _ in isotopes])
        p = np.array([b for _, b in isotopes])
        idx = _rng(seed + 104729).choice(len(ms), size=N, p=p / p.sum())
        return ms[idx].astype(np.float64)
    return np.full(N, float(m), dtype=np.float64)


def sigma_v(mass: np.ndarray, T_K: float) -> np.ndarray:
    """Maxwell-Boltzmann standard deviation of one velocity component, A/ps."""
    return np.sqrt(KB_EV_PER_K * T_K / mass * A2_PS2_PER_EV_AMU)


def drive_coupling(kappa_wmk: float, T_K: float, V_A3: float, Fe: float,
                   mass: np.ndarray) -> float:
    """Coupling g (eV*ps/A) that makes <J^x> = kappa T V F_e for the drive option."""
    target = kappa_wmk / WMK_PER_EV_PS_A_K * T_K * V_A3 * Fe   # eV*A/ps
    mean_v2 = float(np.sum(3.0 * sigma_v(mass, T_K) ** 2))
    return target / mean_v2


@dataclass
class Trajectory:
    """Seeded stream of (v, W) blocks with AR(1) time correlation.

    next_block(K) returns v [K][N][3] and W [K][N][9] (row-major alpha,beta)
    as float32 -- the precision an MD engine hands to the analysis.
    """
    mass: np.ndarray
    T_K: float = 300.0
    sigma_W: float = 1.0
    rho_v: float = 0.9
    rho_W: float = 0.9
    drive_g: float = 0.0
    seed: int = 0
    _rng: np.random.Generator = field(init=False, repr=False)
    _v: np.ndarray = field(init=False, repr=False)
    _w: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self.mass = np.asarray(self.mass, dtype=np.float64)
        self._rng = _rng(self.seed + 15485863)
        N = self.mass.shape[0]
        self._sv = sigma_v(self.mass, self.T_K)[:, None]
        self._v = self._rng.standard_normal((N, 3)) * self._sv
        self._w = self._rng.standard_normal((N, 9)) * self.sigma_W

    @property
    def N(self) -> int:
        return self.mass.shape[0]

    def next_block(self, K: int):
        N = self.N
        v = np.empty((K, N, 3), dtype=np.float32)
        W = np.empty((K, N, 9), dtype=np.float32)
        cv = math.sqrt(max(0.0, 1.0 - self.rho_v ** 2))
        cw = math.sqrt(max(0.0, 1.0 - self.rho_W ** 2))
        for k in range(K):
            v[k] = self._v
            w = self._w.copy()
            if self.drive_g != 0.0:
                w[:, 0:3] += self.drive_g * self._v
            W[k] = w
            self._v = self.rho_v * self._v + cv * self._sv * self._rng.standard_normal((N, 3))
            self._w = self.rho_W * self._w + cw * self.sigma_W * self._rng.standard_normal((N, 9))
        return v, W


# Workload shapes (stand-ins for the paper's systems; Sec. III.A and III.C).
# Si volume 20.02 A^3/atom; graphene / CNT wall 2.619 A^2 x 3.35 A = 8.77 A^3/atom.
WORKLOADS = {
    # K is autotuned here (the block length is not fixed by the workload): candidates that
    # divide the 1000-step run
    "gkma_si_n512": dict(N=512, M=1536, mass=28.085, f=(0.0, 16.0), B=100,
                         T_s=1000, K=250, L=200, dt_ps=0.010, V_per_atom=20.02,
                         T_K=300.0, Fe=(1e-5, 0.0, 0.0), gkma=True, seed=20210205,
                         K_candidates=(125, 250, 500, 1000)),
    "hnema_graphene_n4096": dict(N=4096, M=12288, mass=12.011, f=(0.0, 50.0), B=200,
                                 T_s=20000, K=128, L=0, dt_ps=0.008, V_per_atom=8.77,
                                 T_K=300.0, Fe=(1e-5, 0.0, 0.0), gkma=False,
                                 kappa_drive=3000.0, seed=20210206),
    "gkma_si_n8000": dict(N=8000, M=24000, mass=28.085, f=(0.0, 16.0), B=64,
                          T_s=10000, K=256, L=500, dt_ps=0.010, V_per_atom=20.02,
                          T_K=300.0, Fe=(1e-5, 0.0, 0.0), gkma=True, seed=20210207),
    "subset_si_n20000_m6000": dict(N=20000, M=6000, mass=28.085, f=(0.0, 16.0), B=64,
                                   T_s=50000, K=512, L=1000, dt_ps=0.010, V_per_atom=20.02,
                                   T_K=300.0, Fe=(1e-5, 0.0, 0.0), gkma=True, seed=20210209),
    # small case of the Si shape for profiler captures (E hi+lo 578 MB, 752 tiles)
    "profile_si_n4000_m12000": dict(N=4000, M=12000, mass=28.085, f=(0.0, 16.0), B=64,
                                    T_s=4096, K=512, L=500, dt_ps=0.010, V_per_atom=20.02,
                                    T_K=300.0, Fe=(1e-5, 0.0, 0.0), gkma=True, seed=20210210),
}


def cnt_group_sizes(n_systems: int = 16, seed: int = 20210208) -> list[int]:
    """Atom counts of the uneven CNT (10,10) batch: 40 atoms per unit cell times
    a seeded number of cells in [12, 100], i.e. N in [480, 4000]."""
    u = _rng(seed).integers(12, 101, size=n_systems)
    return [int(40 * x) for x in u]
