"""FP64 CPU oracle for the modal heat current -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  The CUDA library never calls it and shares no code
with it.  ``mhc_oracle.c`` holds the plain FP64 loops (Eqs. 10, 13, 16, 17,
19 and frequency binning; the direction split of Sec. II.A; bin-bin cross-correlations; the SHC correlation and spectrum of Eqs. 20-23);
``brute.py`` restates the same definitions with per-atom 3-vectors in scalar
Python for tiny systems.  ``modal_current_mm`` below writes the projections of Eqs. 13
and 16 as FP64 matrix products for full-size systems.  ``lattice_modes`` is the Gamma-point
lattice-dynamics eigen-solve (cyclic Jacobi) that produces eigenvectors and frequencies
from force constants (Sec. II.B).

This module compiles ``mhc_oracle.c`` with gcc on first use (or through
``build()``) and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile mhc_oracle.c into oracle/liboracle.so (gcc, OpenMP, no fast-math,
    no FMA contraction so x86 and Arm give identical results)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_bins_uniform.argtypes = [_i64, _p, _dbl, _dbl, _i32, _p]
            L.orc_modal_current.argtypes = [_i64, _i64, _p, _p, _i64, _p, _p, _p, _i32,
                                            _p, _p, _p, _p]
            L.orc_modal_current_dir.argtypes = [_i64, _i64, _p, _p, _i64, _p, _p, _p, _i32,
                                                _p, _p, _p]
            L.orc_gkma_corr.argtypes = [_i64, _i32, _p, _p, _i32, _p, _p]
            L.orc_gkma_xcorr.argtypes = [_i64, _i32, _p, _i32, _p]
            L.orc_gk_kappa.argtypes = [_i32, _i32, _p, _p, _dbl, _dbl, _dbl, _p]
            L.orc_kappa_window.argtypes = [_i32, _i32, _p, _dbl, _dbl, _dbl, _p]
            L.orc_kappa_window.restype = _i32
            L.orc_hnema.argtypes = [_i64, _i32, _p, _dbl, _dbl, _p, _p, _p]
            L.orc_shc_corr.argtypes = [_i64, _i64, _p, _p, _i32, _p, _p]
            L.orc_shc_kappa.argtypes = [_i32, _p, _p, _dbl, _dbl, _dbl, _dbl, _i32, _i32, _p, _p]
            L.orc_orthonormality.argtypes = [_i64, _i64, _p]
            L.orc_orthonormality.restype = _dbl
            L.orc_lattice_modes.argtypes = [_i64, _p, _p, _i32, _dbl, _p, _p, _p]
            L.orc_lattice_modes.restype = _i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def bins_uniform(f_THz, f_min: float, f_max: float, B: int) -> np.ndarray:
    f = np.ascontiguousarray(f_THz, dtype=np.float64)
    out = np.empty(f.shape[0], dtype=np.int32)
    lib().orc_bins_uniform(f.shape[0], _ptr(f), f_min, f_max, B, _ptr(out))
    return out


def modal_current(E: np.ndarray, mass, v, W, bin_of_mode, B: int,
                  want_modes: bool = False):
    """E: dof-major [3N][M] float64 (E[3i+b, n] = e^b_{i,n}); v [T][N][3] and
    W [T][N][9] float32.  Returns dict with Jb [T][B][3], J [T][3] and, when
    want_modes, xdot [T][M] and Jn [T][M][3]."""
    E = np.asarray(E, dtype=np.float64)
    D, M = E.shape
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    N = mass.shape[0]
    if D != 3 * N:
        raise ValueError("E must have 3N rows")
    Et = np.ascontiguousarray(E.T)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, N, 3)
    W = np.ascontiguousarray(W, dtype=np.float32).reshape(-1, N, 9)
    T = v.shape[0]
    bins = np.ascontiguousarray(bin_of_mode, dtype=np.int32)
    Jb = np.empty((T, B, 3))
    J = np.empty((T, 3))
    xd = np.empty((T, M)) if want_modes else None
    Jn = np.empty((T, M, 3)) if want_modes else None
    lib().orc_modal_current(N, M, _ptr(Et), _ptr(mass), T, _ptr(v), _ptr(W), _ptr(bins),
                            B, _ptr(Jb), _ptr(J), _ptr(xd), _ptr(Jn))
    out = {"Jb": Jb, "J": J}
    if want_modes:
        out["xdot"] = xd
        out["Jn"] = Jn
    return out


def modal_current_mm(E: np.ndarray, mass, v, W, bin_of_mode, B: int, parts: bool = False,
                     direction: bool = False, steps_per_product: int = 256):
    """The outputs of modal_current (Eqs. 10, 13, 16 and the frequency binning) for systems
    too large for the loops of mhc_oracle.c, with each group of steps' projections written as
    FP64 matrix products (numpy's matmul serves as the projection step; nothing is blocked,
    fused or reordered beyond the definitions):

      Eq. 13       X[t][n]    = sum_d (sqrt(m_i) v_i^b(t))[d] E[d, n]          (d = 3i + b)
      Eq. 16       Y^a[t][n]  = sum_d (W_i^{ab}(t) / sqrt(m_i))[d] E[d, n]
                   J_n^a(t)   = X[t][n] Y^a[t][n]
      binning      J_b^a(t)   = sum_{n: bin(n) = b} J_n^a(t)   (product with a 0/1 indicator)
      Eq. 10       J^a(t)     = sum_i sum_b W_i^{ab}(t) v_i^b(t)

    With direction=True the bracket keeps the direction b of the motion (Sec. II.A split):
    Y^{ab}[t][n] = sum_i W_i^{ab}(t) e^b_{i,n} / sqrt(m_i) and J_n^{ab} = X Y^{ab}; the binned
    output is then [T][3 (b)][B][3 (a)] as for modal_current_dir.

    E is dof-major [3N][M] (float64); v [T][N][3], W [T][N][9] float32.  Returns dict with Jb,
    J and, with parts=True, the factors of Eq. 16: xdot [T][M] and y [T][M][3] (direction:
    [T][M][3 (b)][3 (a)]).  Called on the absolute values of E, v and W it gives the sums of
    the absolute values of the terms of Eq. 13 and of the Eq. 16 bracket."""
    E = np.asarray(E, dtype=np.float64)
    D, M = E.shape
    mass = np.asarray(mass, dtype=np.float64)
    N = mass.shape[0]
    if D != 3 * N:
        raise ValueError("E must have 3N rows")
    v = np.asarray(v, dtype=np.float32).reshape(-1, N, 3)
    W = np.asarray(W, dtype=np.float32).reshape(-1, N, 3, 3)
    T = v.shape[0]
    bins = np.asarray(bin_of_mode, dtype=np.int64)
    ind = np.zeros((M, B))
    kept = (bins >= 0) & (bins < B)
    ind[np.nonzero(kept)[0], bins[kept]] = 1.0
    sqm = np.sqrt(mass)
    J = np.empty((T, 3))
    Jb = np.empty((T, 3, B, 3)) if direction else np.empty((T, B, 3))
    xs = np.empty((T, M)) if parts else None
    ys = (np.empty((T, M, 3, 3)) if direction else np.empty((T, M, 3))) if parts else None
    for t0 in range(0, T, steps_per_product):
        t1 = min(T, t0 + steps_per_product)
        vt = v[t0:t1].astype(np.float64)                       # [S][N][3]
        Wt = W[t0:t1].astype(np.float64)                       # [S][N][3 (a)][3 (b)]
        S = t1 - t0
        X = (vt * sqm[None, :, None]).reshape(S, D) @ E          # Eq. 13
        U = Wt / sqm[None, :, None, None]                       # W_i^{ab} / sqrt(m_i)
        J[t0:t1] = np.einsum("siab,sib->sa", Wt, vt)            # Eq. 10
        if direction:
            Y = np.empty((S, M, 3, 3))
            for b in range(3):
                Eb = E[b::3]                                    # rows d = 3i + b
                for a in range(3):
                    Y[:, :, b, a] = U[:, :, a, b] @ Eb
            Jn = X[:, :, None, None] * Y                        # [S][M][b][a]
            Jb[t0:t1] = (Jn.transpose(0, 2, 3, 1) @ ind).transpose(0, 1, 3, 2)
        else:
            Y = np.stack([U[:, :, a, :].reshape(S, D) @ E for a in range(3)], axis=-1)
            Jn = X[:, :, None] * Y                              # Eq. 16, [S][M][3]
            Jb[t0:t1] = (Jn.transpose(0, 2, 1) @ ind).transpose(0, 2, 1)
        if parts:
            xs[t0:t1] = X
            ys[t0:t1] = Y
    out = {"Jb": Jb, "J": J}
    if parts:
        out["xdot"] = xs
        out["y"] = ys
    return out


def modal_current_dir(E: np.ndarray, mass, v, W, bin_of_mode, B: int,
                      want_modes: bool = False):
    """Direction-resolved currents (Sec. II.A split by the velocity component b).
    Returns dict with Jbd [T][3][B][3] (index [t][b][bin][a]), Jd [T][3][3] ([t][b][a],
    J^{ab} = sum_i W_i^{ab} v_i^b) and, when want_modes, Jnd [T][M][3][3] ([t][n][b][a])."""
    E = np.asarray(E, dtype=np.float64)
    D, M = E.shape
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    N = mass.shape[0]
    if D != 3 * N:
        raise ValueError("E must have 3N rows")
    Et = np.ascontiguousarray(E.T)
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1, N, 3)
    W = np.ascontiguousarray(W, dtype=np.float32).reshape(-1, N, 9)
    T = v.shape[0]
    bins = np.ascontiguousarray(bin_of_mode, dtype=np.int32)
    Jbd = np.empty((T, 3, B, 3))
    Jd = np.empty((T, 3, 3))
    Jnd = np.empty((T, M, 3, 3)) if want_modes else None
    lib().orc_modal_current_dir(N, M, _ptr(Et), _ptr(mass), T, _ptr(v), _ptr(W), _ptr(bins), B,
                                _ptr(Jbd), _ptr(Jd), _ptr(Jnd))
    out = {"Jbd": Jbd, "Jd": Jd}
    if want_modes:
        out["Jnd"] = Jnd
    return out


def gkma_corr(Jb: np.ndarray, J: np.ndarray, L: int):
    """Raw correlation sums Csum [B][3][3][L] and origin counts [L] (Eq. 17)."""
    Jb = np.ascontiguousarray(Jb, dtype=np.float64)
    J = np.ascontiguousarray(J, dtype=np.float64)
    T, B, _ = Jb.shape
    C = np.empty((B, 3, 3, L))
    cnt = np.empty(L, dtype=np.int64)
    lib().orc_gkma_corr(T, B, _ptr(Jb), _ptr(J), L, _ptr(C), _ptr(cnt))
    return C, cnt


def gkma_xcorr(Jb: np.ndarray, L: int):
    """Bin-bin cross-correlation sums Xsum [B][B][3][3][L] (first bin lagged, as in Eq. 17)."""
    Jb = np.ascontiguousarray(Jb, dtype=np.float64)
    T, B, _ = Jb.shape
    X = np.empty((B, B, 3, 3, L))
    lib().orc_gkma_xcorr(T, B, _ptr(Jb), L, _ptr(X))
    return X


def gk_kappa(Csum: np.ndarray, count: np.ndarray, dt_ps: float, T_K: float, V_A3: float):
    """Running Green-Kubo integral kappa_b^{mu nu}(l) in W/(m K) (Eq. 17)."""
    Csum = np.ascontiguousarray(Csum, dtype=np.float64)
    count = np.ascontiguousarray(count, dtype=np.int64)
    B, _, _, L = Csum.shape
    out = np.empty_like(Csum)
    lib().orc_gk_kappa(B, L, _ptr(Csum), _ptr(count), dt_ps, T_K, V_A3, _ptr(out))
    return out


def kappa_window(kappa: np.ndarray, dt_ps: float, tau_lo: float, tau_hi: float):
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    B, _, _, L = kappa.shape
    out = np.empty((B, 3, 3))
    n = lib().orc_kappa_window(B, L, _ptr(kappa), dt_ps, tau_lo, tau_hi, _ptr(out))
    return out, int(n)


def hnema(Jb: np.ndarray, T_K: float, V_A3: float, Fe):
    """Time-averaged binned current and kappa_b^mu (Eq. 19), W/(m K)."""
    Jb = np.ascontiguousarray(Jb, dtype=np.float64)
    T, B, _ = Jb.shape
    fe = np.ascontiguousarray(Fe, dtype=np.float64)
    mean = np.empty((B, 3))
    kap = np.empty((B, 3))
    lib().orc_hnema(T, B, _ptr(Jb), T_K, V_A3, _ptr(fe), _ptr(mean), _ptr(kap))
    return mean, kap


def orthonormality(E: np.ndarray) -> float:
    Et = np.ascontiguousarray(np.asarray(E, dtype=np.float64).T)
    M, D = Et.shape
    return float(lib().orc_orthonormality(D, M, _ptr(Et)))


def shc_corr(v, W, nc: int):
    """SHC correlation sums Ksum [9][nc] (pair 3a+b) and origin counts [nc] (Eq. 20-21)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    T, N, _ = v.shape
    W = np.ascontiguousarray(W, dtype=np.float32).reshape(T, N, 9)
    K = np.empty((9, nc))
    cnt = np.empty(nc, dtype=np.int64)
    lib().orc_shc_corr(N, T, _ptr(v), _ptr(W), nc, _ptr(K), _ptr(cnt))
    return K, cnt


def shc_kappa(Ksum, count, dt_ps: float, T_K: float, V_A3: float, Fe: float, f_THz,
              window: int = 0):
    """SHC spectral conductivity kappa [9][n_freq] in W/(m K THz) (Eq. 22-23)."""
    Ksum = np.ascontiguousarray(Ksum, dtype=np.float64)
    nc = Ksum.shape[1]
    count = np.ascontiguousarray(count, dtype=np.int64)
    f = np.ascontiguousarray(f_THz, dtype=np.float64)
    out = np.empty((9, f.shape[0]))
    lib().orc_shc_kappa(nc, _ptr(Ksum), _ptr(count), dt_ps, T_K, V_A3, Fe, window, f.shape[0],
                        _ptr(f), _ptr(out))
    return out


def lattice_modes(Phi, mass, max_sweeps: int = 60, tol: float = 1e-15):
    """Gamma-point eigenmodes of the force constants Phi [3N][3N] (eV/A^2) and masses [N] (amu)
    (Sec. II.B): w2 [3N] ascending (eV/(A^2 amu)), f_THz [3N], E [3N][3N] dof-major (column n
    = eigenvector n, sign fixed by its first largest-magnitude component), and the sweeps taken
    (cyclic Jacobi, FP64; -1 if max_sweeps ran out)."""
    Phi = np.ascontiguousarray(Phi, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    N = mass.shape[0]
    D = 3 * N
    if Phi.shape != (D, D):
        raise ValueError("Phi must be [3N][3N]")
    w2 = np.empty(D)
    f = np.empty(D)
    E = np.empty((D, D))
    sweeps = lib().orc_lattice_modes(N, _ptr(Phi), _ptr(mass), max_sweeps, tol, _ptr(w2), _ptr(f),
                                     _ptr(E))
    return w2, f, E, int(sweeps)
