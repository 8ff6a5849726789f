"""Python binding of libmhc.so (include/mhc.h): argument marshalling only.

Every step of the modal heat-current path runs in the CUDA library; this
module converts numpy arrays (host memory) and torch CUDA tensors (device
memory) into the plain pointers and sizes of the C ABI, and status codes into
exceptions.  There is no fallback: if the compiled library is missing the
import of a handle fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmhc.so")

MHC_OK = 0
MHC_WARN_NOT_ORTHONORMAL = 100
PRECISIONS = {"fp32": 0, "bf16x3": 1, "fp16x3": 2}
MEM_HOST, MEM_DEVICE, MEM_HOST_ASYNC = 0, 1, 2
F32, F64 = 0, 1
DOF_MAJOR, MODE_MAJOR = 0, 1
FLAG_GKMA, FLAG_NO_GRAPH, FLAG_PROFILE, FLAG_TEST_STALL = 0x1, 0x2, 0x4, 0x8
FLAG_DIRECTION = 0x10
FLAG_XCORR = 0x20

# Every entry point declared in include/mhc.h.
EXPORTS = (
    "mhc_default_params", "mhc_create", "mhc_destroy", "mhc_last_error", "mhc_status_string",
    "mhc_set_modes", "mhc_set_bins_uniform", "mhc_set_bin_ids", "mhc_push", "mhc_sync",
    "mhc_autotune_k", "mhc_lattice_modes", "mhc_group_autotune_k", "mhc_measure_fp32_fma",
    "mhc_read_binned_current", "mhc_read_total_current", "mhc_read_hnema", "mhc_read_corr",
    "mhc_read_kappa_gk", "mhc_check_orthonormality", "mhc_get_info", "mhc_set_flags",
    "mhc_kernel_time", "mhc_read_xcorr", "mhc_read_kappa_xcorr",
    "mhc_reset",
    "mhc_state_size", "mhc_get_state", "mhc_set_state", "mhc_group_create",
    "mhc_group_destroy", "mhc_group_push", "mhc_group_read_hnema", "mhc_binned_current_noalloc",
    "mhc_shc_create", "mhc_shc_destroy", "mhc_shc_last_error", "mhc_shc_push", "mhc_shc_read_corr",
    "mhc_shc_read_kappa", "mhc_shc_set_precision", "mhc_shc_set_profile", "mhc_shc_kernel_time",
)


class MhcParams(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("k_max", ctypes.c_int32), ("n_lags", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tile_config", ctypes.c_int32), ("ortho_probe", ctypes.c_int32),
                ("dt_ps", ctypes.c_double), ("T_K", ctypes.c_double), ("V_A3", ctypes.c_double),
                ("F_e", ctypes.c_double * 3), ("split_d", ctypes.c_int32)]


class MhcInfo(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("n_dof", ctypes.c_int64),
                ("n_modes_in", ctypes.c_int64), ("n_modes_kept", ctypes.c_int64),
                ("n_bins", ctypes.c_int32), ("n_lags", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("steps_pushed", ctypes.c_int64), ("pushes", ctypes.c_int64),
                ("n_slots", ctypes.c_int64), ("tile_n", ctypes.c_int32), ("tile_k", ctypes.c_int32),
                ("tile_pair", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("grid", ctypes.c_int32), ("e_exp", ctypes.c_int32),
                ("ortho_err", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("tile_split", ctypes.c_int32)]


class MhcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mhc status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmhc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.mhc_default_params.argtypes = [ctypes.POINTER(MhcParams)]
    L.mhc_default_params.restype = None
    L.mhc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(MhcParams)]
    L.mhc_destroy.argtypes = [vp]
    L.mhc_destroy.restype = None
    L.mhc_last_error.argtypes = [vp]
    L.mhc_last_error.restype = ctypes.c_char_p
    L.mhc_status_string.argtypes = [ctypes.c_int]
    L.mhc_status_string.restype = ctypes.c_char_p
    L.mhc_set_modes.argtypes = [vp, i64, i64, vp, i32, i32, i64, i32, vp, vp]
    L.mhc_set_bins_uniform.argtypes = [vp, dbl, dbl, i32]
    L.mhc_set_bin_ids.argtypes = [vp, vp, i32]
    L.mhc_push.argtypes = [vp, vp, vp, i32, i32]
    L.mhc_sync.argtypes = [vp]
    L.mhc_autotune_k.argtypes = [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    L.mhc_lattice_modes.argtypes = [i32, vp, i64, vp, vp, i32, dbl, i32, vp, vp, vp, i32,
                                    ctypes.POINTER(i32)]
    L.mhc_measure_fp32_fma.argtypes = [i32, vp, ctypes.POINTER(dbl)]
    L.mhc_read_binned_current.argtypes = [vp, vp, i32]
    L.mhc_read_total_current.argtypes = [vp, vp, i32]
    L.mhc_read_hnema.argtypes = [vp, vp, vp, i32]
    L.mhc_read_corr.argtypes = [vp, vp, vp, i32]
    L.mhc_read_kappa_gk.argtypes = [vp, vp, dbl, dbl, vp, i32]
    L.mhc_read_xcorr.argtypes = [vp, vp, vp, i32]
    L.mhc_read_kappa_xcorr.argtypes = [vp, vp, dbl, dbl, vp, i32]
    L.mhc_check_orthonormality.argtypes = [vp, dbl, ctypes.POINTER(dbl)]
    L.mhc_get_info.argtypes = [vp, ctypes.POINTER(MhcInfo)]
    L.mhc_kernel_time.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
    L.mhc_set_flags.argtypes = [vp, i32]
    L.mhc_reset.argtypes = [vp]
    L.mhc_state_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.mhc_get_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.mhc_set_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.mhc_group_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i32]
    L.mhc_group_destroy.argtypes = [vp]
    L.mhc_group_destroy.restype = None
    L.mhc_group_push.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 ctypes.POINTER(i32), i32]
    L.mhc_group_read_hnema.argtypes = [vp, vp, vp, i32]
    L.mhc_group_autotune_k.argtypes = [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
    L.mhc_shc_create.argtypes = [ctypes.POINTER(vp), i32, vp, i64, i32, i32, dbl, dbl, dbl, vp]
    L.mhc_shc_destroy.argtypes = [vp]
    L.mhc_shc_destroy.restype = None
    L.mhc_shc_last_error.argtypes = [vp]
    L.mhc_shc_last_error.restype = ctypes.c_char_p
    L.mhc_shc_push.argtypes = [vp, vp, vp, i32, i32]
    L.mhc_shc_read_corr.argtypes = [vp, vp, vp, i32]
    L.mhc_shc_read_kappa.argtypes = [vp, vp, i32, i32, vp, i32]
    L.mhc_shc_set_precision.argtypes = [vp, i32]
    L.mhc_shc_set_profile.argtypes = [vp, i32]
    L.mhc_shc_kernel_time.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
    L.mhc_binned_current_noalloc.argtypes = [i32, i32, vp, i64, vp, i32, vp, vp, vp, i32, vp, vp,
                                             i32, vp]
    for name in EXPORTS:
        if name not in ("mhc_default_params", "mhc_destroy", "mhc_last_error",
                        "mhc_status_string", "mhc_group_destroy", "mhc_shc_destroy",
                        "mhc_shc_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class ModalHeatCurrentGroup:
    """mhc_group_*: one grouped tensor-core launch over several ModalHeatCurrent handles."""

    def __init__(self, members):
        self._L = load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h for m in self.members])
        g = ctypes.c_void_p()
        st = self._L.mhc_group_create(ctypes.byref(g), arr, len(self.members))
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_last_error(self.members[0]._h).decode())
        self._g = g

    def autotune_k(self, candidates):
        """mhc_group_autotune_k: the block length (for every member) with the most
        mode*atom*steps per second, and that rate."""
        c = np.ascontiguousarray(candidates, dtype=np.int32)
        best = ctypes.c_int32()
        rate = ctypes.c_double()
        st = self._L.mhc_group_autotune_k(self._g, c.ctypes.data_as(ctypes.c_void_p), c.size,
                                          ctypes.byref(best), ctypes.byref(rate))
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_last_error(self.members[0]._h).decode())
        for m in self.members:
            m._lastK = 0
        return int(best.value), float(rate.value)

    def push(self, vs, Ws, async_inputs: bool = False):
        """async_inputs: host inputs are uploaded after the call returns and must stay unchanged
        until the next push of the group or a sync of its handles returns (references to them
        are kept until then)."""
        n = len(self.members)
        keep, pv, pw, ks, where = [], [], [], [], None
        for m, v, W in zip(self.members, vs, Ws):
            a, wa, ka = _ptr(v, np.float32)
            b, wb, kb = _ptr(W, np.float32)
            if where is None:
                where = wa
            if wa != where or wb != where:
                raise ValueError("all inputs of a group push must be in the same memory space")
            keep += [ka, kb]
            pv.append(a)
            pw.append(b)
            ks.append(int(ka.shape[0]))
        if async_inputs and where == MEM_HOST:
            where = MEM_HOST_ASYNC
        st = self._L.mhc_group_push(self._g, (ctypes.c_void_p * n)(*pv), (ctypes.c_void_p * n)(*pw),
                                    (ctypes.c_int32 * n)(*ks), where)
        self._keep = keep   # after the call: the previous inputs may have been read in it
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_last_error(self.members[0]._h).decode())
        for m, k in zip(self.members, ks):
            m._lastK = k

    def read_hnema(self, kappa=None, mean=None):
        """All members' HNEMA kappa (and mean current) in one call: numpy arrays (host, one
        synchronisation) or CUDA tensors (device, asynchronous), concatenated [sum B_j * 3]."""
        n = sum(m.B * 3 for m in self.members)
        if kappa is None:
            kappa = np.empty(n)
        pk, where, kk = _ptr(kappa, np.float64)
        pm = None if mean is None else _ptr(mean, np.float64)[0]
        st = self._L.mhc_group_read_hnema(self._g, pk, pm, where)
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_last_error(self.members[0]._h).decode())
        return kk

    def close(self):
        if getattr(self, "_g", None):
            self._L.mhc_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SpectralHeatCurrent:
    """mhc_shc_*: run-time SHC correlation K^{ab}(l) (Eq. 20-21) and spectrum (Eq. 22-23)."""

    def __init__(self, n_atoms: int, n_lags: int, k_max: int = 256, dt_ps: float = 0.002,
                 T_K: float = 300.0, V_A3: float = 1.0, F_e=(1e-5, 0.0, 0.0), device: int = 0,
                 stream=None, precision: str = "fp16x3"):
        self._L = load()
        fe = (ctypes.c_double * 3)(*F_e)
        st_ptr = stream if isinstance(stream, ctypes.c_void_p) else (
            ctypes.c_void_p(stream) if stream is not None else _current_stream(device))
        s = ctypes.c_void_p()
        st = self._L.mhc_shc_create(ctypes.byref(s), device, st_ptr, n_atoms, n_lags, k_max, dt_ps,
                                    T_K, V_A3, fe)
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_shc_last_error(None).decode())
        self._s = s
        self.N, self.n_lags = n_atoms, n_lags
        if precision != "fp16x3":
            self._check(self._L.mhc_shc_set_precision(s, PRECISIONS[precision]))

    def _check(self, st):
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_shc_last_error(self._s).decode())

    def push(self, v, W):
        pv, wv, kv = _ptr(v, np.float32)
        pw, ww, kw = _ptr(W, np.float32)
        if wv != ww:
            raise ValueError("v and W must be in the same memory space")
        self._keep = (kv, kw)
        self._check(self._L.mhc_shc_push(self._s, pv, pw, int(kv.shape[0]), wv))

    def set_profile(self, on: bool):
        self._check(self._L.mhc_shc_set_profile(self._s, 1 if on else 0))

    def kernel_time(self):
        """(total ms, launches) of the correlation kernel since the last call (profiling on)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._L.mhc_shc_kernel_time(self._s, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def read_corr(self):
        K = np.empty((9, self.n_lags))
        cnt = np.empty(self.n_lags, np.int64)
        self._check(self._L.mhc_shc_read_corr(self._s, K.ctypes.data_as(ctypes.c_void_p),
                                              cnt.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return K, cnt

    def read_kappa(self, f_THz, window: int = 0, out=None):
        f = np.ascontiguousarray(f_THz, dtype=np.float64)
        if out is None:
            out = np.empty((9, f.shape[0]))
        p, where, keep = _ptr(out, np.float64)
        self._check(self._L.mhc_shc_read_kappa(self._s, f.ctypes.data_as(ctypes.c_void_p),
                                               f.shape[0], window, p, where))
        return keep

    def close(self):
        if getattr(self, "_s", None):
            self._L.mhc_shc_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_fma(device: int = 0, stream=None) -> float:
    """mhc_measure_fp32_fma: the device's measured FP32 FMA throughput, TFLOP/s."""
    L = load()
    out = ctypes.c_double()
    st = L.mhc_measure_fp32_fma(device, stream if stream is not None else _current_stream(device),
                                ctypes.byref(out))
    if st != 0:
        raise MhcError(st, L.mhc_last_error(None).decode())
    return out.value


def lattice_modes(Phi, mass_amu, E_out=None, device: int = 0, stream=None, tol: float = 1e-14,
                  max_sweeps: int = 60):
    """mhc_lattice_modes: Gamma-point eigenmodes of the force constants Phi [3N][3N] (float64,
    numpy or CUDA tensor) with masses [N].  Returns (w2, freq_THz, E, sweeps): w2 and the
    frequencies as numpy arrays; E [3N][3N] dof-major float64 written into E_out (a CUDA tensor,
    so that the basis stays on the GPU) or returned as a numpy array when E_out is None."""
    L = load()
    pphi, wphi, kphi = _ptr(Phi, np.float64)
    mass = np.ascontiguousarray(mass_amu, dtype=np.float64)
    N = mass.shape[0]
    D = 3 * N
    n_phi = kphi.numel() if _is_torch(kphi) else kphi.size
    if n_phi != D * D:
        raise ValueError(f"Phi must be [{D}][{D}]")
    w2 = np.empty(D)
    f = np.empty(D)
    if E_out is None:
        E = np.empty((D, D))
        pe, we, ke = E.ctypes.data_as(ctypes.c_void_p), MEM_HOST, E
    else:
        pe, we, ke = _ptr(E_out, np.float64)
        E = E_out
    sweeps = ctypes.c_int32()
    st = L.mhc_lattice_modes(device, stream if stream is not None else _current_stream(device), N,
                             pphi, mass.ctypes.data_as(ctypes.c_void_p), wphi, tol, max_sweeps,
                             w2.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p),
                             pe, we, ctypes.byref(sweeps))
    if st != MHC_OK:
        raise MhcError(st, L.mhc_last_error(None).decode())
    return w2, f, E, int(sweeps.value)


def binned_current_noalloc(E_mode_major, bin_of_mode, n_bins: int, mass_amu, v, W, Jb, J,
                           device: int = 0, stream=None) -> None:
    """mhc_binned_current_noalloc on torch CUDA tensors (see include/mhc.h): one block's
    binned modal current computed with no device allocation."""
    L = load()
    M, ld = E_mode_major.shape
    N = mass_amu.shape[0]
    K = v.shape[0]
    st = L.mhc_binned_current_noalloc(
        N, M, ctypes.c_void_p(E_mode_major.data_ptr()), ld, ctypes.c_void_p(bin_of_mode.data_ptr()),
        n_bins, ctypes.c_void_p(mass_amu.data_ptr()), ctypes.c_void_p(v.data_ptr()),
        ctypes.c_void_p(W.data_ptr()), K, ctypes.c_void_p(Jb.data_ptr()),
        ctypes.c_void_p(J.data_ptr()), device,
        stream if stream is not None else _current_stream(device))
    if st != MHC_OK:
        raise MhcError(st, "mhc_binned_current_noalloc failed")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, where, keepalive) for a numpy array or a torch CUDA tensor."""
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64,
                np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), MEM_HOST, a


def _current_stream(device: int):
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(None)


class ModalHeatCurrent:
    """One system: eigenvectors, bins and the GKMA / HNEMA accumulators (see include/mhc.h).

    With direction=True (MHC_FLAG_DIRECTION) every per-bin result gains a leading axis for the
    direction b of the atoms' motion: binned current [K][3][B][3], HNEMA [3][B][3], GKMA
    [3][B][3][3][L]; summing that axis gives the results without the split."""

    def __init__(self, precision: str = "bf16x3", k_max: int = 256, n_lags: int = 0,
                 gkma: bool | None = None, dt_ps: float = 0.01, T_K: float = 300.0,
                 V_A3: float = 1.0, F_e=(1e-5, 0.0, 0.0), device: int = 0, stream=None,
                 tile_config: int = 0, ortho_probe: int = -1, flags: int = 0,
                 direction: bool = False, xcorr: bool = False, split_d: int = 0):
        self._L = load()
        p = MhcParams()
        self._L.mhc_default_params(ctypes.byref(p))
        p.device = device
        p.stream = stream if isinstance(stream, ctypes.c_void_p) else (
            ctypes.c_void_p(stream) if stream is not None else _current_stream(device))
        p.k_max = k_max
        p.n_lags = n_lags
        p.precision = PRECISIONS[precision]
        gk = (n_lags > 0) if gkma is None else gkma
        p.flags = (flags | (FLAG_GKMA if gk else 0) | (FLAG_DIRECTION if direction else 0)
                   | (FLAG_XCORR if xcorr else 0))
        p.tile_config = tile_config
        p.split_d = split_d
        p.ortho_probe = ortho_probe
        p.dt_ps, p.T_K, p.V_A3 = dt_ps, T_K, V_A3
        for i in range(3):
            p.F_e[i] = F_e[i]
        self.params = p
        self.device = device
        h = ctypes.c_void_p()
        st = self._L.mhc_create(ctypes.byref(h), ctypes.byref(p))
        if st != MHC_OK:
            raise MhcError(st, self._L.mhc_last_error(None).decode())
        self._h = h
        self.B = 0
        self.N = 0
        self._lastK = 0
        self.direction = bool(p.flags & FLAG_DIRECTION)

    # ------------------------------------------------------------------ plumbing
    def _check(self, st: int):
        if st == MHC_OK:
            return st
        msg = self._L.mhc_last_error(self._h).decode()
        if st == MHC_WARN_NOT_ORTHONORMAL:
            warnings.warn(f"eigenvectors not orthonormal: {msg}")
            return st
        raise MhcError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._L.mhc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ setup
    def set_modes(self, E, mass_amu, freq_THz=None, layout: str = "dof"):
        """E: [3N][M] (layout 'dof') or [M][3N] ('mode'), float32/float64, numpy or CUDA tensor."""
        lay = DOF_MAJOR if layout == "dof" else MODE_MAJOR
        is_f64 = (str(E.dtype) in ("float64", "torch.float64"))
        ptr, where, keep = _ptr(E, np.float64 if is_f64 else np.float32)
        rows, cols = keep.shape
        mass = np.ascontiguousarray(mass_amu, dtype=np.float64)
        N = mass.shape[0]
        M = cols if lay == DOF_MAJOR else rows
        f = None if freq_THz is None else np.ascontiguousarray(freq_THz, dtype=np.float64)
        st = self._L.mhc_set_modes(self._h, N, M, ptr, F64 if is_f64 else F32, lay, cols, where,
                                   None if f is None else f.ctypes.data_as(ctypes.c_void_p),
                                   mass.ctypes.data_as(ctypes.c_void_p))
        self.N = N
        self.M = M
        return self._check(st)

    def set_modes_from_force_constants(self, Phi, mass_amu, tol: float = 1e-14):
        """Gamma-point lattice dynamics of the force constants on the GPU (mhc_lattice_modes)
        and its eigenvectors loaded with mhc_set_modes straight from device memory; returns
        the frequencies (THz) for the binning."""
        import torch
        N = np.asarray(mass_amu).shape[0]
        E = torch.empty((3 * N, 3 * N), dtype=torch.float64, device=f"cuda:{self.device}")
        _, f, _, _ = lattice_modes(Phi, mass_amu, E_out=E, device=self.device,
                                   stream=self.params.stream, tol=tol)
        self.set_modes(E, mass_amu, f)
        return f

    def set_bins_uniform(self, f_min: float, f_max: float, n_bins: int):
        self._check(self._L.mhc_set_bins_uniform(self._h, f_min, f_max, n_bins))
        self.B = n_bins

    def set_bin_ids(self, bin_of_mode, n_bins: int):
        b = np.ascontiguousarray(bin_of_mode, dtype=np.int32)
        self._check(self._L.mhc_set_bin_ids(self._h, b.ctypes.data_as(ctypes.c_void_p), n_bins))
        self.B = n_bins

    # ------------------------------------------------------------------ stream
    def push(self, v, W, async_inputs: bool = False):
        """v [K][N][3], W [K][N][9] float32 (numpy: host, torch CUDA tensor: device).
        async_inputs: host inputs are uploaded after the call returns and must stay unchanged
        until the next push or sync() returns (references to them are kept until then)."""
        pv, wv, kv = _ptr(v, np.float32)
        pw, ww, kw = _ptr(W, np.float32)
        if wv != ww:
            raise ValueError("v and W must be in the same memory space")
        K = int(kv.shape[0])
        nv = int(np.prod(kv.shape)) if not _is_torch(kv) else kv.numel()
        nw = int(np.prod(kw.shape)) if not _is_torch(kw) else kw.numel()
        if nv != K * self.N * 3 or nw != K * self.N * 9:
            raise ValueError(f"v must be [K][{self.N}][3] and W [K][{self.N}][9]")
        if async_inputs and wv == MEM_HOST:
            wv = MEM_HOST_ASYNC
        st = self._L.mhc_push(self._h, pv, pw, K, wv)
        self._keep = (kv, kw)   # after the call: the previous inputs may have been read in it
        self._check(st)
        self._lastK = K

    def sync(self):
        self._check(self._L.mhc_sync(self._h))

    # ------------------------------------------------------------------ reads
    def _rows(self):
        """Leading shape of a per-bin result: (B,) or (3, B) with the direction split."""
        return (3, self.B) if self.direction else (self.B,)

    def read_binned_current(self, out=None):
        if out is None:
            out = np.empty((self._lastK, *self._rows(), 3), np.float32)
        p, where, keep = _ptr(out, np.float32)
        self._check(self._L.mhc_read_binned_current(self._h, p, where))
        return keep

    def read_total_current(self, out=None):
        if out is None:
            out = np.empty((self._lastK, 3), np.float64)
        p, where, keep = _ptr(out, np.float64)
        self._check(self._L.mhc_read_total_current(self._h, p, where))
        return keep

    def read_hnema(self):
        kap = np.empty((*self._rows(), 3))
        mean = np.empty((*self._rows(), 3))
        self._check(self._L.mhc_read_hnema(self._h, kap.ctypes.data_as(ctypes.c_void_p),
                                           mean.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return mean, kap

    def read_hnema_into(self, kappa, mean=None):
        pk, where, _ = _ptr(kappa, np.float64)
        pm = None if mean is None else _ptr(mean, np.float64)[0]
        self._check(self._L.mhc_read_hnema(self._h, pk, pm, where))

    def read_corr(self):
        L_ = self.params.n_lags
        C = np.empty((*self._rows(), 3, 3, L_))
        cnt = np.empty(L_, np.int64)
        self._check(self._L.mhc_read_corr(self._h, C.ctypes.data_as(ctypes.c_void_p),
                                          cnt.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return C, cnt

    def read_kappa_gk(self, tau_lo: float, tau_hi: float):
        L_ = self.params.n_lags
        kt = np.empty((*self._rows(), 3, 3, L_))
        kw = np.empty((*self._rows(), 3, 3))
        self._check(self._L.mhc_read_kappa_gk(self._h, kt.ctypes.data_as(ctypes.c_void_p), tau_lo,
                                              tau_hi, kw.ctypes.data_as(ctypes.c_void_p),
                                              MEM_HOST))
        return kt, kw

    def read_kappa_window(self, tau_lo: float, tau_hi: float):
        """The window averages of read_kappa_gk alone [rows][3][3] (no kappa(tau) output, so the
        library evaluates them as one weighted sum of C(l) a row)."""
        kw = np.empty((*self._rows(), 3, 3))
        self.read_kappa_gk_into(kw, tau_lo, tau_hi)
        return kw

    def read_xcorr(self):
        """Bin-bin cross-correlation sums [rows][rows][3][3][L] and origin counts [L]
        (rows = B, or (3, B) with the direction split)."""
        L_ = self.params.n_lags
        X = np.empty((*self._rows(), *self._rows(), 3, 3, L_))
        cnt = np.empty(L_, np.int64)
        self._check(self._L.mhc_read_xcorr(self._h, X.ctypes.data_as(ctypes.c_void_p),
                                           cnt.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return X, cnt

    def read_kappa_xcorr(self, tau_lo: float, tau_hi: float, with_tau: bool = True):
        """Eq. 17 running integral of every bin pair: kappa_tau [rows][rows][3][3][L] (None
        without with_tau: then only the window averages are evaluated) and its tau-window
        average [rows][rows][3][3], W/(m K)."""
        L_ = self.params.n_lags
        kt = np.empty((*self._rows(), *self._rows(), 3, 3, L_)) if with_tau else None
        kw = np.empty((*self._rows(), *self._rows(), 3, 3))
        self._check(self._L.mhc_read_kappa_xcorr(
            self._h, kt.ctypes.data_as(ctypes.c_void_p) if with_tau else None, tau_lo, tau_hi,
            kw.ctypes.data_as(ctypes.c_void_p), MEM_HOST))
        return kt, kw

    def check_orthonormality(self, tol: float = 1e-6) -> float:
        e = ctypes.c_double()
        st = self._L.mhc_check_orthonormality(self._h, tol, ctypes.byref(e))
        if st not in (MHC_OK, MHC_WARN_NOT_ORTHONORMAL):
            self._check(st)
        return e.value

    def autotune_k(self, candidates):
        """mhc_autotune_k: the candidate block length with the most steps per second, and that
        rate (the last block's currents are unreadable until the next push)."""
        c = np.ascontiguousarray(candidates, dtype=np.int32)
        best = ctypes.c_int32()
        rate = ctypes.c_double()
        self._check(self._L.mhc_autotune_k(self._h, c.ctypes.data_as(ctypes.c_void_p), c.size,
                                           ctypes.byref(best), ctypes.byref(rate)))
        self._lastK = 0
        return int(best.value), float(rate.value)

    def info(self) -> dict:
        i = MhcInfo()
        self._check(self._L.mhc_get_info(self._h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in MhcInfo._fields_}

    def set_flags(self, runtime_flags: int):
        """Set the run-time flags (FLAG_NO_GRAPH, FLAG_PROFILE, FLAG_TEST_STALL); the other
        bits are kept."""
        rt = FLAG_NO_GRAPH | FLAG_PROFILE | FLAG_TEST_STALL
        flags = (self.params.flags & ~rt) | (runtime_flags & rt)
        self._check(self._L.mhc_set_flags(self._h, flags))
        self.params.flags = flags

    def kernel_time(self):
        """(total ms, launches) of the projection kernel since the last call (FLAG_PROFILE)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._L.mhc_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def read_kappa_gk_into(self, kappa_w, tau_lo: float, tau_hi: float, kappa_tau=None):
        pw, where, _ = _ptr(kappa_w, np.float64)
        pt = None if kappa_tau is None else _ptr(kappa_tau, np.float64)[0]
        self._check(self._L.mhc_read_kappa_gk(self._h, pt, tau_lo, tau_hi, pw, where))

    def reset(self):
        self._check(self._L.mhc_reset(self._h))

    def get_state(self) -> bytes:
        n = ctypes.c_size_t()
        self._check(self._L.mhc_state_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._L.mhc_get_state(self._h, buf, n.value))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._L.mhc_set_state(self._h, buf, len(blob)))
