"""Error metrics of the GPU-vs-oracle parity tests.

The spec bar is 1e-5 relative on every binned modal current and every
kappa bin.  A binned current J_b^a(t) is a signed, zero-crossing signal, so
its relative error is taken over the compared time series of that bin and
component: max_t |g - o| / max_t |o|.  A bin whose oracle series is exactly
zero (no modes) must be exactly zero on the GPU.  kappa values (one number
per bin and component) are compared the same way across the spectrum of the
component: |g_b - o_b| / max_b |o_b|.
"""
import numpy as np

REL_TOL = 1e-5


def series_rel_err(g, o, t_axis=0):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    num = np.abs(g - o).max(axis=t_axis)
    den = np.abs(o).max(axis=t_axis)
    err = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))
    return err


def spectrum_rel_err(g, o, bin_axis=0):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    den = np.abs(o).max(axis=bin_axis, keepdims=True)
    num = np.abs(g - o)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))
