"""The no-allocation entry point against the handle-based FP32 path.

mhc_binned_current_noalloc serves callers that cannot allocate device memory (an MD
engine calling from inside its time-step loop, or an application that hands out device
memory only from its own pool): it keeps every intermediate in one static device
buffer.  This file is named so that pytest collects it last.  It checks, on two calls
in a row with different inputs (the buffer keeps the first call's contents), that the
binned modal current and the total current equal what mhc_push and the read calls of
the existing entry points give, within the parity tolerance of the other tests, and
that a problem too large for the buffer is refused.
"""
import ctypes

import numpy as np
import pytest

from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, series_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(seed):
    N, M, B, K = 64, 180, 8, 24
    E = synth.eigvecs(3 * N, M, seed)
    f = synth.frequencies(M, 0.0, 16.0, seed)
    bins = np.minimum((f / 2.0).astype(np.int32), B - 1)
    order = np.argsort(bins, kind="stable")          # modes ordered by bin
    E, bins = E[:, order], bins[order]
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=seed)
    tr = synth.Trajectory(mass, seed=seed)
    blocks = [tr.next_block(K), tr.next_block(K)]
    return N, M, B, K, E.astype(np.float32), bins, mass, blocks


def test_noalloc_matches_handle_path_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent, binned_current_noalloc
    N, M, B, K, E, bins, mass, blocks = _case(seed=211)
    dev = torch.device("cuda", 0)
    E_mm = torch.from_numpy(np.ascontiguousarray(E.T)).to(dev)          # mode-major [M][3N]
    bins_d = torch.from_numpy(bins.astype(np.int32)).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    h = ModalHeatCurrent(precision="fp32", k_max=K)
    h.set_modes(E, mass, None)
    h.set_bin_ids(bins, B)
    for v, W in blocks:                                # two calls in a row
        vd = torch.from_numpy(v).to(dev)
        Wd = torch.from_numpy(W).to(dev)
        Jb = torch.full((K, B, 3), float("nan"), dtype=torch.float32, device=dev)
        J = torch.full((K, 3), float("nan"), dtype=torch.float64, device=dev)
        binned_current_noalloc(E_mm, bins_d, B, mass_d, vd, Wd, Jb, J, device=0)
        h.push(vd, Wd)
        ref_Jb = h.read_binned_current()
        ref_J = h.read_total_current()
        got_Jb = Jb.cpu().numpy()
        got_J = J.cpu().numpy()
        assert np.all(np.isfinite(got_Jb)) and np.all(np.isfinite(got_J))
        assert np.all(series_rel_err(got_Jb, ref_Jb) <= REL_TOL)
        np.testing.assert_allclose(got_J, ref_J, rtol=1e-12, atol=1e-9)
    h.close()


def test_noalloc_refuses_oversized_problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_03691_gb300 import mhc
    L = mhc.load()
    N, M, K, B = 4000, 12000, 64, 4              # ~190 MB of intermediates > 32 MiB
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")   # the size check comes first
    p = ctypes.c_void_p(buf.data_ptr())
    st = L.mhc_binned_current_noalloc(N, M, p, 3 * N, p, B, p, p, p, K, p, p, 0, None)
    assert st == 1
