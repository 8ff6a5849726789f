"""The no-allocation entry point against the FP64 oracle and the handle-based FP32 path.

mhc_binned_current_noalloc serves callers that cannot allocate device memory (an MD
engine calling from inside its time-step loop, where a cudaMalloc would stall the whole
device, or an application that hands out device memory only from its own pool): it keeps
every intermediate in one static device buffer.  This file is named so that pytest
collects it last.  It checks, on calls in a row with different inputs (the buffer keeps
the previous call's contents):
  - the binned modal current and the total current against the FP64 oracle (the
    conditioned metric of tests/parity.py) and against what mhc_push and the read calls of
    the existing entry points give;
  - that a call with decreasing bins, made right after a valid call of the same size,
    is refused with MHC_ERR_INVALID_ARG and leaves its outputs untouched, and that the next
    valid call is still right;
  - that a problem too large for the buffer is refused.
"""
import ctypes

import numpy as np
import pytest

from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, ModalRef, check

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
    blocks = [tr.next_block(K) for _ in range(3)]
    return N, M, B, K, E.astype(np.float32), bins, mass, blocks


def _call(E_mm, bins_d, B, mass_d, v, W, K, dev):
    from paper_2102_03691_gb300.mhc import binned_current_noalloc
    vd = torch.from_numpy(v).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    Jb = torch.full((K, B, 3), float("nan"), dtype=torch.float32, device=dev)
    J = torch.full((K, 3), float("nan"), dtype=torch.float64, device=dev)
    binned_current_noalloc(E_mm, bins_d, B, mass_d, vd, Wd, Jb, J, device=0)
    return Jb.cpu().numpy(), J.cpu().numpy()


def test_noalloc_matches_oracle_and_handle_path_on_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_03691_gb300.mhc import MhcError, ModalHeatCurrent, binned_current_noalloc
    N, M, B, K, E, bins, mass, blocks = _case(seed=211)
    dev = torch.device("cuda", 0)
    E_mm = torch.from_numpy(np.ascontiguousarray(E.T)).to(dev)          # mode-major [M][3N]
    bins_d = torch.from_numpy(bins.astype(np.int32)).to(dev)
    mass_d = torch.from_numpy(mass).to(dev)
    h = ModalHeatCurrent(precision="fp32", k_max=K)
    h.set_modes(E, mass, None)
    h.set_bin_ids(bins, B)
    E64 = E.astype(np.float64)                         # the float32 basis both sides use

    def valid_call(v, W, what):
        got_Jb, got_J = _call(E_mm, bins_d, B, mass_d, v, W, K, dev)
        assert np.all(np.isfinite(got_Jb)) and np.all(np.isfinite(got_J))
        ref = ModalRef(E64, mass, v, W, bins, B)
        ref.check_current(got_Jb, REL_TOL, what)
        np.testing.assert_allclose(got_J, ref.J, rtol=1e-12, atol=1e-9)
        # the existing entry point on the same block, within the same bound of the oracle
        h.push(torch.from_numpy(v).to(dev), torch.from_numpy(W).to(dev))
        check(got_Jb, h.read_binned_current(), 2 * ref.S, 2 * ref.Sd, REL_TOL,
              what + " vs handle")
        np.testing.assert_allclose(got_J, h.read_total_current(), rtol=1e-12, atol=1e-9)

    valid_call(*blocks[0], "no-alloc call 1")
    valid_call(*blocks[1], "no-alloc call 2")

    # decreasing bins after a valid call of the same size: refused, outputs untouched
    bad = bins.copy()
    bad[-1] = 0
    assert bins[-1] > 0
    bad_d = torch.from_numpy(bad.astype(np.int32)).to(dev)
    v, W = blocks[2]
    Jb = torch.full((K, B, 3), float("nan"), dtype=torch.float32, device=dev)
    J = torch.full((K, 3), float("nan"), dtype=torch.float64, device=dev)
    with pytest.raises(MhcError) as err:
        binned_current_noalloc(E_mm, bad_d, B, mass_d, torch.from_numpy(v).to(dev),
                               torch.from_numpy(W).to(dev), Jb, J, device=0)
    assert err.value.status == 1                        # MHC_ERR_INVALID_ARG
    assert torch.isnan(Jb).all() and torch.isnan(J).all()

    # the next valid call is right again
    valid_call(*blocks[2], "no-alloc call after a refused call")
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
