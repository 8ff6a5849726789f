"""Failure detection on the GPU without a fault: every barrier wait of the tensor-core
kernels is bounded.  MHC_FLAG_TEST_STALL arms the first stage barrier to expect 16 bytes
more than its copies deliver, so the wait runs out (0.1 s), the kernel writes the sticky
status word and returns; the host reports MHC_ERR_TIMEOUT, and after mhc_reset the same
handle computes correct results again (the context stays usable)."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import REL_TOL, ModalRef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile_config", [1, 5])   # one-SM tile, two-SM (CTA pair) tile
def test_bounded_wait_times_out_and_context_survives(tile_config):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_03691_gb300.mhc import FLAG_TEST_STALL, MhcError, ModalHeatCurrent
    N, M, K, B = 128, 384, 32, 8
    E = synth.eigvecs(3 * N, M, 401)
    f = synth.frequencies(M, 0.0, 16.0, 401)
    mass = synth.masses(N, 28.085)
    v, W = synth.Trajectory(mass, seed=401).next_block(K)
    h = ModalHeatCurrent(precision="fp16x3", k_max=K, tile_config=tile_config)
    h.set_modes(E, mass, f)
    h.set_bins_uniform(0.0, 16.0, B)
    h.set_flags(FLAG_TEST_STALL)
    h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())   # asynchronous: OK
    with pytest.raises(MhcError) as err:
        h.sync()
    assert err.value.status == 4          # MHC_ERR_TIMEOUT
    h.set_flags(0)
    h.reset()                              # clears the sticky status
    h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
    Jb = h.read_binned_current()
    o = ModalRef(E, mass, v, W, oracle.bins_uniform(f, 0.0, 16.0, B), B)
    o.check_current(Jb, REL_TOL, f"after the timeout, tile {tile_config}")
    h.close()
