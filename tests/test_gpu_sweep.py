"""Seeded random sweep of shapes and options through the C ABI against the FP64 oracle: atoms,
kept modes, block length, bins, lags, excluded modes, precision, the direction split and the
cross-correlations and the d-axis split drawn at random, every output compared (binned currents, total current,
Eq. 17 sums, HNEMA means, cross-correlations)."""
import numpy as np
import pytest

import oracle
from paper_2102_03691_gb300 import synth
from tests.parity import ModalRef
from tests.test_gpu_parity import TOL, need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def draw(i):
    rng = np.random.default_rng(1000 + i)
    N = int(rng.integers(1, 260))
    M = int(rng.integers(1, 3 * N + 1))
    K = int(rng.integers(1, 70))
    T = int(rng.integers(1, 4)) * K + int(rng.integers(0, K))
    T = max(T, 1)
    B = int(rng.integers(1, 12))
    L = int(rng.integers(1, 40))
    d = dict(N=N, M=M, K=K, T=T, B=B, L=L, f_hi=float(rng.uniform(10, 20)),
             cut=float(rng.uniform(0.6, 1.0)), precision=["fp32", "fp16x3"][i % 2],
             direction=bool(rng.integers(0, 2)), xcorr=bool(rng.integers(0, 2)),
             layout=["dof", "mode"][int(rng.integers(0, 2))], host=bool(rng.integers(0, 2)))
    # d-axis split of the tensor-core path: autotuned, none, uniform or balanced (the direction
    # split takes none)
    split = [0, 1, 2, 3, -1][int(rng.integers(0, 5))]
    d["split_d"] = split if d["precision"] != "fp32" and not d["direction"] else 0
    return d


@pytest.mark.parametrize("i", range(20))
def test_random_shapes_and_options(i):
    need_gpu()
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    d = draw(i)
    N, M, K, T, B, L = d["N"], d["M"], d["K"], d["T"], d["B"], d["L"]
    E = synth.eigvecs(3 * N, M, 2000 + i)
    f = synth.frequencies(M, 0.0, d["f_hi"], 2000 + i)
    mass = synth.masses(N, isotopes=synth.SI_ISOTOPES, seed=2000 + i)
    v, W = synth.Trajectory(mass, drive_g=1e-3, seed=2000 + i).next_block(T)
    f_max = d["cut"] * d["f_hi"]   # modes above f_max are excluded
    bins = oracle.bins_uniform(f, 0.0, f_max, B)
    h = ModalHeatCurrent(precision=d["precision"], k_max=K, n_lags=L, direction=d["direction"],
                         xcorr=d["xcorr"], split_d=d["split_d"])
    Ein = E if d["layout"] == "dof" else np.ascontiguousarray(E.T)
    h.set_modes(Ein, mass, f, layout=d["layout"])
    h.set_bins_uniform(0.0, f_max, B)
    Jb, J = [], []
    for t0 in range(0, T, K):
        a, b = np.ascontiguousarray(v[t0:t0 + K]), np.ascontiguousarray(W[t0:t0 + K])
        if not d["host"]:
            a, b = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        h.push(a, b)
        Jb.append(h.read_binned_current().copy())
        J.append(h.read_total_current().copy())
    Jb, J = np.concatenate(Jb), np.concatenate(J)
    tol = TOL[d["precision"]]
    print(d)
    o = ModalRef(E, mass, v, W, bins, B, direction=d["direction"])
    np.testing.assert_allclose(J, o.J, rtol=1e-12, atol=1e-9 * max(1.0, np.abs(o.J).max()))
    o.check_current(Jb, tol, f"sweep {i} currents")
    C, cnt = h.read_corr()
    _, cnt0 = o.check_corr(C, L, tol, f"sweep {i} Eq. 17 sums")
    np.testing.assert_array_equal(cnt, cnt0)
    mean, _ = h.read_hnema()
    o.check_hnema(mean, None, 300.0, 1.0, [1e-5, 0.0, 0.0], tol, f"sweep {i} HNEMA")
    if d["xcorr"]:
        X, _ = h.read_xcorr()
        o.check_xcorr(X, L, tol, f"sweep {i} bin-bin sums")
    h.close()
