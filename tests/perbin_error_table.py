#!/usr/bin/env python
"""Per-bin error table of the library against the FP64 oracle on a long prefix of a
benchmark workload (writes JSON and Markdown; run on a machine with the GPU).

Every step of the prefix is pushed through the C ABI in the workload's blocks (autotuned
tile, graph replay), and recomputed by the oracle from the same seeded inputs with the
projections of Eqs. 13 and 16 written as FP64 matrix products (oracle.modal_current_mm).
For every output the conditioned metric of tests/parity.py is evaluated per bin:

  binned current J_b^a(t)      scale S_b^a(t) = sum_{n in b} |J_n^a(t)|
  Eq. 17 sums C_b^{mu nu}(l)   scale sum_t S_b^mu(t) |J^nu(t - l)|
  kappa_b^{mu nu}(tau), the tau-window kappa_b^{mu nu} (kappa(omega) of Sec. III.A), and the
  HNEMA kappa_b^mu (Eq. 19), each with the same integral / average of the scale.

Per bin it reports the largest scaled error |g - o| / S, the largest plain relative error
|g - o| / |o| over the well-conditioned values (tests/parity.py: |o| >= 0.1 S on bins of at
least 48 modes -- every bin of these workloads), the ratio S / |o| at the worst element, and
the median; and, over all bins, which bin is worst.

  python tests/perbin_error_table.py --workload gkma_si_n8000 --steps 2048 \
      --precision fp16x3 bf16x3 --out perbin_gkma_si_n8000
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2102_03691_gb300 import synth  # noqa: E402
from tests.parity import WELL_CONDITIONED, ModalRef  # noqa: E402



def per_bin_stats(g, o, S, Swc, bin_axis):
    """Per-bin maxima of the scaled and (well-conditioned) relative errors; bin_axis is the
    axis of g, o, S and Swc (the scale of conditioning) that indexes bins."""
    g = np.moveaxis(np.asarray(g, np.float64), bin_axis, 0)
    o = np.moveaxis(np.asarray(o, np.float64), bin_axis, 0)
    S = np.moveaxis(np.asarray(S, np.float64), bin_axis, 0)
    Sw = np.moveaxis(np.asarray(Swc, np.float64), bin_axis, 0)
    nb = g.shape[0]
    d = np.abs(g - o).reshape(nb, -1)
    o2 = np.abs(o).reshape(nb, -1)
    S2 = S.reshape(nb, -1)
    Sw2 = Sw.reshape(nb, -1)
    empty = S2 == 0
    scaled = np.where(empty, np.where(d == 0, 0.0, np.inf), d / np.where(empty, 1.0, S2))
    wc = ~empty & (o2 >= WELL_CONDITIONED * Sw2)
    rel = np.where(wc, d / np.where(wc, o2, 1.0), 0.0)
    nz = o2 > 0
    plain = np.where(nz, d / np.where(nz, o2, 1.0), 0.0)
    out = []
    for b in range(nb):
        k = int(np.argmax(scaled[b]))
        out.append({"bin": b, "scaled_max": float(scaled[b].max()),
                    "scaled_median": float(np.median(scaled[b])),
                    "rel_wc_max": float(rel[b].max()), "n_wc": int(wc[b].sum()),
                    "plain_rel_median": float(np.median(plain[b][nz[b]])) if nz[b].any() else 0.0,
                    "cond_at_worst": float(S2[b, k] / o2[b, k]) if o2[b, k] > 0 else float("inf")})
    return out


def summary(rows):
    sc = np.array([r["scaled_max"] for r in rows])
    rl = np.array([r["rel_wc_max"] for r in rows])
    w = int(np.argmax(np.maximum(sc, rl)))
    return {"bins": len(rows), "scaled_max": float(sc.max()), "scaled_median_of_bins": float(np.median(sc)),
            "rel_wc_max": float(rl.max()), "rel_wc_median_of_bins": float(np.median(rl)),
            "n_wc": int(sum(r["n_wc"] for r in rows)),
            "worst_bin": rows[w]["bin"], "worst_cond": rows[w]["cond_at_worst"],
            "pass_1e-5": bool(sc.max() <= 1e-5 and rl.max() <= 1e-5)}


def run(args):
    import torch
    from paper_2102_03691_gb300.mhc import ModalHeatCurrent
    w = synth.WORKLOADS[args.workload]
    N, M, K, L, B = w["N"], w["M"], w["K"], w["L"], w["B"]
    T = args.steps
    assert T % K == 0
    V = N * w["V_per_atom"]
    t0 = time.time()
    Ed = synth.eigvecs_device(3 * N, M, w["seed"])
    f = synth.frequencies(M, *w["f"], w["seed"])
    mass = synth.masses(N, w["mass"])
    drive = synth.drive_coupling(w["kappa_drive"], w["T_K"], V, w["Fe"][0], mass) \
        if w.get("kappa_drive") else 0.0
    tr = synth.Trajectory(mass, drive_g=drive, seed=w["seed"])
    blocks = [tr.next_block(K) for _ in range(T // K)]
    print(f"inputs {time.time() - t0:.1f} s", flush=True)
    tau_hi = (L - 1) * w["dt_ps"] if L else 0.0
    tau_lo = 0.8 * tau_hi
    gpu = {}
    for prec in args.precision:
        t1 = time.time()
        h = ModalHeatCurrent(precision=prec, k_max=K, n_lags=L, dt_ps=w["dt_ps"], T_K=w["T_K"],
                             V_A3=V, F_e=w["Fe"])
        h.set_modes(Ed, mass, f)
        h.set_bins_uniform(w["f"][0], w["f"][1], B)
        Jb, J = [], []
        for v, W in blocks:
            h.push(torch.from_numpy(v).cuda(), torch.from_numpy(W).cuda())
            Jb.append(h.read_binned_current().copy())
            J.append(h.read_total_current().copy())
        r = {"Jb": np.concatenate(Jb), "J": np.concatenate(J)}
        r["mean"], r["kap_h"] = h.read_hnema()
        if L:
            r["C"], r["cnt"] = h.read_corr()
            r["kt"], r["kw"] = h.read_kappa_gk(tau_lo, tau_hi)
        r["tile"] = {k: h.info()[k] for k in ("tile_n", "tile_k", "tile_pair", "stages")}
        h.close()
        gpu[prec] = r
        print(f"GPU {prec} {time.time() - t1:.1f} s", flush=True)
    E = Ed.double().cpu().numpy()          # the float32 basis the library was given
    del Ed
    torch.cuda.empty_cache()
    t2 = time.time()
    bins = oracle.bins_uniform(f, w["f"][0], w["f"][1], B)
    v = np.concatenate([b[0] for b in blocks])
    W = np.concatenate([b[1] for b in blocks])
    del blocks
    ref = ModalRef(E, mass, v, W, bins, B, mm=True)
    del E, v, W
    print(f"oracle {time.time() - t2:.1f} s on {os.cpu_count()} cores", flush=True)
    res = {"workload": args.workload, "N": N, "M": M, "K": K, "B": B, "L": L, "steps": T,
           "modes_per_bin": {"min": int(ref.counts.min()), "max": int(ref.counts.max())},
           "tau_window_ps": [tau_lo, tau_hi], "precisions": {}}
    if L:
        C, cnt, SC, SCd = ref.corr(L, full=True)
        kt, st, sd, kw, sw, swd, _ = ref.kappa(L, w["dt_ps"], w["T_K"], V, tau_lo, tau_hi,
                                               full=True)
    mean, kap, smean, skap, dmean, dkap = ref.hnema(w["T_K"], V, w["Fe"], full=True)
    for prec, r in gpu.items():
        out = {"tile": r["tile"],
               "total_current_max_rel": float(np.abs(r["J"] - ref.J).max() / np.abs(ref.J).max())}
        tabs = {"binned current J_b(t)": per_bin_stats(r["Jb"], ref.Jb, ref.S, ref.Swc, 1),
                "HNEMA kappa_b (Eq. 19)": per_bin_stats(r["kap_h"], kap, skap, dkap, 0)}
        if L:
            tabs["Eq. 17 sums C_b(l)"] = per_bin_stats(r["C"].reshape(C.shape), C, SC, SCd, 0)
            tabs["kappa_b(tau) (Eq. 17)"] = per_bin_stats(r["kt"].reshape(kt.shape), kt, st, sd,
                                                          0)
            tabs["kappa_b window (kappa(omega))"] = per_bin_stats(r["kw"].reshape(kw.shape), kw,
                                                                  sw, swd, 0)
        out["outputs"] = {k: {"summary": summary(v), "per_bin": v} for k, v in tabs.items()}
        res["precisions"][prec] = out
    return res


def markdown(res, cmd):
    lines = [f"# Per-bin error against the FP64 oracle: {res['workload']}", "",
             f"N = {res['N']} atoms, M = {res['M']} modes, {res['B']} bins "
             f"({res['modes_per_bin']['min']}-{res['modes_per_bin']['max']} modes per bin), "
             f"{res['L']} lags, {res['steps']} steps pushed in blocks of K = {res['K']}; "
             "every step of the prefix recomputed by the oracle.", "",
             "Metric (tests/parity.py): scaled = |g - o| / S with S the same sum over the "
             "absolute values of its terms; rel(wc) = |g - o| / |o| over the n well-conditioned "
             "values, |o| >= 0.1 S (bins of at least 48 modes); S/|o| at the worst element of "
             "the worst bin.", "",
             f"Command: `{cmd}`", ""]
    for prec, out in res["precisions"].items():
        lines += [f"## {prec} (tile {out['tile']}; total current max rel "
                  f"{out['total_current_max_rel']:.1e})", "",
                  "| output | max scaled | median over bins of max scaled | max rel (wc) | n | "
                  "median over bins of max rel (wc) | worst bin | its S/abs(o) | 1e-5 |",
                  "|---|---|---|---|---|---|---|---|---|"]
        for name, t in out["outputs"].items():
            s = t["summary"]
            lines.append(f"| {name} | {s['scaled_max']:.2e} | {s['scaled_median_of_bins']:.2e} | "
                         f"{s['rel_wc_max']:.2e} | {s['n_wc']} | {s['rel_wc_median_of_bins']:.2e} | "
                         f"{s['worst_bin']} | {s['worst_cond']:.1f} | "
                         f"{'pass' if s['pass_1e-5'] else 'MISS'} |")
        lines.append("")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="gkma_si_n8000", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--steps", type=int, default=2048)
    ap.add_argument("--precision", nargs="+", default=["fp16x3", "bf16x3"])
    ap.add_argument("--out", required=True, help="output path without extension")
    args = ap.parse_args()
    res = run(args)
    cmd = "python tests/perbin_error_table.py " + " ".join(sys.argv[1:])
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out + ".json", "w") as fh:
        json.dump(res, fh, indent=1)
    md = markdown(res, cmd)
    with open(args.out + ".md", "w") as fh:
        fh.write(md)
    print(md)


if __name__ == "__main__":
    main()
