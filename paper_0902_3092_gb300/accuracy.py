"""Equal-accuracy comparison of the transport modes on one disk (GPU).

Runs a long plain Monte Carlo reference, then plain MC, plain MC + PDA, MRW and MRW + PDA at several
packet counts and per-packet event caps, and reports for each the relative error of the midplane
temperatures (the two polar rows next to theta = pi/2) against the reference -- RMS and maximum, as
in Sect. 3.1-3.2 -- together with the GPU time of the transport kernel and of the PDA solve.

    python -m paper_0902_3092_gb300.accuracy [--ref-packets 1e9] [--out results.json]

The reference is a long plain Monte Carlo run whose cells with fewer than `--ref-min-visits` packet
entries take the PDA temperature, as the paper does for its intrinsic-error test (Sect. 3.1).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import disks, mcrt


def midplane_rows(d):
    j = d.ntheta // 2
    return [j - 1, j]


def errors(T, T_ref, rows, sel=None):
    """RMS and maximum relative error over the midplane cells (optionally a subset `sel` of them)."""
    t, r = T[:, rows], T_ref[:, rows]
    ok = r > 0
    if sel is not None:
        ok &= sel
    if not ok.any():
        return float("nan"), float("nan"), 0
    rel = np.abs(np.where(ok, t / np.where(ok, r, 1.0) - 1.0, 0.0))[ok]
    return float(np.sqrt(np.mean(rel ** 2))), float(rel.max()), int(ok.sum())


def run_mode(g, n, seed, mrw, pda, cap, gamma=2.0):
    g.reset()
    st = g.run_photons(n, seed=seed, mrw=mrw, gamma=gamma, max_events=int(cap), want_sed=False)
    t_pda = 0.0
    n_pda = 0
    if pda:
        t0 = time.perf_counter()
        n_pda, _ = g.solve_pda()
        t_pda = time.perf_counter() - t0
        T, _, _ = g.temperatures(mcrt.T_PDA)
    else:
        T, _, _ = g.temperatures()
    return T, st, t_pda, n_pda


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--ref-packets", type=float, default=1e9)
    p.add_argument("--ref-cap", type=float, default=1e7)
    p.add_argument("--packets", default="1e5,1e6,1e7,1e8")
    p.add_argument("--caps", default="1e4,1e6")
    p.add_argument("--out", default=None)
    p.add_argument("--fields", default=None, help="npz file for the midplane temperature fields")
    p.add_argument("--ref-min-visits", type=int, default=3000,
                   help="the reference uses the PDA below this many packet entries (0: no PDA)")
    p.add_argument("--ref-tol", type=float, default=0.02,
                   help="evaluate only midplane cells whose two reference halves agree to this")
    a = p.parse_args(argv)
    d = disks.config_thick_gray(200, 120, 1e6)
    g = mcrt.Disk.from_model(d)
    rows = midplane_rows(d)
    # reference: two independent halves, so that its own noise is measured too; their integer tallies
    # add up to the full reference through checkpoints
    halves, blobs = [], []
    t_ref = 0.0
    nh = int(a.ref_packets / 2)
    for h in range(2):
        T, st, _, _ = run_mode(g, nh, 1000 + h, False, False, a.ref_cap)
        halves.append((T, st))
        blobs.append(np.frombuffer(g.checkpoint(), np.uint64).copy())
        t_ref += st["seconds"]
    comb = blobs[0].copy()
    comb[8:] = blobs[0][8:] + blobs[1][8:]
    comb[5] = 2 * nh
    comb[6] = np.frombuffer(np.array([float(2 * nh)]).tobytes(), np.uint64)[0]
    g.restore(comb.tobytes())
    T_mc_ref, _, vis_ref = g.temperatures()
    T_ref = T_mc_ref
    ref_pda = 0
    if a.ref_min_visits > 0:
        ref_pda, _ = g.solve_pda(min_visits=a.ref_min_visits)
        T_ref, _, _ = g.temperatures(mcrt.T_PDA)
    half_rms, half_max, n_cells = errors(halves[0][0], halves[1][0], rows)
    h0, h1 = halves[0][0][:, rows], halves[1][0][:, rows]
    with np.errstate(divide="ignore", invalid="ignore"):
        conv = (h0 > 0) & (h1 > 0) & (np.abs(h0 / h1 - 1) <= a.ref_tol)
    fields = {"T_ref": T_ref[:, rows], "T_mc_ref": T_mc_ref[:, rows], "h0": h0, "h1": h1,
              "vis_ref": vis_ref[:, rows].astype(np.float64)}
    out = {"disk": d.name, "midplane_rows": rows, "reference": {
        "packets": int(a.ref_packets), "cap": int(a.ref_cap), "kernel_s": t_ref,
        "capped": int(halves[0][1]["capped"] + halves[1][1]["capped"]),
        "half_vs_half_rms": half_rms, "half_vs_half_max": half_max, "cells": n_cells,
        "min_midplane_visits": int(vis_ref[:, rows].min()), "converged_cells": int(conv.sum()),
        "pda_min_visits": a.ref_min_visits, "pda_cells": ref_pda,
        "ref_tol": a.ref_tol}, "runs": []}
    print(json.dumps(out["reference"]), flush=True)
    for cap in [float(c) for c in a.caps.split(",")]:
        for n in [int(float(x)) for x in a.packets.split(",")]:
            for mrw, pda in ((False, False), (False, True), (True, False), (True, True)):
                T, st, t_pda, n_pda = run_mode(g, n, 7, mrw, pda, cap)
                rms, mx, _ = errors(T, T_ref, rows)
                crms, cmax, ncv = errors(T, T_ref, rows, conv)
                mode = ("MRW" if mrw else "plain") + ("+PDA" if pda else "")
                fields[f"{mode}_{n}_{int(cap)}"] = T[:, rows]
                rec = {"mode": mode, "packets": n, "cap": int(cap), "rms_all": rms, "max_all": mx,
                       "rms": crms, "max": cmax, "cells": ncv,
                       "kernel_s": st["seconds"], "pda_s": t_pda, "pda_cells": n_pda,
                       "capped": st["capped"], "events": st["events"], "time_s": st["seconds"] + t_pda}
                out["runs"].append(rec)
                print(json.dumps(rec), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)
    if a.fields:
        np.savez_compressed(a.fields, **fields)
    return out


if __name__ == "__main__":
    main(sys.argv[1:])
