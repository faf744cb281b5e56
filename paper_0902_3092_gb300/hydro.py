"""Vertical hydrostatic structure iteration (Sect. 2.5, Eq. 20).

Transport -> temperatures (Monte Carlo + PDA) -> density in hydrostatic equilibrium with them
(`Disk.hydrostatic_density`, one GPU thread per radial shell) -> transport again, until the mean
change of the temperatures between two iterations is below `tol_sigma` (3) of their Monte Carlo
errors, as the paper's convergence criterion states. Each radial shell keeps its dust mass.

    python -m paper_0902_3092_gb300.hydro [--packets 1e7] [--iterations 8]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import disks, mcrt


def temperature_change(T_old, err_old, T_new, err_new):
    """Mean |T_new - T_old| / sqrt(sigma_old^2 + sigma_new^2), sigma = T * relative error, over the cells
    that have a Monte Carlo error estimate in both iterations."""
    s_old, s_new = T_old * err_old, T_new * err_new
    ok = (T_old > 0) & (T_new > 0) & np.isfinite(s_old) & np.isfinite(s_new) & (s_old > 0) & (s_new > 0)
    if not ok.any():
        return float("inf")
    return float(np.mean(np.abs(T_new[ok] - T_old[ok]) / np.hypot(s_old[ok], s_new[ok])))


def iterate(model, packets, max_iter=8, seed=1, mrw=True, gamma=2.0, max_events=1e6, pda=True, min_visits=30,
            M_star_g=None, tol_sigma=3.0, disk=None):
    """Runs the iteration on `model` (a disks.Disk); returns the mcrt.Disk and one record per iteration."""
    g = disk if disk is not None else mcrt.Disk.from_model(model)
    hist, prev = [], None
    for it in range(max_iter):
        t0 = time.perf_counter()
        g.reset()
        st = g.run_photons(packets, seed=seed + it, mrw=mrw, gamma=gamma, max_events=max_events, want_sed=False)
        T_mc, err, _ = g.temperatures()
        npda = 0
        if pda:
            npda, _ = g.solve_pda(min_visits=min_visits)
            T = g.temperatures(mcrt.T_PDA)[0]
        else:
            T = T_mc
        change = temperature_change(prev[0], prev[1], T_mc, err) if prev is not None else float("inf")
        rec = {"iteration": it, "transport_s": st["seconds"], "pda_cells": npda, "change_sigma": change,
               "midplane_T_mean": float(np.mean(T[:, [g.ntheta // 2 - 1, g.ntheta // 2]]))}
        prev = (T_mc, err)
        if change < tol_sigma:
            rec["wall_s"] = time.perf_counter() - t0
            hist.append(rec)
            break
        rho = g.hydrostatic_density(M_star_g=M_star_g, which=mcrt.T_PDA if pda else mcrt.T_MC)
        g.set_density(rho)
        rec["wall_s"] = time.perf_counter() - t0
        hist.append(rec)
    return g, hist


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--packets", type=float, default=1e7)
    p.add_argument("--iterations", type=int, default=8)
    p.add_argument("--nr", type=int, default=200)
    p.add_argument("--ntheta", type=int, default=120)
    p.add_argument("--tau", type=float, default=1e6)
    a = p.parse_args(argv)
    d = disks.config_thick_gray(a.nr, a.ntheta, a.tau)
    _, hist = iterate(d, int(a.packets), max_iter=a.iterations,
                      min_visits=max(30, int(30 * a.packets / 1e5)))
    for h in hist:
        print(json.dumps(h), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
