"""Vertical hydrostatic structure iteration (Sect. 2.5, Eq. 20).

Transport -> temperatures (Monte Carlo + PDA) -> density in hydrostatic equilibrium with them
(`Disk.hydrostatic_density`, one GPU thread per radial shell) -> transport again, until the mean
change of the temperatures between two iterations is below `tol_sigma` (3) of their Monte Carlo
errors, as the paper's convergence criterion states (the statistic, a driver-side reading, is
`temperature_change`, with the counting error of each cell as its sigma, or `temperature_change_halves`,
with sigma measured from two independent halves of each iteration's packets). Each radial shell keeps
its dust mass.

Two schemes. "picard", the paper's: the next density is the Eq. 20 density of the last temperatures.
"adjoint": a damped step per radial shell, log rho <- log rho + a_i (log rho_Eq20 - log rho), with
a_i = min(1, 1/k) / (1 - g_i) at update k. g_i is the shell's loop gain, the response of its midplane
temperature to itself through one update: the PDA adjoint (Sect. 2.2.1; d T_mid / d log rho of every
cell, the Monte Carlo boundary held) times the response of the Eq. 20 density to a uniform scaling of
the shell's temperatures at fixed mass. 1/(1 - g_i) is the Newton step of that linear map, and the 1/k
factor (a Robbins-Monro schedule) averages the Monte Carlo noise of the successive temperature fields
instead of letting the density follow it.

    python -m paper_0902_3092_gb300.hydro [--packets 1e7] [--iterations 8] [--scheme adjoint]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import disks, dist, mcrt


def temperature_change(T_old, err_old, T_new, err_new):
    """Mean |T_new - T_old| / sqrt(sigma_old^2 + sigma_new^2), sigma = T * relative error, over the cells
    that have a Monte Carlo error estimate in both iterations (a reading of the paper's 3-sigma criterion:
    the relative error is the counting error 1/(4 sqrt N) of each cell)."""
    ok = (T_old > 0) & (T_new > 0) & np.isfinite(err_old) & np.isfinite(err_new) & (err_old > 0) & (err_new > 0)
    if not ok.any():
        return float("inf")
    s_old, s_new = T_old[ok] * err_old[ok], T_new[ok] * err_new[ok]
    return float(np.mean(np.abs(T_new[ok] - T_old[ok]) / np.hypot(s_old, s_new)))


def temperature_change_halves(T_old, s_old, T_new, s_new):
    """Mean |T_new - T_old| over the mean of sqrt(sigma_old^2 + sigma_new^2), over the cells with a
    temperature and a sigma in both iterations, where sigma = |T_a - T_b| / 2 is measured from the two
    independent halves a, b of an iteration's packets (the error of their mean). In optically thick
    cells a packet is absorbed many times, and the MRW deposits many packet energies at once, so the
    counting error 1/(4 sqrt N) understates the scatter; the halves measure it. A single pair gives each
    cell's sigma with one degree of freedom, so the statistic is a ratio of means over the cells rather
    than a mean of per-cell ratios; when the temperatures change by noise alone it is near 1."""
    ok = (T_old > 0) & (T_new > 0) & np.isfinite(s_old) & np.isfinite(s_new)
    if not ok.any():
        return float("inf")
    den = float(np.mean(np.hypot(s_old[ok], s_new[ok])))
    if not den > 0:
        return float("inf")
    return float(np.mean(np.abs(T_new[ok] - T_old[ok]))) / den


def transport_halves(g, packets, seed, **kw):
    """One iteration's transport in two independent halves of the packet ids (each its own run, with its
    own packet energy), then their sum: returns the run statistics of both, the temperatures of the sum,
    their Monte Carlo relative errors, and sigma = |T_a - T_b| / 2 per cell (NaN where a half has no
    temperature). Gray tallies of the sum equal one run over all the packets."""
    half = packets // 2
    blobs, Ts, sts = [], [], []
    for first, n in ((0, half), (half, packets - half)):
        g.reset()
        sts.append(g.run_photons(n, seed=seed, first_id=first, n_total=n, **kw))
        Ts.append(g.temperatures()[0])
        blobs.append(g.checkpoint())
    g.restore(dist.combine_blobs(blobs))
    T, err, _ = g.temperatures()
    with np.errstate(invalid="ignore"):
        sig = np.where((Ts[0] > 0) & (Ts[1] > 0), np.abs(Ts[0] - Ts[1]) / 2.0, np.nan)
    return sts, T, err, sig


def midplane_rows(ntheta):
    j = ntheta // 2
    return [j - 1, j]


def shell_gains(g, T, rho_h, T_floor=10.0):
    """Loop gain g_i of each radial shell: sum_j (d log T_mid,i / d log rho_ij) delta_ij.

    d log T_mid,i / d log rho_ij: the PDA adjoint of J_i = the shell's mean midplane temperature (the two
    polar rows next to theta = pi/2), divided by J_i; zero where the midplane has no PDA cell (the Monte
    Carlo temperatures are held). delta_ij = d log rho_ij / d log T of the Eq. 20 density rho_h for a
    uniform scaling of the shell's temperatures at fixed mass: rho_j is proportional to exp(Phi_j) / T_j
    with Phi inversely proportional to T, so delta_j = -(Phi_j - <Phi>), <.> weighted by cell mass, and
    Phi_j = log(rho_j T_j) up to a constant of the shell."""
    nr, nt = T.shape
    rows = midplane_rows(nt)
    Tc = np.maximum(T, T_floor)
    V = g_cell_volumes(g)
    gains = np.zeros(nr)
    for i in range(nr):
        J = float(np.mean(T[i, rows]))
        m = rho_h[i] > 0
        if not (J > 0) or not m.any():
            continue
        w = np.zeros((nr, nt))
        w[i, rows] = 1.0 / len(rows)
        dlr, _ = g.pda_adjoint(w)
        phi = np.log(rho_h[i][m] * Tc[i][m])
        wm = rho_h[i][m] * V[i][m]
        delta = -(phi - np.sum(wm * phi) / np.sum(wm))
        gains[i] = float(np.sum(dlr[i][m] * delta)) / J
    return gains


def g_cell_volumes(g):
    rf, tf = g._rf, g._tf
    return (2.0 * np.pi / 3.0) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]


def iterate(model, packets, max_iter=8, seed=1, mrw=True, gamma=2.0, max_events=1e6, pda=True, min_visits=30,
            M_star_g=None, tol_sigma=3.0, disk=None, scheme="picard", on_update=None, sigma="counting"):
    """Runs the iteration on `model` (a disks.Disk); returns the mcrt.Disk and one record per iteration.
    scheme: "picard" or "adjoint" (see the module docstring; "adjoint" needs the PDA). on_update(g, rho_cur,
    relax, rho_new): called with the disk, each update's current density, step factors (None for Picard)
    and new density, before the new density is installed, e.g. to check them. sigma: "counting" (each
    cell's counting error, `temperature_change`) or "halves" (each iteration's packets in two independent
    halves, `temperature_change_halves`; the record then carries both statistics)."""
    if scheme not in ("picard", "adjoint"):
        raise ValueError("scheme must be picard or adjoint")
    if sigma not in ("counting", "halves"):
        raise ValueError("sigma must be counting or halves")
    if scheme == "adjoint" and not pda:
        raise ValueError("the adjoint scheme needs the PDA")
    g = disk if disk is not None else mcrt.Disk.from_model(model)
    hist, prev, k = [], None, 0
    for it in range(max_iter):
        t0 = time.perf_counter()
        kw = dict(mrw=mrw, gamma=gamma, max_events=max_events, want_sed=False)
        if sigma == "halves":
            sts, T_mc, err, sig = transport_halves(g, packets, seed + it, **kw)
            st = {"seconds": sum(x["seconds"] for x in sts)}
        else:
            g.reset()
            st = g.run_photons(packets, seed=seed + it, **kw)
            T_mc, err, _ = g.temperatures()
            sig = None
        npda = 0
        if pda:
            npda, _ = g.solve_pda(min_visits=min_visits)
            T = g.temperatures(mcrt.T_PDA)[0]
        else:
            T = T_mc
        counting = temperature_change(prev[0], prev[1], T_mc, err) if prev is not None else float("inf")
        change = counting
        rec = {"iteration": it, "transport_s": st["seconds"], "pda_cells": npda,
               "midplane_T_mean": float(np.mean(T[:, [g.ntheta // 2 - 1, g.ntheta // 2]]))}
        if sigma == "halves":
            change = temperature_change_halves(prev[0], prev[2], T_mc, sig) if prev is not None else float("inf")
            rec["change_sigma_counting"] = counting
        rec["change_sigma"] = change
        prev = (T_mc, err, sig)
        if change < tol_sigma:
            rec["wall_s"] = time.perf_counter() - t0
            hist.append(rec)
            break
        which = mcrt.T_PDA if pda else mcrt.T_MC
        rho_cur = g.density() if on_update is not None or scheme == "adjoint" else None
        relax = None
        if scheme == "adjoint":
            k += 1
            rho_h = g.hydrostatic_density(M_star_g=M_star_g, which=which)
            gains = shell_gains(g, T, rho_h)
            relax = np.clip(min(1.0, 1.0 / k) / (1.0 - gains), 0.05, 2.0)
            rec["gain_range"] = [float(gains.min()), float(gains.max())]
            rec["relax_mean"] = float(relax.mean())
        rho = g.hydrostatic_density(M_star_g=M_star_g, which=which, relax=relax)
        if on_update is not None:
            on_update(g, rho_cur, relax, rho)
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
    p.add_argument("--scheme", default="picard", choices=["picard", "adjoint"])
    p.add_argument("--sigma", default="counting", choices=["counting", "halves"])
    a = p.parse_args(argv)
    d = disks.config_thick_gray(a.nr, a.ntheta, a.tau)
    _, hist = iterate(d, int(a.packets), max_iter=a.iterations,
                      min_visits=max(30, int(30 * a.packets / 1e5)), scheme=a.scheme, sigma=a.sigma)
    for h in hist:
        print(json.dumps(h), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
