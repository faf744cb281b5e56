"""Diffusion coefficient, Sect. 2.2.3: eta fixed point (Eq. 13), <d>, <d^2> (Eq. 14-15),
D (Eq. 12), kappa_bar (Eq. 10) and the anisotropic-scattering correction (Eq. 16).

Closed form used as the pin (derived by substitution into Eq. 13): the fixed point is
eta_b = a chi_b dB_b/dT with a = sum kappa dB/dT / sum chi dB/dT; then D = 1/(3 rho chi_R)
with chi_R the Rosseland mean of the extinction (Eq. 2-3), and kappa_bar = sum kappa dB/dT /
sum dB/dT."""
import dataclasses
import math

import numpy as np

from paper_0902_3092_gb300 import disks


def _disk(g=0.6):
    d = disks.config_plain_gray(nr=4, ntheta=4)
    op = disks.powerlaw_opacity(g=g)
    return dataclasses.replace(d, opacity=op)


def test_eta_fixed_point_closed_form(oracle):
    d = _disk(g=0.0)
    op = d.opacity
    for T in [20.0, 150.0, 900.0]:
        eta = oracle.eta_iterate(d, T, iters=2000)
        dB = oracle.dplanck_bins(op.lam_edges_um, T)
        chi = op.kappa_abs + op.kappa_sca
        a = np.sum(op.kappa_abs * dB) / np.sum(chi * dB)
        ref = a * chi * dB
        assert np.allclose(eta, ref, rtol=1e-10, atol=1e-14 * ref.max())
        # the normalisation that Eq. 13 fixes: sum eta = sum kappa dB/dT
        assert math.isclose(eta.sum(), np.sum(op.kappa_abs * dB), rel_tol=1e-12)


def test_D_is_rosseland_and_kbar(oracle):
    for g in (0.0, 0.6):
        d = _disk(g=g)
        op = d.opacity
        chi = op.kappa_abs + (1 - g) * op.kappa_sca  # Eq. 16 with g' = 0
        for T in [30.0, 300.0]:
            rho = 3.7e-12
            D, kb = oracle.diffusion(d, T, rho)
            dB = oracle.dplanck_bins(op.lam_edges_um, T)
            chiR = dB.sum() / np.sum(dB / chi)
            assert math.isclose(D, 1 / (3 * rho * chiR), rel_tol=1e-10)
            assert math.isclose(kb, np.sum(op.kappa_abs * dB) / dB.sum(), rel_tol=1e-10)


def test_no_scattering_reduces_to_rosseland(oracle):
    d = _disk(g=0.0)
    op = dataclasses.replace(d.opacity, kappa_sca=np.zeros(d.opacity.nlam))
    d = dataclasses.replace(d, opacity=op)
    T, rho = 80.0, 1e-13
    D, kb = oracle.diffusion(d, T, rho)
    dB = oracle.dplanck_bins(op.lam_edges_um, T)
    chiR = dB.sum() / np.sum(dB / op.kappa_abs)
    assert math.isclose(D, 1 / (3 * rho * chiR), rel_tol=1e-10)


def test_anisotropic_equals_isotropic_with_reduced_sigma(oracle):
    d6 = _disk(g=0.6)
    op0 = dataclasses.replace(d6.opacity, kappa_sca=0.4 * d6.opacity.kappa_sca, g=np.zeros(d6.opacity.nlam))
    d0 = dataclasses.replace(d6, opacity=op0)
    for T in (40.0, 400.0):
        a = oracle.diffusion(d6, T, 1e-12)
        b = oracle.diffusion(d0, T, 1e-12)
        assert math.isclose(a[0], b[0], rel_tol=1e-12) and math.isclose(a[1], b[1], rel_tol=1e-12)


def test_gray(oracle):
    d = disks.config_plain_gray(nr=4, ntheta=4)
    D, kb = oracle.diffusion(d, 100.0, 2e-12)
    assert math.isclose(D, 1 / (3 * 2e-12 * 1000.0), rel_tol=1e-14)
    assert kb == 500.0


def test_monochromatic_path_moments():
    """Sect. 2.2.3: for one frequency <d> = 1/(rho chi), <d^2> = 2/(rho chi)^2, so D = 1/(3 rho chi);
    checked against samples of an exponential free path."""
    rng = np.random.default_rng(3)
    a = 2.5
    d = rng.exponential(1 / a, 2_000_000)
    D = (d ** 2).mean() / (6 * d.mean())
    assert abs(D * 3 * a - 1) < 5e-3
