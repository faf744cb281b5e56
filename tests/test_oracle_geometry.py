"""Face distances of the (r, theta) grid: straight rays through the oracle's marcher."""
import math

import numpy as np

from paper_0902_3092_gb300 import disks


def _cell_of(d, p):
    r = np.linalg.norm(p)
    th = math.acos(max(-1.0, min(1.0, p[2] / r)))
    ir = int(np.searchsorted(d.r_faces_cm, r, side="right") - 1)
    it = int(np.searchsorted(d.theta_faces, th, side="right") - 1)
    return ir, min(it, d.ntheta - 1)


def test_volumes_sum(oracle):
    d = disks.config_thick_gray(nr=30, ntheta=20)
    rf, tf = d.r_faces_cm, d.theta_faces
    V = (2 * math.pi / 3) * (rf[1:] ** 3 - rf[:-1] ** 3)[:, None] * (np.cos(tf[:-1]) - np.cos(tf[1:]))[None, :]
    assert math.isclose(V.sum(), 4 * math.pi / 3 * (rf[-1] ** 3 - rf[0] ** 3), rel_tol=1e-12)


def test_random_rays_segments(oracle):
    """Each segment's midpoint lies in the cell the marcher assigned, and the segment lengths add
    up to the chord from the start point to the outer sphere (or to the inner cavity)."""
    d = disks.config_thick_gray(nr=24, ntheta=16)
    rng = np.random.default_rng(11)
    rf = d.r_faces_cm
    n_checked = 0
    for k in range(300):
        r = math.exp(rng.uniform(math.log(rf[0] * 1.01), math.log(rf[-1] * 0.99)))
        mu = rng.uniform(-1, 1)
        if k % 5 == 0:
            mu = rng.uniform(-0.02, 0.02)  # near the midplane
        ph = rng.uniform(0, 2 * math.pi)
        st = math.sqrt(1 - mu * mu)
        p = np.array([r * st * math.cos(ph), r * st * math.sin(ph), r * mu])
        mu2 = rng.uniform(-1, 1)
        ph2 = rng.uniform(0, 2 * math.pi)
        s2 = math.sqrt(1 - mu2 * mu2)
        u = np.array([s2 * math.cos(ph2), s2 * math.sin(ph2), mu2])
        ir, it = _cell_of(d, p)
        cells, lens = oracle.march(d, p, u, ir, it)
        assert len(cells) > 0 and np.all(lens >= 0)
        pos = p.copy()
        for c, l in zip(cells, lens):
            mid = pos + 0.5 * l * u
            if l > 1e-9 * r:
                assert _cell_of(d, mid) == (c // d.ntheta, c % d.ntheta)
                n_checked += 1
            pos = pos + l * u
        total = lens.sum()
        b = p @ u
        c = p @ p
        s_out = -b + math.sqrt(b * b - c + rf[-1] ** 2)
        disc_in = b * b - c + rf[0] ** 2
        s_in = -b - math.sqrt(disc_in) if (b < 0 and disc_in >= 0) else math.inf
        assert math.isclose(total, min(s_out, s_in), rel_tol=1e-10)
    assert n_checked > 2000


def test_cone_exit_matches_bisection(oracle):
    """Distance to a polar face against bisection on theta(s) along the ray."""
    rng = np.random.default_rng(2)
    L = oracle.lib()
    import ctypes as C
    for _ in range(300):
        th_f = rng.uniform(0.05, math.pi - 0.05)
        if abs(th_f - math.pi / 2) < 1e-3:
            continue
        # start at theta slightly below or above the face
        down = bool(rng.integers(0, 2))
        th0 = th_f + (rng.uniform(1e-3, 0.3) if down else -rng.uniform(1e-3, 0.3))
        th0 = min(max(th0, 1e-3), math.pi - 1e-3)
        r0 = 1.0
        p = np.array([r0 * math.sin(th0), 0.0, r0 * math.cos(th0)])
        mu = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * math.pi)
        st = math.sqrt(1 - mu * mu)
        u = np.array([st * math.cos(ph), st * math.sin(ph), mu])
        pd = C.POINTER(C.c_double)
        s = L.oracle_cone_exit(p.ctypes.data_as(pd), u.ctypes.data_as(pd), th_f, int(down))
        theta = lambda s_: math.atan2(math.hypot(*(p[:2] + s_ * u[:2])), p[2] + s_ * u[2])
        # brute force: first s where theta crosses th_f in the leaving direction
        ss = np.linspace(0, 20, 200001)
        pts = p[None, :] + ss[:, None] * u[None, :]
        th = np.arctan2(np.hypot(pts[:, 0], pts[:, 1]), pts[:, 2])
        if down:
            hit = np.flatnonzero((th[:-1] >= th_f) & (th[1:] < th_f))
        else:
            hit = np.flatnonzero((th[:-1] <= th_f) & (th[1:] > th_f))
        if hit.size == 0:
            assert s == math.inf or s > 19.9
            continue
        lo, hi = ss[hit[0]], ss[hit[0] + 1]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if (theta(mid) >= th_f) == down:
                lo = mid
            else:
                hi = mid
        assert math.isclose(s, 0.5 * (lo + hi), rel_tol=1e-9, abs_tol=1e-12)


def test_dmin_is_distance_to_cell_boundary(oracle):
    """d_min of Eq. 11 against the smallest distance to points sampled on the cell's faces."""
    d = disks.config_plain_gray(nr=6, ntheta=6)
    rng = np.random.default_rng(4)
    rf, tf = d.r_faces_cm, d.theta_faces
    for _ in range(40):
        ir, it = int(rng.integers(0, 6)), int(rng.integers(1, 5))
        r = rng.uniform(rf[ir], rf[ir + 1])
        th = rng.uniform(tf[it], tf[it + 1])
        p = np.array([r * math.sin(th), 0.0, r * math.cos(th)])
        dm = oracle.dmin(d, p, ir, it)
        # brute-force: dense sampling of the 4 boundary curves in the meridional plane
        rs = np.linspace(rf[ir], rf[ir + 1], 4001)
        ts = np.linspace(tf[it], tf[it + 1], 4001)
        pts = []
        for t_ in (tf[it], tf[it + 1]):
            pts.append(np.stack([rs * math.sin(t_), rs * math.cos(t_)], 1))
        for r_ in (rf[ir], rf[ir + 1]):
            pts.append(np.stack([r_ * np.sin(ts), r_ * np.cos(ts)], 1))
        pts = np.concatenate(pts)
        q = np.array([p[0], p[2]])
        bf = np.min(np.linalg.norm(pts - q, axis=1))
        assert dm <= bf * (1 + 1e-9)
        assert dm >= bf - 2e-3 * (rf[ir + 1] - rf[ir])
