"""Oracle random streams: Philox4x32-10 words -> 23-bit uniforms in (0, 1)."""
import numpy as np


def test_uniform_grid_and_range(oracle):
    u = oracle.uniforms(seed=1, model=0, packet=0, n=40000)
    assert np.all(u > 0) and np.all(u < 1)
    k = u * 2 ** 23 - 0.5  # exactly integers
    assert np.all(k == np.round(k))
    # 1 - u lies on the same grid (symmetry used by tau = -ln u)
    k2 = (1 - u) * 2 ** 23 - 0.5
    assert np.all(k2 == np.round(k2))


def test_uniform_statistics(oracle):
    u = np.concatenate([oracle.uniforms(7, 0, p, 1000) for p in range(200)])
    n = len(u)
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * 0.0745 / np.sqrt(n)  # sd of sample variance of U(0,1)
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    e = n / 64
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)
    # lag-1 correlation within a stream
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(n)


def test_streams_are_distinct(oracle):
    a = oracle.uniforms(1, 0, 0, 64)
    b = oracle.uniforms(1, 0, 1, 64)
    c = oracle.uniforms(1, 1, 0, 64)
    d = oracle.uniforms(2, 0, 0, 64)
    for x in (b, c, d):
        assert not np.any(a == x) or np.mean(a == x) < 0.05


def test_counter_layout(oracle):
    """uniform i of a stream is word i%4 of Philox(block=i//4, model, packet_lo, packet_hi; seed)."""
    seed, model, packet = 0x123456789ABCDEF0, 3, (5 << 32) + 17
    u = oracle.uniforms(seed, model, packet, 12)
    for blk in range(3):
        w = oracle.philox([blk, model, packet & 0xFFFFFFFF, packet >> 32], [seed & 0xFFFFFFFF, seed >> 32])
        for j in range(4):
            assert u[4 * blk + j] == ((w[j] >> 9) + 0.5) / 2 ** 23


def test_philox_avalanche(oracle):
    """Flipping one counter bit flips about half of the 128 output bits (bijective mixing)."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(200):
        c = [int(x) for x in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)]
        k = [int(x) for x in rng.integers(0, 2 ** 32, 2, dtype=np.uint64)]
        o1 = oracle.philox(c, k)
        bit = int(rng.integers(0, 128))
        c2 = list(c)
        c2[bit // 32] ^= 1 << (bit % 32)
        o2 = oracle.philox(c2, k)
        flips.append(sum(bin(a ^ b).count("1") for a, b in zip(o1, o2)))
    assert abs(np.mean(flips) - 64) < 2.0


def test_henyey_greenstein_moments(oracle):
    """HG phase function: <cos> = g and <cos^2> = (1 + 2 g^2)/3 for the oracle's inverse-CDF sampling."""
    L = oracle.lib()
    u = (np.arange(200000) + 0.5) / 200000
    for g in (0.6, -0.3, 0.9):
        mu = np.array([L.oracle_hg_mu(g, float(x)) for x in u])
        assert abs(mu.mean() - g) < 2e-4
        assert abs((mu ** 2).mean() - (1 + 2 * g * g) / 3) < 2e-4
