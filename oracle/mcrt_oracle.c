/*
 * mcrt_oracle.c -- plain, slow FP64 CPU oracle for Monte Carlo dust radiative
 * transfer with Bjorkman-Wood re-emission and the modified random walk (MRW) of
 * Min et al. 2009 (A&A 497, 155), Sect. 2.1-2.2.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code with the
 * CUDA path and is not part of the product.
 *
 * Everything is computed in double precision, one packet after another, in the
 * order the method describes. Units: cgs (cm, g, s, K); wavelengths in micron.
 *
 * Random numbers: Philox4x32-10 written from Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3" (SC'11), Sect. 4. Key =
 * (seed_lo, seed_hi); counter = (block, model, packet_lo, packet_hi). Each
 * 32-bit output word w gives one uniform u = (floor(w / 2^9) + 1/2) * 2^-23,
 * exactly representable in binary32 and binary64, in (0, 1). One stream per
 * packet; every event takes the next whole block (blocks 0, 1, 2, ...), so the
 * block an event uses depends only on how many events came before it.
 *
 * Uniforms (w0, w1, w2, w3) of each event's block (the CUDA path uses them
 * identically):
 *   launch:      w0 stellar bin, (w1, w2) isotropic direction, w3 first tau
 *   interaction: w0 albedo test a: scatter if a < omega, else absorb, and the BW
 *                bin is drawn with (a - omega) / (1 - omega), the same uniform
 *                conditioned on absorption; (w1, w2) new direction (isotropic, or
 *                HG cosine and azimuth); w3 the next tau (-ln u), taken after the
 *                interaction's MRW chain
 *   MRW jump:    two blocks: w0 escape-time quantile P, (w1, w2) point on the
 *                sphere, w3 exit bin; then (w0, w1) new direction, w2 and w3 unused
 *   polarization: with a Mueller matrix (Sect. 2.3), a scattering takes w1 for the
 *                scattering angle (inverse CDF of S11 sin theta on the table) and w2
 *                for the azimuth of the scattering plane (inverse CDF of
 *                1 + (S12/S11)(q cos 2phi + u sin 2phi)), in place of the direction
 *                pair of the unpolarized case
 *   source:      only when the model has internal sources (viscous heating, Sect. 5):
 *                a block before the launch, w0 and w1 one uniform of 46 bits
 *                u = (w0 - 2^-24) + w1 2^-23 that picks the star (u L_tot < L_star)
 *                or the cell (the first c whose cumulative source luminosity passes
 *                u L_tot - L_star), w2 the radius (uniform in r^3 across the cell),
 *                w3 the polar position (uniform in cos theta); the star's packets
 *                then take the launch block, a cell's packet is released at that
 *                point by an absorption with omega = 0 (the interaction block: w0
 *                the BW bin, (w1, w2) direction, w3 tau)
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_H 6.62607015e-27
#define OR_C 2.99792458e10
#define OR_KB 1.380649e-16
/* Stefan-Boltzmann constant from its definition 2 pi^5 k^4 / (15 h^3 c^2) */
#define OR_SIGMA (2.0 * OR_PI * OR_PI * OR_PI * OR_PI * OR_PI * OR_KB * OR_KB * OR_KB * OR_KB / (15.0 * OR_H * OR_H * OR_H * OR_C * OR_C))
#define OR_EUNIT 65536.0 /* fixed-point counts per packet energy */
#define OR_NINC 10       /* inclination bins of the escape SED, uniform in |cos i| */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al. 2011, Sect. 4)                               */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* Weyl key schedule */
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  uint32_t buf[4];
  int pos;
} or_rng;

static void rng_init(or_rng *r, uint64_t seed, uint32_t model, uint64_t packet) {
  r->key[0] = (uint32_t)seed;
  r->key[1] = (uint32_t)(seed >> 32);
  r->ctr[0] = 0;
  r->ctr[1] = model;
  r->ctr[2] = (uint32_t)packet;
  r->ctr[3] = (uint32_t)(packet >> 32);
  r->pos = 4;
}

static double word_to_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

static double U(or_rng *r) {
  if (r->pos == 4) {
    oracle_philox4x32_10(r->ctr, r->key, r->buf);
    r->ctr[0] += 1u;
    r->pos = 0;
  }
  return word_to_uniform(r->buf[r->pos++]);
}

/* the four uniforms of the stream's next block */
static void U4(or_rng *r, double w[4]) {
  uint32_t b[4];
  oracle_philox4x32_10(r->ctr, r->key, b);
  r->ctr[0] += 1u;
  for (int i = 0; i < 4; ++i) w[i] = word_to_uniform(b[i]);
}

/* First n uniforms of the stream of (seed, model, packet); used by tests. */
void oracle_uniforms(uint64_t seed, uint32_t model, uint64_t packet, int n, double *out) {
  or_rng r;
  rng_init(&r, seed, model, packet);
  for (int i = 0; i < n; ++i) out[i] = U(&r);
}

/* ------------------------------------------------------------------------- */
/* Planck function integrated over wavelength bins                           */
/* ------------------------------------------------------------------------- */
/* Bernoulli numbers B_0..B_20 (odd ones beyond B_1 vanish). */
static const double BERN[21] = {1.0, -0.5, 1.0 / 6, 0, -1.0 / 30, 0, 1.0 / 42, 0, -1.0 / 30, 0, 5.0 / 66,
                                0, -691.0 / 2730, 0, 7.0 / 6, 0, -3617.0 / 510, 0, 43867.0 / 798, 0,
                                -174611.0 / 330};

/* G3(x) = int_x^inf t^3/(e^t-1) dt.  x >= 1: sum_n e^{-nx}(x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4);
 * x < 1: pi^4/15 - sum_k B_k x^{k+3} / (k! (k+3)) (Taylor series of t/(e^t-1)). */
double oracle_G3(double x) {
  if (x <= 0.0) return pow(OR_PI, 4) / 15.0;
  if (x >= 1.0) {
    double s = 0.0;
    for (int n = 1; n < 400; ++n) {
      double e = exp(-n * x);
      double term = e * (x * x * x / n + 3.0 * x * x / ((double)n * n) + 6.0 * x / ((double)n * n * n) +
                         6.0 / ((double)n * n * n * n));
      s += term;
      if (term < 1e-18 * s) break;
    }
    return s;
  }
  double s = 0.0, fact = 1.0;
  for (int k = 0; k <= 20; ++k) {
    if (k > 0) fact *= k;
    if (BERN[k] != 0.0) s += BERN[k] * pow(x, k + 3) / (fact * (k + 3));
  }
  return pow(OR_PI, 4) / 15.0 - s;
}

/* G4(x) = int_x^inf t^4 e^t/(e^t-1)^2 dt.  x >= 1: sum_n e^{-nx}(x^4 + 4x^3/n + 12x^2/n^2 + 24x/n^3 + 24/n^4);
 * x < 1: 4 pi^4/15 - sum_k B_k (1-k) x^{k+3} / (k! (k+3)). */
double oracle_G4(double x) {
  if (x <= 0.0) return 4.0 * pow(OR_PI, 4) / 15.0;
  if (x >= 1.0) {
    double s = 0.0;
    for (int n = 1; n < 400; ++n) {
      double e = exp(-n * x);
      double term = e * (x * x * x * x + 4.0 * x * x * x / n + 12.0 * x * x / ((double)n * n) +
                         24.0 * x / ((double)n * n * n) + 24.0 / ((double)n * n * n * n));
      s += term;
      if (term < 1e-18 * s) break;
    }
    return s;
  }
  double s = 0.0, fact = 1.0;
  for (int k = 0; k <= 20; ++k) {
    if (k > 0) fact *= k;
    if (BERN[k] != 0.0) s += BERN[k] * (1.0 - k) * pow(x, k + 3) / (fact * (k + 3));
  }
  return 4.0 * pow(OR_PI, 4) / 15.0 - s;
}

/* x at a wavelength edge: h c / (lambda k T); edge 0 is taken at lambda -> 0 and
 * edge nlam at lambda -> infinity, so the bins cover the whole spectrum. */
static double edge_x(const double *lam_e, int nlam, int e, double T) {
  if (e == 0) return INFINITY;
  if (e == nlam) return 0.0;
  return OR_H * OR_C / (lam_e[e] * 1e-4 * OR_KB * T);
}

/* Bin-integrated Planck function int_bin B_nu(T) dnu (erg s^-1 cm^-2 sr^-1), per bin. */
void oracle_planck_bins(const double *lam_e, int nlam, double T, double *out) {
  if (T <= 0.0) {
    for (int b = 0; b < nlam; ++b) out[b] = 0.0;
    return;
  }
  double pref = 2.0 * pow(OR_KB * T, 4) / (pow(OR_H, 3) * OR_C * OR_C);
  double gprev = 0.0; /* G3 at edge 0 (x = inf) */
  for (int b = 0; b < nlam; ++b) {
    double x = edge_x(lam_e, nlam, b + 1, T);
    double g = oracle_G3(x);
    out[b] = pref * (g - gprev);
    gprev = g;
  }
}

/* Bin-integrated dB_nu/dT (erg s^-1 cm^-2 sr^-1 K^-1), per bin. */
void oracle_dplanck_bins(const double *lam_e, int nlam, double T, double *out) {
  double pref = 2.0 * pow(OR_KB, 4) * T * T * T / (pow(OR_H, 3) * OR_C * OR_C);
  double gprev = 0.0;
  for (int b = 0; b < nlam; ++b) {
    double x = edge_x(lam_e, nlam, b + 1, T);
    double g = oracle_G4(x);
    out[b] = pref * (g - gprev);
    gprev = g;
  }
}

/* ------------------------------------------------------------------------- */
/* Model                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
  int nr, nt, nlam;
  const double *rf;   /* nr+1 radial faces (cm) */
  const double *tf;   /* nt+1 polar faces (rad) */
  const double *rho;  /* nr*nt, [ir*nt + it] */
  const double *lam_e;/* nlam+1 (micron) */
  const double *kabs, *ksca, *g; /* nlam */
  double Tstar, Rstar;
  const double *Lsrc; /* nr*nt internal source luminosity (erg/s) or NULL */
  /* Mueller matrix per bin for polarized transport, or NULL: [nlam][4][nmu] = S11, S12, S33, S34 at the
   * scattering angles theta_k = k pi / (nmu - 1); S22 = S11, S44 = S33 (Sect. 2.3) */
  const double *mueller;
  int nmu;
} oracle_model;

typedef struct {
  int mrw;              /* 0/1 */
  double gamma;         /* Eq. 11 */
  int nmin;             /* interactions in a cell before MRW may start */
  uint64_t max_events;  /* per packet */
  int want_sed;         /* gray dust: sample BW / exit bins only when the SED is wanted */
  int mrw_exit_dir;     /* 0 isotropic, 1 cosine-weighted outward */
} oracle_opts;

typedef struct {
  uint64_t *tally;  /* nr*nt fixed-point absorbed energy, 2^16 per packet energy */
  uint64_t *visits; /* nr*nt packet entries */
  uint64_t *nabs;   /* nr*nt absorption events */
  uint64_t *sed;    /* nlam*NINC escaped packets [lam*NINC + incl] */
  int64_t *sed_q, *sed_u; /* with a Mueller matrix: Stokes Q/I and U/I of the escaped packets in the sky
                             frame (reference: the projected disk axis), 2^20 per packet, or NULL */
  double *Tcell;    /* nr*nt current temperature (K) */
  uint64_t cnt[10]; /* packets, events, absorptions, scatterings, crossings, mrw_jumps, capped, escaped,
                       deposit_sum_lo32-free (sum of per-packet deposits), error flags */
  /* optional event trace */
  int trace_packets;     /* trace the first trace_packets packets of this call */
  int trace_max;         /* events per traced packet */
  int32_t *tr_type, *tr_cell, *tr_lam, *tr_n;
  double *tr_pos;        /* [packet][event][3] */
  /* optional path-length estimator of the mean intensity: path length (cm) per [cell][bin] of all
   * flights and MRW jumps, J = E_pkt * jtally / (4 pi V) per bin (Lucy 1999); NULL: not kept */
  double *jtally;
  /* optional escape spectrum of the packets that scattered at least once, [lam*NINC + incl]; NULL: not
   * kept */
  uint64_t *sed_sca;
} oracle_state;

enum { EV_LAUNCH = 0, EV_CROSS = 1, EV_SCATTER = 2, EV_ABSORB = 3, EV_MRW = 4, EV_ESCAPE = 5, EV_CAPPED = 6 };
enum { CNT_PACKETS, CNT_EVENTS, CNT_ABS, CNT_SCA, CNT_CROSS, CNT_MRW, CNT_CAPPED, CNT_ESCAPED, CNT_DEPSUM, CNT_ERR };

static int is_gray(const oracle_model *m) {
  for (int b = 1; b < m->nlam; ++b)
    if (m->kabs[b] != m->kabs[0] || m->ksca[b] != m->ksca[0] || m->g[b] != m->g[0]) return 0;
  return 1;
}

static double cell_volume(const oracle_model *m, int ir, int it) {
  double r1 = m->rf[ir], r2 = m->rf[ir + 1];
  return 2.0 * OR_PI / 3.0 * (r2 * r2 * r2 - r1 * r1 * r1) * (cos(m->tf[it]) - cos(m->tf[it + 1]));
}

/* Absorbed luminosity per unit mass -> temperature. Radiative equilibrium
 * 4 pi kappa_P(T) B(T) = 4 pi sum_b kappa_b Bbar_b(T) = q (Sect. 2.1, BW method). */
static double Q_of_T(const oracle_model *m, double T, double *Bb) {
  oracle_planck_bins(m->lam_e, m->nlam, T, Bb);
  double s = 0.0;
  for (int b = 0; b < m->nlam; ++b) s += m->kabs[b] * Bb[b];
  return 4.0 * OR_PI * s;
}

static double dQ_of_T(const oracle_model *m, double T, double *Bb) {
  oracle_dplanck_bins(m->lam_e, m->nlam, T, Bb);
  double s = 0.0;
  for (int b = 0; b < m->nlam; ++b) s += m->kabs[b] * Bb[b];
  return 4.0 * OR_PI * s;
}

double oracle_T_of_q(const oracle_model *m, double q) {
  if (!(q > 0.0)) return 0.0;
  if (is_gray(m)) return pow(q / (4.0 * OR_SIGMA * m->kabs[0]), 0.25);
  double *Bb = (double *)malloc(sizeof(double) * m->nlam);
  double lo = 1e-3, hi = 1e7;
  while (Q_of_T(m, hi, Bb) < q) hi *= 10.0;
  while (lo > 1e-300 && Q_of_T(m, lo, Bb) > q) lo *= 0.1;
  double T = pow(q / (4.0 * OR_SIGMA * m->kabs[0]), 0.25);
  if (!(T > lo && T < hi)) T = sqrt(lo * hi);
  for (int it = 0; it < 200; ++it) {
    double f = Q_of_T(m, T, Bb) - q;
    if (f > 0) hi = T; else lo = T;
    double d = dQ_of_T(m, T, Bb);
    double Tn = T - f / d;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    if (fabs(Tn - T) <= 1e-15 * T) { T = Tn; break; }
    T = Tn;
  }
  free(Bb);
  return T;
}

static double star_lum(const oracle_model *m) {
  return 4.0 * OR_PI * m->Rstar * m->Rstar * OR_SIGMA * pow(m->Tstar, 4);
}

/* Luminosity the packets carry: the star plus every internal source. */
double oracle_packet_lum(const oracle_model *m) {
  double L = 0.0;
  if (m->Lsrc)
    for (int c = 0; c < m->nr * m->nt; ++c) L += m->Lsrc[c];
  return star_lum(m) + L;
}

/* Temperature of cell c from its fixed-point tally; L_abs = tally/EUNIT * Lpkt/N (Lpkt: the
 * luminosity the packets carry). A cell's own source releases count as absorbed energy, so the
 * balance is emission = absorption + heating. */
static double cell_T(const oracle_model *m, int c, uint64_t tally, double n_total, double Lpkt) {
  if (tally == 0) return 0.0;
  int ir = c / m->nt, it = c % m->nt;
  double mass = m->rho[c] * cell_volume(m, ir, it);
  double Labs = ((double)tally / OR_EUNIT) * Lpkt / n_total;
  return oracle_T_of_q(m, Labs / mass);
}

/* Per-cell temperature and statistical error 1/(4 sqrt(N_abs,eq)). */
void oracle_temperatures(const oracle_model *m, const uint64_t *tally, double n_total, double *T, double *relerr) {
  const double Lpkt = oracle_packet_lum(m);
  for (int c = 0; c < m->nr * m->nt; ++c) {
    T[c] = (m->rho[c] > 0.0) ? cell_T(m, c, tally[c], n_total, Lpkt) : 0.0;
    if (relerr) {
      double n = (double)tally[c] / OR_EUNIT;
      relerr[c] = n > 0 ? 0.25 / sqrt(n) : INFINITY;
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Diffusion coefficient and mean opacities, Sect. 2.2.3                     */
/* ------------------------------------------------------------------------- */
/* chi' = kappa + (1-g) sigma: isotropic-equivalent extinction, Eq. 16 with g' = 0. */
static double chi_prime(const oracle_model *m, int b) { return m->kabs[b] + (1.0 - m->g[b]) * m->ksca[b]; }

/* Iterate Eq. 13 as written, from the initial guess eta = kappa dB/dT. The right-hand
 * side is affine in eta (the ratio term is scale free, the scattering term is not), so the
 * iterate is not rescaled; at the fixed point sum eta = sum kappa dB/dT. */
void oracle_eta_iterate(const oracle_model *m, double T, int iters, double *eta) {
  int n = m->nlam;
  double *dB = (double *)malloc(sizeof(double) * n), *nxt = (double *)malloc(sizeof(double) * n);
  oracle_dplanck_bins(m->lam_e, n, T, dB);
  for (int b = 0; b < n; ++b) eta[b] = m->kabs[b] * dB[b];
  for (int k = 0; k < iters; ++k) {
    double num = 0.0, den = 0.0;
    for (int b = 0; b < n; ++b) { num += eta[b] * m->kabs[b] / chi_prime(m, b); den += eta[b]; }
    double ratio = num / den, diff = 0.0, scale = 0.0;
    for (int b = 0; b < n; ++b) {
      double sig = (1.0 - m->g[b]) * m->ksca[b];
      nxt[b] = m->kabs[b] * dB[b] * ratio + sig / chi_prime(m, b) * eta[b];
    }
    for (int b = 0; b < n; ++b) {
      diff = fmax(diff, fabs(nxt[b] - eta[b]));
      scale = fmax(scale, fabs(nxt[b]));
      eta[b] = nxt[b];
    }
    if (diff <= 1e-17 * scale) break;
  }
  free(dB);
  free(nxt);
}

/* D (cm^2 per unit c t) from Eq. 12, 14, 15, and kappa_bar from Eq. 10, at density rho. */
void oracle_diffusion(const oracle_model *m, double T, double rho, double *D, double *kbar) {
  int n = m->nlam;
  if (is_gray(m)) {
    *D = 1.0 / (3.0 * rho * chi_prime(m, 0));
    *kbar = m->kabs[0];
    return;
  }
  double *eta = (double *)malloc(sizeof(double) * n);
  oracle_eta_iterate(m, T, 500, eta);
  double d1 = 0.0, d2 = 0.0, e0 = 0.0, kn = 0.0, kd = 0.0;
  for (int b = 0; b < n; ++b) {
    double chi = chi_prime(m, b);
    e0 += eta[b];
    d1 += eta[b] / (rho * chi);
    d2 += eta[b] / (rho * rho * chi * chi);
    kn += m->kabs[b] / chi * eta[b];
    kd += eta[b] / chi;
  }
  double avd = d1 / e0, avd2 = 2.0 * d2 / e0;
  *D = avd2 / (6.0 * avd);
  *kbar = kn / kd;
  free(eta);
}

/* ------------------------------------------------------------------------- */
/* MRW escape-time law, Eq. 7-8                                              */
/* ------------------------------------------------------------------------- */
/* P(x) = 2 sum_{n>=1} (-1)^{n+1} y^{n^2}, y = exp(-pi^2 x), x = D c t / R0^2. */
double oracle_mrw_P(double x) {
  if (x <= 0.0) return 1.0;
  double s = 0.0;
  for (int n = 1; n < 100000; ++n) {
    double term = exp(-(double)n * n * OR_PI * OR_PI * x);
    s += (n & 1) ? term : -term;
    if (term < 1e-300 || term < 1e-19 * fabs(s)) break;
  }
  return 2.0 * s;
}

/* Solve P(x) = P0 by bisection. */
double oracle_mrw_x(double P0) {
  double lo = 0.0, hi = 1.0;
  while (oracle_mrw_P(hi) > P0) hi *= 2.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (oracle_mrw_P(mid) > P0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------- */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------- */
static int is_midplane_face(double th) { return fabs(th - 0.5 * OR_PI) < 1e-12; }

/* Distance along u from p to the sphere |x| = R where the ray leaves the ball: the larger
 * root of s^2 + 2 b s + c = 0 (b = p.u, c = |p|^2 - R^2), from the cancellation-free pair
 * q = -(b + sign(b) sqrt(b^2 - c)) and c/q. */
static double sphere_far(const double p[3], const double u[3], double R) {
  double b = p[0] * u[0] + p[1] * u[1] + p[2] * u[2];
  double c = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - R * R;
  double disc = b * b - c;
  if (disc < 0) disc = 0;
  double q = -(b + copysign(sqrt(disc), b));
  if (q == 0.0) return 0.0;
  double s = fmax(q, c / q);
  return s > 0 ? s : 0.0;
}

/* Distance to the sphere |x| = R hit from outside (smaller root), or infinity. */
static double sphere_near(const double p[3], const double u[3], double R) {
  double b = p[0] * u[0] + p[1] * u[1] + p[2] * u[2];
  if (!(b < 0)) return INFINITY;
  double c = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - R * R;
  double disc = b * b - c;
  if (disc < 0) return INFINITY;
  double q = -b + sqrt(disc);
  double s = c / q;
  return s > 0 ? s : 0.0;
}

/* Distance to cone face theta_f, crossing in the direction that leaves the cell.
 * G(s) = sig*(cos^2 th (x^2+y^2) - sin^2 th z^2) along the ray; G >= 0 <=> theta >= th (own nappe).
 * leaving_down = 1: cell lies at theta >= th, exit where G goes + -> -. */
static double cone_exit(const double p[3], const double u[3], double th, int leaving_down) {
  if (is_midplane_face(th)) {
    /* plane z = 0 */
    if (leaving_down) { /* cell below the plane (z < 0), exit upward */
      if (u[2] <= 0) return INFINITY;
    } else {
      if (u[2] >= 0) return INFINITY;
    }
    double s = -p[2] / u[2];
    return s > 0 ? s : 0.0;
  }
  double ct = cos(th), st = sin(th);
  double c2 = ct * ct, s2 = st * st;
  double sig = th < 0.5 * OR_PI ? 1.0 : -1.0;
  double A = sig * (c2 * (u[0] * u[0] + u[1] * u[1]) - s2 * u[2] * u[2]);
  double B = sig * (c2 * (p[0] * u[0] + p[1] * u[1]) - s2 * p[2] * u[2]);
  double C = sig * (c2 * (p[0] * p[0] + p[1] * p[1]) - s2 * p[2] * p[2]);
  double disc = B * B - A * C;
  if (disc < 0) return INFINITY;
  double q = -(B + copysign(sqrt(disc), B));
  if (q == 0.0) return INFINITY;
  double r1 = q / A, r2 = C / q;
  /* sign bit of B clear: r1 is the + -> - root; set: r2 is (signbit, not B >= 0, so that
   * B = -0 picks the root that copysign built). */
  int bpos = !signbit(B);
  double s;
  if (leaving_down) s = bpos ? r1 : r2;
  else s = bpos ? r2 : r1;
  if (!(s >= 0.0) && !(s < 0.0)) return INFINITY; /* NaN */
  if (s < 0) {
    if (s > -1e-9 * sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])) s = 0.0; /* rounding on the face */
    else return INFINITY;
  }
  double z = p[2] + s * u[2];
  if (sig * z < 0) return INFINITY; /* mirror nappe */
  return s;
}

/* Smallest distance from p to the faces of cell (ir, it), Sect. 2.2.2 (d_min of Eq. 11). */
double oracle_dmin(const oracle_model *m, const double p[3], int ir, int it) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  double rc = sqrt(p[0] * p[0] + p[1] * p[1]);
  double d = fmin(r - m->rf[ir], m->rf[ir + 1] - r);
  if (it > 0) {
    double th = m->tf[it];
    d = fmin(d, fabs(rc * cos(th) - p[2] * sin(th)));
  }
  if (it + 1 < m->nt) {
    double th = m->tf[it + 1];
    d = fmin(d, fabs(rc * cos(th) - p[2] * sin(th)));
  }
  return d > 0 ? d : 0.0;
}

/* Distance along u to the face through which the ray leaves cell (ir, it);
 * face = 0 inner sphere, 1 outer sphere, 2 lower polar face, 3 upper polar face. */
static double next_face(const oracle_model *m, const double p[3], const double u[3], int ir, int it, int *face) {
  double s_face = sphere_far(p, u, m->rf[ir + 1]);
  *face = 1;
  double sn = sphere_near(p, u, m->rf[ir]);
  if (sn < s_face) { s_face = sn; *face = 0; }
  if (it > 0) {
    double sc = cone_exit(p, u, m->tf[it], 1);
    if (sc < s_face) { s_face = sc; *face = 2; }
  }
  if (it + 1 < m->nt) {
    double sc = cone_exit(p, u, m->tf[it + 1], 0);
    if (sc < s_face) { s_face = sc; *face = 3; }
  }
  return s_face;
}

static int theta_cell(const oracle_model *m, const double p[3]) {
  double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  double mu = p[2] / r;
  int j = 0;
  for (int k = 1; k < m->nt; ++k)
    if (cos(m->tf[k]) >= mu) j = k;
  return j;
}

/* isotropic direction from two uniforms: cos(theta) = 2 u1 - 1, phi = 2 pi u2 */
static void iso_dir(double u1, double u2, double u[3]) {
  double mu = 2.0 * u1 - 1.0;
  double phi = 2.0 * OR_PI * u2;
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  u[0] = st * cos(phi);
  u[1] = st * sin(phi);
  u[2] = mu;
}

/* Rotate u by polar angle acos(mu) and azimuth phi about itself. */
static void turn(double u[3], double mu, double phi) {
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  if (fabs(u[2]) < 0.99999) {
    double w = sqrt(1.0 - u[2] * u[2]);
    double nx = st * (u[0] * u[2] * cp - u[1] * sp) / w + u[0] * mu;
    double ny = st * (u[1] * u[2] * cp + u[0] * sp) / w + u[1] * mu;
    double nz = -st * cp * w + u[2] * mu;
    u[0] = nx; u[1] = ny; u[2] = nz;
  } else {
    double sgn = u[2] > 0 ? 1.0 : -1.0;
    u[0] = st * cp;
    u[1] = st * sp;
    u[2] = sgn * mu;
  }
  double n = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] /= n; u[1] /= n; u[2] /= n;
}

/* Henyey-Greenstein cosine by inversion of its CDF. */
static double hg_mu(double g, double xi) {
  if (fabs(g) < 1e-6) return 2.0 * xi - 1.0;
  double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
  double mu = (1.0 + g * g - t * t) / (2.0 * g);
  return fmin(1.0, fmax(-1.0, mu));
}

/* ------------------------------------------------------------------------- */
/* Polarization: Stokes (q, u, v) = (Q, U, V) / I of a packet relative to a  */
/* reference unit vector e perpendicular to its direction (Q > 0: E along e) */
/* ------------------------------------------------------------------------- */
#define OR_QUNIT 1048576.0 /* fixed-point Stokes tallies: 2^20 per packet */

/* the reference of an unpolarized packet: the horizontal direction z x u (x - (x.u) u near the axis) */
static void ref_perp(const double u[3], double e[3]) {
  if (fabs(u[2]) < 0.999999) {
    e[0] = -u[1];
    e[1] = u[0];
    e[2] = 0.0;
  } else {
    e[0] = 1.0 - u[0] * u[0];
    e[1] = -u[0] * u[1];
    e[2] = -u[0] * u[2];
  }
  double n = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  e[0] /= n; e[1] /= n; e[2] /= n;
}

/* Stokes in the frame whose reference is e turned by psi about u (e' = e cos psi + (u x e) sin psi). */
static void rotate_stokes(double st[3], double psi) {
  double c = cos(2.0 * psi), s = sin(2.0 * psi);
  double q = st[0] * c + st[1] * s;
  double uu = -st[0] * s + st[1] * c;
  st[0] = q;
  st[1] = uu;
}

/* Element k (0: S11, 1: S12, 2: S33, 3: S34) of bin table t at scattering angle th, linear in theta. */
static double mueller_at(const double *t, int nmu, int k, double th) {
  double x = th / OR_PI * (nmu - 1);
  int j = (int)floor(x);
  if (j < 0) j = 0;
  if (j > nmu - 2) j = nmu - 2;
  double f = x - j;
  return (1.0 - f) * t[k * nmu + j] + f * t[k * nmu + j + 1];
}

/* Scattering angle from S11 sin(theta): cumulative by the trapezoid rule on the table's grid, inverted
 * linearly in theta within the bracketing interval. */
double oracle_pol_sample_theta(const double *S11, int nmu, double xi) {
  double *c = (double *)malloc(sizeof(double) * nmu);
  double h = OR_PI / (nmu - 1);
  c[0] = 0.0;
  for (int k = 1; k < nmu; ++k)
    c[k] = c[k - 1] + 0.5 * h * (S11[k - 1] * sin((k - 1) * h) + S11[k] * sin(k * h));
  double target = xi * c[nmu - 1], th = OR_PI;
  for (int k = 1; k < nmu; ++k) {
    if (c[k] >= target && c[k] > c[k - 1]) {
      th = (k - 1) * h + (target - c[k - 1]) / (c[k] - c[k - 1]) * h;
      break;
    }
  }
  free(c);
  return th;
}

/* Azimuth of the scattering plane from p(phi) = (1 + a (q cos 2phi + u sin 2phi)) / (2 pi): the root of
 * F(phi) = phi / (2 pi) + a (q sin 2phi + u (1 - cos 2phi)) / (4 pi) = xi by Newton steps kept inside a
 * bisection bracket (F rises monotonically from 0 to 1 on [0, 2 pi]). */
double oracle_pol_sample_phi(double a, double q, double u, double xi) {
  double lo = 0.0, hi = 2.0 * OR_PI, phi = 2.0 * OR_PI * xi;
  for (int it = 0; it < 200; ++it) {
    double F = phi / (2.0 * OR_PI) + a * (q * sin(2.0 * phi) + u * (1.0 - cos(2.0 * phi))) / (4.0 * OR_PI) - xi;
    if (F > 0) hi = phi; else lo = phi;
    double dF = (1.0 + a * (q * cos(2.0 * phi) + u * sin(2.0 * phi))) / (2.0 * OR_PI);
    double nx = dF > 0 ? phi - F / dF : 0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
    if (fabs(nx - phi) < 1e-13) { phi = nx; break; }
    phi = nx;
  }
  return phi;
}

/* One scattering with bin table t: angle from w1, plane azimuth (measured from e about u) from w2; the
 * Stokes vector is turned into the scattering plane, multiplied by the Mueller matrix and renormalised,
 * and the new reference is the in-plane direction perpendicular to the new direction. */
void oracle_pol_scatter(const double *t, int nmu, double u[3], double e[3], double st[3], double w1, double w2) {
  double th = oracle_pol_sample_theta(t, nmu, w1);
  double s11 = mueller_at(t, nmu, 0, th), s12 = mueller_at(t, nmu, 1, th);
  double s33 = mueller_at(t, nmu, 2, th), s34 = mueller_at(t, nmu, 3, th);
  double a = s11 > 0 ? s12 / s11 : 0.0;
  double phi = oracle_pol_sample_phi(a, st[0], st[1], w2);
  rotate_stokes(st, phi);
  double cp = cos(phi), sp = sin(phi), ct = cos(th), sn = sin(th);
  double uxe[3] = {u[1] * e[2] - u[2] * e[1], u[2] * e[0] - u[0] * e[2], u[0] * e[1] - u[1] * e[0]};
  double ep[3], un[3], en[3];
  for (int d = 0; d < 3; ++d) ep[d] = e[d] * cp + uxe[d] * sp;
  for (int d = 0; d < 3; ++d) un[d] = u[d] * ct + ep[d] * sn;
  for (int d = 0; d < 3; ++d) en[d] = ep[d] * ct - u[d] * sn;
  double nu = sqrt(un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
  for (int d = 0; d < 3; ++d) un[d] /= nu;
  double dot = en[0] * un[0] + en[1] * un[1] + en[2] * un[2];
  for (int d = 0; d < 3; ++d) en[d] -= dot * un[d];
  double ne = sqrt(en[0] * en[0] + en[1] * en[1] + en[2] * en[2]);
  for (int d = 0; d < 3; ++d) { u[d] = un[d]; e[d] = en[d] / ne; }
  double I = s11 + s12 * st[0];
  double Q = s12 + s11 * st[0];
  double U = s33 * st[1] + s34 * st[2];
  double V = -s34 * st[1] + s33 * st[2];
  if (I > 0) {
    st[0] = Q / I; st[1] = U / I; st[2] = V / I;
  } else {
    st[0] = st[1] = st[2] = 0.0;
  }
}

/* Stokes q, u of a packet in the sky frame of an observer along its direction u: the reference turned
 * from e to the disk axis projected on the sky (north); unchanged along the axis itself. */
void oracle_pol_observer(const double u[3], const double e[3], const double st[3], double *q, double *uu) {
  double n[3] = {-u[2] * u[0], -u[2] * u[1], 1.0 - u[2] * u[2]};
  double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  double s[3] = {st[0], st[1], st[2]};
  if (nn > 1e-12) {
    for (int d = 0; d < 3; ++d) n[d] /= nn;
    double uxe[3] = {u[1] * e[2] - u[2] * e[1], u[2] * e[0] - u[0] * e[2], u[0] * e[1] - u[1] * e[0]};
    double c = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
    double sn = uxe[0] * n[0] + uxe[1] * n[1] + uxe[2] * n[2];
    rotate_stokes(s, atan2(sn, c));
  }
  *q = s[0];
  *uu = s[1];
}

/* smallest b with cumulative(w) >= xi * total */
static int sample_bins(const double *w, int n, double xi) {
  double tot = 0.0;
  for (int b = 0; b < n; ++b) tot += w[b];
  double target = xi * tot, c = 0.0;
  for (int b = 0; b < n; ++b) {
    c += w[b];
    if (c >= target && w[b] > 0) return b;
  }
  for (int b = n - 1; b >= 0; --b)
    if (w[b] > 0) return b;
  return n - 1;
}

/* ------------------------------------------------------------------------- */
/* Transport                                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  const oracle_model *m;
  const oracle_opts *o;
  oracle_state *st;
  int gray;
  double n_total;
  double Lpkt;    /* luminosity the packets carry */
  double *w, *w2; /* nlam scratch */
  double *star_w;
  double *src_cum; /* nr*nt+1 cumulative source luminosity, or NULL */
  int pol;         /* Mueller matrix given: packets carry Stokes q, u, v and a reference vector */
  int par;         /* packet-parallel run: other threads deposit into the same tallies */
} ctx_t;

static void trace(ctx_t *x, int tp, int *ntr, int type, int cell, const double p[3], int lam) {
  oracle_state *s = x->st;
  if (tp < 0 || *ntr >= s->trace_max) return;
  int k = tp * s->trace_max + *ntr;
  s->tr_type[k] = type;
  s->tr_cell[k] = cell;
  s->tr_lam[k] = lam;
  s->tr_pos[3 * k + 0] = p[0];
  s->tr_pos[3 * k + 1] = p[1];
  s->tr_pos[3 * k + 2] = p[2];
  (*ntr)++;
  s->tr_n[tp] = *ntr;
}

/* BW re-emission bin from kappa_b [Bbar_b(T_new) - Bbar_b(T_old)]. */
static int bw_bin(ctx_t *x, double Told, double Tnew, double xi) {
  const oracle_model *m = x->m;
  oracle_planck_bins(m->lam_e, m->nlam, Tnew, x->w);
  oracle_planck_bins(m->lam_e, m->nlam, Told, x->w2);
  double tot = 0.0;
  for (int b = 0; b < m->nlam; ++b) {
    x->w[b] = m->kabs[b] * (x->w[b] - x->w2[b]);
    if (x->w[b] < 0) x->w[b] = 0;
    tot += x->w[b];
  }
  if (!(tot > 0)) {
    oracle_dplanck_bins(m->lam_e, m->nlam, fmax(Tnew, 1.0), x->w);
    for (int b = 0; b < m->nlam; ++b) x->w[b] *= m->kabs[b];
  }
  return sample_bins(x->w, m->nlam, xi);
}

/* MRW exit bin from the diffusion flux spectrum dBbar_b/dT / chi'_b. */
static int exit_bin(ctx_t *x, double T, double xi) {
  const oracle_model *m = x->m;
  oracle_dplanck_bins(m->lam_e, m->nlam, fmax(T, 1.0), x->w);
  for (int b = 0; b < m->nlam; ++b) x->w[b] /= chi_prime(m, b);
  return sample_bins(x->w, m->nlam, xi);
}

/* Adds `units` to the tally of cell c and returns the tally before it (in a packet-parallel run the
 * addition is atomic, so the returned value is the one this deposit followed). */
static uint64_t deposit(ctx_t *x, int c, uint64_t units, uint64_t *pkt_dep) {
  oracle_state *s = x->st;
  uint64_t old;
  if (x->par) {
    old = __atomic_fetch_add(&s->tally[c], units, __ATOMIC_RELAXED);
  } else {
    old = s->tally[c];
    s->tally[c] = old + units;
  }
  if (old + units < old) s->cnt[CNT_ERR] |= 1u; /* overflow */
  *pkt_dep += units;
  return old;
}

/* Temperatures of cell c before and after a deposit of `units` onto the tally value `before`: the cell's
 * temperature follows its absorbed energy (Sect. 2.1). A serial run keeps the current temperature of every
 * cell in Tcell; in a packet-parallel run the other threads move the tallies, so both are inverted from
 * the tally values of this deposit. */
static void cell_T_step(ctx_t *x, int c, uint64_t before, uint64_t units, double *Told, double *Tnew) {
  oracle_state *s = x->st;
  if (x->par) {
    *Told = cell_T(x->m, c, before, x->n_total, x->Lpkt);
    *Tnew = cell_T(x->m, c, before + units, x->n_total, x->Lpkt);
  } else {
    *Told = s->Tcell[c];
    *Tnew = cell_T(x->m, c, s->tally[c], x->n_total, x->Lpkt);
    s->Tcell[c] = *Tnew;
  }
}

/* the current temperature of cell c */
static double cell_T_now(ctx_t *x, int c) {
  if (x->par) return cell_T(x->m, c, __atomic_load_n(&x->st->tally[c], __ATOMIC_RELAXED), x->n_total, x->Lpkt);
  return x->st->Tcell[c];
}

/* The chain of MRW jumps from the packet's point in cell (ir, it) while Eq. 11 holds (Sect. 2.2.2). */
static void mrw_walk(ctx_t *x, or_rng *r, double p[3], double u[3], double e[3], double st[3], int *lam, int ir,
                     int it, uint64_t *events, int tp, int *ntr, uint64_t *dep) {
  const oracle_model *m = x->m;
  const oracle_opts *o = x->o;
  oracle_state *s = x->st;
  const int c = ir * m->nt + it;
  for (;;) {
    if (*events >= o->max_events) break;
    double dmin = oracle_dmin(m, p, ir, it);
    double T = fmax(cell_T_now(x, c), 1.0);
    double D, kbar;
    oracle_diffusion(m, T, m->rho[c], &D, &kbar);
    /* Eq. 11 with rho chi_R = 1/(3 D) */
    if (!(dmin > o->gamma * 3.0 * D)) break;
    double ja[4], jb[4];
    U4(r, ja);
    U4(r, jb);
    double x0 = oracle_mrw_x(ja[0]);
    double ct = x0 * dmin * dmin / D;           /* path length c t */
    if (s->jtally) {
      /* the walk's path length counts in J spread over the bins as Eq. 10 spreads it, by the distance
       * travelled at each frequency, eta_b / chi'_b (eta: the fixed point of Eq. 13 at the cell's
       * temperature), so that sum_b kappa_b J_b gives back the absorption of Eq. 9 */
      oracle_eta_iterate(m, T, 500, x->w);
      double tot = 0.0;
      for (int b = 0; b < m->nlam; ++b) {
        x->w[b] /= chi_prime(m, b);
        tot += x->w[b];
      }
      if (!(tot > 0)) { /* no absorption: the closed-form fixed point, eta / chi' ~ dB/dT */
        oracle_dplanck_bins(m->lam_e, m->nlam, T, x->w);
        tot = 0.0;
        for (int b = 0; b < m->nlam; ++b) tot += x->w[b];
      }
      for (int b = 0; b < m->nlam; ++b) s->jtally[(size_t)c * m->nlam + b] += ct * x->w[b] / tot;
    }
    double E = ct * m->rho[c] * kbar;             /* Eq. 9, in packet energies */
    double units = floor(E * OR_EUNIT + 0.5);
    if (units >= 1.8e19) { s->cnt[CNT_ERR] |= 2u; units = 1.8e19; }
    const uint64_t before = deposit(x, c, (uint64_t)units, dep);
    double Tb, Ta; /* before and after the deposit */
    cell_T_step(x, c, before, (uint64_t)units, &Tb, &Ta);
    double uh[3];
    iso_dir(ja[1], ja[2], uh);
    for (int d = 0; d < 3; ++d) p[d] += dmin * uh[d];
    if (o->mrw_exit_dir == 1) {
      double mu = sqrt(jb[0]);
      double phi = 2.0 * OR_PI * jb[1];
      u[0] = uh[0]; u[1] = uh[1]; u[2] = uh[2];
      turn(u, mu, phi);
    } else {
      iso_dir(jb[0], jb[1], u);
    }
    double xl = ja[3];
    if (!x->gray || o->want_sed) *lam = exit_bin(x, Ta, xl);
    if (x->pol) { /* a diffusing packet leaves the sphere unpolarized */
      st[0] = st[1] = st[2] = 0.0;
      ref_perp(u, e);
    }
    (*events)++;
    s->cnt[CNT_MRW]++;
    trace(x, tp, ntr, EV_MRW, c, p, *lam);
  }
}

static void run_packet(ctx_t *x, uint64_t k, uint64_t seed, uint32_t model, int tp) {
  const oracle_model *m = x->m;
  const oracle_opts *o = x->o;
  oracle_state *s = x->st;
  const int nt = m->nt;
  or_rng r;
  rng_init(&r, seed, model, k);
  int ntr = 0;
  uint64_t dep = 0, events = 0, crossings = 0;
  double p[3] = {0, 0, 0}, u[3], w[4];
  double e[3] = {1, 0, 0}, st[3] = {0, 0, 0}; /* polarization: reference vector and Stokes q, u, v */
  int ir = -1, it = -1, ninc = 0, lam = 0, scattered = 0;
  double tau = 0.0;
  int released = 0;
  if (x->src_cum) {
    /* internal sources: the star or a cell, chosen in proportion to their luminosities */
    const int n = m->nr * nt;
    const double Lstar = star_lum(m);
    const double Ltot = Lstar + x->src_cum[n];
    U4(&r, w);
    const double us = (w[0] - 0.5 / 8388608.0) + w[1] * (1.0 / 8388608.0);
    const double t = us * Ltot;
    if (t >= Lstar) {
      const double tt = t - Lstar;
      int c = 0;
      while (c < n - 1 && !(x->src_cum[c + 1] > tt)) ++c;
      while (c > 0 && !(x->src_cum[c + 1] > x->src_cum[c])) --c; /* rounding past the end: the last source */
      ir = c / nt;
      it = c % nt;
      /* a point uniform in the cell's volume (at azimuth 0: the grid is axisymmetric) */
      const double r1 = m->rf[ir], r2 = m->rf[ir + 1];
      const double rr = cbrt(r1 * r1 * r1 + w[2] * (r2 * r2 * r2 - r1 * r1 * r1));
      const double c1 = cos(m->tf[it]), c2 = cos(m->tf[it + 1]);
      const double mu = c1 + w[3] * (c2 - c1);
      p[0] = rr * sqrt(1.0 - mu * mu);
      p[1] = 0.0;
      p[2] = rr * mu;
      s->visits[c]++;
      trace(x, tp, &ntr, EV_LAUNCH, c, p, lam);
      s->cnt[CNT_PACKETS]++;
      /* the release: an absorption with omega = 0 at that point */
      U4(&r, w);
      const uint64_t before = deposit(x, c, (uint64_t)OR_EUNIT, &dep);
      s->nabs[c]++;
      double Told, Tnew;
      cell_T_step(x, c, before, (uint64_t)OR_EUNIT, &Told, &Tnew);
      if (!x->gray || o->want_sed) lam = bw_bin(x, Told, Tnew, w[0]);
      iso_dir(w[1], w[2], u);
      if (x->pol) ref_perp(u, e);
      s->cnt[CNT_ABS]++;
      trace(x, tp, &ntr, EV_ABSORB, c, p, lam);
      events++;
      ninc++;
      if (o->mrw && ninc >= o->nmin) mrw_walk(x, &r, p, u, e, st, &lam, ir, it, &events, tp, &ntr, &dep);
      released = 1;
      if (events >= o->max_events) {
        s->cnt[CNT_CAPPED]++;
        trace(x, tp, &ntr, EV_CAPPED, c, p, lam);
        s->cnt[CNT_EVENTS] += events;
        s->cnt[CNT_DEPSUM] += dep;
        return;
      }
      tau = -log(w[3]);
    }
  }
  if (!released) {
    U4(&r, w);
    lam = sample_bins(x->star_w, m->nlam, w[0]);
    iso_dir(w[1], w[2], u);
    if (x->pol) ref_perp(u, e);
    trace(x, tp, &ntr, EV_LAUNCH, -1, p, lam);
    tau = -log(w[3]);
    s->cnt[CNT_PACKETS]++;
  }
  for (;;) {
    if (++crossings > 4000000000ull) { s->cnt[CNT_ERR] |= 4u; s->cnt[CNT_CAPPED]++; break; }
    if (ir < 0) {
      /* inner cavity: free flight out to r_in */
      double sf = sphere_far(p, u, m->rf[0]);
      for (int d = 0; d < 3; ++d) p[d] += sf * u[d];
      ir = 0;
      it = theta_cell(m, p);
      ninc = 0;
      s->visits[ir * nt + it]++;
      s->cnt[CNT_CROSS]++;
      trace(x, tp, &ntr, EV_CROSS, ir * nt + it, p, lam);
      continue;
    }
    int c = ir * nt + it;
    double chi = m->kabs[lam] + m->ksca[lam];
    double alpha = m->rho[c] * chi;
    int face;
    double s_face = next_face(m, p, u, ir, it, &face);
    double s_int = alpha > 0 ? tau / alpha : INFINITY;
    if (s_int < s_face) {
      for (int d = 0; d < 3; ++d) p[d] += s_int * u[d];
      if (s->jtally) s->jtally[(size_t)c * m->nlam + lam] += s_int;
      /* interaction */
      double omega = m->ksca[lam] / chi;
      U4(&r, w);
      if (w[0] < omega && x->pol) {
        oracle_pol_scatter(m->mueller + (size_t)lam * 4 * m->nmu, m->nmu, u, e, st, w[1], w[2]);
        scattered = 1;
        s->cnt[CNT_SCA]++;
        trace(x, tp, &ntr, EV_SCATTER, c, p, lam);
      } else if (w[0] < omega) {
        double g = m->g[lam];
        scattered = 1;
        if (g != 0.0) {
          double mu = hg_mu(g, w[1]);
          double phi = 2.0 * OR_PI * w[2];
          turn(u, mu, phi);
        } else {
          iso_dir(w[1], w[2], u);
        }
        s->cnt[CNT_SCA]++;
        trace(x, tp, &ntr, EV_SCATTER, c, p, lam);
      } else {
        const uint64_t before = deposit(x, c, (uint64_t)OR_EUNIT, &dep);
        s->nabs[c]++;
        double Told, Tnew;
        cell_T_step(x, c, before, (uint64_t)OR_EUNIT, &Told, &Tnew);
        double xl = (w[0] - omega) / (1.0 - omega);
        if (!x->gray || o->want_sed) lam = bw_bin(x, Told, Tnew, xl);
        iso_dir(w[1], w[2], u);
        if (x->pol) { /* re-emission is unpolarized */
          st[0] = st[1] = st[2] = 0.0;
          ref_perp(u, e);
        }
        s->cnt[CNT_ABS]++;
        trace(x, tp, &ntr, EV_ABSORB, c, p, lam);
      }
      events++;
      ninc++;
      /* modified random walk, Sect. 2.2.2 */
      if (o->mrw && ninc >= o->nmin) mrw_walk(x, &r, p, u, e, st, &lam, ir, it, &events, tp, &ntr, &dep);
      if (events >= o->max_events) {
        s->cnt[CNT_CAPPED]++;
        trace(x, tp, &ntr, EV_CAPPED, c, p, lam);
        break;
      }
      tau = -log(w[3]);
    } else {
      for (int d = 0; d < 3; ++d) p[d] += s_face * u[d];
      if (s->jtally && alpha > 0) s->jtally[(size_t)c * m->nlam + lam] += s_face;
      tau -= alpha * s_face;
      if (tau < 0) tau = 0;
      s->cnt[CNT_CROSS]++;
      if (face == 1) ir++;
      else if (face == 0) ir--;
      else if (face == 2) it--;
      else it++;
      if (ir >= m->nr) {
        double az = fabs(u[2]);
        int ib = (int)(az * OR_NINC);
        if (ib >= OR_NINC) ib = OR_NINC - 1;
        s->sed[lam * OR_NINC + ib]++;
        if (s->sed_sca && scattered) s->sed_sca[lam * OR_NINC + ib]++;
        if (x->pol) {
          double qo, uo;
          oracle_pol_observer(u, e, st, &qo, &uo);
          s->sed_q[lam * OR_NINC + ib] += (int64_t)floor(qo * OR_QUNIT + 0.5);
          s->sed_u[lam * OR_NINC + ib] += (int64_t)floor(uo * OR_QUNIT + 0.5);
        }
        s->cnt[CNT_ESCAPED]++;
        trace(x, tp, &ntr, EV_ESCAPE, -1, p, lam);
        break;
      }
      if (ir < 0) {
        trace(x, tp, &ntr, EV_CROSS, -1, p, lam);
        continue;
      }
      ninc = 0;
      s->visits[ir * nt + it]++;
      trace(x, tp, &ntr, EV_CROSS, ir * nt + it, p, lam);
    }
  }
  s->cnt[CNT_EVENTS] += events;
  s->cnt[CNT_DEPSUM] += dep;
}

/* Run packets first_id .. first_id+n-1. n_total sets the packet energy Lstar/n_total.
 * The tallies and Tcell carry over between calls (resume). Returns 0. */
static void ctx_init(ctx_t *x, const oracle_model *m, const oracle_opts *o, oracle_state *s, uint64_t n_total,
                     int par) {
  x->m = m;
  x->o = o;
  x->st = s;
  x->gray = is_gray(m);
  x->n_total = (double)n_total;
  x->Lpkt = oracle_packet_lum(m);
  x->pol = m->mueller != NULL && m->nmu >= 2 && s->sed_q != NULL && s->sed_u != NULL;
  x->par = par;
  x->src_cum = NULL;
  if (m->Lsrc) {
    const int n = m->nr * m->nt;
    x->src_cum = (double *)malloc(sizeof(double) * (n + 1));
    x->src_cum[0] = 0.0;
    for (int c = 0; c < n; ++c) x->src_cum[c + 1] = x->src_cum[c] + m->Lsrc[c];
    if (!(x->src_cum[n] > 0.0)) {
      free(x->src_cum);
      x->src_cum = NULL;
    }
  }
  x->w = (double *)malloc(sizeof(double) * m->nlam);
  x->w2 = (double *)malloc(sizeof(double) * m->nlam);
  x->star_w = (double *)malloc(sizeof(double) * m->nlam);
  oracle_planck_bins(m->lam_e, m->nlam, m->Tstar, x->star_w);
}

static void ctx_free(ctx_t *x) {
  free(x->w);
  free(x->w2);
  free(x->star_w);
  free(x->src_cum);
}

int oracle_run(const oracle_model *m, const oracle_opts *o, oracle_state *s, uint64_t n, uint64_t first_id,
               uint64_t n_total, uint64_t seed, uint32_t model) {
  ctx_t x;
  ctx_init(&x, m, o, s, n_total, 0);
  for (uint64_t i = 0; i < n; ++i) {
    int tp = (i < (uint64_t)s->trace_packets) ? (int)i : -1;
    run_packet(&x, first_id + i, seed, model, tp);
  }
  ctx_free(&x);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Packet-parallel runs: the same packets on several host threads, for the    */
/* CPU baseline's timing and for runs too long for one core. The threads take */
/* chunks of packet ids from a shared counter; the energy tallies are shared  */
/* and added to atomically (integers, so the sums do not depend on the order), */
/* every other count is kept per thread and summed at the end. For gray dust  */
/* the trajectories do not depend on the temperatures, so the tallies, counts */
/* and escapes per inclination equal the serial run's bit for bit (only the   */
/* wavelength bins drawn at re-emission follow the order of the deposits);    */
/* for non-gray dust each re-emission sees the tally that its own deposit     */
/* followed, which another thread may have moved since the serial order would */
/* have it.                                                                   */
/* ------------------------------------------------------------------------- */
typedef struct {
  const oracle_model *m;
  const oracle_opts *o;
  oracle_state st; /* this thread's counts; the tally pointer is the shared one */
  uint64_t n, first_id, n_total, seed;
  uint32_t model;
  uint64_t *next;  /* shared: the next packet index to hand out */
  char pad[256];   /* keeps the counters of neighbouring threads off each other's cache lines */
} par_job;

#define OR_PAR_CHUNK 16

static void *par_worker(void *arg) {
  par_job *j = (par_job *)arg;
  ctx_t x;
  ctx_init(&x, j->m, j->o, &j->st, j->n_total, 1);
  for (;;) {
    const uint64_t i0 = __atomic_fetch_add(j->next, (uint64_t)OR_PAR_CHUNK, __ATOMIC_RELAXED);
    if (i0 >= j->n) break;
    const uint64_t i1 = i0 + OR_PAR_CHUNK < j->n ? i0 + OR_PAR_CHUNK : j->n;
    for (uint64_t i = i0; i < i1; ++i) run_packet(&x, j->first_id + i, j->seed, j->model, -1);
  }
  ctx_free(&x);
  return NULL;
}

/* oracle_run on `threads` host threads. No event trace or mean-intensity tally (returns -1 if asked). The
 * cell temperatures Tcell are set from the final tallies, so that a serial run may continue. */
int oracle_run_par(const oracle_model *m, const oracle_opts *o, oracle_state *s, uint64_t n, uint64_t first_id,
                   uint64_t n_total, uint64_t seed, uint32_t model, int threads) {
  if (threads < 1 || s->trace_packets > 0 || s->jtally) return -1;
  const size_t nc = (size_t)m->nr * m->nt, ns = (size_t)m->nlam * OR_NINC;
  par_job *jobs = (par_job *)aligned_alloc(256, ((sizeof(par_job) * (size_t)threads + 255) / 256) * 256);
  memset(jobs, 0, sizeof(par_job) * (size_t)threads);
  pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
  uint64_t next = 0;
  /* gray dust without an escape spectrum: no temperature steers a packet (D and kappa_bar are constants,
   * no re-emission bin is drawn), so every thread deposits into a tally of its own, added at the end,
   * instead of contending for the shared one */
  const int own_tally = is_gray(m) && !o->want_sed;
  for (int t = 0; t < threads; ++t) {
    par_job *j = &jobs[t];
    j->m = m;
    j->o = o;
    j->n = n;
    j->first_id = first_id;
    j->n_total = n_total;
    j->seed = seed;
    j->model = model;
    j->next = &next;
    j->st.tally = own_tally ? (uint64_t *)calloc(nc, sizeof(uint64_t)) : s->tally;
    j->st.visits = (uint64_t *)calloc(nc, sizeof(uint64_t));
    j->st.nabs = (uint64_t *)calloc(nc, sizeof(uint64_t));
    j->st.sed = (uint64_t *)calloc(ns, sizeof(uint64_t));
    j->st.sed_sca = s->sed_sca ? (uint64_t *)calloc(ns, sizeof(uint64_t)) : NULL;
    j->st.sed_q = s->sed_q ? (int64_t *)calloc(ns, sizeof(int64_t)) : NULL;
    j->st.sed_u = s->sed_u ? (int64_t *)calloc(ns, sizeof(int64_t)) : NULL;
    j->st.Tcell = NULL;
  }
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    if (pthread_create(&tid[t], NULL, par_worker, &jobs[t]) != 0) break;
    ++started;
  }
  if (started == 0) par_worker(&jobs[0]); /* no thread could be started: run them here */
  for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
  for (int t = 0; t < threads; ++t) {
    par_job *j = &jobs[t];
    for (size_t c = 0; c < nc; ++c) {
      if (own_tally) {
        const uint64_t old = s->tally[c];
        s->tally[c] = old + j->st.tally[c];
        if (s->tally[c] < old) s->cnt[CNT_ERR] |= 1u; /* overflow */
      }
      s->visits[c] += j->st.visits[c];
      s->nabs[c] += j->st.nabs[c];
    }
    if (own_tally) free(j->st.tally);
    for (size_t k = 0; k < ns; ++k) {
      s->sed[k] += j->st.sed[k];
      if (s->sed_sca) s->sed_sca[k] += j->st.sed_sca[k];
      if (s->sed_q) s->sed_q[k] += j->st.sed_q[k];
      if (s->sed_u) s->sed_u[k] += j->st.sed_u[k];
    }
    for (int k = 0; k < 10; ++k) {
      if (k == CNT_ERR) s->cnt[k] |= j->st.cnt[k];
      else s->cnt[k] += j->st.cnt[k];
    }
    free(j->st.visits);
    free(j->st.nabs);
    free(j->st.sed);
    free(j->st.sed_sca);
    free(j->st.sed_q);
    free(j->st.sed_u);
  }
  free(jobs);
  free(tid);
  const double Lpkt = oracle_packet_lum(m);
  for (size_t c = 0; c < nc; ++c) s->Tcell[c] = cell_T(m, (int)c, s->tally[c], (double)n_total, Lpkt);
  return 0;
}

/* Stellar bin of the first draw, for tests of the launch spectrum. */
int oracle_star_bin(const oracle_model *m, double xi) {
  double *w = (double *)malloc(sizeof(double) * m->nlam);
  oracle_planck_bins(m->lam_e, m->nlam, m->Tstar, w);
  int b = sample_bins(w, m->nlam, xi);
  free(w);
  return b;
}

/* Exposed for tests: face distances and HG sampling. */
double oracle_cone_exit(const double p[3], const double u[3], double th, int leaving_down) {
  return cone_exit(p, u, th, leaving_down);
}
double oracle_sphere_far(const double p[3], const double u[3], double R) { return sphere_far(p, u, R); }
double oracle_sphere_near(const double p[3], const double u[3], double R) { return sphere_near(p, u, R); }
double oracle_hg_mu(double g, double xi) { return hg_mu(g, xi); }

/* Straight ray from p (inside cell (ir, it)) along u until it leaves the grid or
 * enters the inner cavity; records up to nmax (cell, length) segments. Returns the
 * number of segments. Used by tests of the face-distance geometry. */
int oracle_march(const oracle_model *m, const double p0[3], const double u[3], int ir, int it, int nmax,
                 int32_t *cells, double *lens) {
  double p[3] = {p0[0], p0[1], p0[2]};
  int n = 0;
  while (n < nmax && ir >= 0 && ir < m->nr) {
    int face;
    double s = next_face(m, p, u, ir, it, &face);
    cells[n] = ir * m->nt + it;
    lens[n] = s;
    n++;
    for (int d = 0; d < 3; ++d) p[d] += s * u[d];
    if (face == 1) ir++;
    else if (face == 0) ir--;
    else if (face == 2) it--;
    else it++;
  }
  return n;
}
