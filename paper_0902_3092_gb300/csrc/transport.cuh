// transport.cuh -- persistent Monte Carlo packet kernel (Sect. 2.1 and 2.2.2).
//
// One thread carries one packet at a time. When its packet escapes (or is capped) the thread takes
// the next packet id from a global queue (ids handed out per warp with one atomic), so warps stay
// full until the queue drains. Per step a packet either enters a cell, interacts, or escapes:
//   * distance to interaction s = tau / (rho chi);
//   * the exact ray/face distance (two spheres, two cones or the midplane plane) is computed only
//     when s exceeds a safety distance (a lower bound of the distance to the cell boundary, kept
//     from the last d_min evaluation), so deep inside optically thick cells interactions need no
//     face arithmetic at all;
//   * interaction: scatter with the albedo (isotropic or Henyey-Greenstein), else absorb: one
//     packet energy (2^16 counts) is atomically added to the 64-bit cell tally; the returned old
//     value gives the cell temperature before and after, and the packet is re-emitted at once with
//     a wavelength from kappa_nu [B_nu(T_new) - B_nu(T_old)] (Bjorkman & Wood 2001); for gray dust,
//     where the wavelength only shapes the escape spectrum, the bin is drawn at escape instead;
//   * MRW (Sect. 2.2.2): after at least `nmin` interactions in the cell, while d_min > gamma/(rho
//     chi_R) (Eq. 11), the packet jumps to the surface of the sphere of radius R0 = d_min, the time
//     spent inside comes from the inverse of Eq. 7 (table), and E_gamma c t rho kappa_bar (Eq. 9)
//     is deposited;
//   * leaving r_out adds the packet to the escape spectrum.
// Random numbers: each packet owns a Philox4x32-10 stream (key = seed; counter = block, model, packet
// id), and every event takes the next whole block: launch (stellar bin, direction, tau), interaction
// (albedo test whose conditional value also draws the BW bin, direction, next tau), MRW jump (two
// blocks: escape-time quantile, point on the sphere, exit bin; new direction). The FP64 CPU oracle
// uses the same layout, so gray trajectories of the FP64 build match it event by event.
#pragma once
#include "common.cuh"

namespace mcrt {

template <class R>
struct Pkt;

template <class R>
struct KParams {
  DevModel<R> m0;              // the model of single-disk launches
  const DevModel<R>* models;   // batch launches: descriptors in global memory
  int nmodels;
  int mrw;                     // MRW on
  int nmin;                    // interactions in a cell before MRW
  int exit_dir;                // 0 isotropic, 1 cosine-weighted outward
  int want_lam;                // sample emission bins (1), or skip them for gray dust without SED (0)
  int refill;                  // refill finished lanes every `refill` steps
  int defer;                   // a warp runs the interaction code once this many lanes wait at one
  R gamma;
  unsigned long long total;    // packets in the queue
  unsigned long long* queue;   // queue head (global counter)
  // batch launches whose models' packets are interleaved: per chunk of 32 queue slots, model << 48 | the
  // model's first packet of the chunk (slots past a model's last packet are padding); NULL: each model's
  // packets one range of the queue (q_begin)
  const unsigned long long* qmap;
  uint64_t seed;
  unsigned long long max_events;
  unsigned long long max_steps;  // loop guard per packet
  const float* mrw_tab;        // 2*kMrwTab: x(ln u) for u <= 1/2, then 1/x(ln(1-u)) for u > 1/2
  float mrw_t0, mrw_dt;        // table abscissae t = t0 + i dt
  // packets in flight when the queue drains, handed to the tail kernel (single-disk launches)
  Pkt<R>* pool;                // one slot per thread of the launch: long packets from the front,
  unsigned* pool_ctr;          // the others from the back; [0] long, [1] others, [2] taken by the tail
  unsigned pool_cap;
  // the first packet that a step guard drops (kTripWords words, word 0 claims it; NULL: not kept)
  unsigned long long* trip;
  // debug trace (TRACE builds)
  int trace_n, trace_max;
  int32_t *tr_type, *tr_cell, *tr_lam, *tr_n;
  double* tr_pos;
  double l_unit;
};

// Per-lane packet state. The Philox key (the seed) is a launch parameter, not lane state.
template <class R>
struct Pkt {
  R px, py, pz, ux, uy, uz, tau, dsafe;
  R alpha;   // extinction per unit length in the current cell at the current wavelength
  R ialpha;  // 1 / alpha (0 where alpha = 0)
  int ir, it, lam, ninc;
  unsigned events, steps, xcross;  // interactions + jumps, all steps, crossings since the last interaction
  uint32_t model, plo, phi, blk;  // stream counter of the packet; blk: the next event's Philox block
  // gray dust: the wavelength only matters for the escape spectrum, so the bin of the last re-emission
  // is sampled at escape. 0: bin known; 1: BW bin of cell pend_cell; 2: MRW exit bin of pend_cell
  int pend_mode;
  int pend_cell;
  float pend_u;
  int tslot, ntr;
  int pend;  // 1: moved to an interaction point whose interaction has not run yet; 2: an internal
            // source's packet waiting for its release
  // polarized transport only: Stokes (Q, U, V) / I relative to the reference vector (ex, ey, ez),
  // perpendicular to the direction (Q > 0: electric field along it)
  R sq, su, sv, ex, ey, ez;
};

// packets that had taken this many steps when the queue drained go first in the tail kernel
constexpr unsigned kTailLongSteps = 20000u;
// 32-thread blocks of the tail kernel resident per SM by default (its register budget: 65536 / (32 x 20))
constexpr int kTailBlocksPerSm = 20;

// Per-lane run counters, flushed once per launch (32-bit: a lane's share of a launch stays far below 2^32)
struct Acc {
  unsigned packets, abs, sca, cross, mrw, capped, escaped, err;
  unsigned long long depsum;
  unsigned long long longest;  // (steps << 24) | (packet id & 0xffffff) of the lane's longest packet
};

// Counts a fixed-point deposit. Tally overflow is detected on the sum of all deposits instead of on
// every atomic's returned value (which would put an L2 round trip on each deposit's critical path):
// the library adds the run's deposit sum to the energy the tallies already hold, and since every
// cell's tally is at most that total, no cell wrapped while it stays below 2^64.
__device__ __forceinline__ void add_deposit(Acc& acc, unsigned long long du) {
  const unsigned long long t = acc.depsum + du;
  if (t < du) acc.err |= kErrOverflow;
  acc.depsum = t;
}

// next Philox block of a stream: one out-of-line copy, so the 10 rounds are not inlined at every draw
static __device__ __noinline__ uint4 philox_block(uint32_t blk, uint32_t model, uint32_t plo, uint32_t phi, uint32_t k0,
                                          uint32_t k1) {
  uint32_t c0 = blk, c1 = model, c2 = plo, c3 = phi;
  philox4x32_10(c0, c1, c2, c3, k0, k1);
  return make_uint4(c0, c1, c2, c3);
}

// the key of every stream of a launch
struct Key {
  uint32_t k0, k1;
};

// Sources of the packet's next event's four random words (every event takes one whole block, so an
// event's words depend only on how many events the packet had before it).
// SerialRng: each lane computes its packet's blocks itself.
struct SerialRng {
  Key key;
  static constexpr bool coop = false;
  template <class R>
  __device__ __forceinline__ uint4 next(Pkt<R>& s) {
    return philox_block(s.blk++, s.model, s.plo, s.phi, key.k0, key.k1);
  }
};

// WarpRng: all 32 lanes of a warp carry the same packet (tail kernel); lane j holds block base + j,
// computed by the 32 lanes at once whenever the packet has used the window, and an event's block is
// read from its lane by shuffles. Needs a converged warp.
struct WarpRng {
  Key key;
  uint32_t base;
  uint4 mine;
  static constexpr bool coop = true;
  template <class R>
  __device__ __forceinline__ uint4 next(Pkt<R>& s) {
    if (s.blk - base >= 32u) {
      base = s.blk;
      mine = philox_block(base + (threadIdx.x & 31u), s.model, s.plo, s.phi, key.k0, key.k1);
    }
    const int j = (int)(s.blk - base);
    ++s.blk;
    return make_uint4(__shfl_sync(0xffffffffu, mine.x, j), __shfl_sync(0xffffffffu, mine.y, j),
                      __shfl_sync(0xffffffffu, mine.z, j), __shfl_sync(0xffffffffu, mine.w, j));
  }
  // The packet's next blocks side by side, lane j holding block s.blk + j for j < count: the window the
  // lanes already hold, shifted down, while at least `need` of its blocks are unused; 32 new blocks
  // otherwise. Does not advance s.blk.
  template <class R>
  __device__ __forceinline__ uint4 window(const Pkt<R>& s, unsigned need, unsigned& count) {
    const unsigned off = s.blk - base;  // (wraps to a large value when the lanes hold no block of s)
    if (off > 32u - need) {
      base = s.blk;
      mine = philox_block(base + (threadIdx.x & 31u), s.model, s.plo, s.phi, key.k0, key.k1);
      count = 32u;
      return mine;
    }
    count = 32u - off;
    return make_uint4(__shfl_down_sync(0xffffffffu, mine.x, off), __shfl_down_sync(0xffffffffu, mine.y, off),
                      __shfl_down_sync(0xffffffffu, mine.z, off), __shfl_down_sync(0xffffffffu, mine.w, off));
  }
};

// the lane that performs a packet's memory side effects (atomics): every lane, except in a warp that
// carries one packet in all its lanes
template <class RNG>
__device__ __forceinline__ bool lead() { return !RNG::coop || (threadIdx.x & 31u) == 0u; }

// Record of the first packet dropped by a step guard: its full id, which guard, where it was and how it
// was moving, so that the packet can be replayed. Words: 0 claim, 1 packet id, 2 guard (1: step limit,
// 2: face crossings without an interaction) | 256 in the tail kernel, 3 ir, 4 itheta, 5 events, 6 steps,
// 7 crossings since the last interaction, 8-13 position and direction (FP64 bits, internal units),
// 14 optical depth left, 15 safety distance.
constexpr int kTripWords = 16;
template <class R, class RNG>
__device__ __forceinline__ void note_trip(const KParams<R>& P, const DevModel<R>& M, const Pkt<R>& s, unsigned kind) {
  if (!lead<RNG>()) return;
  atomicAdd(M.cnt + C_GUARDS, 1ull);
  unsigned long long* t = P.trip;
  if (!t || atomicCAS(t, 0ull, 1ull) != 0ull) return;
  t[1] = ((unsigned long long)s.phi << 32) | s.plo;
  t[2] = kind | (RNG::coop ? 256u : 0u);
  t[3] = (unsigned long long)(long long)s.ir;
  t[4] = (unsigned long long)(long long)s.it;
  t[5] = s.events;
  t[6] = s.steps;
  t[7] = s.xcross;
  const double v[8] = {(double)s.px, (double)s.py, (double)s.pz, (double)s.ux, (double)s.uy, (double)s.uz,
                       (double)s.tau, (double)s.dsafe};
  for (int i = 0; i < 8; ++i) t[8 + i] = (unsigned long long)__double_as_longlong(v[i]);
}

template <class R>
__device__ __forceinline__ R uni(uint32_t w) { return to_uniform<R>(w); }

template <class R>
__device__ __forceinline__ R neg_log(R u);
template <>
__device__ __forceinline__ float neg_log<float>(float u) { return -__logf(u); }
template <>
__device__ __forceinline__ double neg_log<double>(double u) { return -log(u); }

// direction (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu) with phi = 2 pi u2
template <class R>
__device__ __forceinline__ void polar_dir(R mu, R u2, R& x, R& y, R& z);
template <>
__device__ __forceinline__ void polar_dir<float>(float mu, float u2, float& x, float& y, float& z) {
  const float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
  float sp, cp;
  __sincosf(6.283185307179586f * u2 - 3.141592653589793f, &sp, &cp);  // argument in [-pi, pi]
  x = -st * cp;
  y = -st * sp;
  z = mu;
}
template <>
__device__ __forceinline__ void polar_dir<double>(double mu, double u2, double& x, double& y, double& z) {
  const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  const double phi = 2.0 * kPi * u2;
  x = st * cos(phi);
  y = st * sin(phi);
  z = mu;
}

// isotropic direction from two random words: cos theta = 2 u1 - 1, phi = 2 pi u2
template <class R>
__device__ __forceinline__ void iso_dir(uint32_t w1, uint32_t w2, R& x, R& y, R& z) {
  polar_dir<R>((R)2 * uni<R>(w1) - (R)1, uni<R>(w2), x, y, z);
}

// rotate (x,y,z) by polar angle acos(mu) and azimuth 2 pi u2 about itself
template <class R>
__device__ __forceinline__ void turn(R& x, R& y, R& z, R mu, R u2) {
  R a, b, c;
  polar_dir<R>(mu, u2, a, b, c);  // a = st cos phi, b = st sin phi
  if (fabs(z) < (R)0.99999) {
    const R w = sqrt((R)1 - z * z);
    const R iw = (R)1 / w;
    const R nx = (a * x * z - b * y) * iw + x * mu;
    const R ny = (a * y * z + b * x) * iw + y * mu;
    const R nz = -a * w + z * mu;
    x = nx; y = ny; z = nz;
  } else {
    const R sg = z > (R)0 ? (R)1 : (R)-1;
    x = a; y = b; z = sg * mu;
  }
  const R n = rsqrt_<R>(x * x + y * y + z * z);
  x *= n; y *= n; z *= n;
}

// ------------------------------------------------------------------------------------------------
// Polarization (Sect. 2.3: the full Mueller matrix of each scattering); host and device, so that the
// same code can be checked against the oracle on the CPU
// ------------------------------------------------------------------------------------------------
// the reference of an unpolarized packet: the horizontal direction z x u (x - (x.u) u near the axis)
template <class R>
__host__ __device__ __forceinline__ void pol_reset(Pkt<R>& s) {
  R ex, ey, ez;
  if (fabs(s.uz) < (R)0.999999) {
    ex = -s.uy;
    ey = s.ux;
    ez = (R)0;
  } else {
    ex = (R)1 - s.ux * s.ux;
    ey = -s.ux * s.uy;
    ez = -s.ux * s.uz;
  }
  const R n = sqrt(ex * ex + ey * ey + ez * ez);
  s.ex = ex / n;
  s.ey = ey / n;
  s.ez = ez / n;
  s.sq = s.su = s.sv = (R)0;
}

// Stokes q, u in the frame whose reference is turned by psi about the direction
template <class R>
__host__ __device__ __forceinline__ void pol_rotate(R& q, R& u, R psi) {
  const R c = cos((R)2 * psi), sn = sin((R)2 * psi);
  const R qn = q * c + u * sn;
  u = -q * sn + u * c;
  q = qn;
}

// scattering angle from the normalised cumulative S11 sin(theta) of bin lam (linear in theta between
// the grid's angles)
template <class R>
__host__ __device__ __forceinline__ R pol_theta(const DevModel<R>& M, int lam, R xi) {
  const R* c = M.mcdf + (size_t)lam * M.nmu;
  int lo = 1, hi = M.nmu - 1;  // the first k >= 1 with c[k] >= xi
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (c[mid] >= xi) hi = mid; else lo = mid + 1;
  }
  const R h = (R)3.14159265358979323846 / (R)(M.nmu - 1);
  const R d = c[lo] - c[lo - 1];
  return (R)(lo - 1) * h + (d > (R)0 ? (xi - c[lo - 1]) / d : (R)0) * h;
}

template <class R>
__host__ __device__ __forceinline__ R mueller_at(const DevModel<R>& M, int lam, int k, R th) {
  const R* t = M.mtab + ((size_t)lam * 4 + k) * M.nmu;
  R x = th / (R)3.14159265358979323846 * (R)(M.nmu - 1);
  int j = (int)floor(x);
  j = j < 0 ? 0 : (j > M.nmu - 2 ? M.nmu - 2 : j);
  const R f = x - (R)j;
  return ((R)1 - f) * t[j] + f * t[j + 1];
}

// azimuth of the scattering plane: the root of F(phi) = phi / 2pi + a (q sin 2phi + u (1 - cos 2phi)) / 4pi
// = xi by Newton steps kept inside a bisection bracket
template <class R>
__host__ __device__ __forceinline__ R pol_phi(R a, R q, R u, R xi) {
  const R tp = (R)6.283185307179586476925;
  R lo = (R)0, hi = tp, phi = tp * xi;
  for (int it = 0; it < 200; ++it) {
    const R s2 = sin((R)2 * phi), c2 = cos((R)2 * phi);
    const R F = phi / tp + a * (q * s2 + u * ((R)1 - c2)) / ((R)2 * tp) - xi;
    if (F > (R)0) hi = phi; else lo = phi;
    const R dF = ((R)1 + a * (q * c2 + u * s2)) / tp;
    R nx = dF > (R)0 ? phi - F / dF : (R)0.5 * (lo + hi);
    if (!(nx > lo && nx < hi)) nx = (R)0.5 * (lo + hi);
    if (fabs(nx - phi) < (sizeof(R) == 8 ? (R)1e-13 : (R)1e-6)) {
      phi = nx;
      break;
    }
    phi = nx;
  }
  return phi;
}

// one polarized scattering of bin lam with uniforms (w1, w2): angle, plane, Stokes update, new direction
// and reference (the in-plane direction perpendicular to the new direction)
template <class R>
__host__ __device__ __forceinline__ void pol_scatter(const DevModel<R>& M, Pkt<R>& s, R w1, R w2) {
  const R th = pol_theta(M, s.lam, w1);
  const R s11 = mueller_at(M, s.lam, 0, th), s12 = mueller_at(M, s.lam, 1, th);
  const R s33 = mueller_at(M, s.lam, 2, th), s34 = mueller_at(M, s.lam, 3, th);
  const R a = s11 > (R)0 ? s12 / s11 : (R)0;
  const R phi = pol_phi(a, s.sq, s.su, w2);
  R q = s.sq, u = s.su;
  pol_rotate(q, u, phi);
  const R cp = cos(phi), sp = sin(phi), ct = cos(th), st = sin(th);
  const R cx = s.uy * s.ez - s.uz * s.ey, cy = s.uz * s.ex - s.ux * s.ez, cz = s.ux * s.ey - s.uy * s.ex;
  const R px = s.ex * cp + cx * sp, py = s.ey * cp + cy * sp, pz = s.ez * cp + cz * sp;
  R nx = s.ux * ct + px * st, ny = s.uy * ct + py * st, nz = s.uz * ct + pz * st;
  R ex = px * ct - s.ux * st, ey = py * ct - s.uy * st, ez = pz * ct - s.uz * st;
  const R nn = sqrt(nx * nx + ny * ny + nz * nz);
  nx /= nn;
  ny /= nn;
  nz /= nn;
  const R dot = ex * nx + ey * ny + ez * nz;
  ex -= dot * nx;
  ey -= dot * ny;
  ez -= dot * nz;
  const R ne = sqrt(ex * ex + ey * ey + ez * ez);
  s.ux = nx;
  s.uy = ny;
  s.uz = nz;
  s.ex = ex / ne;
  s.ey = ey / ne;
  s.ez = ez / ne;
  const R I = s11 + s12 * q;
  const R Q = s12 + s11 * q;
  const R U = s33 * u + s34 * s.sv;
  const R V = -s34 * u + s33 * s.sv;
  if (I > (R)0) {
    s.sq = Q / I;
    s.su = U / I;
    s.sv = V / I;
  } else {
    s.sq = s.su = s.sv = (R)0;
  }
}

// Stokes q, u of an escaping packet in the sky frame (reference: the disk axis projected on the sky)
template <class R>
__host__ __device__ __forceinline__ void pol_observer(const Pkt<R>& s, R& q, R& u) {
  q = s.sq;
  u = s.su;
  R nx = -s.uz * s.ux, ny = -s.uz * s.uy, nz = (R)1 - s.uz * s.uz;
  const R nn = sqrt(nx * nx + ny * ny + nz * nz);
  if (nn > (R)1e-12) {
    nx /= nn;
    ny /= nn;
    nz /= nn;
    const R cx = s.uy * s.ez - s.uz * s.ey, cy = s.uz * s.ex - s.ux * s.ez, cz = s.ux * s.ey - s.uy * s.ex;
    const R c = s.ex * nx + s.ey * ny + s.ez * nz;
    const R sn = cx * nx + cy * ny + cz * nz;
    pol_rotate(q, u, atan2(sn, c));
  }
}

template <class R>
__device__ __forceinline__ R hg_mu(R g, R xi) {
  if (fabs(g) < (R)1e-6) return (R)2 * xi - (R)1;
  const R t = ((R)1 - g * g) / ((R)1 - g + (R)2 * g * xi);
  const R mu = ((R)1 + g * g - t * t) / ((R)2 * g);
  return fmin((R)1, fmax((R)-1, mu));
}

// inverse of the MRW survival law P(x) = u (Eq. 7-8) from the two tables
template <class R>
__host__ __device__ __forceinline__ R mrw_x(const KParams<R>& P, R u) {
  const bool lower = u <= (R)0.5;
  const float a = lower ? (float)u : (float)((R)1 - u);
  const float t = sizeof(R) == 4 ? fast_logf(a) : logf(a);
  float f = (t - P.mrw_t0) / P.mrw_dt;
  f = fminf(fmaxf(f, 0.f), (float)(kMrwTab - 1) - 1e-3f);
  const int i = (int)f;
  const float w = f - (float)i;
  const float* T = P.mrw_tab + (lower ? 0 : kMrwTab);
  const float v = ldg(T + i) * (1.f - w) + ldg(T + i + 1) * w;
  return lower ? (R)v : (R)1 / (R)v;
}

// position on the temperature grid of the absorbed energy `tally` of cell c: interval k and weight
// w, linear in log q. tally = 0 (or below the first grid temperature) gives k = 0, w = 0.
template <class R>
__host__ __device__ __forceinline__ void qpos(const DevModel<R>& M, unsigned long long tally, int c, int& k, float& w) {
  k = 0;
  w = 0.f;
  if (tally == 0ull) return;
  const float lq = (sizeof(R) == 4 ? fast_logf((float)tally) : logf((float)tally)) + ldg(M.lqm + c) + M.lq_run;
  if (!(lq >= ldg(M.lQk + 1))) return;
  const int nT = M.nT;
  if (lq >= ldg(M.lQk + nT - 1)) {
    k = nT - 2;
    w = 1.f;
    return;
  }
  int lo = 1, hi = nT - 1;  // lQk[lo] <= lq < lQk[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ldg(M.lQk + mid) <= lq) lo = mid; else hi = mid;
  }
  k = lo;
  const float a = ldg(M.lQk + lo), b = ldg(M.lQk + lo + 1);
  w = (lq - a) / (b - a);
}

// BW re-emission bin: smallest b with D(b) >= u D(last), D the cumulative difference spectrum
// kappa [Bbar(T_new) - Bbar(T_old)] from the tabulated rows C[k] = cumulative kappa Bbar(T_k) (nT rows),
// arranged so that nearby temperatures do not cancel in FP32:
//   both in interval k:       D = the derivative spectrum at the pair's position w in the interval,
//                             linear between the derivative spectra C[j+1] - C[j] of interval k and of
//                             its neighbour on w's side (each taken at its interval's middle): second
//                             order in the grid spacing; the interval's own alone next to the grid's ends
//   adjacent intervals:       D = (1 - w_old)(C[k_old+1] - C[k_old]) + w_new (C[k_new+1] - C[k_new])
//   further apart:            D = C(T_new) - C(T_old), both interpolated
// Below the first grid temperature (k = 0) the spectrum is the one of the first interval.
static __host__ __device__ __noinline__ int sample_bw_rows(const float* __restrict__ C, int nl, int nT, int ko, float wo,
                                                           int kn, float wn, float u) {
  int mode = kn <= ko ? 0 : (kn == ko + 1 ? 1 : 2);
  // mode 0: interval j2 weighs a2 against interval kn (j2 = kn and a2 = 0 at the grid's ends, where the
  // first interval, from 0 K, is no derivative)
  const float w = kn == ko ? 0.5f * (wo + wn) : wn;
  int j2 = kn;
  float a2 = 0.f;
  if (w >= 0.5f && kn + 2 <= nT - 1) {
    j2 = kn + 1;
    a2 = w - 0.5f;
  } else if (w < 0.5f && kn >= 2) {
    j2 = kn - 1;
    a2 = 0.5f - w;
  }
  auto D = [&](int b) -> float {
    if (mode == 0) {
      const float* r = C + (size_t)kn * nl;
      const float* r2 = C + (size_t)j2 * nl;
      return (1.f - a2) * (ldg(r + nl + b) - ldg(r + b)) + a2 * (ldg(r2 + nl + b) - ldg(r2 + b));
    }
    if (mode == 1) {
      const float* ro = C + (size_t)ko * nl;
      const float c0 = ldg(ro + b), c1 = ldg(ro + nl + b), c2 = ldg(ro + 2 * nl + b);
      return (1.f - wo) * (c1 - c0) + wn * (c2 - c1);
    }
    const float* ro = C + (size_t)ko * nl;
    const float* rn = C + (size_t)kn * nl;
    return ((1.f - wn) * ldg(rn + b) + wn * ldg(rn + nl + b)) - ((1.f - wo) * ldg(ro + b) + wo * ldg(ro + nl + b));
  };
  float tot = D(nl - 1);
  if (!(tot > 0.f)) {
    mode = 0;
    tot = D(nl - 1);
  }
  const float target = u * tot;
  int lo = -1, hi = nl - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (D(mid) >= target) hi = mid; else lo = mid;
  }
  return hi;
}

// MRW exit bin from the cumulative dBbar/dT / chi' row at (k, w)
static __host__ __device__ __noinline__ int sample_exit_rows(const float* __restrict__ cexit, int nl, int k, float w, float u) {
  const float* X = cexit + (size_t)k * nl;
  auto cum = [&](int b) { return (1.f - w) * ldg(X + b) + w * ldg(X + nl + b); };
  const float target = u * cum(nl - 1);
  int lo = -1, hi = nl - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cum(mid) >= target) hi = mid; else lo = mid;
  }
  return hi;
}

template <class R>
__host__ __device__ __forceinline__ int sample_bw(const DevModel<R>& M, int ko, float wo, int kn, float wn, float u) {
  return sample_bw_rows(M.cbw, M.nlam, M.nT, ko, wo, kn, wn, u);
}

template <class R>
__host__ __device__ __forceinline__ int sample_exit(const DevModel<R>& M, int k, float w, float u) {
  return sample_exit_rows(M.cexit, M.nlam, k, w, u);
}

template <class R>
__host__ __device__ __forceinline__ int sample_star(const DevModel<R>& M, R u) {
  const int nl = M.nlam;
  const R target = u * M.star_cum[nl - 1];
  int lo = -1, hi = nl - 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (M.star_cum[mid] >= target) hi = mid; else lo = mid;
  }
  return hi;
}

template <class R, bool TRACE>
__device__ __forceinline__ void trace_ev(const KParams<R>& P, Pkt<R>& s, int type, int cell) {
  if (!TRACE) return;
  if (s.tslot < 0 || s.ntr >= P.trace_max) return;
  const size_t k = (size_t)s.tslot * P.trace_max + s.ntr;
  P.tr_type[k] = type;
  P.tr_cell[k] = cell;
  P.tr_lam[k] = s.lam;
  P.tr_pos[3 * k + 0] = (double)s.px * P.l_unit;
  P.tr_pos[3 * k + 1] = (double)s.py * P.l_unit;
  P.tr_pos[3 * k + 2] = (double)s.pz * P.l_unit;
  ++s.ntr;
  P.tr_n[s.tslot] = s.ntr;
}

// Samples a pending gray re-emission bin from the cell's tally t at the packet's escape: the BW step
// from t - EUNIT to t (the last packet energy the cell received), or the MRW exit spectrum at t. The
// tally then includes the deposits other packets made since the re-emission; waiting for each
// deposit's returned old value instead would stall every absorption for an L2 round trip.
template <class R>
__device__ __forceinline__ void resolve_pending(const DevModel<R>& M, Pkt<R>& s) {
  if (s.pend_mode == 0) return;
  const unsigned long long t = *(volatile unsigned long long*)(M.tally + s.pend_cell);
  if (s.pend_mode == 1) {
    int ko, kn;
    float wo, wn;
    qpos(M, t >= kEUnit ? t - kEUnit : 0ull, s.pend_cell, ko, wo);
    qpos(M, t, s.pend_cell, kn, wn);
    s.lam = sample_bw(M, ko, wo, kn, wn, s.pend_u);
  } else {
    int k;
    float w;
    qpos(M, t, s.pend_cell, k, w);
    s.lam = sample_exit(M, k, w, s.pend_u);
  }
  s.pend_mode = 0;
}

// extinction per unit length of the packet's cell at its wavelength
template <class R, bool G>
__device__ __forceinline__ void set_alpha(const DevModel<R>& M, Pkt<R>& s) {
  const R rho = M.rho[s.ir * M.nt + s.it];
  s.alpha = rho * ((G || M.gray) ? M.chi0 : M.chi[s.lam]);
  s.ialpha = s.alpha > (R)0 ? (R)1 / s.alpha : (R)0;
}

template <class R, bool TRACE, bool G, bool POL = false, bool JT = false, class RNG>
__device__ __forceinline__ void launch_packet(const KParams<R>& P, RNG& rng, const DevModel<R>& M, Pkt<R>& s,
                              unsigned long long k, int tslot, Acc& acc) {
  s.model = M.model_id;
  s.plo = (uint32_t)k;
  s.phi = (uint32_t)(k >> 32);
  s.blk = 0;
  if (M.n_src) {
    // internal sources (viscous heating, Sect. 5): a first block picks the star or a cell in proportion
    // to the luminosities (one 46-bit uniform from two words) and the point in the cell
    const uint4 v = rng.next(s);
    const double us = (to_uniform<double>(v.x) - 0x1p-24) + to_uniform<double>(v.y) * 0x1p-23;
    const double t = us * M.src_Ltot;
    if (t >= M.src_Lstar) {
      const double tt = t - M.src_Lstar;
      int lo = 0, hi = M.n_src - 1;  // the first cell whose cumulative luminosity passes tt
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (M.src_cum[mid + 1] > tt) hi = mid; else lo = mid + 1;
      }
      int c = lo;
      while (c > 0 && !(M.src_cum[c + 1] > M.src_cum[c])) --c;  // rounding past the end: the last source
      const int ir = c / M.nt, it = c - ir * M.nt;
      // uniform in the cell's volume: r^3 and cos(theta) uniform across the cell, azimuth 0
      const R r1 = M.rf[ir], r2 = M.rf[ir + 1];
      const R rr = cbrt(r1 * r1 * r1 + uni<R>(v.z) * (r2 * r2 * r2 - r1 * r1 * r1));
      const R c1 = M.cf[it], c2 = M.cf[it + 1];
      const R mu = c1 + uni<R>(v.w) * (c2 - c1);
      s.px = rr * sqrt((R)1 - mu * mu);
      s.py = (R)0;
      s.pz = rr * mu;
      s.ux = (R)0;
      s.uy = (R)0;
      s.uz = (R)1;
      s.ir = ir;
      s.it = it;
      s.lam = 0;
      s.ninc = 0;
      s.events = 0;
      s.steps = 0;
      s.xcross = 0;
      s.dsafe = (R)0;
      set_alpha<R, G>(M, s);
      s.pend_mode = 0;
      s.tslot = tslot;
      s.ntr = 0;
      s.tau = (R)0;
      s.pend = 2;  // the next event releases the packet: an absorption with omega = 0 at this point
      if (lead<RNG>()) atomicAdd(M.visits + c, 1ull);
      trace_ev<R, TRACE>(P, s, EV_LAUNCH, c);
      acc.packets++;
      return;
    }
  }
  const uint4 w = rng.next(s);  // stellar bin, direction, first optical depth
  s.lam = sample_star(M, uni<R>(w.x));
  iso_dir<R>(w.y, w.z, s.ux, s.uy, s.uz);
  s.px = s.py = s.pz = (R)0;
  s.ir = -1;
  s.it = -1;
  s.ninc = 0;
  s.events = 0;
  s.steps = 0;
  s.xcross = 0;
  s.dsafe = (R)0;
  s.alpha = (R)0;
  s.ialpha = (R)0;
  s.pend_mode = 0;
  s.tslot = tslot;
  s.ntr = 0;
  s.pend = 0;
  if (POL) pol_reset(s);
  trace_ev<R, TRACE>(P, s, EV_LAUNCH, -1);
  s.tau = neg_log<R>(uni<R>(w.w));
  acc.packets++;
}

// safety margin applied to d_min when it serves as the lower bound of the distance to the cell boundary
template <class R>
__device__ __forceinline__ R dsafe_margin() { return sizeof(R) == 4 ? (R)(1.0 - 1e-5) : (R)(1.0 - 1e-12); }

// Path-length estimator of the mean intensity (the scattering field of the observables, Sect. 2.3):
// every flight adds its length to the tally of its cell and bin.
template <class R, class RNG>
__device__ __forceinline__ void j_flight(const DevModel<R>& M, int c, int lam, R len) {
  if (lead<RNG>()) atomicAdd(M.jlen + (size_t)c * M.nlam + lam, (double)len);
}

// An MRW walk of path length ct in cell c adds it spread over the bins with the weights of Eq. 10 (the
// distance travelled at each frequency, eta_b / chi'_b), interpolated at the cell's T-grid position
// (k, w); the lanes of a warp that carries one packet share the bins.
template <class R, class RNG>
__device__ __forceinline__ void j_walk(const DevModel<R>& M, int c, R ct, int k, float w) {
  const float* w0 = M.jw + (size_t)k * M.nlam;
  const float* w1 = w0 + M.nlam;
  double* dst = M.jlen + (size_t)c * M.nlam;
  const int first = RNG::coop ? (int)(threadIdx.x & 31u) : 0;
  const int stride = RNG::coop ? 32 : 1;
  for (int b = first; b < M.nlam; b += stride) {
    const float wb = (1.f - w) * __ldg(w0 + b) + w * __ldg(w1 + b);
    if (wb > 0.f) atomicAdd(dst + b, (double)ct * (double)wb);
  }
}

// The faces of one cell as d_min needs them, loaded once for a chain of jumps inside the cell.
struct CellFaces {
  float rlo, rhi, cl, sl, cu, su;
  bool hasl, hasu;
};

__device__ __forceinline__ CellFaces cell_faces(const DevModel<float>& M, int ir, int it) {
  CellFaces f;
  f.rlo = M.rf[ir];
  f.rhi = M.rf[ir + 1];
  f.cl = M.cf[it];
  f.sl = M.sf[it];
  f.cu = M.cf[it + 1];
  f.su = M.sf[it + 1];
  f.hasl = M.fk[it] != 2;
  f.hasu = M.fk[it + 1] != 2;
  return f;
}

// dmin_cell<float> with the cell's faces in registers (the same arithmetic)
__device__ __forceinline__ float dmin_faces(const CellFaces& f, float px, float py, float pz) {
  const float rc2 = px * px + py * py;
  const float r = sqrtf(rc2 + pz * pz);
  const float rc = sqrtf(rc2);
  const float d0 = fminf(r - f.rlo, f.rhi - r);
  const float dl = f.hasl ? fabsf(rc * f.cl - pz * f.sl) : inf_<float>();
  const float du = f.hasu ? fabsf(rc * f.cu - pz * f.su) : inf_<float>();
  return fmaxf(fminf(d0, fminf(dl, du)), 0.f);
}

// The MRW chain of a packet that all 32 lanes of a warp carry (tail kernel; gray dust, FP32, isotropic
// direction after a jump). What a jump draws -- its escape-time quantile, the point on the sphere, the exit
// bin's uniform and the new direction -- does not depend on where the packet is, so the lanes evaluate the
// next jumps at once (lane 2k the first of jump k's two blocks, lane 2k+1 the second; up to 16 jumps
// from the blocks the lanes hold); only p <- p + d_min(p) h_k, with the Eq. 11 test at every point, runs
// jump after jump, and each jump's deposit (Eq. 9) is computed after the loop by the lane that holds its
// first block. The draws and the arithmetic of each jump are mrw_chain's; the deposits of the jumps of
// one window are one atomic.
__device__ __forceinline__ void mrw_chain_warp(const KParams<float>& P, WarpRng& rng, const DevModel<float>& M,
                                               Pkt<float>& s, int c, Acc& acc) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned full = 0xffffffffu;
  const float rho = M.rho[c];
  const float chiR = M.chiR0, kb = M.kbar0;
  const CellFaces f = cell_faces(M, s.ir, s.it);
  bool more = true;
  while (more) {
    const uint32_t blk0 = s.blk;
    unsigned m;
    const uint4 w = rng.window(s, 4u, m);
    const int kmax = (int)(m >> 1);
    // even lanes: jump k's first block (quantile, point on the sphere, exit-bin uniform); odd lanes: its
    // second block (new direction). Every lane evaluates both forms; each keeps the one it serves.
    const float x = mrw_x(P, uni<float>(w.x));
    float hx, hy, hz, nx, ny, nz;
    iso_dir<float>(w.y, w.z, hx, hy, hz);
    iso_dir<float>(w.x, w.y, nx, ny, nz);
    const float ul = uni<float>(w.w);
    int k = 0;
    more = false;
    float mydm = 0.f;  // lane 2k: d_min of jump k
    for (; k < kmax; ++k) {
      if (s.events >= P.max_events) break;
      const float dm = dmin_faces(f, s.px, s.py, s.pz);
      s.dsafe = dm * dsafe_margin<float>();
      if (!(dm * rho * chiR > P.gamma)) break;  // Eq. 11
      mydm = (int)lane == 2 * k ? dm : mydm;
      s.px += dm * __shfl_sync(full, hx, 2 * k);
      s.py += dm * __shfl_sync(full, hy, 2 * k);
      s.pz += dm * __shfl_sync(full, hz, 2 * k);
      s.events++;
      acc.mrw++;
      s.dsafe = 0.f;
      more = k == kmax - 1;
    }
    // the deposits of the jumps made (lane 2j: jump j), summed over the warp
    unsigned long long du = 0ull;
    bool clip = false;
    if ((lane & 1u) == 0u && (int)lane < 2 * k) {
      const float tau0 = mydm * rho;
      const float E = 3.f * x * tau0 * tau0 * chiR * kb;  // Eq. 9, as mrw_chain
      float units = floorf(E * (float)kEUnit + 0.5f);
      if (!(units < 1.8e19f)) {
        units = 1.8e19f;
        clip = true;
      }
      du = (unsigned long long)units;
    }
    unsigned long long dep = du;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dep += __shfl_xor_sync(full, dep, o);
    if (__any_sync(full, clip)) acc.err |= kErrMrwClip;
    if (k > 0) {
      if (lane == 0) atomicAdd(M.tally + c, dep);
      add_deposit(acc, dep);
      const int last = 2 * (k - 1);
      s.ux = __shfl_sync(full, nx, last + 1);
      s.uy = __shfl_sync(full, ny, last + 1);
      s.uz = __shfl_sync(full, nz, last + 1);
      if (P.want_lam) {  // the exit bin of the last jump, drawn at escape
        s.pend_mode = 2;
        s.pend_cell = c;
        s.pend_u = __shfl_sync(full, ul, last);
      }
      s.blk = blk0 + 2u * (unsigned)k;
    }
  }
}

template <class R, bool TRACE, bool G, bool POL = false, bool JT = false, class RNG>
__device__ __forceinline__ void mrw_chain(const KParams<R>& P, RNG& rng, const DevModel<R>& M, Pkt<R>& s, int c,
                                          Acc& acc) {
  if constexpr (RNG::coop && sizeof(R) == 4 && !TRACE && !POL && !JT) {
    if ((G || M.gray) && P.exit_dir == 0) {
      mrw_chain_warp(P, rng, M, s, c, acc);
      return;
    }
  }
  const R rho = M.rho[c];
  for (;;) {
    if (s.events >= P.max_events) break;
    const R dm = dmin_cell(M, s.ir, s.it, s.px, s.py, s.pz);
    s.dsafe = dm * dsafe_margin<R>();  // d_min at the current position bounds the next flight's face test
    R chiR, kb;
    int kq = 0;  // the cell's position on the T grid (non-gray dust, or the J weights)
    float wq = 0.f;
    if (G || M.gray) {
      chiR = M.chiR0;
      kb = M.kbar0;
      if (JT) qpos(M, *(volatile unsigned long long*)(M.tally + c), c, kq, wq);
    } else {
      qpos(M, *(volatile unsigned long long*)(M.tally + c), c, kq, wq);
      chiR = (R)((1.f - wq) * __ldg(M.chiR + kq) + wq * __ldg(M.chiR + kq + 1));
      kb = (R)((1.f - wq) * __ldg(M.kbar + kq) + wq * __ldg(M.kbar + kq + 1));
    }
    if (!(dm * rho * chiR > P.gamma)) break;  // Eq. 11
    const uint4 ja = rng.next(s);  // escape-time quantile, point on the sphere, exit bin
    const uint4 jb = rng.next(s);  // new direction
    const R x = mrw_x(P, uni<R>(ja.x));
    const R tau0 = dm * rho;
    const R E = (R)3 * x * tau0 * tau0 * chiR * kb;  // Eq. 9 with c t = x R0^2 / D, D = 1/(3 rho chi_R)
    if (JT) j_walk<R, RNG>(M, c, (R)3 * x * dm * dm * rho * chiR, kq, wq);
    R units = floor(E * (R)kEUnit + (R)0.5);
    if (!(units < (R)1.8e19)) {
      units = (R)1.8e19;
      acc.err |= kErrMrwClip;
    }
    const unsigned long long du = (unsigned long long)units;
    // the exit bin needs the tally now (the J tally needs the bin of every flight)
    const bool lam_now = P.want_lam && (!(G || M.gray) || TRACE || JT);
    unsigned long long old = 0;
    if (lam_now) {
      if (lead<RNG>()) old = atomicAdd(M.tally + c, du);
      if (RNG::coop) old = __shfl_sync(0xffffffffu, old, 0);
    } else if (lead<RNG>()) {
      atomicAdd(M.tally + c, du);
    }
    add_deposit(acc, du);
    R hx, hy, hz;
    iso_dir<R>(ja.y, ja.z, hx, hy, hz);
    s.px += dm * hx;
    s.py += dm * hy;
    s.pz += dm * hz;
    if (P.exit_dir == 1) {
      const R mu = sqrt(uni<R>(jb.x));
      const R u2 = uni<R>(jb.y);
      s.ux = hx; s.uy = hy; s.uz = hz;
      turn<R>(s.ux, s.uy, s.uz, mu, u2);
    } else {
      iso_dir<R>(jb.x, jb.y, s.ux, s.uy, s.uz);
    }
    if (POL) pol_reset(s);  // a packet leaves the diffusion sphere unpolarized
    const R ul = uni<R>(ja.w);
    if (lam_now) {
      int k;
      float w;
      qpos(M, old + du, c, k, w);
      s.lam = sample_exit(M, k, w, (float)ul);
      s.pend_mode = 0;
      if (!(G || M.gray)) set_alpha<R, G>(M, s);
    } else if (P.want_lam) {
      s.pend_mode = 2;
      s.pend_cell = c;
      s.pend_u = (float)ul;
    }
    s.events++;
    acc.mrw++;
    s.dsafe = (R)0;  // set again from d_min at the landing point by the next pass of the loop
    trace_ev<R, TRACE>(P, s, EV_MRW, c);
  }
}

// position of the (i+1)-th set bit of m (0 <= i < popc(m))
__device__ __forceinline__ int nth_set_bit(unsigned m, int i) {
  int pos = 0;
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const int c = __popc(m & ((1u << b) - 1u));
    if (c <= i) {
      i -= c;
      m >>= b;
      pos += b;
    }
  }
  return pos;
}

// The MRW chains of the lanes in `want` (one packet per lane; transport kernel, single gray FP32 disk,
// isotropic direction after a jump), made together by the whole warp: the Eq. 11 test at each chain's
// point, then the 32 lanes compute the next random blocks of every chain that goes on (up to 16 chains,
// 2 to 32 blocks each: lane j a block of chain j / per) and each chain lane makes its jumps from them, one
// after another, with the blocks read from the lanes that hold them. The draws and the arithmetic of
// every jump are mrw_chain's; a chain's deposits of one pass are one atomic. Needs a converged warp.
__device__ __forceinline__ void mrw_chains_lanes(const KParams<float>& P, const Key& key, const DevModel<float>& M,
                                                 Pkt<float>& s, Acc& acc, bool want) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned full = 0xffffffffu;
  const int c = s.ir * M.nt + s.it;
  const float rho = want ? M.rho[c] : 0.f;
  const float chiR = M.chiR0, kb = M.kbar0;
  for (;;) {
    // the test that opens each pass of mrw_chain's loop: event cap, d_min (the safety distance), Eq. 11
    float dm = 0.f;
    if (want) {
      if (s.events >= P.max_events) {
        want = false;
      } else {
        dm = dmin_cell(M, s.ir, s.it, s.px, s.py, s.pz);
        s.dsafe = dm * dsafe_margin<float>();
        want = dm * rho * chiR > P.gamma;
      }
    }
    const unsigned gm = __ballot_sync(full, want);
    if (!gm) break;
    const int k = __popc(gm);
    const int served = k < 16 ? k : 16;  // the others wait for the next pass (their test stands)
    const int per = k > 16 ? 2 : (int)((32u / (unsigned)k) & ~1u);
    const int rank = __popc(gm & ((1u << lane) - 1u));
    const int ci = (int)lane / per, co = (int)lane - ci * per;
    const int src = ci < served ? nth_set_bit(gm, ci) : (int)lane;
    const uint32_t plo = __shfl_sync(full, s.plo, src), phi = __shfl_sync(full, s.phi, src);
    const uint32_t mdl = __shfl_sync(full, s.model, src), blk = __shfl_sync(full, s.blk, src);
    const uint4 w = philox_block(blk + (uint32_t)co, mdl, plo, phi, key.k0, key.k1);
    // even slots: a jump's first block (quantile, point on the sphere, exit-bin uniform); odd: its second
    // (new direction). Every lane evaluates both forms.
    const float x = mrw_x(P, uni<float>(w.x));
    float hx, hy, hz, nx, ny, nz;
    iso_dir<float>(w.y, w.z, hx, hy, hz);
    iso_dir<float>(w.x, w.y, nx, ny, nz);
    const float ul = uni<float>(w.w);
    const int base = rank * per;
    bool go = want && rank < served;
    unsigned long long dep = 0ull;
    int kk = 0;
    for (int j = 0; j < per / 2; ++j) {
      if (go && j > 0) {
        if (s.events >= P.max_events) {
          go = false;
        } else {
          dm = dmin_cell(M, s.ir, s.it, s.px, s.py, s.pz);
          s.dsafe = dm * dsafe_margin<float>();
          go = dm * rho * chiR > P.gamma;
        }
      }
      const int sl = go ? base + 2 * j : (int)lane;
      const float xk = __shfl_sync(full, x, sl);
      const float jx = __shfl_sync(full, hx, sl), jy = __shfl_sync(full, hy, sl), jz = __shfl_sync(full, hz, sl);
      if (go) {
        const float tau0 = dm * rho;
        const float E = 3.f * xk * tau0 * tau0 * chiR * kb;  // Eq. 9, as mrw_chain
        float units = floorf(E * (float)kEUnit + 0.5f);
        if (!(units < 1.8e19f)) {
          units = 1.8e19f;
          acc.err |= kErrMrwClip;
        }
        dep += (unsigned long long)units;
        s.px += dm * jx;
        s.py += dm * jy;
        s.pz += dm * jz;
        s.events++;
        acc.mrw++;
        s.dsafe = 0.f;
        kk = j + 1;
      }
      if (!__any_sync(full, go)) break;
    }
    const int l1 = kk > 0 ? base + 2 * kk - 2 : (int)lane;
    const int l2 = kk > 0 ? l1 + 1 : (int)lane;
    const float ex = __shfl_sync(full, nx, l2), ey = __shfl_sync(full, ny, l2), ez = __shfl_sync(full, nz, l2);
    const float eu = __shfl_sync(full, ul, l1);
    if (kk > 0) {
      atomicAdd(M.tally + c, dep);
      add_deposit(acc, dep);
      s.ux = ex;
      s.uy = ey;
      s.uz = ez;
      if (P.want_lam) {  // the exit bin of the last jump, drawn at escape
        s.pend_mode = 2;
        s.pend_cell = c;
        s.pend_u = eu;
      }
      s.blk += 2u * (unsigned)kk;
    }
    // a served chain goes on only after jumps in all its slots (its next test opens the next pass)
    want = want && (rank >= served || go);
  }
}

// Crosses face `face` of the packet's cell at distance s_face along its direction (alpha: the extinction
// of the cell it leaves): the packet enters the next cell (1), or leaves the grid (0, escaped).
template <class R, bool TRACE, bool G, bool POL = false, class RNG>
__device__ __forceinline__ int cross_face(const KParams<R>& P, const DevModel<R>& M, Pkt<R>& s, Acc& acc, R s_face,
                                          int face, R alpha) {
  s.px += s_face * s.ux;
  s.py += s_face * s.uy;
  s.pz += s_face * s.uz;
  s.tau -= alpha * s_face;
  if (s.tau < (R)0) s.tau = (R)0;
  acc.cross++;
  if (face == 1) s.ir++;
  else if (face == 0) s.ir--;
  else if (face == 2) s.it--;
  else s.it++;
  if (s.ir >= M.nr) {
    if (P.want_lam) resolve_pending(M, s);
    int ib = (int)(fabs(s.uz) * (R)kNInc);
    ib = ib < kNInc ? ib : kNInc - 1;
    if (lead<RNG>()) atomicAdd(M.sed + s.lam * kNInc + ib, 1ull);
    if (POL) {
      R q, u;
      pol_observer(s, q, u);
      const long long iq = (long long)floor(q * (R)1048576 + (R)0.5), iu = (long long)floor(u * (R)1048576 + (R)0.5);
      if (lead<RNG>()) {
        atomicAdd(M.sed_q + s.lam * kNInc + ib, (unsigned long long)iq);
        atomicAdd(M.sed_u + s.lam * kNInc + ib, (unsigned long long)iu);
      }
    }
    acc.escaped++;
    trace_ev<R, TRACE>(P, s, EV_ESCAPE, -1);
    return 0;
  }
  if (s.ir < 0) {
    s.alpha = (R)0;
    s.ialpha = (R)0;
    trace_ev<R, TRACE>(P, s, EV_CROSS, -1);
    return 1;
  }
  s.ninc = 0;
  set_alpha<R, G>(M, s);
  const int cn = s.ir * M.nt + s.it;
  if (lead<RNG>()) atomicAdd(M.visits + cn, 1ull);
  trace_ev<R, TRACE>(P, s, EV_CROSS, cn);
  return 1;
}

// Moves a packet to its next event: enters the next cell (1), reaches an interaction point (2, the
// interaction itself is left to interact()), or ends (0: escaped, or a step guard).
template <class R, bool TRACE, bool G, bool POL = false, bool JT = false, class RNG>
__device__ __forceinline__ int advance(const KParams<R>& P, RNG& rng, const DevModel<R>& M, Pkt<R>& s, Acc& acc) {
  if (++s.steps > P.max_steps) {
    acc.err |= kErrStepGuard;
    acc.capped++;
    note_trip<R, RNG>(P, M, s, 1u);
    return 0;
  }
  if (s.ir < 0) {  // inner cavity: straight to r_in
    const R b = s.px * s.ux + s.py * s.uy + s.pz * s.uz;
    const R r2 = s.px * s.px + s.py * s.py + s.pz * s.pz;
    const R sf = sphere_far(b, r2 - M.rf2[0]);
    s.px += sf * s.ux;
    s.py += sf * s.uy;
    s.pz += sf * s.uz;
    s.ir = 0;
    s.it = theta_cell(M, s.px, s.py, s.pz);
    s.ninc = 0;
    s.dsafe = (R)0;
    set_alpha<R, G>(M, s);
    const int c = s.it;
    if (lead<RNG>()) atomicAdd(M.visits + c, 1ull);
    acc.cross++;
    trace_ev<R, TRACE>(P, s, EV_CROSS, c);
    return 1;
  }
  const R alpha = s.alpha;
  R s_int;
  if (!(alpha > (R)0)) s_int = inf_<R>();
  else if (sizeof(R) == 8) s_int = s.tau / alpha;  // the FP64 path divides like the CPU reference
  else s_int = s.tau * s.ialpha;
  bool hit;  // the interaction comes before the cell boundary
  R s_face = (R)0;
  int face = 1;
  if (s_int < s.dsafe) {
    hit = true;
  } else {
    // right after a face crossing the packet lies on a face, where d_min is 0: go to the face test
    const R dm = s.xcross ? (R)0 : dmin_cell(M, s.ir, s.it, s.px, s.py, s.pz) * dsafe_margin<R>();
    if (s_int < dm) {
      hit = true;
      s.dsafe = dm;
    } else {
      s_face = next_face(M, s.ir, s.it, s.px, s.py, s.pz, s.ux, s.uy, s.uz, face);
      if (sizeof(R) == 4 && s.xcross) {
        // FP32: a crossing that follows another one moves at least 1e-6 of the radius (about 16 ulps of
        // the position). A ray that grazes a face can otherwise step back and forth across it without
        // moving: at a sphere the rounded p.u says "inward" while |p| rounds onto the face, so the face
        // is met at distance 0 and the chord back out (2|p.u|) is below the position's resolution.
        const R mv = (R)1e-6 * (fabs(s.px) + fabs(s.py) + fabs(s.pz));
        s_face = s_face > mv ? s_face : mv;
      }
      hit = s_int < s_face;
      s.dsafe = (R)0;
    }
  }
  if (hit) {
    if (JT) j_flight<R, RNG>(M, s.ir * M.nt + s.it, s.lam, s_int);
    s.xcross = 0;
    s.px += s_int * s.ux;
    s.py += s_int * s.uy;
    s.pz += s_int * s.uz;
    s.dsafe = s.dsafe > s_int ? s.dsafe - s_int : (R)0;
    return 2;
  }
  // cross a face
  if (++s.xcross > 100000u) {
    acc.err |= kErrStepGuard;
    acc.capped++;
    note_trip<R, RNG>(P, M, s, 2u);
    return 0;
  }
  if (JT && alpha > (R)0) j_flight<R, RNG>(M, s.ir * M.nt + s.it, s.lam, s_face);
  return cross_face<R, TRACE, G, POL, RNG>(P, M, s, acc, s_face, face, alpha);
}

// The interaction at the packet's current point (Sect. 2.1): scattering or absorption with immediate
// re-emission, then the MRW chain (Sect. 2.2.2) and the next optical depth. A release (the first event
// of an internal source's packet) is an absorption with omega = 0. False: capped. With tau_out, the
// interaction stops after the scattering or re-emission: the caller runs the MRW chain, the cap test and
// sets the next optical depth (*tau_out).
template <class R, bool TRACE, bool G, bool POL = false, bool JT = false, class RNG>
__device__ __forceinline__ bool interact(const KParams<R>& P, RNG& rng, const DevModel<R>& M, Pkt<R>& s, Acc& acc,
                                         bool release = false, R* tau_out = nullptr) {
  const int c = s.ir * M.nt + s.it;
  const uint4 w = rng.next(s);  // albedo test, new direction, next optical depth
  const R om = release ? (R)0 : ((G || M.gray) ? M.alb0 : M.alb[s.lam]);
  const R a = uni<R>(w.x);
  const bool sca = a < om;
  const R g = sca ? ((G || M.gray) ? M.g0 : M.gq[s.lam]) : (R)0;
  const R tau_next = neg_log<R>(uni<R>(w.w));
  if (!sca) {
    const R ul = (a - om) / ((R)1 - om);  // the albedo uniform conditioned on absorption: the BW bin draw
    if (P.want_lam && (!(G || M.gray) || TRACE || JT)) {
      // the old tally sets T_old / T_new of the BW re-emission
      unsigned long long old = 0;
      if (lead<RNG>()) old = atomicAdd(M.tally + c, kEUnit);
      if (RNG::coop) old = __shfl_sync(0xffffffffu, old, 0);
      int ko, kn;
      float wo, wn;
      qpos(M, old, c, ko, wo);
      qpos(M, old + kEUnit, c, kn, wn);
      s.lam = sample_bw(M, ko, wo, kn, wn, (float)ul);
      s.pend_mode = 0;
      if (!(G || M.gray)) set_alpha<R, G>(M, s);
    } else {
      if (lead<RNG>()) atomicAdd(M.tally + c, kEUnit);  // nothing waits for the old value
      if (P.want_lam) {
        s.pend_mode = 1;
        s.pend_cell = c;
        s.pend_u = (float)ul;
      }
    }
    if (lead<RNG>()) atomicAdd(M.nabs + c, 1ull);
    add_deposit(acc, kEUnit);
    acc.abs++;
  } else {
    acc.sca++;
  }
  // new direction: Henyey-Greenstein turn for anisotropic scattering, isotropic otherwise (scattering
  // with g = 0 and re-emission share this code)
  if (POL && sca) {
    pol_scatter(M, s, uni<R>(w.y), uni<R>(w.z));  // the Mueller matrix of bin lam (Sect. 2.3)
  } else if (g != (R)0) {
    const R mu = hg_mu(g, uni<R>(w.y));
    const R u2 = uni<R>(w.z);
    turn<R>(s.ux, s.uy, s.uz, mu, u2);
  } else {
    iso_dir<R>(w.y, w.z, s.ux, s.uy, s.uz);
  }
  if (POL && !sca) pol_reset(s);  // re-emission is unpolarized
  trace_ev<R, TRACE>(P, s, sca ? EV_SCATTER : EV_ABSORB, c);
  s.events++;
  s.ninc++;
  if (tau_out) {
    *tau_out = tau_next;
    return true;
  }
  if (P.mrw && s.ninc >= P.nmin) mrw_chain<R, TRACE, G, POL, JT>(P, rng, M, s, c, acc);
  if (s.events >= P.max_events) {
    acc.capped++;
    trace_ev<R, TRACE>(P, s, EV_CAPPED, c);
    return false;
  }
  s.tau = tau_next;
  return true;
}

// One event of a packet, an interaction run at once. False when the packet has ended.
template <class R, bool TRACE, bool G, bool POL = false, bool JT = false, class RNG>
__device__ __forceinline__ bool step(const KParams<R>& P, RNG& rng, const DevModel<R>& M, Pkt<R>& s, Acc& acc) {
  if (s.pend) {
    const bool release = s.pend == 2;
    s.pend = 0;
    return interact<R, TRACE, G, POL, JT>(P, rng, M, s, acc, release);
  }
  const int r = advance<R, TRACE, G, POL, JT>(P, rng, M, s, acc);
  if (r == 2) return interact<R, TRACE, G, POL, JT>(P, rng, M, s, acc);
  return r == 1;
}

template <class R>
__device__ __forceinline__ void note_end(const Pkt<R>& s, Acc& acc) {
  const unsigned long long packed = ((unsigned long long)s.steps << 24) | (s.plo & 0xffffffu);
  if (packed > acc.longest) acc.longest = packed;
}

__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// warp sum that reports a wrap of any partial sum in `carry`
__device__ __forceinline__ unsigned long long warp_sum64_carry(unsigned long long v, bool& carry) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    carry |= v + w < v;
    v += w;
  }
  return v;
}

// adds the lane counters to the model's run counters (warp-reduced when the whole warp flushes)
template <class R>
__device__ __forceinline__ void flush(const DevModel<R>& M, Acc& acc, bool warp_uniform) {
  unsigned long long v[C_NCNT];
  v[C_PACKETS] = acc.packets;
  v[C_EVENTS] = 0;
  v[C_ABS] = acc.abs;
  v[C_SCA] = acc.sca;
  v[C_CROSS] = acc.cross;
  v[C_MRW] = acc.mrw;
  v[C_CAPPED] = acc.capped;
  v[C_ESCAPED] = acc.escaped;
  v[C_DEPSUM] = acc.depsum;
  v[C_ERR] = acc.err;
  v[C_MAXSTEPS] = acc.longest >> 24;
  v[C_LONGEST] = acc.longest;
  // the deposit sum first: a wrap of it sets the overflow bit of the error word
  {
    bool carry = false;
    unsigned long long x = v[C_DEPSUM];
    if (warp_uniform) x = warp_sum64_carry(x, carry);
    if (!warp_uniform || (threadIdx.x & 31) == 0) {
      if (x && atomicAdd(M.cnt + C_DEPSUM, x) + x < x) carry = true;
    }
    if (carry) v[C_ERR] |= kErrOverflow;
  }
#pragma unroll
  for (int i = 0; i < C_LONGEST + 1; ++i) {
    if (i == C_EVENTS || i == C_DEPSUM) continue;
    unsigned long long x = v[i];
    const bool is_max = (i == C_MAXSTEPS || i == C_LONGEST);
    if (warp_uniform) {
      if (i == C_ERR) x = __reduce_or_sync(0xffffffffu, (unsigned)x);
      else if (is_max) x = warp_max64(x);
      else x = warp_sum64(x);
      if ((threadIdx.x & 31) != 0) continue;
    }
    if (!x) continue;
    if (i == C_ERR) atomicOr(M.cnt + i, x);
    else if (is_max) atomicMax(M.cnt + i, x);
    else atomicAdd(M.cnt + i, x);
  }
  acc = Acc{};
}

// model of queue position q (batch launches): largest m with q_begin <= q
template <class R>
__device__ __forceinline__ int find_model(const KParams<R>& P, unsigned long long q) {
  int lo = 0, hi = P.nmodels;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.models[mid].q_begin <= q) lo = mid; else hi = mid;
  }
  return lo;
}

// fewest blocks a run of interactions starts from before the lanes compute a new window of 32
constexpr unsigned kMinRun = 24u;

// Several interactions of one packet at once, in a warp whose 32 lanes all carry the packet (gray,
// isotropic dust). Lane k evaluates the packet's k-th next interaction: its Philox block (the packet's
// blocks are consumed one per interaction), the flight that leads to it (direction and optical depth
// drawn at interaction k-1, lane 0: the packet's current ones) and, by a warp prefix sum of the flight
// vectors, its position. The interactions are the packet's own, with its own random blocks, up to the
// first flight that meets a cell face (the exact face distance decides, as in advance()) or the first
// interaction after which Eq. 11 starts an MRW chain; their deposits are one atomic. A run that ends at
// a face ends with that crossing, as advance() makes it, and so does a call whose first flight leaves the
// cell. False when the call did nothing (advance()'s guard on crossings is due; the caller then takes a
// normal step); sets `ended` when the packet ended (its MRW chain reached the event cap, or the crossing
// left the grid).
template <class R, bool G>
__device__ __forceinline__ bool interactions_at_once(const KParams<R>& P, WarpRng& rng, const DevModel<R>& M, Pkt<R>& s,
                                                    Acc& acc, bool& ended) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned full = 0xffffffffu;
  const int c = s.ir * M.nt + s.it;
  const R om = M.alb0;
  const R rho_c = __ldg(M.rho + c);
  // lane k: block of interaction k; what it draws for interaction k (albedo test) and for flight k+1.
  // Lanes from m on hold no block of this packet's run: the run stops at interaction m - 1 at the latest.
  const uint32_t blk0 = s.blk;
  unsigned m;
  const uint4 w = rng.window(s, kMinRun, m);
  const unsigned win = m == 32u ? full : ((1u << m) - 1u);
  const R a = uni<R>(w.x);
  R nx, ny, nz;
  iso_dir<R>(w.y, w.z, nx, ny, nz);
  const R tnext = neg_log<R>(uni<R>(w.w));
  // flight k: direction and optical depth drawn at interaction k-1
  R ux = __shfl_up_sync(full, nx, 1), uy = __shfl_up_sync(full, ny, 1), uz = __shfl_up_sync(full, nz, 1);
  R tau = __shfl_up_sync(full, tnext, 1);
  if (lane == 0) {
    ux = s.ux;
    uy = s.uy;
    uz = s.uz;
    tau = s.tau;
  }
  const R f = sizeof(R) == 8 ? tau / s.alpha : tau * s.ialpha;
  // start of flight k (exclusive prefix sum of the flight vectors) and interaction point k (inclusive)
  R qx = f * ux, qy = f * uy, qz = f * uz;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const R tx = __shfl_up_sync(full, qx, o), ty = __shfl_up_sync(full, qy, o), tz = __shfl_up_sync(full, qz, o);
    if ((int)lane >= o) {
      qx += tx;
      qy += ty;
      qz += tz;
    }
  }
  qx += s.px;
  qy += s.py;
  qz += s.pz;
  // start of flight k: interaction point k - 1 as lane k - 1 holds it (the packet's position after the
  // run), so that the face distance of a flight that leaves the cell is the one advance() would find
  R px = __shfl_up_sync(full, qx, 1), py = __shfl_up_sync(full, qy, 1), pz = __shfl_up_sync(full, qz, 1);
  if (lane == 0) {
    px = s.px;
    py = s.py;
    pz = s.pz;
  }
  // d_min at the interaction point: the MRW test there and the safety distance of the next flight
  const R dq = dmin_cell(M, s.ir, s.it, qx, qy, qz);
  R dstart = __shfl_up_sync(full, dq * dsafe_margin<R>(), 1);
  if (lane == 0) dstart = s.dsafe;
  // the face distance of every flight, whether or not d_min already decides (it overlaps with d_min)
  int face = 1;
  R sf = next_face(M, s.ir, s.it, px, py, pz, ux, uy, uz, face);
  if (sizeof(R) == 4 && lane == 0 && s.xcross) {
    // flight 0 after a crossing: advance()'s minimum move
    const R mv = (R)1e-6 * (fabs(s.px) + fabs(s.py) + fabs(s.pz));
    sf = sf > mv ? sf : mv;
  }
  const bool hit = f < dstart || f < sf;
  const unsigned miss = __ballot_sync(full, !hit) & win;
  const int h = miss ? __ffs(miss) - 1 : (int)m;  // flights 0 .. h-1 end inside the cell
  if (h == 0) {
    // the packet's flight leaves the cell: the crossing advance() would make (its face distance is lane
    // 0's), unless advance()'s guard on crossings without an interaction is due
    if (s.xcross >= 100000u) return false;
    const R s_face = __shfl_sync(full, sf, 0);
    const int fc = __shfl_sync(full, face, 0);
    s.steps++;
    s.xcross++;
    s.dsafe = (R)0;
    if (!cross_face<R, false, G, false, WarpRng>(P, M, s, acc, s_face, fc, s.alpha)) ended = true;
    return true;
  }
  const bool mrw = P.mrw && s.ninc + (int)lane + 1 >= P.nmin && dq * rho_c * M.chiR0 > P.gamma;  // Eq. 11
  const unsigned mrws = __ballot_sync(full, mrw) & (h == 32 ? full : ((1u << h) - 1u));
  const int n = mrws ? __ffs(mrws) : h;  // interactions done; an MRW chain follows interaction n-1 if mrws
  const unsigned done_mask = n == 32 ? full : ((1u << n) - 1u);
  const unsigned absm = __ballot_sync(full, !(a < om)) & done_mask;
  const int nabs = __popc(absm);
  if (nabs) {
    const unsigned long long dep = (unsigned long long)nabs * kEUnit;
    if (lane == 0) {
      atomicAdd(M.tally + c, dep);
      atomicAdd(M.nabs + c, (unsigned long long)nabs);
    }
    add_deposit(acc, dep);
    if (P.want_lam) {  // the bin of the last absorption's re-emission, drawn at escape
      const R al = __shfl_sync(full, a, 31 - __clz(absm));
      s.pend_mode = 1;
      s.pend_cell = c;
      s.pend_u = (float)((al - om) / ((R)1 - om));
    }
  }
  acc.abs += nabs;
  acc.sca += n - nabs;
  // the packet after interaction n-1
  const int l = n - 1;
  s.px = __shfl_sync(full, qx, l);
  s.py = __shfl_sync(full, qy, l);
  s.pz = __shfl_sync(full, qz, l);
  s.ux = __shfl_sync(full, nx, l);
  s.uy = __shfl_sync(full, ny, l);
  s.uz = __shfl_sync(full, nz, l);
  const R tau_next = __shfl_sync(full, tnext, l);
  s.dsafe = __shfl_sync(full, dq, l) * dsafe_margin<R>();
  s.blk = blk0 + n;
  s.events += n;
  s.steps += n;
  s.ninc += n;
  s.xcross = 0;
  if (!mrws && h < (int)m) {
    // flight h leaves the cell (h = m: the window ended, not the run): the crossing advance() would make
    // next (no interaction before the face; d_min at the start of the flight is the safety distance the
    // run's last interaction left, and the face distance is lane h's)
    const R s_face = __shfl_sync(full, sf, h);
    const int fc = __shfl_sync(full, face, h);
    s.tau = tau_next;
    s.steps++;
    s.xcross = 1;
    s.dsafe = (R)0;
    if (!cross_face<R, false, G, false, WarpRng>(P, M, s, acc, s_face, fc, s.alpha)) ended = true;
    return true;
  }
  if (mrws) {
    mrw_chain<R, false, G>(P, rng, M, s, c, acc);
    if (s.events >= P.max_events) {
      acc.capped++;
      ended = true;
      return true;
    }
  }
  s.tau = tau_next;
  return true;
}

// Tail of a transport launch (single disk or batch). When the queue drains, the packets still in flight are mostly long
// ones (a lane holds a long packet for long), and lanes of one warp that follow different branches
// share its issue slots, so in the transport kernel a long packet would then advance at a fraction of
// its speed alone. The transport kernel therefore stores them (state unchanged, so the random stream
// and the result are the same) and this kernel runs them one per warp: lane 0 of each 32-thread block
// takes packets from the pool, those that had taken at least kTailLongSteps steps first.
template <class R, bool TRACE, bool G, bool BATCH, bool POL = false, bool JT = false>
__global__ void __launch_bounds__(32, kTailBlocksPerSm) transport_tail_kernel(const KParams<R> P) {
  const unsigned lane = threadIdx.x & 31u;
  if (TRACE && lane != 0) return;  // the debug trace runs one lane per packet
  Acc acc = Acc{};
  const unsigned nlong = P.pool_ctr[0], nshort = P.pool_ctr[1];
  for (;;) {
    unsigned k = 0;
    if (lane == 0) k = atomicAdd(P.pool_ctr + 2, 1u);
    if (!TRACE) k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= nlong + nshort) break;
    Pkt<R> s = P.pool[k < nlong ? k : P.pool_cap - 1u - (k - nlong)];
    const DevModel<R>& M = BATCH ? P.models[s.model] : P.m0;  // batches: the packet's model index
    if (TRACE) {
      SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
      while (step<R, TRACE, G, POL, JT>(P, rng, M, s, acc)) {
      }
    } else {
      // all 32 lanes carry the packet: the same arithmetic in every lane, the random blocks computed
      // 32 at a time, side effects by lane 0; gray isotropic dust takes runs of interactions at once
      WarpRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}, s.blk - 32u, make_uint4(0u, 0u, 0u, 0u)};
      bool ended = false;
      for (;;) {
        // (FP32 only: the FP64 debug path keeps the oracle's order of floating-point operations)
        if (!POL && !JT && (G || M.gray) && sizeof(R) == 4 && !s.pend && s.ir >= 0 && s.alpha > (R)0 && M.g0 == (R)0 &&
            s.events + 33u < P.max_events && s.steps + 33u < P.max_steps) {
          const bool moved = interactions_at_once<R, G>(P, rng, M, s, acc, ended);
          if (ended) break;
          if (moved) continue;
        }
        if (!step<R, TRACE, G, POL, JT>(P, rng, M, s, acc)) break;
      }
    }
    if (lane == 0) {
      note_end(s, acc);
      if (BATCH) flush(M, acc, false);  // counters of the packet's model
    }
  }
  if (!BATCH && lane == 0) flush(P.m0, acc, false);
}

// resident 256-thread blocks per SM the FP32 kernel is compiled for (register budget 65536 / (256 n))
#ifndef MCRT_TRANSPORT_MIN_BLOCKS
#define MCRT_TRANSPORT_MIN_BLOCKS 3
#endif
template <class R>
constexpr int transport_min_blocks() { return sizeof(R) == 4 ? MCRT_TRANSPORT_MIN_BLOCKS : 1; }

// transport kernels whose MRW chains run warp-wide (mrw_chains_lanes): single gray FP32 disk
template <class R, bool TRACE, bool BATCH, bool G, bool POL, bool JT>
__host__ __device__ constexpr bool kLaneChains() { return sizeof(R) == 4 && !TRACE && !BATCH && G && !POL && !JT; }

// G: gray dust known at compile time (single-disk gray runs); otherwise M.gray is read at run time.
template <class R, bool TRACE, bool BATCH, bool G, bool POL = false, bool JT = false>
__global__ void __launch_bounds__(256, transport_min_blocks<R>()) transport_kernel(const KParams<R> P) {
  Pkt<R> s;
  Acc acc = Acc{};
  SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
  bool active = false, done = false;
  int model = 0;
  const unsigned lane = threadIdx.x & 31;
  int until_refill = 0;
  for (;;) {
    if (--until_refill < 0) {
      until_refill = P.refill - 1;
      const unsigned need = __ballot_sync(0xffffffffu, !active && !done);
      if (need) {
        const int leader = __ffs(need) - 1;
        unsigned long long base = 0;
        if ((int)lane == leader) base = atomicAdd(P.queue, (unsigned long long)__popc(need));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (!active && !done) {
          const unsigned long long q = base + __popc(need & ((1u << lane) - 1u));
          if (q < P.total) {
            int m = 0;
            unsigned long long local = q;
            if (BATCH) {
              if (P.qmap) {
                const unsigned long long e = __ldg(P.qmap + (q >> 5));
                m = (int)(e >> 48);
                local = (e & 0xffffffffffffull) + (q & 31ull);
              } else {
                m = find_model(P, q);
                local = q - P.models[m].q_begin;
              }
              if (m != model) {
                flush(P.models[model], acc, false);
                model = m;
              }
            }
            const DevModel<R>& M = BATCH ? P.models[m] : P.m0;
            if (local < M.n_packets) {  // (a padding slot of an interleaved queue launches nothing)
              const int tslot = (TRACE && local < (unsigned long long)P.trace_n) ? (int)local : -1;
              launch_packet<R, TRACE, G, POL, JT>(P, rng, M, s, M.first_id + local, tslot, acc);
              active = true;
            }
          } else {
            done = true;
          }
        }
      }
      if (__all_sync(0xffffffffu, done && !active)) break;
      // a lane that found the queue empty means it is empty for every lane: the packets still in
      // flight go to the tail kernel (or, without its pool, run to the end here)
      if (__any_sync(0xffffffffu, done)) {
        if (P.pool) {
          if (active) {
            const bool longp = s.steps >= kTailLongSteps;
            const unsigned k = atomicAdd(P.pool_ctr + (longp ? 0 : 1), 1u);
            const unsigned slot = longp ? k : P.pool_cap - 1u - k;  // the two ends never meet: one per thread
            P.pool[slot] = s;
          }
          break;
        }
        const DevModel<R>& M = BATCH ? P.models[model] : P.m0;
        while (active) {
          active = step<R, TRACE, G, POL, JT>(P, rng, M, s, acc);
          if (!active) note_end(s, acc);
        }
        break;
      }
    }
    // Lanes that reach an interaction point wait there until `defer` lanes of the warp (or every
    // moving lane) do, so the long interaction code runs for many lanes at once while the others
    // keep crossing cells; a packet's own sequence of events and random draws is unchanged.
    const DevModel<R>& M = BATCH ? P.models[model] : P.m0;
    if (active && !s.pend) {
      const int r = advance<R, TRACE, G, POL, JT>(P, rng, M, s, acc);
      if (r == 0) {
        active = false;
        note_end(s, acc);
      } else if (r == 2) {
        s.pend = 1;
      }
    }
    const unsigned waiting = __ballot_sync(0xffffffffu, active && s.pend);
    if (waiting) {
      const unsigned moving = __ballot_sync(0xffffffffu, active && !s.pend);
      bool batch_now = __popc(waiting) >= P.defer || !moving;
      if constexpr (kLaneChains<R, TRACE, BATCH, G, POL, JT>()) {
        if (batch_now && P.exit_dir == 0) {
          // the MRW chains that follow the interactions run warp-wide
          batch_now = false;
          const bool inter = active && s.pend;
          bool chain = false;
          R tau_next = (R)0;
          if (inter) {
            const bool release = s.pend == 2;
            s.pend = 0;
            interact<R, TRACE, G, POL, JT>(P, rng, M, s, acc, release, &tau_next);
            chain = P.mrw && s.ninc >= P.nmin;
          }
          if (__any_sync(0xffffffffu, chain)) mrw_chains_lanes(P, rng.key, M, s, acc, chain);
          if (inter) {
            if (s.events >= P.max_events) {
              acc.capped++;
              active = false;
              note_end(s, acc);
            } else {
              s.tau = tau_next;
            }
          }
        }
      }
      if (batch_now) {
        if (active && s.pend) {
          const bool release = s.pend == 2;
          s.pend = 0;
          if (!interact<R, TRACE, G, POL, JT>(P, rng, M, s, acc, release)) {
            active = false;
            note_end(s, acc);
          }
        }
      }
    }
  }
  __syncwarp();
  if (BATCH) flush(P.models[model], acc, false);
  else flush(P.m0, acc, true);
}

}  // namespace mcrt
