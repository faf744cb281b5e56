// common.cuh -- device-side building blocks shared by the transport, temperature and PDA kernels:
// counter-based random numbers, the per-disk model descriptor and the (r, theta) cell geometry.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mcrt {

constexpr unsigned long long kEUnit = 65536ull;  // fixed-point counts per packet energy
constexpr int kNInc = 10;                          // inclination bins, uniform in |cos i|
constexpr int kMrwTab = 2048;                      // entries of each MRW inverse table
constexpr double kPi = 3.14159265358979323846;

// error flag bits (mcrt_run_stats.error_flags)
constexpr unsigned kErrOverflow = 1u, kErrMrwClip = 2u, kErrStepGuard = 4u;

// Read-only load through the non-coherent cache on the device, a plain load on the host; the fast
// logarithm intrinsic on the device, logf on the host. They let table lookups be compiled for the host.
template <class T>
__host__ __device__ __forceinline__ T ldg(const T* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}
__host__ __device__ __forceinline__ float fast_logf(float x) {
#ifdef __CUDA_ARCH__
  return __logf(x);
#else
  return logf(x);
#endif
}

// event types of the debug trace
enum EventType { EV_LAUNCH = 0, EV_CROSS = 1, EV_SCATTER = 2, EV_ABSORB = 3, EV_MRW = 4, EV_ESCAPE = 5, EV_CAPPED = 6 };

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): 10 rounds of two 32x32->64 multiplies with a
// Weyl-sequence key schedule. Counter (block, model, packet_lo, packet_hi), key = seed.
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                                       uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit product gives both halves
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// One stream per packet. The four words of a block are consumed in order w0..w3 by shifting, so
// the buffer stays in registers.
struct Rng {
  uint32_t k0, k1, model, plo, phi, blk;
  uint32_t w0, w1, w2, w3;
  int left;
  __device__ __forceinline__ void init(uint64_t seed, uint32_t m, uint64_t packet) {
    k0 = (uint32_t)seed;
    k1 = (uint32_t)(seed >> 32);
    model = m;
    plo = (uint32_t)packet;
    phi = (uint32_t)(packet >> 32);
    blk = 0;
    left = 0;
  }
  __device__ __forceinline__ uint32_t next() {
    if (left == 0) {
      uint32_t c0 = blk, c1 = model, c2 = plo, c3 = phi;
      philox4x32_10(c0, c1, c2, c3, k0, k1);
      w0 = c0; w1 = c1; w2 = c2; w3 = c3;
      ++blk;
      left = 4;
    }
    const uint32_t w = w0;
    w0 = w1; w1 = w2; w2 = w3;
    --left;
    return w;
  }
};

// u = (floor(w / 2^9) + 1/2) 2^-23: exact in binary32 and binary64, in (0, 1), and 1-u is exact too.
template <class R>
__device__ __forceinline__ R to_uniform(uint32_t w) {
  return (R)(w >> 9) * (R)(1.0 / 8388608.0) + (R)(1.0 / 16777216.0);
}

// ------------------------------------------------------------------------------------------------
// Model descriptor: one disk's geometry, dust, tables and tallies, all device pointers.
// Lengths are in units of the inner radius r_faces[0]; rho is stored as rho * l_unit so that
// alpha = rho * chi is an opacity per unit length.
// ------------------------------------------------------------------------------------------------
template <class R>
struct DevModel {
  int nr, nt, nlam, nT;
  int gray;
  int pad_;
  // geometry
  const R* rf;            // nr+1 radial faces
  const R* rf2;           // squared
  const R* c2;            // nt+1 cos^2 theta_f
  const R* s2;            // nt+1 sin^2 theta_f
  const R* cf;            // nt+1 cos theta_f
  const R* sf;            // nt+1 sin theta_f
  const signed char* fk;  // nt+1: +1 theta_f < pi/2, -1 theta_f > pi/2, 0 midplane plane, 2 axis
  const R* rho;           // nr*nt, rho * l_unit (g cm^-2)
  // dust per wavelength bin
  const R* chi;           // extinction kappa + sigma
  const R* alb;           // albedo sigma / chi
  const R* gq;            // Henyey-Greenstein g
  const R* star_cum;      // cumulative stellar bin luminosity (unnormalised)
  R chi0, alb0, g0;       // gray values
  R chiR0, kbar0;         // gray: chi' = kappa + (1-g) sigma and kappa
  // temperature tables on the T grid
  const float* lQk;       // nT: log Q(T_k), Q = 4 pi sum_b kappa_b Bbar_b(T) (erg/s/g); lQk[0] = -inf
  const float* cbw;       // nT*nlam: cumulative kappa_b Bbar_b(T_k)
  const float* cexit;     // nT*nlam: cumulative dBbar_b/dT / chi'_b
  const float* chiR;      // nT: Rosseland mean of chi' (cm^2/g)
  const float* kbar;      // nT: kappa_bar of Eq. 10
  const float* lqm;       // nr*nt: log(1 / m_cell) (1/g)
  float lq_run;           // log(L_pkt / (N EUNIT)): log q = log(tally) + lqm[c] + lq_run
  // internal sources (viscous heating): cumulative luminosity over the cells (n_src + 1 entries, FP64),
  // the star's luminosity and the total the packets carry; n_src = 0 without sources
  const double* src_cum;
  double src_Lstar, src_Ltot;
  int n_src;
  // polarization (Sect. 2.3): Mueller matrix per bin [nlam][4][nmu] (S11, S12, S33, S34 at theta_k =
  // k pi / (nmu - 1)), the normalised cumulative S11 sin(theta) per bin [nlam][nmu], and the escaping
  // Stokes Q/I, U/I per [lam][incl] in fixed point (2^20 per packet, two's complement)
  const R* mtab;
  const R* mcdf;
  int nmu;
  unsigned long long* sed_q;
  unsigned long long* sed_u;
  // path-length estimator of the mean intensity: path length (internal units) of flights and MRW walks
  // per [cell][bin], NULL when not kept; the weights of Eq. 10 that spread a walk over the bins, per
  // [T_k][bin] (dBbar_b/dT normalised: eta_b / chi'_b at the fixed point of Eq. 13)
  double* jlen;
  const float* jw;
  // tallies
  unsigned long long* tally;   // nr*nt fixed-point absorbed energy
  unsigned long long* visits;  // nr*nt packet entries
  unsigned long long* nabs;    // nr*nt absorption events
  unsigned long long* sed;     // nlam*kNInc escaped packets
  unsigned long long* cnt;     // 16 run counters (see CntIdx)
  // packet range of this model in the run
  unsigned long long first_id;
  unsigned long long n_packets;
  unsigned long long q_begin;  // offset of this model in the shared packet queue
  uint32_t model_id;
  uint32_t pad2_;
};

enum CntIdx {
  C_PACKETS = 0, C_EVENTS, C_ABS, C_SCA, C_CROSS, C_MRW, C_CAPPED, C_ESCAPED, C_DEPSUM, C_ERR,
  C_MAXSTEPS,  // steps (interactions + jumps + crossings) of the longest packet
  C_LONGEST,   // (steps << 24) | (packet id & 0xffffff) of the longest packet
  C_GUARDS,    // packets dropped by a step guard (also counted as capped)
  C_NCNT = 16
};

// ------------------------------------------------------------------------------------------------
// Geometry helpers (templated on the floating type; host and device, so that the same code can be
// checked against the oracle on the CPU)
// ------------------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R rsqrt_(R x);
template <>
__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }

template <class R>
__host__ __device__ __forceinline__ R inf_() { return (R)INFINITY; }

// Larger root of s^2 + 2 b s + c = 0 (leaving the sphere |x|^2 = R^2), from q = -(b + sign(b) sqrt(disc))
// and c/q; the sign bit of b (not b >= 0) picks the branch, so b = -0 is handled like copysign does.
template <class R>
__host__ __device__ __forceinline__ R sphere_far(R b, R c) {
  R disc = b * b - c;
  disc = disc > (R)0 ? disc : (R)0;
  const R q = -(b + copysign(sqrt(disc), b));
  if (q == (R)0) return (R)0;
  R s = fmax(q, c / q);
  return s > (R)0 ? s : (R)0;
}

// Smaller root when the sphere is hit from outside (b < 0), else infinity.
template <class R>
__host__ __device__ __forceinline__ R sphere_near(R b, R c) {
  if (!(b < (R)0)) return inf_<R>();
  const R disc = b * b - c;
  if (disc < (R)0) return inf_<R>();
  const R q = -b + sqrt(disc);
  const R s = c / q;
  return s > (R)0 ? s : (R)0;
}

// Distance to the polar face f when leaving the cell across it. leaving_down: the cell lies at
// theta >= theta_f and the ray leaves towards smaller theta. G(s) = sig (cos^2 (x^2+y^2) - sin^2 z^2)
// is >= 0 exactly where theta >= theta_f on the face's own nappe; the exit is where G changes sign
// in the leaving direction, on that nappe.
template <class R>
__host__ __device__ __forceinline__ R cone_exit(const DevModel<R>& M, int f, R px, R py, R pz, R ux, R uy, R uz,
                                       bool leaving_down) {
  const int kind = M.fk[f];
  if (kind == 2) return inf_<R>();
  if (kind == 0) {  // midplane: plane z = 0
    if (leaving_down) {
      if (!(uz > (R)0)) return inf_<R>();
    } else {
      if (!(uz < (R)0)) return inf_<R>();
    }
    const R s = -pz / uz;
    return s > (R)0 ? s : (R)0;
  }
  const R sig = (R)kind;
  const R cc = M.c2[f], ss = M.s2[f];
  const R A = sig * (cc * (ux * ux + uy * uy) - ss * uz * uz);
  const R B = sig * (cc * (px * ux + py * uy) - ss * pz * uz);
  const R C = sig * (cc * (px * px + py * py) - ss * pz * pz);
  const R disc = B * B - A * C;
  if (disc < (R)0) return inf_<R>();
  const R q = -(B + copysign(sqrt(disc), B));
  if (q == (R)0) return inf_<R>();
  const bool bpos = !signbit(B);
  R s = (leaving_down == bpos) ? q / A : C / q;
  if (!(s == s)) return inf_<R>();
  if (s < (R)0) {
    const R r2 = px * px + py * py + pz * pz;
    if (s * s < (R)1e-18 * r2) s = (R)0;  // on the face within rounding
    else return inf_<R>();
  }
  const R z = pz + s * uz;
  if (sig * z < (R)0) return inf_<R>();
  return s;
}

// Distance to the boundary of cell (ir, it) along the ray, and which face: 0 inner sphere,
// 1 outer sphere, 2 lower polar face, 3 upper polar face.
template <class R>
__host__ __device__ __forceinline__ R next_face(const DevModel<R>& M, int ir, int it, R px, R py, R pz, R ux, R uy, R uz,
                                       int& face) {
  const R b = px * ux + py * uy + pz * uz;
  const R r2 = px * px + py * py + pz * pz;
  R s = sphere_far(b, r2 - M.rf2[ir + 1]);
  face = 1;
  const R sn = sphere_near(b, r2 - M.rf2[ir]);
  if (sn < s) { s = sn; face = 0; }
  if (it > 0) {
    const R sc = cone_exit(M, it, px, py, pz, ux, uy, uz, true);
    if (sc < s) { s = sc; face = 2; }
  }
  if (it + 1 < M.nt) {
    const R sc = cone_exit(M, it + 1, px, py, pz, ux, uy, uz, false);
    if (sc < s) { s = sc; face = 3; }
  }
  return s;
}

// Smallest distance from p to the faces of cell (ir, it): d_min of Eq. 11. Also a lower bound on the
// distance to the cell boundary along any direction.
template <class R>
__host__ __device__ __forceinline__ R dmin_cell(const DevModel<R>& M, int ir, int it, R px, R py, R pz) {
  const R rc2 = px * px + py * py;
  const R r = sqrt(rc2 + pz * pz);
  const R rc = sqrt(rc2);
  R d = fmin(r - M.rf[ir], M.rf[ir + 1] - r);
  if (M.fk[it] != 2) d = fmin(d, fabs(rc * M.cf[it] - pz * M.sf[it]));
  if (M.fk[it + 1] != 2) d = fmin(d, fabs(rc * M.cf[it + 1] - pz * M.sf[it + 1]));
  return d > (R)0 ? d : (R)0;
}

// FP32 versions of the three geometry functions above without branches: every candidate is computed
// and the valid one selected, so the dependency chains of the four faces overlap (a packet that
// runs alone on its SM is latency bound). They return what the generic versions return.
template <>
__host__ __device__ __forceinline__ float sphere_far<float>(float b, float c) {
  const float disc = fmaxf(b * b - c, 0.f);
  const float q = -(b + copysignf(sqrtf(disc), b));
  const float s = fmaxf(q, c / q);
  return q == 0.f ? 0.f : fmaxf(s, 0.f);
}

template <>
__host__ __device__ __forceinline__ float sphere_near<float>(float b, float c) {
  const float disc = b * b - c;
  const float q = -b + sqrtf(fmaxf(disc, 0.f));
  const float s = fmaxf(c / q, 0.f);
  return (b < 0.f && disc >= 0.f) ? s : inf_<float>();
}

template <>
__host__ __device__ __forceinline__ float cone_exit<float>(const DevModel<float>& M, int f, float px, float py, float pz, float ux,
                                                  float uy, float uz, bool leaving_down) {
  const int kind = M.fk[f];
  const float sig = (float)kind, cc = M.c2[f], ss = M.s2[f];
  // cone nappe (kind +-1)
  const float A = sig * (cc * (ux * ux + uy * uy) - ss * uz * uz);
  const float B = sig * (cc * (px * ux + py * uy) - ss * pz * uz);
  const float C = sig * (cc * (px * px + py * py) - ss * pz * pz);
  const float disc = B * B - A * C;
  const float q = -(B + copysignf(sqrtf(fmaxf(disc, 0.f)), B));
  const bool first = leaving_down == !signbit(B);
  float s = (first ? q : C) / (first ? A : q);
  const float r2 = px * px + py * py + pz * pz;
  s = (s < 0.f && s * s < 1e-18f * r2) ? 0.f : s;
  const bool cone_ok = disc >= 0.f && q != 0.f && s >= 0.f && sig * (pz + s * uz) >= 0.f;  // s >= 0 is false for NaN
  // midplane plane (kind 0)
  const bool toward = leaving_down ? uz > 0.f : uz < 0.f;
  const float sp = fmaxf(-pz / uz, 0.f);
  float res = cone_ok ? s : inf_<float>();
  res = kind == 0 ? (toward ? sp : inf_<float>()) : res;
  return kind == 2 ? inf_<float>() : res;
}

template <>
__host__ __device__ __forceinline__ float next_face<float>(const DevModel<float>& M, int ir, int it, float px, float py, float pz,
                                                  float ux, float uy, float uz, int& face) {
  const float b = px * ux + py * uy + pz * uz;
  const float r2 = px * px + py * py + pz * pz;
  const float so = sphere_far<float>(b, r2 - M.rf2[ir + 1]);
  const float si = sphere_near<float>(b, r2 - M.rf2[ir]);
  // the axis faces (theta = 0, pi) have kind 2, so the first and last polar cells need no guard
  const float sl = cone_exit<float>(M, it, px, py, pz, ux, uy, uz, true);
  const float su = cone_exit<float>(M, it + 1, px, py, pz, ux, uy, uz, false);
  float s = so;
  face = 1;
  if (si < s) { s = si; face = 0; }
  if (sl < s) { s = sl; face = 2; }
  if (su < s) { s = su; face = 3; }
  return s;
}

template <>
__host__ __device__ __forceinline__ float dmin_cell<float>(const DevModel<float>& M, int ir, int it, float px, float py, float pz) {
  const float rc2 = px * px + py * py;
  const float r = sqrtf(rc2 + pz * pz);
  const float rc = sqrtf(rc2);
  const float d0 = fminf(r - M.rf[ir], M.rf[ir + 1] - r);
  const float dl = M.fk[it] != 2 ? fabsf(rc * M.cf[it] - pz * M.sf[it]) : inf_<float>();
  const float du = M.fk[it + 1] != 2 ? fabsf(rc * M.cf[it + 1] - pz * M.sf[it + 1]) : inf_<float>();
  return fmaxf(fminf(d0, fminf(dl, du)), 0.f);
}

// Polar cell containing the direction of p: the last face k in 1..nt-1 with cos theta_k >= z/r.
template <class R>
__host__ __device__ __forceinline__ int theta_cell(const DevModel<R>& M, R px, R py, R pz) {
  const R mu = pz / sqrt(px * px + py * py + pz * pz);
  int lo = 0, hi = M.nt;  // invariant: answer in [lo, hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (M.cf[mid] >= mu) lo = mid; else hi = mid;
  }
  return lo;
}

}  // namespace mcrt
