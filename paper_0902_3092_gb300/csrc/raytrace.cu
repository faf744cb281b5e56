// raytrace.cu -- ray-traced observables: images, the SED and interferometric visibilities, by integrating
// the source function along straight rays through the (r, theta) grid with the Monte Carlo temperatures
// (Sect. 2.3: observables from the computed source function, free of Monte Carlo noise; Sect. 4.1: SED at
// 45 degrees, N-band visibilities at a 100 m baseline).
//
// Readings: the source function of a cell in bin b is S_b = kappa_b Bbar_b(T) / chi_b with chi = kappa +
// sigma (thermal emission over the total extinction; scattering takes light out of a ray and adds none);
// S and the extinction are constant in a cell, so a segment of optical depth dtau updates the intensity
// carried towards the observer exactly: I <- S + (I - S) exp(-dtau). The star is a point source at the
// origin, dimmed along the radial line towards the observer, and occults no ray.
//
// Layout: one thread per ray and chunk of up to 25 wavelength bins (intensities and extinctions in
// registers); the thread marches its ray (raymarch.cuh: closed-form crossings, one square root or one
// quadratic per cell) and reads CH contiguous values of the source table row S[cell][bin] per segment.
// Consecutive threads take rays that are neighbours on the sky (Morton order of the sky positions, built
// by mcrt_set_rays), whose paths cross the same cells.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "internal.h"
#include "planck.cuh"
#include "raymarch.cuh"
#include "source.cuh"

namespace mcrt {

struct RayState {
  DBuf p, q, w;   // rays: sky-plane coordinates (cm) and areas (cm^2), FP64
  DBuf order;     // the rays in Morton order of their sky positions (int32): neighbours share warps
  long long n = 0;
  double incl = 0, dist = 0;
  DBuf S;         // cells x nlam source table of the last trace (float or double)
  int S_prec = 0, S_which = -1;
  unsigned long long S_epoch = ~0ull;
  DBuf img;       // n x nlam image of the last trace
  int img_prec = 0;
  bool have_img = false;
  DBuf part, F, Fs, cnt;  // SED partial sums, disk + star flux, star flux, counters
  DBuf vis_par;           // per visibility: bin, fu, fv
  DBuf vis_out;
};

void ray_free(RayState* r) { delete r; }

namespace {

constexpr int kRayBlock = 256;
constexpr int kSedBlock = 128;

// One segment of optical depth x through a cell of source function s: I <- I e^-x + s (1 - e^-x).
// 1 - e^-x is not formed as a difference where x is small (optically thin segments, where the FP32
// exponential's absolute error of ~2e-7 would be a large part of it): below 0.1 it is the series
// x (1 - x/2 + x^2/6 - x^3/24), whose truncation is below 1e-6 of it; in FP64, expm1.
template <class R>
__device__ __forceinline__ R segment(R I, R s, R x);
template <>
__device__ __forceinline__ float segment<float>(float I, float s, float x) {
  const float e = __expf(-x);
  const float ser = x * (1.f - x * (0.5f - x * (1.f / 6.f - x * (1.f / 24.f))));
  const bool small = x < 0.1f;
  const float om = small ? ser : 1.f - e;
  return (small ? 1.f - ser : e) * I + om * s;
}
template <>
__device__ __forceinline__ double segment<double>(double I, double s, double x) {
  return exp(-x) * I - expm1(-x) * s;
}

// One thread per (ray, chunk of CH wavelength bins), grid-stride over the items, consecutive threads on
// consecutive rays of the same chunk. Each thread marches its ray (march_ray: closed-form crossings of
// the straight ray with the spheres and cones) and applies every segment to its CH bins, whose
// intensities and extinctions stay in registers; a ray with nlam bins is marched ceil(nlam / CH) times.
// Per bin the sequence of segment updates is the same for any chunking. cnt[0] += segments with dust
// (counted by chunk 0), cnt[1] |= 1 when a ray took more events than the bound.
template <class R, int CH>
__global__ void __launch_bounds__(kRayBlock) k_raytrace(const DevModel<R> M, const R* __restrict__ chi,
                                                        const R* __restrict__ S, long long n, int nchunk,
                                                        const int* __restrict__ order,
                                                        const double* __restrict__ p, const double* __restrict__ q,
                                                        double inv_l, R si, R ci, int max_events,
                                                        R* __restrict__ img, unsigned long long* __restrict__ cnt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FaceCoef<R>* face = reinterpret_cast<FaceCoef<R>*>(smem_raw);  // nt+1 entries for this inclination
  R* chs = reinterpret_cast<R*>(smem_raw + (size_t)(M.nt + 1) * sizeof(FaceCoef<R>));  // nlam extinctions
  for (int j = threadIdx.x; j <= M.nt; j += blockDim.x) face[j] = face_coef<R>(M.c2[j], M.s2[j], M.fk[j], si, ci);
  for (int b = threadIdx.x; b < M.nlam; b += blockDim.x) chs[b] = chi[b];
  __syncthreads();
  const int nlam = M.nlam, nt = M.nt;
  const RayGrid<R> G{M.nr, M.nt, M.rf2, M.cf, face};
  const long long items = n * nchunk;
  unsigned long long segs = 0;
  bool err = false;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < items;
       w += (long long)gridDim.x * blockDim.x) {
    const int chunk = (int)(w / n);
    const long long ray = order[w - (long long)chunk * n];
    const int b0 = chunk * CH;
    R I[CH], ch[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      I[k] = (R)0;
      ch[k] = b0 + k < nlam ? chs[b0 + k] : (R)0;
    }
    const int rc = march_ray(G, (R)(p[ray] * inv_l), (R)(q[ray] * inv_l), si, ci, max_events,
                             [&](int ir, int it, R L) {
                               const int c = ir * nt + it;
                               const R a = M.rho[c] * L;  // optical depth per unit chi
                               if (a > (R)0) {
                                 const R* Sc = S + (size_t)c * nlam + b0;
#pragma unroll
                                 for (int k = 0; k < CH; ++k)
                                   if (b0 + k < nlam) I[k] = segment<R>(I[k], Sc[k], a * ch[k]);
                                 segs += chunk == 0;
                               }
                             });
    if (rc < 0) err = true;
    R* o = img + (size_t)ray * nlam + b0;
#pragma unroll
    for (int k = 0; k < CH; ++k)
      if (b0 + k < nlam) o[k] = I[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) segs += __shfl_xor_sync(0xffffffffu, segs, o);
  const bool any_err = __any_sync(0xffffffffu, err);
  if ((threadIdx.x & 31) == 0) {
    if (segs) atomicAdd(cnt, segs);
    if (any_err) atomicOr(cnt + 1, 1ull);
  }
}

// bins per thread for nlam bins: the candidate that minimises chunks x (bins + a march's worth of work);
// the environment variable MCRT_RAY_CHUNK (4, 8, 16, 20 or 25) overrides the choice, for tuning
inline int ray_chunk(int nlam) {
  const int cand[5] = {4, 8, 16, 20, 25};
  if (const char* env = std::getenv("MCRT_RAY_CHUNK")) {
    const int v = std::atoi(env);
    for (int c : cand)
      if (v == c) return c;
  }
  int best = 25;
  long long cost = -1;
  for (int c : cand) {
    const long long k = ((long long)nlam + c - 1) / c * (c + 6);
    if (cost < 0 || k < cost) {
      cost = k;
      best = c;
    }
  }
  return best;
}

// Flux of the star per bin at distance d: pi R*^2 Bbar_b(T*) / d^2, dimmed by chi_b times the column
// sum rho dr of polar row `it` (the row that holds the line of sight).
__global__ void k_star(int nr, int nt, int it, int nlam, const double* __restrict__ rho_l,
                       const double* __restrict__ rf_l, const double* __restrict__ lam_e,
                       const double* __restrict__ chi, double Tstar, double Rstar, double dist,
                       double* __restrict__ Fs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nlam) return;
  double col = 0.0;
  for (int ir = 0; ir < nr; ++ir) col += rho_l[ir * nt + it] * (rf_l[ir + 1] - rf_l[ir]);
  const double k4 = kKB * kKB * kKB * kKB;
  const double pref3 = 2.0 * k4 * Tstar * Tstar * Tstar * Tstar / (kH * kH * kH * kC * kC);
  double g_short = 0.0, g_long, g4;
  if (b > 0) tails(kH * kC / (lam_e[b] * 1e-4 * kKB * Tstar), g_short, g4);
  if (b + 1 == nlam) tails(0.0, g_long, g4);
  else tails(kH * kC / (lam_e[b + 1] * 1e-4 * kKB * Tstar), g_long, g4);
  const double B = pref3 * (g_long - g_short);
  Fs[b] = 3.14159265358979323846 * Rstar * Rstar * B / (dist * dist) * exp(-col * chi[b]);
}

// Weighted image sums per bin over a contiguous range of rays (one block per range, threads over bins,
// so each ray's row is read contiguously).
template <class R>
__global__ void k_sed_part(long long n, int nlam, long long per_blk, const R* __restrict__ img,
                           const double* __restrict__ w, double* __restrict__ part) {
  const long long r0 = (long long)blockIdx.x * per_blk;
  const long long r1 = r0 + per_blk < n ? r0 + per_blk : n;
  for (int b = threadIdx.x; b < nlam; b += blockDim.x) {
    double s = 0.0;
    for (long long r = r0; r < r1; ++r) s += w[r] * (double)img[r * nlam + b];
    part[(size_t)blockIdx.x * nlam + b] = s;
  }
}

// F_b = sum of the partial sums (fixed order) / d^2 + star.
__global__ void k_sed_final(int nblk, int nlam, const double* __restrict__ part, double inv_d2,
                            const double* __restrict__ Fs, double* __restrict__ F) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nlam) return;
  double s = 0.0;
  for (int j = 0; j < nblk; ++j) s += part[(size_t)j * nlam + b];
  F[b] = s * inv_d2 + Fs[b];
}

// One block per visibility: sums over the rays of w I exp(-2 pi i t), t = fu p + fv q in turns (fu, fv:
// spatial frequency over distance, cycles per cm at the source), reduced to its fractional part in FP64
// before the sine and cosine.
template <class R>
__global__ void k_vis(long long n, int nlam, const R* __restrict__ img, const double* __restrict__ p,
                      const double* __restrict__ q, const double* __restrict__ w, const double* __restrict__ par,
                      const double* __restrict__ Fs, int with_star, double inv_d2, double* __restrict__ out) {
  const int j = blockIdx.x;
  const int b = (int)par[3 * j];
  const double fu = par[3 * j + 1], fv = par[3 * j + 2];
  double re = 0.0, im = 0.0, tot = 0.0;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) {
    const double f = w[r] * (double)img[r * nlam + b];
    double t = fu * p[r] + fv * q[r];
    t -= rint(t);
    double sn, cs;
    if (sizeof(R) == 8) {
      sincospi(2.0 * t, &sn, &cs);
    } else {
      float s32, c32;
      sincospif(2.0f * (float)t, &s32, &c32);
      sn = s32;
      cs = c32;
    }
    re += f * cs;
    im -= f * sn;
    tot += f;
  }
  __shared__ double sh[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
    tot += __shfl_down_sync(0xffffffffu, tot, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = re;
    sh[1][wid] = im;
    sh[2][wid] = tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0, t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      c += sh[1][k];
      t += sh[2][k];
    }
    const double fs = with_star ? Fs[b] : 0.0;
    a = a * inv_d2 + fs;
    c = c * inv_d2;
    t = t * inv_d2 + fs;
    out[j] = t > 0.0 ? sqrt(a * a + c * c) / t : 0.0;
  }
}

int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v > 0 ? v : 1;
}

template <class R, int CH>
cudaError_t launch_trace_ch(mcrt_disk* d, RayState* rs, const DevModel<R>& M, const R* chi, int sms) {
  const R si = (R)std::sin(rs->incl), ci = (R)std::cos(rs->incl);
  const int max_events = 4 * (d->nr + d->nt) + 64;
  const double inv_l = 1.0 / d->l_unit;
  const int nchunk = (d->nlam + CH - 1) / CH;
  const size_t smem = (size_t)(d->nt + 1) * sizeof(FaceCoef<R>) + (size_t)d->nlam * sizeof(R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_raytrace<R, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raytrace<R, CH>, kRayBlock, smem);
  long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
  const long long need = (rs->n * nchunk + kRayBlock - 1) / kRayBlock;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_raytrace<R, CH><<<(int)grid, kRayBlock, smem, d->stream>>>(M, chi, rs->S.as<R>(), rs->n, nchunk,
                                                               rs->order.as<int>(), rs->p.as<double>(), rs->q.as<double>(), inv_l, si, ci,
                                                               max_events, rs->img.as<R>(),
                                                               rs->cnt.as<unsigned long long>());
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_trace(mcrt_disk* d, RayState* rs, const DevModel<R>& M, const R* chi, int sms) {
  switch (ray_chunk(d->nlam)) {
    case 4: return launch_trace_ch<R, 4>(d, rs, M, chi, sms);
    case 8: return launch_trace_ch<R, 8>(d, rs, M, chi, sms);
    case 16: return launch_trace_ch<R, 16>(d, rs, M, chi, sms);
    case 20: return launch_trace_ch<R, 20>(d, rs, M, chi, sms);
    default: return launch_trace_ch<R, 25>(d, rs, M, chi, sms);
  }
}

}  // namespace
}  // namespace mcrt

using namespace mcrt;

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(d, e_, what); \
  } while (0)

namespace {

template <class R>
DevModel<R> model_of(const mcrt_disk* d);
template <>
DevModel<float> model_of<float>(const mcrt_disk* d) { return d->model32(); }
template <>
DevModel<double> model_of<double>(const mcrt_disk* d) { return d->model64(); }
template <class R>
const R* chi_of(const mcrt_disk* d) { return static_cast<const R*>(sizeof(R) == 8 ? d->chi64.p : d->chi32.p); }

static double j_factor(const mcrt_disk* d) {
  return j_factor_of(d->Lpkt(), d->n_total, d->l_unit, d->packets_done);
}

template <class R>
mcrt_status trace_impl(mcrt_disk* d, int which) {
  RayState* rs = d->rays;
  const size_t nc = (size_t)d->nr * d->nt;
  const int nlam = d->nlam;
  const bool scat = (which & MCRT_WITH_SCATTERING) != 0;
  const double* T = (which & ~MCRT_WITH_SCATTERING) == MCRT_T_PDA ? d->T_pda.as<double>() : d->T_mc.as<double>();
  const int prec = sizeof(R) == 8 ? 64 : 32;
  if (rs->S_epoch != d->T_epoch || rs->S_which != which || rs->S_prec != prec || !rs->S.p) {
    if (rs->S.n < nc * nlam * sizeof(R)) CK(rs->S.alloc(nc * nlam * sizeof(R)), "cudaMalloc");
    const int blocks = (int)((nc * 32 + 255) / 256);
    k_source<R><<<blocks, 256, 0, d->stream>>>((int)nc, nlam, T, d->lam_e_d.as<double>(), d->kabs_d.as<double>(),
                                               d->chi64.as<double>(), rs->S.as<R>(),
                                               scat ? d->jlen.as<double>() : nullptr, j_factor(d),
                                               d->alb64.as<double>(), d->rf64.as<double>(), d->cf64.as<double>(),
                                               d->nt);
    d->launches++;
    CK(cudaGetLastError(), "source kernel");
    rs->S_epoch = d->T_epoch;
    rs->S_which = which;
    rs->S_prec = prec;
  }
  const size_t img_bytes = (size_t)rs->n * nlam * sizeof(R);
  if (rs->img.n < img_bytes) CK(rs->img.alloc(img_bytes), "cudaMalloc");
  CK(cudaMemsetAsync(rs->cnt.p, 0, 2 * sizeof(unsigned long long), d->stream), "memset");
  const int sms = sm_count(d->device);
  const size_t smem = (size_t)(d->nt + 1) * sizeof(FaceCoef<R>) + (size_t)nlam * sizeof(R);
  if (smem > 200 * 1024) return set_error(d, MCRT_EINVAL, "too many polar cells for the ray-tracing face table");
  CK(launch_trace<R>(d, rs, model_of<R>(d), chi_of<R>(d), sms), "ray-trace kernel");
  d->launches++;
  rs->img_prec = prec;
  rs->have_img = true;
  // star, then the SED from the image
  int it = 0;
  while (it + 1 < d->nt && d->tf[it + 1] <= rs->incl) ++it;
  k_star<<<(nlam + 127) / 128, 128, 0, d->stream>>>(d->nr, d->nt, it, nlam, d->rho64.as<double>(), d->rf64.as<double>(),
                                                    d->lam_e_d.as<double>(), d->chi64.as<double>(), d->Tstar, d->Rstar,
                                                    rs->dist, rs->Fs.as<double>());
  d->launches++;
  const int nblk = (int)std::min<long long>(rs->n, (long long)sms * 4);
  const long long per_blk = (rs->n + nblk - 1) / nblk;
  if (rs->part.n < (size_t)nblk * nlam * 8) CK(rs->part.alloc((size_t)nblk * nlam * 8), "cudaMalloc");
  k_sed_part<R><<<nblk, kSedBlock, 0, d->stream>>>(rs->n, nlam, per_blk, rs->img.as<R>(), rs->w.as<double>(),
                                                  rs->part.as<double>());
  k_sed_final<<<(nlam + 127) / 128, 128, 0, d->stream>>>(nblk, nlam, rs->part.as<double>(), 1.0 / (rs->dist * rs->dist),
                                                         rs->Fs.as<double>(), rs->F.as<double>());
  d->launches += 2;
  CK(cudaGetLastError(), "SED kernels");
  return MCRT_OK;
}

}  // namespace

extern "C" {

mcrt_status mcrt_set_rays(mcrt_disk* d, double incl_rad, double dist_cm, int64_t n, const double* p_cm,
                          const double* q_cm, const double* w_cm2) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  if (!(incl_rad >= 0.0 && incl_rad <= 3.14159265358979323846))
    return set_error(d, MCRT_EINVAL, "inclination must lie in [0, pi]");
  if (!(dist_cm > 0.0) || !std::isfinite(dist_cm)) return set_error(d, MCRT_EINVAL, "distance must be > 0");
  if (n < 1 || n > (int64_t)1 << 27) return set_error(d, MCRT_EINVAL, "rays: 1 .. 2^27");
  if (!p_cm || !q_cm || !w_cm2) return set_error(d, MCRT_EINVAL, "p, q, w must not be NULL");
  if (d->nlam > 256) return set_error(d, MCRT_EINVAL, "ray tracing takes at most 256 wavelength bins");
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(p_cm[k]) || !std::isfinite(q_cm[k]) || !(w_cm2[k] >= 0.0) || !std::isfinite(w_cm2[k]))
      return set_error(d, MCRT_EINVAL, "rays: p, q finite and w >= 0");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (!d->rays) d->rays = new RayState();
  RayState* rs = d->rays;
  const size_t bytes = (size_t)n * 8;
  if (rs->p.n < bytes) CK(rs->p.alloc(bytes), "cudaMalloc");
  if (rs->q.n < bytes) CK(rs->q.alloc(bytes), "cudaMalloc");
  if (rs->w.n < bytes) CK(rs->w.alloc(bytes), "cudaMalloc");
  if (!rs->F.p) CK(rs->F.alloc(256 * 8), "cudaMalloc");
  if (!rs->Fs.p) CK(rs->Fs.alloc(256 * 8), "cudaMalloc");
  if (!rs->cnt.p) CK(rs->cnt.alloc(2 * 8), "cudaMalloc");
  // Morton order of the sky positions (16 bits per axis over the square of side 2 r_out): consecutive
  // threads take neighbouring rays, whose paths cross the same cells
  std::vector<std::pair<uint32_t, int>> key((size_t)n);
  const double rmax = d->rf[d->nr];
  for (int64_t k = 0; k < n; ++k) {
    auto quant = [&](double x) {
      const double t = std::min(std::max((x / rmax + 1.0) * 0.5, 0.0), 1.0);
      return (uint32_t)std::min(65535.0, std::floor(t * 65536.0));
    };
    uint32_t x = quant(p_cm[k]), y = quant(q_cm[k]), m = 0;
    for (int bit = 0; bit < 16; ++bit) m |= ((x >> bit) & 1u) << (2 * bit) | ((y >> bit) & 1u) << (2 * bit + 1);
    key[(size_t)k] = {m, (int)k};
  }
  std::stable_sort(key.begin(), key.end(), [](const auto& u, const auto& v) { return u.first < v.first; });
  std::vector<int> order((size_t)n);
  for (int64_t k = 0; k < n; ++k) order[(size_t)k] = key[(size_t)k].second;
  if (rs->order.n < (size_t)n * 4) CK(rs->order.alloc((size_t)n * 4), "cudaMalloc");
  CK(cudaMemcpyAsync(rs->order.p, order.data(), (size_t)n * 4, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaMemcpyAsync(rs->p.p, p_cm, bytes, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaMemcpyAsync(rs->q.p, q_cm, bytes, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaMemcpyAsync(rs->w.p, w_cm2, bytes, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  rs->n = n;
  rs->incl = incl_rad;
  rs->dist = dist_cm;
  rs->have_img = false;
  return MCRT_OK;
}

mcrt_status mcrt_mean_intensity(mcrt_disk* d, double* J_out) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!J_out) return set_error(d, MCRT_EINVAL, "J_out must not be NULL");
  if (!d->keep_j) return set_error(d, MCRT_ESTATE, "mcrt_keep_mean_intensity must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  const size_t nc = (size_t)d->nr * d->nt, n = nc * d->nlam;
  DBuf J;
  CK(J.alloc(n * 8), "cudaMalloc");
  const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count(d->device) * 8);
  k_mean_intensity<<<blocks, 256, 0, d->stream>>>((int)nc, d->nt, d->nlam, d->rf64.as<double>(), d->cf64.as<double>(),
                                                  d->jlen.as<double>(), j_factor(d), J.as<double>());
  d->launches++;
  CK(cudaGetLastError(), "mean-intensity kernel");
  CK(cudaMemcpyAsync(J_out, J.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_raytrace(mcrt_disk* d, int which, int precision, double* F_out, double* F_star_out, double* I_out,
                          uint64_t* n_segments) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->rays || d->rays->n < 1) return set_error(d, MCRT_ESTATE, "mcrt_set_rays must come first");
  const int base = which & ~MCRT_WITH_SCATTERING;
  if (base != MCRT_T_MC && base != MCRT_T_PDA) return set_error(d, MCRT_EINVAL, "which");
  if (precision != 0 && precision != 32 && precision != 64) return set_error(d, MCRT_EINVAL, "precision: 32 or 64");
  if (base == MCRT_T_PDA && !d->have_pda) return set_error(d, MCRT_ESTATE, "no PDA solution");
  if ((which & MCRT_WITH_SCATTERING) && !d->keep_j)
    return set_error(d, MCRT_ESTATE, "scattered light needs the mean-intensity tally (mcrt_keep_mean_intensity)");
  if (d->nlam > 256) return set_error(d, MCRT_EINVAL, "ray tracing takes at most 256 wavelength bins");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (!d->have_T) {
    mcrt_status s = compute_temperatures(d);
    if (s != MCRT_OK) return s;
  }
  RayState* rs = d->rays;
  mcrt_status s = precision == 64 ? trace_impl<double>(d, which) : trace_impl<float>(d, which);
  if (s != MCRT_OK) return s;
  unsigned long long c[2];
  CK(cudaMemcpyAsync(c, rs->cnt.p, sizeof(c), cudaMemcpyDeviceToHost, d->stream), "copy");
  if (F_out) CK(cudaMemcpyAsync(F_out, rs->F.p, (size_t)d->nlam * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (F_star_out)
    CK(cudaMemcpyAsync(F_star_out, rs->Fs.p, (size_t)d->nlam * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  if (I_out) {
    const size_t m = (size_t)rs->n * d->nlam;
    if (rs->img_prec == 64) {
      CK(cudaMemcpy(I_out, rs->img.p, m * 8, cudaMemcpyDeviceToHost), "copy");
    } else {
      std::vector<float> tmp(m);
      CK(cudaMemcpy(tmp.data(), rs->img.p, m * 4, cudaMemcpyDeviceToHost), "copy");
      for (size_t k = 0; k < m; ++k) I_out[k] = tmp[k];
    }
  }
  if (n_segments) *n_segments = c[0];
  if (c[1]) return set_error(d, MCRT_ETIMEOUT, "a ray took more than 4 (nr + ntheta) + 64 events");
  return MCRT_OK;
}

mcrt_status mcrt_visibilities(mcrt_disk* d, int n_vis, const int* bins, const double* baseline_cm,
                              const double* pa_rad, int with_star, double* vis_out) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->rays || !d->rays->have_img) return set_error(d, MCRT_ESTATE, "mcrt_raytrace must come first");
  if (n_vis < 1 || n_vis > (1 << 20) || !bins || !baseline_cm || !pa_rad || !vis_out)
    return set_error(d, MCRT_EINVAL, "bad arguments");
  RayState* rs = d->rays;
  std::vector<double> par((size_t)3 * n_vis);
  for (int j = 0; j < n_vis; ++j) {
    if (bins[j] < 0 || bins[j] >= d->nlam) return set_error(d, MCRT_EINVAL, "bin out of range");
    if (!(baseline_cm[j] >= 0.0) || !std::isfinite(baseline_cm[j]) || !std::isfinite(pa_rad[j]))
      return set_error(d, MCRT_EINVAL, "baselines: finite, >= 0");
    // bin centre lambda = sqrt(lambda_lo lambda_hi); frequency over distance in cycles per cm at the source
    const double lam_cm = std::sqrt(d->lam_e[bins[j]] * d->lam_e[bins[j] + 1]) * 1e-4;
    const double f = baseline_cm[j] / (lam_cm * rs->dist);
    par[3 * j] = bins[j];
    par[3 * j + 1] = f * std::cos(pa_rad[j]);
    par[3 * j + 2] = f * std::sin(pa_rad[j]);
  }
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (rs->vis_par.n < par.size() * 8) CK(rs->vis_par.alloc(par.size() * 8), "cudaMalloc");
  if (rs->vis_out.n < (size_t)n_vis * 8) CK(rs->vis_out.alloc((size_t)n_vis * 8), "cudaMalloc");
  CK(cudaMemcpyAsync(rs->vis_par.p, par.data(), par.size() * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  const double inv_d2 = 1.0 / (rs->dist * rs->dist);
  if (rs->img_prec == 64)
    k_vis<double><<<n_vis, 256, 0, d->stream>>>(rs->n, d->nlam, rs->img.as<double>(), rs->p.as<double>(),
                                                rs->q.as<double>(), rs->w.as<double>(), rs->vis_par.as<double>(),
                                                rs->Fs.as<double>(), with_star, inv_d2, rs->vis_out.as<double>());
  else
    k_vis<float><<<n_vis, 256, 0, d->stream>>>(rs->n, d->nlam, rs->img.as<float>(), rs->p.as<double>(),
                                               rs->q.as<double>(), rs->w.as<double>(), rs->vis_par.as<double>(),
                                               rs->Fs.as<double>(), with_star, inv_d2, rs->vis_out.as<double>());
  d->launches++;
  CK(cudaGetLastError(), "visibility kernel");
  CK(cudaMemcpyAsync(vis_out, rs->vis_out.p, (size_t)n_vis * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

}  // extern "C"
