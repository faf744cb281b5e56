// api.cu -- the C ABI of include/mcrt.h: disk objects, opacity tables, transport runs, temperatures,
// escape spectrum, checkpoints and test hooks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "internal.h"
#include "planck.cuh"
#include "tables.h"
#include "temperature.cuh"

using mcrt::DBuf;

namespace {
thread_local std::string g_err;
}

namespace mcrt {

mcrt_status set_error(mcrt_disk* d, mcrt_status s, const std::string& msg) {
  g_err = msg;
  if (d) d->err = msg;
  return s;
}

mcrt_status cuda_fail(mcrt_disk* d, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_error(d, MCRT_ENOMEM, m);
  return set_error(d, MCRT_ECUDA, m);
}

// ------------------------------------------------------------------------------------------------
// MRW inverse escape-time tables (Eq. 7-8; built by tables.h), once per process, uploaded per device.
// ------------------------------------------------------------------------------------------------
const float kMrwT0 = mrw_table_t0();
const float kMrwDT = mrw_table_dt();

const float* mrw_table(int device, cudaError_t* err) {
  static std::mutex mu;
  static std::vector<float> host;
  static std::vector<std::pair<int, float*>> per_dev;
  std::lock_guard<std::mutex> lock(mu);
  *err = cudaSuccess;
  for (auto& pr : per_dev)
    if (pr.first == device) return pr.second;
  if (host.empty()) {
    host.resize(2 * kMrwTab);
    build_mrw_table(host.data());
  }
  float* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(float) * host.size());
  if (e == cudaSuccess) e = cudaMemcpy(p, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    *err = e;
    if (p) cudaFree(p);
    return nullptr;
  }
  per_dev.push_back({device, p});
  return p;
}

// ------------------------------------------------------------------------------------------------
// Temperatures (a7): 4 pi m sum_b kappa_b Bbar_b(T) = L_abs, FP64
// ------------------------------------------------------------------------------------------------
__global__ void k_temperature(int n, const unsigned long long* __restrict__ tally, const double* __restrict__ mass,
                              double lfac, int gray, double kabs0, int nlam, const double* __restrict__ lam_e,
                              const double* __restrict__ kabs, const double* __restrict__ lQk,
                              const double* __restrict__ slQ, int nT, double Tmin, double dlnT,
                              double* __restrict__ T, double* __restrict__ relerr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const unsigned long long t = tally[c];
  const double neq = (double)t / (double)kEUnit;
  if (relerr) relerr[c] = t ? 0.25 / sqrt(neq) : (double)INFINITY;
  const double m = mass[c];
  if (t == 0ull || !(m > 0.0)) {
    T[c] = 0.0;
    return;
  }
  const double q = neq * lfac / m;
  T[c] = cell_temperature(q, gray, kabs0, nlam, lam_e, kabs, lQk, slQ, nT, Tmin, dlnT);
}

mcrt_status compute_temperatures(mcrt_disk* d) {
  const int n = d->nr * d->nt;
  const double lfac = d->Lpkt() / (d->n_total > 0 ? d->n_total : 1.0);
  const double dlnT = std::log(d->Tmax / d->Tmin) / (d->nT - 2);
  k_temperature<<<(n + 255) / 256, 256, 0, d->stream>>>(
      n, d->tally.as<unsigned long long>(), d->mass_d.as<double>(), lfac, d->gray ? 1 : 0, d->kabs[0], d->nlam,
      d->lam_e_d.as<double>(), d->kabs_d.as<double>(), d->lQ64.as<double>(), d->slQ64.as<double>(), d->nT, d->Tmin,
      dlnT,
      d->T_mc.as<double>(), d->relerr.as<double>());
  d->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(d, e, "temperature kernel");
  d->have_T = true;
  d->T_epoch++;
  return MCRT_OK;
}

// ------------------------------------------------------------------------------------------------
// test hooks
// ------------------------------------------------------------------------------------------------
__global__ void k_uniforms(uint64_t seed, uint32_t model, uint64_t packet, int n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Rng r;
  r.init(seed, model, packet);
  for (int i = 0; i < n; ++i) out[i] = to_uniform<double>(r.next());
}

__global__ void k_mrw_x(int n, const double* P0, double* out, const float* tab, float t0, float dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  KParams<float> P;
  P.mrw_tab = tab;
  P.mrw_t0 = t0;
  P.mrw_dt = dt;
  out[i] = (double)mrw_x<float>(P, (float)P0[i]);
}

}  // namespace mcrt

using namespace mcrt;

// ------------------------------------------------------------------------------------------------
// model descriptors
// ------------------------------------------------------------------------------------------------
template <class R>
static DevModel<R> make_model(const mcrt_disk* d, bool f64) {
  DevModel<R> m;
  std::memset(&m, 0, sizeof(m));
  m.nr = d->nr;
  m.nt = d->nt;
  m.nlam = d->nlam;
  m.nT = d->nT;
  m.gray = d->gray ? 1 : 0;
  m.rf = (const R*)(f64 ? d->rf64.p : d->rf32.p);
  m.rf2 = (const R*)(f64 ? d->rf2_64.p : d->rf2_32.p);
  m.c2 = (const R*)(f64 ? d->c2_64.p : d->c2_32.p);
  m.s2 = (const R*)(f64 ? d->s2_64.p : d->s2_32.p);
  m.cf = (const R*)(f64 ? d->cf64.p : d->cf32.p);
  m.sf = (const R*)(f64 ? d->sf64.p : d->sf32.p);
  m.fk = (const signed char*)d->fk.p;
  m.rho = (const R*)(f64 ? d->rho64.p : d->rho32.p);
  m.chi = (const R*)(f64 ? d->chi64.p : d->chi32.p);
  m.alb = (const R*)(f64 ? d->alb64.p : d->alb32.p);
  m.gq = (const R*)(f64 ? d->g64.p : d->g32.p);
  m.star_cum = (const R*)(f64 ? d->star64.p : d->star32.p);
  if (d->has_opacity) {
    const double chi = d->kabs[0] + d->ksca[0];
    m.chi0 = (R)chi;
    m.alb0 = (R)(d->ksca[0] / chi);
    m.g0 = (R)d->g[0];
    m.chiR0 = (R)(d->kabs[0] + (1.0 - d->g[0]) * d->ksca[0]);
    m.kbar0 = (R)d->kabs[0];
  }
  m.lQk = d->lQk.as<float>();
  m.cbw = d->cbw.as<float>();
  m.cexit = d->cexit.as<float>();
  m.chiR = d->chiRk.as<float>();
  m.kbar = d->kbark.as<float>();
  m.lqm = d->lqm.as<float>();
  m.lq_run = (float)std::log(d->Lpkt() / ((d->n_total > 0 ? d->n_total : 1.0) * (double)kEUnit));
  m.src_cum = d->n_src ? d->src_cum.as<double>() : nullptr;
  m.src_Lstar = d->Lstar;
  m.src_Ltot = d->Lpkt();
  m.n_src = d->n_src;
  m.mtab = (const R*)(f64 ? d->mtab64.p : d->mtab32.p);
  m.mcdf = (const R*)(f64 ? d->mcdf64.p : d->mcdf32.p);
  m.nmu = d->pol ? d->nmu : 0;
  m.sed_q = d->sed_q.as<unsigned long long>();
  m.sed_u = d->sed_u.as<unsigned long long>();
  m.jlen = d->keep_j ? d->jlen.as<double>() : nullptr;
  m.jw = d->jw.as<float>();
  m.tally = d->tally.as<unsigned long long>();
  m.visits = d->visits.as<unsigned long long>();
  m.nabs = d->nabs.as<unsigned long long>();
  m.sed = d->sed.as<unsigned long long>();
  m.cnt = d->cnt.as<unsigned long long>();
  return m;
}

DevModel<float> mcrt_disk::model32() const { return make_model<float>(this, false); }
DevModel<double> mcrt_disk::model64() const { return make_model<double>(this, true); }

// ------------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------------
template <class T>
static cudaError_t upload(DBuf& b, const std::vector<T>& v) {
  const size_t bytes = sizeof(T) * v.size();
  if (!b.p || b.n != (bytes ? bytes : 16)) {  // an allocation of the right size is kept (its address too)
    cudaError_t e = b.alloc(bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(b.p, v.data(), bytes, cudaMemcpyHostToDevice);
}

template <class A, class B>
static std::vector<A> cast_vec(const std::vector<B>& v) {
  return std::vector<A>(v.begin(), v.end());
}

#define CK(call, what)                                 \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(d, e_, what); \
  } while (0)

static mcrt_status zero_tallies(mcrt_disk* d) {
  const size_t n = (size_t)d->nr * d->nt;
  CK(cudaMemsetAsync(d->tally.p, 0, n * 8, d->stream), "memset");
  CK(cudaMemsetAsync(d->visits.p, 0, n * 8, d->stream), "memset");
  CK(cudaMemsetAsync(d->nabs.p, 0, n * 8, d->stream), "memset");
  if (d->sed.p) CK(cudaMemsetAsync(d->sed.p, 0, d->sed.n, d->stream), "memset");
  if (d->sed_q.p) CK(cudaMemsetAsync(d->sed_q.p, 0, d->sed_q.n, d->stream), "memset");
  if (d->sed_u.p) CK(cudaMemsetAsync(d->sed_u.p, 0, d->sed_u.n, d->stream), "memset");
  if (d->keep_j && d->jlen.p) CK(cudaMemsetAsync(d->jlen.p, 0, d->jlen.n, d->stream), "memset");
  d->have_T = false;
  d->have_pda = false;
  d->packets_done = 0;
  d->tally_held = 0;
  d->tally_wrapped = false;
  return MCRT_OK;
}

namespace mcrt {
bool account_deposits(mcrt_disk* d, const unsigned long long* c) {
  const unsigned long long before = d->tally_held;
  d->tally_held += c[C_DEPSUM];
  if (d->tally_held < before || (c[C_ERR] & kErrOverflow)) d->tally_wrapped = true;
  return !d->tally_wrapped;
}
}  // namespace mcrt

namespace mcrt {
// density-dependent device arrays from d->rho: rho * l_unit (FP32, FP64), cell masses, log(1/m), rho (cgs)
mcrt_status upload_density(mcrt_disk* d) {
  DensityArrays da;
  density_arrays(d->nr, d->nt, d->rf.data(), d->tf.data(), d->rho.data(), da);
  d->mass = da.mass;
  cudaError_t e = upload(d->rho32, cast_vec<float>(da.rhol));
  if (e == cudaSuccess) e = upload(d->rho64, da.rhol);
  if (e == cudaSuccess) e = upload(d->lqm, da.lqm);
  if (e == cudaSuccess) e = upload(d->mass_d, d->mass);
  if (e == cudaSuccess) e = upload(d->rho_cgs_d, d->rho);
  if (e != cudaSuccess) return cuda_fail(d, e, "upload");
  return MCRT_OK;
}
}  // namespace mcrt

extern "C" {

mcrt_status mcrt_set_density(mcrt_disk* d, const double* rho) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!rho) return set_error(d, MCRT_EINVAL, "rho is NULL");
  const size_t n = (size_t)d->nr * d->nt;
  for (size_t c = 0; c < n; ++c)
    if (!(std::isfinite(rho[c]) && rho[c] >= 0)) return set_error(d, MCRT_EINVAL, "rho must be finite and >= 0");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  d->rho.assign(rho, rho + n);
  mcrt_status s = upload_density(d);
  if (s != MCRT_OK) return s;
  s = zero_tallies(d);
  if (s != MCRT_OK) return s;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_set_sources(mcrt_disk* d, const double* L) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  const size_t n = (size_t)d->nr * d->nt;
  std::vector<double> cum(n + 1, 0.0);
  if (L) {
    for (size_t c = 0; c < n; ++c) {
      if (!(std::isfinite(L[c]) && L[c] >= 0)) return set_error(d, MCRT_EINVAL, "source luminosities: finite, >= 0");
      if (L[c] > 0 && !(d->rho[c] > 0)) return set_error(d, MCRT_EINVAL, "a source in a cell without dust");
      cum[c + 1] = cum[c] + L[c];  // in cell order, as the sources are drawn
    }
  }
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  if (cum[n] > 0) {
    cudaError_t e = upload(d->src_cum, cum);
    if (e != cudaSuccess) return cuda_fail(d, e, "upload");
    d->n_src = (int)n;
    d->Lsrc_total = cum[n];
  } else {
    d->n_src = 0;
    d->Lsrc_total = 0;
  }
  mcrt_status s = zero_tallies(d);  // the packet energy changed
  if (s != MCRT_OK) return s;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

void mcrt_default_run_opts(mcrt_run_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = 32;
  o->mrw = 0;
  o->gamma = 2.0;
  o->mrw_min_interactions = 20;
  o->mrw_exit_dir = 0;
  o->max_events_per_packet = 100000000ull;
  o->n_total_packets = 0;
  o->block_size = 0;
  o->refill_interval = 0;
  o->tail_warps_per_sm = 0;
  o->interact_batch = 0;
  o->max_in_flight = 0;
  o->want_sed = 1;
}

mcrt_status mcrt_disk_create(const mcrt_grid* grid, const mcrt_star* star, int device, void* cuda_stream,
                             mcrt_disk** out) {
  if (!out) return set_error(nullptr, MCRT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !star || !grid->r_faces_cm || !grid->theta_faces || !grid->rho_gcm3)
    return set_error(nullptr, MCRT_EINVAL, "NULL grid or star");
  const int nr = grid->nr, nt = grid->ntheta;
  if (nr < 1 || nt < 1 || (long long)nr * nt > (1ll << 30))
    return set_error(nullptr, MCRT_EINVAL, "grid sizes out of range");
  for (int i = 0; i <= nr; ++i) {
    const double r = grid->r_faces_cm[i];
    if (!(std::isfinite(r) && r > 0) || (i && !(r > grid->r_faces_cm[i - 1])))
      return set_error(nullptr, MCRT_EINVAL, "r_faces must be positive, finite and increasing");
  }
  for (int j = 0; j <= nt; ++j) {
    const double t = grid->theta_faces[j];
    if (!std::isfinite(t) || (j && !(t > grid->theta_faces[j - 1])))
      return set_error(nullptr, MCRT_EINVAL, "theta_faces must be finite and increasing");
  }
  if (std::fabs(grid->theta_faces[0]) > 1e-12 || std::fabs(grid->theta_faces[nt] - kPi) > 1e-12)
    return set_error(nullptr, MCRT_EINVAL, "theta_faces must run from 0 to pi");
  for (long long c = 0; c < (long long)nr * nt; ++c)
    if (!(std::isfinite(grid->rho_gcm3[c]) && grid->rho_gcm3[c] >= 0))
      return set_error(nullptr, MCRT_EINVAL, "rho must be finite and >= 0");
  if (!(star->T_star_K > 0 && std::isfinite(star->T_star_K) && star->R_star_cm > 0 && std::isfinite(star->R_star_cm)))
    return set_error(nullptr, MCRT_EINVAL, "star temperature and radius must be positive");

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return set_error(nullptr, MCRT_ECUDA, "no CUDA device");
  if (device < 0 || device >= ndev) return set_error(nullptr, MCRT_EINVAL, "device index out of range");
  mcrt_disk* d = new (std::nothrow) mcrt_disk();
  if (!d) return set_error(nullptr, MCRT_ENOMEM, "host allocation");
  auto fail = [&](mcrt_status s) {
    g_err = d->err;
    mcrt_disk_destroy(d);
    return s;
  };
  d->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(cuda_fail(d, e, "cudaSetDevice"));
  if (cuda_stream) {
    d->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(cuda_fail(d, e, "cudaStreamCreate"));
    d->own_stream = true;
  }
  d->nr = nr;
  d->nt = nt;
  d->rf.assign(grid->r_faces_cm, grid->r_faces_cm + nr + 1);
  d->tf.assign(grid->theta_faces, grid->theta_faces + nt + 1);
  d->rho.assign(grid->rho_gcm3, grid->rho_gcm3 + (size_t)nr * nt);
  d->Tstar = star->T_star_K;
  d->Rstar = star->R_star_cm;
  d->Lstar = 4.0 * kPi * d->Rstar * d->Rstar * MCRT_SIGMA * std::pow(d->Tstar, 4);
  d->l_unit = d->rf[0];
  d->Tmax = std::max(1e4, 2.0 * d->Tstar);

  // geometry in units of r_faces[0]
  GeomArrays geo;
  geometry_arrays(nr, nt, d->rf.data(), d->tf.data(), geo);
  const size_t ncell = (size_t)nr * nt;
  mcrt_status st = MCRT_OK;
#define UP(buf, vec)                                          \
  do {                                                        \
    cudaError_t e2 = upload(buf, vec);                        \
    if (e2 != cudaSuccess) return fail(cuda_fail(d, e2, "upload")); \
  } while (0)
  UP(d->rf32, cast_vec<float>(geo.rf));
  UP(d->rf2_32, cast_vec<float>(geo.rf2));
  UP(d->c2_32, cast_vec<float>(geo.c2));
  UP(d->s2_32, cast_vec<float>(geo.s2));
  UP(d->cf32, cast_vec<float>(geo.cf));
  UP(d->sf32, cast_vec<float>(geo.sf));
  UP(d->rf64, geo.rf);
  UP(d->rf2_64, geo.rf2);
  UP(d->c2_64, geo.c2);
  UP(d->s2_64, geo.s2);
  UP(d->cf64, geo.cf);
  UP(d->sf64, geo.sf);
  UP(d->fk, geo.fk);
#undef UP
  st = upload_density(d);
  if (st != MCRT_OK) return fail(st);
  e = d->tally.alloc(ncell * 8);
  if (e == cudaSuccess) e = d->visits.alloc(ncell * 8);
  if (e == cudaSuccess) e = d->nabs.alloc(ncell * 8);
  if (e == cudaSuccess) e = d->cnt.alloc((C_NCNT + kTripWords) * 8);  // run counters, then the guard record
  if (e == cudaSuccess) e = d->queue.alloc(8);
  if (e == cudaSuccess) e = d->T_mc.alloc(ncell * 8);
  if (e == cudaSuccess) e = d->relerr.alloc(ncell * 8);
  if (e == cudaSuccess) e = d->T_pda.alloc(ncell * 8);
  if (e != cudaSuccess) return fail(cuda_fail(d, e, "cudaMalloc"));
  st = zero_tallies(d);
  if (st != MCRT_OK) return fail(st);
  e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) return fail(cuda_fail(d, e, "synchronize"));
  *out = d;
  return MCRT_OK;
}

mcrt_status mcrt_set_opacity(mcrt_disk* d, int nlam, const double* lam_e, const double* kabs, const double* ksca,
                             const double* g) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (nlam < 1 || nlam > 1024 || !lam_e || !kabs || !ksca) return set_error(d, MCRT_EINVAL, "bad opacity arguments");
  for (int b = 0; b <= nlam; ++b)
    if (!(std::isfinite(lam_e[b]) && lam_e[b] > 0) || (b && !(lam_e[b] > lam_e[b - 1])))
      return set_error(d, MCRT_EINVAL, "wavelength edges must be positive and increasing");
  for (int b = 0; b < nlam; ++b) {
    if (!(std::isfinite(kabs[b]) && kabs[b] > 0)) return set_error(d, MCRT_EINVAL, "kappa_abs must be > 0");
    if (!(std::isfinite(ksca[b]) && ksca[b] >= 0)) return set_error(d, MCRT_EINVAL, "kappa_sca must be >= 0");
    if (g && !(std::isfinite(g[b]) && g[b] > -1 && g[b] < 1)) return set_error(d, MCRT_EINVAL, "g must be in (-1, 1)");
  }
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  d->nlam = nlam;
  d->lam_e.assign(lam_e, lam_e + nlam + 1);
  d->kabs.assign(kabs, kabs + nlam);
  d->ksca.assign(ksca, ksca + nlam);
  d->g.assign(nlam, 0.0);
  if (g) d->g.assign(g, g + nlam);
  d->gray = true;
  for (int b = 1; b < nlam; ++b)
    if (d->kabs[b] != d->kabs[0] || d->ksca[b] != d->ksca[0] || d->g[b] != d->g[0]) d->gray = false;

  DustArrays dust;
  dust_arrays(nlam, d->lam_e.data(), d->kabs.data(), d->ksca.data(), d->g.data(), d->Tstar, dust);
  const std::vector<double>&chi = dust.chi, &alb = dust.alb, &chip = dust.chip, &star = dust.star;
  const int nT = d->nT;
  TGridTables tt;
  build_T_tables(nlam, d->lam_e.data(), d->kabs.data(), chip.data(), nT, d->Tmin, d->Tmax, tt);
  cudaError_t e;
#define UP(buf, vec)                                   \
  do {                                                 \
    e = upload(buf, vec);                              \
    if (e != cudaSuccess) return cuda_fail(d, e, "upload"); \
  } while (0)
  UP(d->chi32, cast_vec<float>(chi));
  UP(d->alb32, cast_vec<float>(alb));
  UP(d->g32, cast_vec<float>(d->g));
  UP(d->star32, cast_vec<float>(star));
  UP(d->chi64, chi);
  UP(d->alb64, alb);
  UP(d->g64, d->g);
  UP(d->star64, star);
  UP(d->lQk, tt.lQk);
  UP(d->lQ64, tt.lQ64);
  UP(d->slQ64, tt.slQ64);
  UP(d->cbw, tt.cbw);
  UP(d->cexit, tt.cexit);
  UP(d->chiRk, tt.chiRk);
  UP(d->kbark, tt.kbark);
  UP(d->jw, tt.jw);
  UP(d->lam_e_d, d->lam_e);
  UP(d->kabs_d, d->kabs);
  UP(d->chip_d, chip);
#undef UP
  d->chiR0 = (float)chip[0];
  d->kbar0 = (float)d->kabs[0];
  e = d->sed.alloc((size_t)nlam * kNInc * 8);
  if (e != cudaSuccess) return cuda_fail(d, e, "cudaMalloc");
  if (d->keep_j) {  // the J tally follows the number of bins
    e = d->jlen.alloc((size_t)d->nr * d->nt * nlam * 8);
    if (e != cudaSuccess) return cuda_fail(d, e, "cudaMalloc");
  }
  d->has_opacity = true;
  mcrt_status st = zero_tallies(d);
  if (st != MCRT_OK) return st;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_reset(mcrt_disk* d) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  mcrt_status s = zero_tallies(d);
  if (s != MCRT_OK) return s;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_launch_count(const mcrt_disk* d, uint64_t* n) {
  if (!d || !n) return set_error(nullptr, MCRT_EINVAL, "bad arguments");
  *n = d->launches;
  return MCRT_OK;
}

mcrt_status mcrt_disk_info(const mcrt_disk* d, int* nr, int* ntheta, int* nlam) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (nr) *nr = d->nr;
  if (ntheta) *ntheta = d->nt;
  if (nlam) *nlam = d->nlam;
  return MCRT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// transport runs
// ------------------------------------------------------------------------------------------------
static mcrt_status check_opts(mcrt_disk* d, const mcrt_run_opts* o) {
  if (!o) return set_error(d, MCRT_EINVAL, "opts is NULL");
  if (o->precision != 32 && o->precision != 64) return set_error(d, MCRT_EINVAL, "precision must be 32 or 64");
  if (o->mrw && !(o->gamma > 0)) return set_error(d, MCRT_EINVAL, "gamma must be > 0");
  if (o->mrw && o->mrw_min_interactions < 0) return set_error(d, MCRT_EINVAL, "mrw_min_interactions < 0");
  if (o->max_events_per_packet == 0) return set_error(d, MCRT_EINVAL, "max_events_per_packet must be > 0");
  if (o->block_size && (o->block_size % 32 || o->block_size > 256))
    return set_error(d, MCRT_EINVAL, "block_size must be a multiple of 32 up to 256");
  if (o->refill_interval < 0) return set_error(d, MCRT_EINVAL, "refill_interval < 0");
  if (o->tail_warps_per_sm < -1 || o->tail_warps_per_sm > 32)
    return set_error(d, MCRT_EINVAL, "tail_warps_per_sm must be -1..32");
  if (o->interact_batch < 0 || o->interact_batch > 32) return set_error(d, MCRT_EINVAL, "interact_batch must be 0..32");
  return MCRT_OK;
}

template <class R>
static void fill_params(KParams<R>& P, const mcrt_run_opts* o, uint64_t seed, const float* tab) {
  P.mrw = o->mrw ? 1 : 0;
  P.nmin = o->mrw_min_interactions;
  P.exit_dir = o->mrw_exit_dir;
  P.refill = o->refill_interval > 0 ? o->refill_interval : 8;  // (single disks; batches tune theirs)
  P.defer = o->interact_batch > 0 ? o->interact_batch : 8;
  P.gamma = (R)o->gamma;
  P.seed = seed;
  // per-packet counters are 32-bit: caps above 2^31 events (4e9 steps) are clamped
  P.max_events = std::min<unsigned long long>(o->max_events_per_packet, 1ull << 31);
  P.max_steps = std::min<unsigned long long>(4ull * P.max_events + 10000000ull, 4000000000ull);
  P.mrw_tab = tab;
  P.mrw_t0 = kMrwT0;
  P.mrw_dt = kMrwDT;
  P.trace_n = 0;
  P.trace_max = 0;
  P.tr_type = P.tr_cell = P.tr_lam = P.tr_n = nullptr;
  P.tr_pos = nullptr;
  P.models = nullptr;
  P.nmodels = 1;
  P.trip = nullptr;
}

static void stats_from(const unsigned long long* c, mcrt_run_stats* s, double secs) {
  s->packets = c[C_PACKETS];
  s->events = c[C_EVENTS];
  s->absorptions = c[C_ABS];
  s->scatterings = c[C_SCA];
  s->crossings = c[C_CROSS];
  s->mrw_jumps = c[C_MRW];
  s->capped = c[C_CAPPED];
  s->escaped = c[C_ESCAPED];
  s->deposit_sum = c[C_DEPSUM];
  s->error_flags = (uint32_t)c[C_ERR];
  s->seconds = secs;
  s->max_packet_steps = c[C_MAXSTEPS];
  s->longest_packet = c[C_LONGEST] & 0xffffffull;
  s->guarded = c[C_GUARDS];
  s->guard_packet = 0;
  s->guard_kind = 0;
  s->guard_in_tail = 0;
  s->guard_cell[0] = s->guard_cell[1] = -1;
  for (int i = 0; i < 3; ++i) s->guard_pos_cm[i] = s->guard_dir[i] = 0.0;
  s->guard_events = s->guard_steps = 0;
}

// the record of the first packet dropped by a step guard (words of note_trip) into the run statistics
static void trip_from(const unsigned long long* t, double l_unit, mcrt_run_stats* s) {
  if (t[0] == 0) return;
  double v[8];
  std::memcpy(v, t + 8, sizeof(v));
  s->guard_packet = t[1];
  s->guard_kind = (int32_t)(t[2] & 255u);
  s->guard_in_tail = (t[2] & 256u) ? 1 : 0;
  s->guard_cell[0] = (int32_t)(long long)t[3];
  s->guard_cell[1] = (int32_t)(long long)t[4];
  s->guard_events = t[5];
  s->guard_steps = t[6];
  for (int i = 0; i < 3; ++i) {
    s->guard_pos_cm[i] = v[i] * l_unit;
    s->guard_dir[i] = v[3 + i];
  }
}

// events = scatterings + absorptions + MRW jumps (the kernel counts the three separately)
static void fix_events(unsigned long long* c) { c[C_EVENTS] = c[C_ABS] + c[C_SCA] + c[C_MRW]; }

// sizes the tail pool for `cap` threads and clears its counters on the disk's stream; without it
// (allocation failure, or tail kernel off) the transport kernel finishes every packet itself
template <class R>
static bool setup_pool(mcrt_disk* d, KParams<R>& P, unsigned cap, int tail_warps) {
  P.pool = nullptr;
  P.pool_ctr = nullptr;
  P.pool_cap = 0;
  if (tail_warps < 0) return false;
  if (d->pool_cap < cap) {
    d->pool_cap = 0;
    if (d->pool.alloc((size_t)cap * sizeof(Pkt<double>)) != cudaSuccess || d->pool_ctr.alloc(16) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    d->pool_cap = cap;
  }
  if (cudaMemsetAsync(d->pool_ctr.p, 0, 16, d->stream) != cudaSuccess) return false;
  P.pool = d->pool.as<Pkt<R>>();
  P.pool_ctr = d->pool_ctr.as<unsigned>();
  P.pool_cap = cap;
  return true;
}

// blocks of a single-disk transport launch: one packet per thread, at most the device's resident blocks,
// and at most max_in_flight threads (whole blocks) when given
static int transport_grid(uint64_t n_packets, int block, int sms, int bps, uint64_t max_in_flight) {
  long long g = (long long)((n_packets + block - 1) / block);
  g = std::min<long long>(g, (long long)sms * std::max(1, bps));
  if (max_in_flight) g = std::min<long long>(g, (long long)((max_in_flight + block - 1) / block));
  return (int)std::max(1ll, g);
}

// packets in flight of a run: the caller's cap, else all threads for gray dust and n_total /
// MCRT_NONGRAY_IN_FLIGHT (at least one warp) for non-gray dust (see mcrt.h)
static uint64_t in_flight_cap(bool gray, double n_total, uint64_t requested) {
  if (requested || gray) return requested;
  return std::max<uint64_t>(32, (uint64_t)(n_total / MCRT_NONGRAY_IN_FLIGHT));
}

// Queue of a batch with non-gray dust: chunks of 32 slots of one model, ordered so that every model moves
// through its packets at the same pace (chunk k of model m at (k + 1/2) / chunks_m, ties by model), so that
// each model has the launch's share of its packets in flight (see MCRT_NONGRAY_IN_FLIGHT in mcrt.h).
// Entry: model << 48 | the model's first packet of the chunk.
static std::vector<unsigned long long> interleaved_queue(const uint64_t* n, int models) {
  std::vector<unsigned long long> out;
  using Item = std::pair<double, int>;
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> next;
  std::vector<uint64_t> chunks(models), k(models, 0);
  for (int i = 0; i < models; ++i) {
    chunks[i] = (n[i] + 31) / 32;
    if (chunks[i]) next.push({0.5 / (double)chunks[i], i});
  }
  while (!next.empty()) {
    const int i = next.top().second;
    next.pop();
    out.push_back(((unsigned long long)i << 48) | (k[i] * 32));
    if (++k[i] < chunks[i]) next.push({((double)k[i] + 0.5) / (double)chunks[i], i});
  }
  return out;
}

static mcrt_status run_impl(mcrt_disk* d, uint64_t n_packets, uint64_t seed, uint64_t first_id,
                            const mcrt_run_opts* o, mcrt_run_stats* stats, int trace_max, int32_t* tr_type,
                            int32_t* tr_cell, int32_t* tr_lam, double* tr_pos, int32_t* tr_n) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  mcrt_status s = check_opts(d, o);
  if (s != MCRT_OK) return s;
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  cudaError_t e;
  const float* tab = mrw_table(d->device, &e);
  if (!tab) return cuda_fail(d, e, "MRW table");
  d->n_total = (double)(o->n_total_packets ? o->n_total_packets : n_packets);
  const bool trace = trace_max > 0;
  const bool f64 = trace || o->precision == 64;
  const bool pol = d->pol, jt = d->keep_j;
  if (pol && trace) return set_error(d, MCRT_EINVAL, "polarized transport has no event trace");
  if (jt && trace) return set_error(d, MCRT_EINVAL, "the mean-intensity tally has no event trace");
  if (jt && pol) return set_error(d, MCRT_EINVAL, "polarized transport does not keep the mean intensity");
  CK(cudaMemsetAsync(d->cnt.p, 0, (C_NCNT + kTripWords) * 8, d->stream), "memset");
  CK(cudaMemsetAsync(d->queue.p, 0, 8, d->stream), "memset");
  DBuf ttype, tcell, tlam, tpos, tn;
  if (trace) {
    const size_t m = (size_t)n_packets * trace_max;
    e = ttype.alloc(m * 4);
    if (e == cudaSuccess) e = tcell.alloc(m * 4);
    if (e == cudaSuccess) e = tlam.alloc(m * 4);
    if (e == cudaSuccess) e = tpos.alloc(m * 24);
    if (e == cudaSuccess) e = tn.alloc(n_packets * 4);
    if (e != cudaSuccess) return cuda_fail(d, e, "trace buffers");
    CK(cudaMemsetAsync(tn.p, 0, n_packets * 4, d->stream), "memset");
  }
  int dev_sms = 0;
  CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, d->device), "attribute");
  const int block = o->block_size ? o->block_size : 128;
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0), "event");
  CK(cudaEventCreate(&ev1), "event");
  CK(cudaEventRecord(ev0, d->stream), "event");
  if (n_packets > 0) {
    if (f64) {
      KParams<double> P;
      std::memset(&P, 0, sizeof(P));
      fill_params(P, o, seed, tab);
      P.m0 = d->model64();
      P.m0.first_id = first_id;
      P.m0.n_packets = n_packets;
      P.m0.q_begin = 0;
      P.m0.model_id = 0;
      P.total = n_packets;
      P.queue = d->queue.as<unsigned long long>();
      P.trip = d->cnt.as<unsigned long long>() + C_NCNT;
      P.want_lam = (!d->gray || o->want_sed) ? 1 : 0;
      if (trace) {
        P.trace_n = (int)n_packets;
        P.trace_max = trace_max;
        P.tr_type = ttype.as<int32_t>();
        P.tr_cell = tcell.as<int32_t>();
        P.tr_lam = tlam.as<int32_t>();
        P.tr_pos = tpos.as<double>();
        P.tr_n = tn.as<int32_t>();
        P.l_unit = d->l_unit;
      }
      const int bps = pol  ? transport_blocks_per_sm_pol<double>(d->gray, block)
                      : jt ? transport_blocks_per_sm_j<double>(d->gray, block)
                           : transport_blocks_per_sm<double>(trace, false, d->gray, block);
      const int grid = transport_grid(n_packets, block, dev_sms, bps, in_flight_cap(d->gray, d->n_total, o->max_in_flight));
      const bool tail = setup_pool(d, P, (unsigned)grid * block, o->tail_warps_per_sm);
      e = pol  ? launch_transport_pol<double>(P, d->gray, grid, block, d->stream)
          : jt ? launch_transport_j<double>(P, d->gray, grid, block, d->stream)
               : launch_transport<double>(P, trace, false, d->gray, grid, block, d->stream);
      d->launches++;
      if (e == cudaSuccess && tail) {
        e = pol  ? launch_transport_tail_pol<double>(P, d->gray, dev_sms, o->tail_warps_per_sm, d->stream)
            : jt ? launch_transport_tail_j<double>(P, d->gray, dev_sms, o->tail_warps_per_sm, d->stream)
                 : launch_transport_tail<double>(P, trace, false, d->gray, dev_sms, o->tail_warps_per_sm, d->stream);
        d->launches++;
      }
    } else {
      KParams<float> P;
      std::memset(&P, 0, sizeof(P));
      fill_params(P, o, seed, tab);
      P.m0 = d->model32();
      P.m0.first_id = first_id;
      P.m0.n_packets = n_packets;
      P.m0.q_begin = 0;
      P.m0.model_id = 0;
      P.total = n_packets;
      P.queue = d->queue.as<unsigned long long>();
      P.trip = d->cnt.as<unsigned long long>() + C_NCNT;
      P.want_lam = (!d->gray || o->want_sed) ? 1 : 0;
      const int bps = pol  ? transport_blocks_per_sm_pol<float>(d->gray, block)
                      : jt ? transport_blocks_per_sm_j<float>(d->gray, block)
                           : transport_blocks_per_sm<float>(false, false, d->gray, block);
      const int grid = transport_grid(n_packets, block, dev_sms, bps, in_flight_cap(d->gray, d->n_total, o->max_in_flight));
      const bool tail = setup_pool(d, P, (unsigned)grid * block, o->tail_warps_per_sm);
      e = pol  ? launch_transport_pol<float>(P, d->gray, grid, block, d->stream)
          : jt ? launch_transport_j<float>(P, d->gray, grid, block, d->stream)
               : launch_transport<float>(P, false, false, d->gray, grid, block, d->stream);
      d->launches++;
      if (e == cudaSuccess && tail) {
        e = pol  ? launch_transport_tail_pol<float>(P, d->gray, dev_sms, o->tail_warps_per_sm, d->stream)
            : jt ? launch_transport_tail_j<float>(P, d->gray, dev_sms, o->tail_warps_per_sm, d->stream)
                 : launch_transport_tail<float>(P, false, false, d->gray, dev_sms, o->tail_warps_per_sm, d->stream);
        d->launches++;
      }
    }
    if (e != cudaSuccess) {
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
      return cuda_fail(d, e, "transport launch");
    }
  }
  CK(cudaEventRecord(ev1, d->stream), "event");
  unsigned long long c[C_NCNT + kTripWords];
  CK(cudaMemcpyAsync(c, d->cnt.p, sizeof(c), cudaMemcpyDeviceToHost, d->stream), "copy counters");
  if (trace) {
    const size_t m = (size_t)n_packets * trace_max;
    if (tr_type) CK(cudaMemcpyAsync(tr_type, ttype.p, m * 4, cudaMemcpyDeviceToHost, d->stream), "copy");
    if (tr_cell) CK(cudaMemcpyAsync(tr_cell, tcell.p, m * 4, cudaMemcpyDeviceToHost, d->stream), "copy");
    if (tr_lam) CK(cudaMemcpyAsync(tr_lam, tlam.p, m * 4, cudaMemcpyDeviceToHost, d->stream), "copy");
    if (tr_pos) CK(cudaMemcpyAsync(tr_pos, tpos.p, m * 24, cudaMemcpyDeviceToHost, d->stream), "copy");
    if (tr_n) CK(cudaMemcpyAsync(tr_n, tn.p, n_packets * 4, cudaMemcpyDeviceToHost, d->stream), "copy");
  }
  e = cudaStreamSynchronize(d->stream);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (e != cudaSuccess) return cuda_fail(d, e, "transport kernel");
  fix_events(c);
  d->packets_done += n_packets;
  d->have_T = false;
  d->have_pda = false;
  if (stats) {
    stats_from(c, stats, ms * 1e-3);
    trip_from(c + C_NCNT, d->l_unit, stats);
  }
  if (!account_deposits(d, c)) return set_error(d, MCRT_EOVERFLOW, "fixed-point tally overflow");
  if (c[C_ERR] & kErrStepGuard) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "packet step guard reached: %llu packet(s) dropped, the first packet id %llu",
                  c[C_GUARDS], c[C_NCNT] ? c[C_NCNT + 1] : 0ull);
    return set_error(d, MCRT_ETIMEOUT, msg);
  }
  return MCRT_OK;
}

extern "C" {

mcrt_status mcrt_run_photons(mcrt_disk* d, uint64_t n_packets, uint64_t seed, uint64_t first_packet_id,
                             const mcrt_run_opts* opts, mcrt_run_stats* stats) {
  return run_impl(d, n_packets, seed, first_packet_id, opts, stats, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
}

mcrt_status mcrt_trace_packets(mcrt_disk* d, uint64_t n_packets, uint64_t seed, uint64_t first_packet_id,
                               const mcrt_run_opts* opts, int max_events, int32_t* type, int32_t* cell, int32_t* lam,
                               double* pos, int32_t* n_events) {
  if (max_events <= 0) return set_error(d, MCRT_EINVAL, "max_events must be > 0");
  if (n_packets > (1ull << 24) || (unsigned long long)n_packets * (unsigned long long)max_events > (1ull << 31))
    return set_error(d, MCRT_EINVAL, "trace too large");
  return run_impl(d, n_packets, seed, first_packet_id, opts, nullptr, max_events, type, cell, lam, pos, n_events);
}

mcrt_status mcrt_run_batch(mcrt_disk* const* disks, int n, const uint64_t* n_packets, uint64_t seed,
                           const mcrt_run_opts* o, mcrt_run_stats* stats) {
  if (!disks || n <= 0 || !n_packets) return set_error(nullptr, MCRT_EINVAL, "bad batch arguments");
  mcrt_disk* d0 = disks[0];
  for (int i = 0; i < n; ++i) {
    if (!disks[i]) return set_error(nullptr, MCRT_EINVAL, "NULL disk in batch");
    if (!disks[i]->has_opacity) return set_error(disks[i], MCRT_ESTATE, "mcrt_set_opacity must come first");
    if (disks[i]->pol) return set_error(disks[i], MCRT_EINVAL, "batches do not take polarized disks");
    if (disks[i]->keep_j) return set_error(disks[i], MCRT_EINVAL, "batches do not keep the mean intensity");
    if (disks[i]->device != d0->device) return set_error(disks[i], MCRT_EINVAL, "batch disks on different devices");
  }
  mcrt_disk* d = d0;
  mcrt_status s = check_opts(d, o);
  if (s != MCRT_OK) return s;
  if (o->precision != 32) return set_error(d, MCRT_EINVAL, "batches run the FP32 path");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  cudaError_t e;
  const float* tab = mrw_table(d->device, &e);
  if (!tab) return cuda_fail(d, e, "MRW table");
  std::vector<DevModel<float>> ms(n);
  unsigned long long q = 0;
  for (int i = 0; i < n; ++i) {
    disks[i]->n_total = (double)n_packets[i];
    ms[i] = disks[i]->model32();
    ms[i].first_id = 0;
    ms[i].n_packets = n_packets[i];
    ms[i].q_begin = q;
    ms[i].model_id = (uint32_t)i;
    q += n_packets[i];
    if (disks[i] != d) {
      // other disks' counters are zeroed on the shared stream below
    }
  }
  DBuf dm;
  e = dm.alloc(sizeof(DevModel<float>) * n);
  if (e != cudaSuccess) return cuda_fail(d, e, "cudaMalloc");
  CK(cudaMemcpyAsync(dm.p, ms.data(), sizeof(DevModel<float>) * n, cudaMemcpyHostToDevice, d->stream), "copy");
  for (int i = 0; i < n; ++i) CK(cudaMemsetAsync(disks[i]->cnt.p, 0, C_NCNT * 8, d->stream), "memset");
  CK(cudaMemsetAsync(d->queue.p, 0, 8, d->stream), "memset");
  KParams<float> P;
  std::memset(&P, 0, sizeof(P));
  fill_params(P, o, seed, tab);
  P.m0 = ms[0];
  P.models = dm.as<DevModel<float>>();
  P.nmodels = n;
  P.total = q;
  P.queue = d->queue.as<unsigned long long>();
  bool any_nongray = false;
  for (int i = 0; i < n; ++i) any_nongray |= !disks[i]->gray;
  P.want_lam = (any_nongray || o->want_sed) ? 1 : 0;
  DBuf qmap;
  if (any_nongray) {  // the models' packets interleaved, each model with the launch's share in flight
    if (n > 65535) return set_error(d, MCRT_EINVAL, "a non-gray batch takes at most 65535 disks");
    const std::vector<unsigned long long> qm = interleaved_queue(n_packets, n);
    CK(qmap.alloc(qm.size() * 8), "cudaMalloc");
    CK(cudaMemcpyAsync(qmap.p, qm.data(), qm.size() * 8, cudaMemcpyHostToDevice, d->stream), "copy");
    P.qmap = qmap.as<unsigned long long>();
    P.total = 32ull * qm.size();
  }
  int dev_sms = 0;
  CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, d->device), "attribute");
  const int block = o->block_size ? o->block_size : 128;
  const int bps = transport_blocks_per_sm<float>(false, true, false, block);
  const int grid = transport_grid(P.total, block, dev_sms, bps, in_flight_cap(!any_nongray, (double)q, o->max_in_flight));
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0), "event");
  CK(cudaEventCreate(&ev1), "event");
  CK(cudaEventRecord(ev0, d->stream), "event");
  if (q > 0) {
    e = launch_transport<float>(P, false, true, false, grid, block, d->stream);
    d->launches++;
    if (e != cudaSuccess) return cuda_fail(d, e, "transport launch");
  }
  CK(cudaEventRecord(ev1, d->stream), "event");
  std::vector<unsigned long long> c((size_t)n * C_NCNT);
  for (int i = 0; i < n; ++i)
    CK(cudaMemcpyAsync(&c[(size_t)i * C_NCNT], disks[i]->cnt.p, C_NCNT * 8, cudaMemcpyDeviceToHost, d->stream),
       "copy");
  e = cudaStreamSynchronize(d->stream);
  float ms_ = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms_, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (e != cudaSuccess) return cuda_fail(d, e, "transport kernel");
  mcrt_status ret = MCRT_OK;
  for (int i = 0; i < n; ++i) {
    unsigned long long* ci = &c[(size_t)i * C_NCNT];
    fix_events(ci);
    disks[i]->packets_done += n_packets[i];
    disks[i]->have_T = false;
    disks[i]->have_pda = false;
    if (stats) stats_from(ci, &stats[i], ms_ * 1e-3);
    if (!account_deposits(disks[i], ci)) ret = set_error(disks[i], MCRT_EOVERFLOW, "fixed-point tally overflow");
  }
  return ret;
}

mcrt_status mcrt_temperatures(mcrt_disk* d, int which, double* T, double* relerr, uint64_t* visits) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!T) return set_error(d, MCRT_EINVAL, "T is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  if (which != MCRT_T_MC && which != MCRT_T_PDA) return set_error(d, MCRT_EINVAL, "which");
  if (which == MCRT_T_PDA && !d->have_pda) return set_error(d, MCRT_ESTATE, "no PDA solution");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (!d->have_T) {
    mcrt_status s = compute_temperatures(d);
    if (s != MCRT_OK) return s;
  }
  const size_t n = (size_t)d->nr * d->nt;
  CK(cudaMemcpyAsync(T, which == MCRT_T_PDA ? d->T_pda.p : d->T_mc.p, n * 8, cudaMemcpyDeviceToHost, d->stream),
     "copy");
  if (relerr) CK(cudaMemcpyAsync(relerr, d->relerr.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (visits) CK(cudaMemcpyAsync(visits, d->visits.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_temperatures_dev(mcrt_disk* d, int which, double* T, double* relerr) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!T) return set_error(d, MCRT_EINVAL, "T is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  if (which == MCRT_T_PDA && !d->have_pda) return set_error(d, MCRT_ESTATE, "no PDA solution");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  if (!d->have_T) {
    mcrt_status s = compute_temperatures(d);
    if (s != MCRT_OK) return s;
  }
  const size_t n = (size_t)d->nr * d->nt;
  CK(cudaMemcpyAsync(T, which == MCRT_T_PDA ? d->T_pda.p : d->T_mc.p, n * 8, cudaMemcpyDeviceToDevice, d->stream),
     "copy");
  if (relerr) CK(cudaMemcpyAsync(relerr, d->relerr.p, n * 8, cudaMemcpyDeviceToDevice, d->stream), "copy");
  return MCRT_OK;
}

mcrt_status mcrt_get_tallies(mcrt_disk* d, uint64_t* tally, uint64_t* visits, uint64_t* nabs) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  const size_t n = (size_t)d->nr * d->nt * 8;
  if (tally) CK(cudaMemcpyAsync(tally, d->tally.p, n, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (visits) CK(cudaMemcpyAsync(visits, d->visits.p, n, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (nabs) CK(cudaMemcpyAsync(nabs, d->nabs.p, n, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_sed(mcrt_disk* d, int n_incl, double* L) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!L || n_incl <= 0 || kNInc % n_incl) return set_error(d, MCRT_EINVAL, "n_incl must divide 10");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  std::vector<unsigned long long> c((size_t)d->nlam * kNInc);
  CK(cudaMemcpyAsync(c.data(), d->sed.p, c.size() * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  const double e = d->Lpkt() / (d->n_total > 0 ? d->n_total : 1.0);
  const int grp = kNInc / n_incl;
  for (int b = 0; b < d->nlam; ++b)
    for (int i = 0; i < n_incl; ++i) {
      unsigned long long s = 0;
      for (int j = 0; j < grp; ++j) s += c[(size_t)b * kNInc + i * grp + j];
      L[(size_t)b * n_incl + i] = (double)s * e;
    }
  return MCRT_OK;
}

// checkpoint layout: 8 x uint64 header (magic, version, nr, nt, nlam, packets_done, n_total bits, 0),
// then tally, visits, nabs (nr*nt each) and sed (nlam*10), all uint64.
mcrt_status mcrt_keep_mean_intensity(mcrt_disk* d, int keep) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  const size_t bytes = (size_t)d->nr * d->nt * d->nlam * 8;
  if (keep && d->jlen.n != bytes) {
    cudaError_t e = d->jlen.alloc(bytes);
    if (e != cudaSuccess) return cuda_fail(d, e, "cudaMalloc");
  }
  if (!keep) d->jlen.release();
  d->keep_j = keep != 0;
  mcrt_status s = zero_tallies(d);
  if (s != MCRT_OK) return s;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_set_mueller(mcrt_disk* d, int nmu, const double* table) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  if (!table) {
    d->pol = false;
    d->nmu = 0;
    return MCRT_OK;
  }
  if (nmu < 2 || nmu > 4097) return set_error(d, MCRT_EINVAL, "nmu: 2 .. 4097 scattering angles");
  const size_t nl = (size_t)d->nlam, m = (size_t)nmu;
  std::vector<double> cdf(nl * m);
  for (size_t b = 0; b < nl; ++b) {
    const double* t = table + b * 4 * m;
    for (size_t k = 0; k < 4 * m; ++k)
      if (!std::isfinite(t[k])) return set_error(d, MCRT_EINVAL, "Mueller matrix: finite values");
    for (size_t k = 0; k < m; ++k)
      if (t[k] < 0) return set_error(d, MCRT_EINVAL, "Mueller matrix: S11 >= 0");
    if (!mueller_cdf(t, nmu, cdf.data() + b * m)) return set_error(d, MCRT_EINVAL, "Mueller matrix: S11 vanishes");
  }
  std::vector<double> tab(table, table + nl * 4 * m);
  cudaError_t e = upload(d->mtab64, tab);
  if (e == cudaSuccess) e = upload(d->mtab32, cast_vec<float>(tab));
  if (e == cudaSuccess) e = upload(d->mcdf64, cdf);
  if (e == cudaSuccess) e = upload(d->mcdf32, cast_vec<float>(cdf));
  if (e == cudaSuccess && d->sed_q.n < nl * kNInc * 8) e = d->sed_q.alloc(nl * kNInc * 8);
  if (e == cudaSuccess && d->sed_u.n < nl * kNInc * 8) e = d->sed_u.alloc(nl * kNInc * 8);
  if (e != cudaSuccess) return cuda_fail(d, e, "upload");
  d->nmu = nmu;
  d->pol = true;
  mcrt_status s = zero_tallies(d);
  if (s != MCRT_OK) return s;
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

mcrt_status mcrt_sed_stokes(mcrt_disk* d, int n_incl, double* L_I, double* L_Q, double* L_U) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!L_I || !L_Q || !L_U || n_incl <= 0 || kNInc % n_incl) return set_error(d, MCRT_EINVAL, "n_incl must divide 10");
  if (!d->pol) return set_error(d, MCRT_ESTATE, "mcrt_set_mueller must come first");
  mcrt_status s = mcrt_sed(d, n_incl, L_I);
  if (s != MCRT_OK) return s;
  const size_t nc = (size_t)d->nlam * kNInc;
  std::vector<unsigned long long> q(nc), u(nc);
  CK(cudaMemcpyAsync(q.data(), d->sed_q.p, nc * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaMemcpyAsync(u.data(), d->sed_u.p, nc * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  const double e = d->Lpkt() / (d->n_total > 0 ? d->n_total : 1.0) / 1048576.0;
  const int grp = kNInc / n_incl;
  for (int b = 0; b < d->nlam; ++b)
    for (int i = 0; i < n_incl; ++i) {
      long long sq = 0, su = 0;
      for (int j = 0; j < grp; ++j) {
        sq += (long long)q[(size_t)b * kNInc + i * grp + j];
        su += (long long)u[(size_t)b * kNInc + i * grp + j];
      }
      L_Q[(size_t)b * n_incl + i] = (double)sq * e;
      L_U[(size_t)b * n_incl + i] = (double)su * e;
    }
  return MCRT_OK;
}

mcrt_status mcrt_checkpoint(mcrt_disk* d, void* buf, size_t* len) {
  if (!d || !len) return set_error(d, MCRT_EINVAL, "bad arguments");
  const size_t n = (size_t)d->nr * d->nt;
  const size_t nsed = (size_t)d->nlam * kNInc;
  const size_t need = 8 * (8 + 3 * n + nsed);
  if (!buf) {
    *len = need;
    return MCRT_OK;
  }
  if (*len < need) return set_error(d, MCRT_EINVAL, "checkpoint buffer too small");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  uint64_t* h = (uint64_t*)buf;
  uint64_t ntb;
  std::memcpy(&ntb, &d->n_total, 8);
  const uint64_t hdr[8] = {0x4D43525443484B31ull, 1, (uint64_t)d->nr, (uint64_t)d->nt, (uint64_t)d->nlam,
                           d->packets_done, ntb, 0};
  std::memcpy(h, hdr, sizeof(hdr));
  CK(cudaMemcpyAsync(h + 8, d->tally.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaMemcpyAsync(h + 8 + n, d->visits.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaMemcpyAsync(h + 8 + 2 * n, d->nabs.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (nsed) CK(cudaMemcpyAsync(h + 8 + 3 * n, d->sed.p, nsed * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  *len = need;
  return MCRT_OK;
}

mcrt_status mcrt_restore(mcrt_disk* d, const void* buf, size_t len) {
  if (!d || !buf) return set_error(d, MCRT_EINVAL, "bad arguments");
  const size_t n = (size_t)d->nr * d->nt;
  const size_t nsed = (size_t)d->nlam * kNInc;
  if (len < 64) return set_error(d, MCRT_EINVAL, "checkpoint too short");
  const uint64_t* h = (const uint64_t*)buf;
  if (h[0] != 0x4D43525443484B31ull || h[1] != 1 || h[2] != (uint64_t)d->nr || h[3] != (uint64_t)d->nt ||
      h[4] != (uint64_t)d->nlam || len < 8 * (8 + 3 * n + nsed))
    return set_error(d, MCRT_EINVAL, "checkpoint does not match this disk");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  CK(cudaMemcpyAsync(d->tally.p, h + 8, n * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaMemcpyAsync(d->visits.p, h + 8 + n, n * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  CK(cudaMemcpyAsync(d->nabs.p, h + 8 + 2 * n, n * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  if (nsed) CK(cudaMemcpyAsync(d->sed.p, h + 8 + 3 * n, nsed * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  // the tallies a checkpoint does not hold (Stokes Q/U, mean-intensity path lengths) start from zero
  if (d->sed_q.p) CK(cudaMemsetAsync(d->sed_q.p, 0, d->sed_q.n, d->stream), "memset");
  if (d->sed_u.p) CK(cudaMemsetAsync(d->sed_u.p, 0, d->sed_u.n, d->stream), "memset");
  if (d->keep_j && d->jlen.p) CK(cudaMemsetAsync(d->jlen.p, 0, d->jlen.n, d->stream), "memset");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  d->packets_done = h[5];
  std::memcpy(&d->n_total, &h[6], 8);
  d->tally_held = 0;
  d->tally_wrapped = false;
  for (size_t c = 0; c < n; ++c) {
    const unsigned long long t = d->tally_held + h[8 + c];
    if (t < d->tally_held) d->tally_wrapped = true;
    d->tally_held = t;
  }
  d->have_T = false;
  d->have_pda = false;
  return MCRT_OK;
}

mcrt_status mcrt_debug_uniforms(int device, uint64_t seed, uint32_t model, uint64_t packet, int n, double* out) {
  if (n <= 0 || n > (1 << 20) || !out) return set_error(nullptr, MCRT_EINVAL, "bad arguments");
  mcrt_disk* d = nullptr;
  CK(cudaSetDevice(device), "cudaSetDevice");
  double* p = nullptr;
  CK(cudaMalloc(&p, sizeof(double) * n), "cudaMalloc");
  k_uniforms<<<1, 32>>>(seed, model, packet, n, p);
  cudaError_t e = cudaMemcpy(out, p, sizeof(double) * n, cudaMemcpyDeviceToHost);
  cudaFree(p);
  if (e != cudaSuccess) return cuda_fail(d, e, "debug uniforms");
  return MCRT_OK;
}

mcrt_status mcrt_debug_mrw_x(int device, int n, const double* P0, double* out) {
  if (n <= 0 || n > (1 << 24) || !P0 || !out) return set_error(nullptr, MCRT_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i)
    if (!(P0[i] > 0 && P0[i] < 1)) return set_error(nullptr, MCRT_EINVAL, "P0 must be in (0, 1)");
  mcrt_disk* d = nullptr;
  CK(cudaSetDevice(device), "cudaSetDevice");
  cudaError_t e;
  const float* tab = mrw_table(device, &e);
  if (!tab) return cuda_fail(d, e, "MRW table");
  double *a = nullptr, *b = nullptr;
  CK(cudaMalloc(&a, sizeof(double) * n), "cudaMalloc");
  e = cudaMalloc(&b, sizeof(double) * n);
  if (e != cudaSuccess) {
    cudaFree(a);
    return cuda_fail(d, e, "cudaMalloc");
  }
  e = cudaMemcpy(a, P0, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_mrw_x<<<(n + 255) / 256, 256>>>(n, a, b, tab, kMrwT0, kMrwDT);
    e = cudaMemcpy(out, b, sizeof(double) * n, cudaMemcpyDeviceToHost);
  }
  cudaFree(a);
  cudaFree(b);
  if (e != cudaSuccess) return cuda_fail(d, e, "debug mrw");
  return MCRT_OK;
}

const char* mcrt_last_error(const mcrt_disk* d) { return d ? d->err.c_str() : g_err.c_str(); }

void mcrt_disk_destroy(mcrt_disk* d) {
  if (!d) return;
  cudaSetDevice(d->device);
  if (d->stream) cudaStreamSynchronize(d->stream);
  if (d->pda) pda_free(d->pda);
  d->pda = nullptr;
  if (d->rays) ray_free(d->rays);
  d->rays = nullptr;
  cudaStream_t st = d->own_stream ? d->stream : nullptr;
  delete d;  // frees the device buffers
  if (st) cudaStreamDestroy(st);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// prepared batches: descriptors built once, autotuned launch shape, CUDA graph replay
// ------------------------------------------------------------------------------------------------
struct mcrt_batch {
  int n = 0, device = 0;
  cudaStream_t stream = nullptr;
  std::vector<mcrt_disk*> disks;
  std::vector<uint64_t> npk;
  unsigned long long total = 0;
  DBuf models, queue, qmap;  // qmap: the interleaved queue of a non-gray batch
  KParams<float> P;
  int block = 256, refill = 1, grid = 0;
  double tune_seconds = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> knodes;  // kernel nodes (their KParams carry the seed)
  DBuf pool, pool_ctr;                   // packets in flight at the drain, for the tail kernel
  int tail_warps = 0, sms = 0;
  std::string err;
  ~mcrt_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace {
// direct (uncaptured) launch of the batch kernel with a given shape, counters zeroed first
cudaError_t batch_launch(mcrt_batch* b, const KParams<float>& P, int block, int grid) {
  cudaError_t e;
  for (auto* dk : b->disks) {
    e = cudaMemsetAsync(dk->cnt.p, 0, C_NCNT * 8, b->stream);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(b->queue.p, 0, 8, b->stream);
  if (e != cudaSuccess) return e;
  if (P.pool) {
    e = cudaMemsetAsync(P.pool_ctr, 0, 16, b->stream);
    if (e != cudaSuccess) return e;
  }
  e = launch_transport<float>(P, false, true, false, grid, block, b->stream);
  if (e != cudaSuccess || !P.pool) return e;
  return launch_transport_tail<float>(P, false, true, false, b->sms, b->tail_warps, b->stream);
}
}  // namespace

extern "C" {

mcrt_status mcrt_batch_create(mcrt_disk* const* disks, int n, const uint64_t* n_packets, const mcrt_run_opts* o,
                              mcrt_batch** out) {
  if (!out) return set_error(nullptr, MCRT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!disks || n <= 0 || !n_packets) return set_error(nullptr, MCRT_EINVAL, "bad batch arguments");
  for (int i = 0; i < n; ++i) {
    if (!disks[i]) return set_error(nullptr, MCRT_EINVAL, "NULL disk in batch");
    if (!disks[i]->has_opacity) return set_error(disks[i], MCRT_ESTATE, "mcrt_set_opacity must come first");
    if (disks[i]->pol) return set_error(disks[i], MCRT_EINVAL, "batches do not take polarized disks");
    if (disks[i]->keep_j) return set_error(disks[i], MCRT_EINVAL, "batches do not keep the mean intensity");
    if (disks[i]->device != disks[0]->device) return set_error(nullptr, MCRT_EINVAL, "disks on different devices");
  }
  mcrt_disk* d = disks[0];
  mcrt_status s = check_opts(d, o);
  if (s != MCRT_OK) return s;
  if (o->precision != 32) return set_error(d, MCRT_EINVAL, "batches run the FP32 path");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  cudaError_t e;
  const float* tab = mrw_table(d->device, &e);
  if (!tab) return cuda_fail(d, e, "MRW table");
  mcrt_batch* b = new (std::nothrow) mcrt_batch();
  if (!b) return set_error(nullptr, MCRT_ENOMEM, "host allocation");
  b->n = n;
  b->device = d->device;
  b->stream = d->stream;
  b->disks.assign(disks, disks + n);
  b->npk.assign(n_packets, n_packets + n);
  std::vector<DevModel<float>> ms(n);
  bool any_nongray = false;
  for (int i = 0; i < n; ++i) {
    disks[i]->n_total = (double)n_packets[i];
    ms[i] = disks[i]->model32();
    ms[i].first_id = 0;
    ms[i].n_packets = n_packets[i];
    ms[i].q_begin = b->total;
    ms[i].model_id = (uint32_t)i;
    b->total += n_packets[i];
    any_nongray |= !disks[i]->gray;
  }
  e = b->models.alloc(sizeof(DevModel<float>) * n);
  if (e == cudaSuccess) e = b->queue.alloc(8);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->models.p, ms.data(), sizeof(DevModel<float>) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(d, e, "batch buffers");
  }
  std::memset(&b->P, 0, sizeof(b->P));
  fill_params(b->P, o, 1, tab);
  b->P.m0 = ms[0];
  b->P.models = b->models.as<DevModel<float>>();
  b->P.nmodels = n;
  b->P.total = b->total;
  b->P.queue = b->queue.as<unsigned long long>();
  b->P.want_lam = (any_nongray || o->want_sed) ? 1 : 0;
  if (any_nongray) {  // the models' packets interleaved, each model with the launch's share in flight
    if (n > 65535) {
      delete b;
      return set_error(d, MCRT_EINVAL, "a non-gray batch takes at most 65535 disks");
    }
    const std::vector<unsigned long long> qm = interleaved_queue(n_packets, n);
    e = b->qmap.alloc(qm.size() * 8);
    if (e == cudaSuccess) e = cudaMemcpy(b->qmap.p, qm.data(), qm.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(d, e, "batch queue");
    }
    b->P.qmap = b->qmap.as<unsigned long long>();
    b->P.total = 32ull * qm.size();
  }
  const uint64_t cap = in_flight_cap(!any_nongray, (double)b->total, o->max_in_flight);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device);
  auto grid_for = [&](int block) {
    return transport_grid(b->P.total, block, sms, transport_blocks_per_sm<float>(false, true, false, block), cap);
  };
  if (o->block_size) {
    b->block = o->block_size;
    b->refill = o->refill_interval > 0 ? o->refill_interval : 1;
  } else {
    // autotune on a short run of about 5 % of the packets (at least one per model)
    std::vector<DevModel<float>> mt = ms;
    unsigned long long tq = 0;
    for (int i = 0; i < n; ++i) {
      const unsigned long long k = std::max<unsigned long long>(1, n_packets[i] / 20);
      mt[i].n_packets = k;
      mt[i].q_begin = tq;
      tq += k;
    }
    DBuf tm;
    e = tm.alloc(sizeof(DevModel<float>) * n);
    if (e == cudaSuccess) e = cudaMemcpy(tm.p, mt.data(), sizeof(DevModel<float>) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(d, e, "tuning buffers");
    }
    KParams<float> T = b->P;
    T.models = tm.as<DevModel<float>>();
    T.total = tq;
    T.qmap = nullptr;  // the tuning run takes each model's packets in one range
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    const int blocks[3] = {64, 128, 256}, refills[3] = {1, 4, 16};
    auto t_start = std::chrono::steady_clock::now();
    for (int bi = 0; bi < 3; ++bi)
      for (int ri = 0; ri < 3; ++ri) {
        T.refill = refills[ri];
        cudaEventRecord(e0, b->stream);
        e = batch_launch(b, T, blocks[bi], grid_for(blocks[bi]));
        cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          delete b;
          return cuda_fail(d, e, "autotune launch");
        }
        float ms_ = 0.f;
        cudaEventElapsedTime(&ms_, e0, e1);
        if (ms_ < best) {
          best = ms_;
          b->block = blocks[bi];
          b->refill = refills[ri];
        }
      }
    b->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int i = 0; i < n; ++i) {
      s = zero_tallies(disks[i]);
      if (s != MCRT_OK) {
        delete b;
        return s;
      }
    }
  }
  b->P.refill = b->refill;
  b->grid = grid_for(b->block);
  // the tail kernel's pool: one slot per thread of the chosen launch (the autotuner ran without it)
  b->sms = sms;
  b->tail_warps = o->tail_warps_per_sm;
  if (o->tail_warps_per_sm >= 0) {
    const size_t cap = (size_t)b->grid * b->block;
    if (b->pool.alloc(cap * sizeof(Pkt<float>)) == cudaSuccess && b->pool_ctr.alloc(16) == cudaSuccess) {
      b->P.pool = b->pool.as<Pkt<float>>();
      b->P.pool_ctr = b->pool_ctr.as<unsigned>();
      b->P.pool_cap = (unsigned)cap;
    } else {
      cudaGetLastError();
    }
  }
  // capture: counter resets + the persistent launch
  e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t el = batch_launch(b, b->P, b->block, b->grid);
    e = cudaStreamEndCapture(b->stream, &b->graph);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e == cudaSuccess) {
    size_t nn = 0;
    e = cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess) e = cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    for (size_t k = 0; e == cudaSuccess && k < nn; ++k) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nodes[k], &ty);
      if (ty == cudaGraphNodeTypeKernel) b->knodes.push_back(nodes[k]);
    }
    if (e == cudaSuccess && b->knodes.empty()) e = cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(d, e, "graph capture");
  }
  *out = b;
  return MCRT_OK;
}

mcrt_status mcrt_batch_run(mcrt_batch* b, uint64_t seed, mcrt_run_stats* stats) {
  if (!b) return set_error(nullptr, MCRT_EINVAL, "batch is NULL");
  mcrt_disk* d = b->disks[0];
  CK(cudaSetDevice(b->device), "cudaSetDevice");
  if (seed != b->P.seed) {
    b->P.seed = seed;
    for (cudaGraphNode_t kn : b->knodes) {  // the transport and the tail kernel both take the KParams
      cudaKernelNodeParams kp;
      CK(cudaGraphKernelNodeGetParams(kn, &kp), "kernel node params");
      void* args[1] = {&b->P};
      kp.kernelParams = args;
      CK(cudaGraphExecKernelNodeSetParams(b->exec, kn, &kp), "kernel node update");
    }
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(cudaEventRecord(e0, b->stream), "event");
  CK(cudaGraphLaunch(b->exec, b->stream), "graph launch");
  CK(cudaEventRecord(e1, b->stream), "event");
  std::vector<unsigned long long> c((size_t)b->n * C_NCNT);
  for (int i = 0; i < b->n; ++i)
    CK(cudaMemcpyAsync(&c[(size_t)i * C_NCNT], b->disks[i]->cnt.p, C_NCNT * 8, cudaMemcpyDeviceToHost, b->stream),
       "copy");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  float ms_ = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms_, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(d, e, "batch kernel");
  d->launches++;
  mcrt_status ret = MCRT_OK;
  for (int i = 0; i < b->n; ++i) {
    unsigned long long* ci = &c[(size_t)i * C_NCNT];
    fix_events(ci);
    b->disks[i]->packets_done += b->npk[i];
    b->disks[i]->n_total = (double)b->npk[i];
    b->disks[i]->have_T = false;
    b->disks[i]->have_pda = false;
    if (stats) stats_from(ci, &stats[i], ms_ * 1e-3);
    if (!account_deposits(b->disks[i], ci)) ret = set_error(b->disks[i], MCRT_EOVERFLOW, "fixed-point tally overflow");
  }
  return ret;
}

mcrt_status mcrt_batch_config(const mcrt_batch* b, int* block, int* refill, int* grid, double* tune_seconds) {
  if (!b) return set_error(nullptr, MCRT_EINVAL, "batch is NULL");
  if (block) *block = b->block;
  if (refill) *refill = b->refill;
  if (grid) *grid = b->grid;
  if (tune_seconds) *tune_seconds = b->tune_seconds;
  return MCRT_OK;
}

void mcrt_batch_destroy(mcrt_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  delete b;
}

}  // extern "C"
