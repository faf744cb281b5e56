// Host build of the transport kernels' per-packet code (transport.cuh: launch_packet, step and what they
// call) in FP64, for a CPU test against the oracle: packets run one after another, as one lane of the FP64
// kernels runs them, over a model built by the library's own host builders (tables.h). Compiled by the host
// compiler with single-lane stand-ins for the CUDA builtins the header names (one lane: warp operations
// return their own lane's value; atomics are plain read-modify-writes).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

struct HostIdx {
  unsigned x, y, z;
};
static HostIdx host_threadIdx{0, 0, 0}, host_blockIdx{0, 0, 0}, host_blockDim{1, 1, 1}, host_gridDim{1, 1, 1};
#define threadIdx host_threadIdx
#define blockIdx host_blockIdx
#define blockDim host_blockDim
#define gridDim host_gridDim
#ifndef __noinline__
#define __noinline__ __attribute__((noinline))
#endif
#define __launch_bounds__(...)
using std::isfinite;
using std::signbit;
template <class T>
inline T __ldg(const T* p) { return *p; }
inline float __logf(float x) { return std::log(x); }
inline float __expf(float x) { return std::exp(x); }
inline void __sincosf(float x, float* s, float* c) {
  *s = std::sin(x);
  *c = std::cos(x);
}
inline float rsqrtf(float x) { return 1.f / std::sqrt(x); }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
template <class T>
inline T atomicAdd(T* p, T v) {
  const T o = *p;
  *p = o + v;
  return o;
}
inline unsigned atomicOr(unsigned* p, unsigned v) {
  const unsigned o = *p;
  *p |= v;
  return o;
}
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
  const unsigned long long o = *p;
  if (v > o) *p = v;
  return o;
}
template <class T>
inline T __shfl_sync(unsigned, T v, int, int = 32) { return v; }
template <class T>
inline T __shfl_up_sync(unsigned, T v, unsigned, int = 32) { return v; }
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int, int = 32) { return v; }
inline unsigned __ballot_sync(unsigned, int p) { return p ? 1u : 0u; }
inline int __any_sync(unsigned, int p) { return p; }
inline int __all_sync(unsigned, int p) { return p; }
inline unsigned __reduce_or_sync(unsigned, unsigned v) { return v; }
inline void __syncwarp(unsigned = 0xffffffffu) {}
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline int __ffs(int v) { return __builtin_ffs(v); }
inline int __clz(int v) { return v ? __builtin_clz((unsigned)v) : 32; }

#include "tables.h"
#include "transport.cuh"

using namespace mcrt;

namespace {

template <bool G, bool JT>
void run_packets(const KParams<double>& P, const DevModel<double>& M, uint64_t n, Acc& acc) {
  for (uint64_t k = 0; k < n; ++k) {
    Pkt<double> s;
    std::memset(&s, 0, sizeof(s));
    SerialRng rng{{(uint32_t)P.seed, (uint32_t)(P.seed >> 32)}};
    launch_packet<double, false, G, false, JT>(P, rng, M, s, k, -1, acc);
    while (step<double, false, G, false, JT>(P, rng, M, s, acc)) {
    }
  }
}

}  // namespace

// Transports packets 0 .. n-1 with Philox key `seed` through the disk (cgs inputs, as mcrt_disk_create and
// mcrt_set_opacity take them) and returns the tallies (nr*nt: fixed-point energy, entries, absorptions),
// the escape counts (nlam * 10), the mean-intensity path lengths (nr*nt*nlam, internal length units;
// NULL: not kept) and the counters {packets, absorptions, scatterings, crossings, MRW jumps, capped,
// escaped, error flags}.
extern "C" void host_transport(int nr, int nt, const double* rf_cm, const double* tf, const double* rho, int nlam,
                               const double* lam_e, const double* kabs, const double* ksca, const double* g,
                               double Tstar, double Rstar, uint64_t n, uint64_t seed, int mrw, double gamma, int nmin,
                               int want_sed, uint64_t* tally, uint64_t* visits, uint64_t* nabs, uint64_t* sed,
                               double* jlen, uint64_t* counters) {
  GeomArrays geo;
  geometry_arrays(nr, nt, rf_cm, tf, geo);
  DensityArrays den;
  density_arrays(nr, nt, rf_cm, tf, rho, den);
  DustArrays dust;
  dust_arrays(nlam, lam_e, kabs, ksca, g, Tstar, dust);
  const int nT = 1024;
  TGridTables tt;
  build_T_tables(nlam, lam_e, kabs, dust.chip.data(), nT, 1.0, std::max(1e4, 2.0 * Tstar), tt);
  std::vector<float> mtab(2 * kMrwTab);
  build_mrw_table(mtab.data());
  std::vector<double> gq(g, g + nlam);
  bool gray = true;
  for (int b = 1; b < nlam; ++b)
    if (kabs[b] != kabs[0] || ksca[b] != ksca[0] || g[b] != g[0]) gray = false;
  std::vector<unsigned long long> cnt(C_NCNT, 0ull);

  DevModel<double> M;
  std::memset(&M, 0, sizeof(M));
  M.nr = nr;
  M.nt = nt;
  M.nlam = nlam;
  M.nT = nT;
  M.gray = gray ? 1 : 0;
  M.rf = geo.rf.data();
  M.rf2 = geo.rf2.data();
  M.c2 = geo.c2.data();
  M.s2 = geo.s2.data();
  M.cf = geo.cf.data();
  M.sf = geo.sf.data();
  M.fk = geo.fk.data();
  M.rho = den.rhol.data();
  M.chi = dust.chi.data();
  M.alb = dust.alb.data();
  M.gq = gq.data();
  M.star_cum = dust.star.data();
  M.chi0 = kabs[0] + ksca[0];
  M.alb0 = ksca[0] / M.chi0;
  M.g0 = g[0];
  M.chiR0 = kabs[0] + (1.0 - g[0]) * ksca[0];
  M.kbar0 = kabs[0];
  M.lQk = tt.lQk.data();
  M.cbw = tt.cbw.data();
  M.cexit = tt.cexit.data();
  M.chiR = tt.chiRk.data();
  M.kbar = tt.kbark.data();
  M.lqm = den.lqm.data();
  const double Lstar = 4.0 * kPi * Rstar * Rstar * MCRT_SIGMA * std::pow(Tstar, 4);
  M.lq_run = (float)std::log(Lstar / ((double)n * (double)kEUnit));
  M.src_Lstar = Lstar;
  M.src_Ltot = Lstar;
  M.jlen = jlen;
  M.jw = tt.jw.data();
  M.tally = (unsigned long long*)tally;
  M.visits = (unsigned long long*)visits;
  M.nabs = (unsigned long long*)nabs;
  M.sed = (unsigned long long*)sed;
  M.cnt = cnt.data();
  M.n_packets = n;

  KParams<double> P;
  std::memset(&P, 0, sizeof(P));
  P.m0 = M;
  P.mrw = mrw ? 1 : 0;
  P.nmin = nmin;
  P.exit_dir = 0;
  P.want_lam = (!gray || want_sed) ? 1 : 0;
  P.refill = 4;
  P.defer = 8;
  P.gamma = gamma;
  P.seed = seed;
  P.max_events = 1ull << 31;
  P.max_steps = 4000000000ull;
  P.mrw_tab = mtab.data();
  P.mrw_t0 = mrw_table_t0();
  P.mrw_dt = mrw_table_dt();
  P.nmodels = 1;

  Acc acc;
  std::memset(&acc, 0, sizeof(acc));
  if (gray && jlen) run_packets<true, true>(P, M, n, acc);
  else if (gray) run_packets<true, false>(P, M, n, acc);
  else if (jlen) run_packets<false, true>(P, M, n, acc);
  else run_packets<false, false>(P, M, n, acc);
  const unsigned long long c[8] = {acc.packets, acc.abs, acc.sca, acc.cross, acc.mrw, acc.capped, acc.escaped, acc.err};
  for (int i = 0; i < 8; ++i) counters[i] = c[i];
}
