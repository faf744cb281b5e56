// internal.h -- the disk object behind the C ABI and the launchers shared between translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mcrt.h"
#include "common.cuh"
#include "transport.cuh"

namespace mcrt {

// Owning device allocation.
struct DBuf {
  void* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t bytes) {
    release();
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) n = bytes; else p = nullptr;
    return e;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

struct PdaState;  // pda.cu
struct RayState;  // raytrace.cu

template <class R>
cudaError_t launch_transport(const KParams<R>& P, bool trace, bool batch, bool gray, int grid, int block,
                             cudaStream_t st);
template <class R>
int transport_blocks_per_sm(bool trace, bool batch, bool gray, int block);
// tail kernel of a single-disk launch: 32-thread blocks, warps_per_sm of them per SM (0: 20)
template <class R>
cudaError_t launch_transport_tail(const KParams<R>& P, bool trace, bool batch, bool gray, int sms, int warps_per_sm,
                                  cudaStream_t st);
// polarized transport (single disk, no event trace)
template <class R>
cudaError_t launch_transport_pol(const KParams<R>& P, bool gray, int grid, int block, cudaStream_t st);
template <class R>
cudaError_t launch_transport_tail_pol(const KParams<R>& P, bool gray, int sms, int warps_per_sm, cudaStream_t st);
template <class R>
int transport_blocks_per_sm_pol(bool gray, int block);
// transport that keeps the path-length estimator of the mean intensity (single disk, no event trace)
template <class R>
cudaError_t launch_transport_j(const KParams<R>& P, bool gray, int grid, int block, cudaStream_t st);
template <class R>
cudaError_t launch_transport_tail_j(const KParams<R>& P, bool gray, int sms, int warps_per_sm, cudaStream_t st);
template <class R>
int transport_blocks_per_sm_j(bool gray, int block);

}  // namespace mcrt

struct mcrt_disk {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nr = 0, nt = 0, nlam = 0;
  bool gray = false, has_opacity = false;
  double l_unit = 1.0;  // cm per internal length unit (= r_faces[0])
  double Tstar = 0, Rstar = 0, Lstar = 0;
  // internal sources (viscous heating): cumulative luminosity over the cells on the device, their total
  double Lsrc_total = 0;
  mcrt::DBuf src_cum;
  int n_src = 0;
  double Lpkt() const { return Lstar + Lsrc_total; }  // luminosity the packets carry
  // polarized transport: Mueller matrix per bin and its cumulative S11 sin(theta) (FP32 and FP64
  // copies), escaping Stokes Q/I and U/I (fixed point, 2^20 per packet)
  bool pol = false;
  int nmu = 0;
  mcrt::DBuf mtab32, mtab64, mcdf32, mcdf64, sed_q, sed_u;
  // path-length estimator of the mean intensity (kept on request): path length per [cell][bin], and the
  // Eq. 10 weights per [T_k][bin] that spread an MRW walk over the bins
  bool keep_j = false;
  mcrt::DBuf jlen, jw;
  std::vector<double> rf, tf, rho, mass;
  std::vector<double> lam_e, kabs, ksca, g;
  // temperature grid
  int nT = 1024;
  double Tmin = 1.0, Tmax = 1e4;
  // device: geometry (float / double), dust, tables
  mcrt::DBuf rf32, rf2_32, c2_32, s2_32, cf32, sf32, rho32;
  mcrt::DBuf rf64, rf2_64, c2_64, s2_64, cf64, sf64, rho64;
  mcrt::DBuf fk;
  mcrt::DBuf chi32, alb32, g32, star32, chi64, alb64, g64, star64;
  mcrt::DBuf lQk, cbw, cexit, chiRk, kbark, lqm;
  mcrt::DBuf lQ64, slQ64;  // FP64 log Q(T_k) and d log Q / d log T on the T grid (temperature guesses)
  mcrt::DBuf lam_e_d, kabs_d, chip_d;  // FP64 per-bin data for exact temperatures / Rosseland means
  mcrt::DBuf mass_d, rho_cgs_d;
  // tallies
  mcrt::DBuf tally, visits, nabs, sed, cnt, queue;
  mcrt::DBuf pool, pool_ctr;  // packets in flight when the queue drains (one slot per thread of the launch)
  unsigned pool_cap = 0;
  // temperatures
  mcrt::DBuf T_mc, relerr, T_pda;
  bool have_T = false, have_pda = false;
  double n_total = 0;         // packet count that sets the packet energy of the tallies
  unsigned long long packets_done = 0;
  // fixed-point energy held by all tallies together: an upper bound of every cell's tally, so no
  // cell has wrapped while it has not (tally_wrapped: the bound itself passed 2^64)
  unsigned long long tally_held = 0;
  bool tally_wrapped = false;
  float chiR0 = 0, kbar0 = 0;
  mcrt::PdaState* pda = nullptr;
  mcrt::RayState* rays = nullptr;   // rays, source table and image of the ray-traced observables
  unsigned long long T_epoch = 0;   // advances whenever T_mc or T_pda is recomputed
  unsigned long long launches = 0;  // kernels launched by this disk
  std::string err;
  mcrt::DevModel<float> model32() const;
  mcrt::DevModel<double> model64() const;
};

namespace mcrt {
mcrt_status set_error(mcrt_disk* d, mcrt_status s, const std::string& msg);
mcrt_status cuda_fail(mcrt_disk* d, cudaError_t e, const char* what);
const float* mrw_table(int device, cudaError_t* err);
extern const float kMrwT0, kMrwDT;
mcrt_status compute_temperatures(mcrt_disk* d);
mcrt_status upload_density(mcrt_disk* d);
// adds a run's deposit sum (counters c) to the disk's held energy; false if a tally may have wrapped
bool account_deposits(mcrt_disk* d, const unsigned long long* c);
void pda_free(PdaState* p);
void ray_free(RayState* r);
}  // namespace mcrt
