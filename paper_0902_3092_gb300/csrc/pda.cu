// pda.cu -- partial diffusion approximation (Sect. 2.2.1, Eq. 4) and its adjoint.
//
// After the Monte Carlo run the cells that fewer than `min_visits` packets entered, or whose
// statistical temperature error exceeds `max_rel_err` (Sect. 3.1), form the PDA region. There
// div(D grad u) = 0 with u = T^4 and D = 1/(3 rho kappa_R) (Eq. 2) frozen at the Monte Carlo
// temperature, so the system is linear; all other dusty cells give Dirichlet values u = T_MC^4.
//
// Discretisation: finite volumes on the (r, theta) cells. The conductance of a face is the series
// resistance of the two half cells, each exact for constant D: radial half cell [a, b] of solid
// angle Omega: (1/a - 1/b)/(D Omega); polar half cell [t1, t2] of radial width dr:
// (ln tan(t2/2) - ln tan(t1/2))/(2 pi D dr). Grid edges and dust-free cells carry no flux.
//
// Solve: FP64 iterative refinement. Each outer step forms r = b - A u in FP64 and solves the
// Jacobi-scaled system (S A S) y = S r / |S r| (unit diagonal) with a matrix-free FP32 conjugate
// gradient; u += |S r| S y. Two kernels per CG iteration: (A) p = r + beta p_old and Ap for the own
// cell and its four neighbours (p recomputed for neighbours from r and p_old, so no extra sweep),
// with a block-reduced p.Ap; (B) y, r updates with a block-reduced r.r. The scalars live in a device
// array indexed by the iteration, so the host only reads back once per chunk of iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "tables.h"
#include "planck.cuh"

namespace mcrt {

struct PdaState {
  int nr = 0, nt = 0, n = 0;
  DBuf mask;                          // int8 per cell: 0 no dust, 1 Dirichlet, 2 PDA unknown
  DBuf hr_in, hr_out, ht_lo, ht_hi;   // geometric half-cell resistances (FP64)
  DBuf ell;                           // smallest cell extent min(dr, r_c dtheta) (cm)
  DBuf kR, D, Cr, Ct;                 // FP64: Rosseland opacity, D, radial / polar face conductances
  DBuf dis;                           // FP64 1/sqrt(diag) on PDA cells
  DBuf ar, at;                        // FP32 scaled couplings between PDA cells
  DBuf u;                             // FP64 T^4 on every cell
  DBuf lam;                           // FP64 adjoint solution
  DBuf b64;                           // FP64 right-hand side (adjoint)
  DBuf rs;                            // FP64 scaled residual S r
  DBuf y, r, p0, p1, Ap;              // FP32 CG vectors
  DBuf tiles;                         // int32 active tiles of the CG kernels
  std::vector<int> htiles;            // their host copy (source of the upload)
  bool vec4 = false;                  // tiles of 128 cells for the 16-byte kernels (ntheta % 4 == 0)
  int ntiles = 0;
  DBuf sc;                            // FP64 CG scalars per iteration
  DBuf kctr;                          // int: index of the CG iteration, on the device (graph replay)
  DBuf red;                           // FP64 reduction slots
  DBuf w, gl, gk;                     // adjoint weights / gradient outputs (device staging)
  int n_pda = 0;
  int max_inner_alloc = 0;
};

void pda_free(PdaState* p) { delete p; }

__device__ __forceinline__ float block_sum_f(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  float s = 0.f;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// ---------------------------------------------------------------------------------------------- setup
// PDA cells (2): dust, optically thick (rho chi'_max ell_c >= min_tau, ell_c = min(dr, r_c dtheta)), and
// fewer than min_visits entries or a statistical error above max_rel. Dirichlet cells (1): the other
// dusty cells that absorbed energy. Dust-free cells and thin cells that absorbed nothing carry no
// temperature and no flux (0).
__global__ void k_mask(int n, const double* rho, const double* ell, double chi_max, double min_tau,
                       const unsigned long long* visits, const double* relerr, const unsigned long long* tally,
                       int min_visits, double max_rel, signed char* mask, double* red) {
  __shared__ double sh[32];
  double cnt = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    signed char m = 0;
    if (rho[c] > 0) {
      const bool thick = rho[c] * chi_max * ell[c] >= min_tau;
      if (thick && (visits[c] < (unsigned long long)min_visits || relerr[c] > max_rel)) m = 2;
      else if (tally[c] > 0ull) m = 1;
    }
    mask[c] = m;
    cnt += m == 2 ? 1.0 : 0.0;
  }
  const double s = block_sum_d(cnt, sh);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(red + 0, s);
}

// mean MC temperature of the Dirichlet cells that border the PDA region
__global__ void k_bnd_mean(int nr, int nt, const signed char* mask, const double* T, double* red) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt || mask[c] != 1) return;
  const int i = c / nt, j = c - i * nt;
  const bool nb = (i > 0 && mask[c - nt] == 2) || (i + 1 < nr && mask[c + nt] == 2) || (j > 0 && mask[c - 1] == 2) ||
                  (j + 1 < nt && mask[c + 1] == 2);
  if (nb) {
    atomicAdd(red + 1, T[c]);
    atomicAdd(red + 2, 1.0);
  }
}

// Rosseland extinction of the cells whose D enters a conductance (PDA cells and their dusty
// neighbours); the others get a placeholder (their D takes part in no face)
__global__ void k_kappaR(int nr, int nt, const signed char* mask, const double* rho, const unsigned long long* tally,
                         const double* T, const double* red, int gray, double chip0, int nlam, const double* lam_e,
                         const double* chip, const double* over, double* kR) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nr * nt;
  if (c >= n) return;
  if (!(rho[c] > 0)) {
    kR[c] = 1.0;
    return;
  }
  if (over) {
    kR[c] = over[c];
    return;
  }
  if (gray) {
    kR[c] = chip0;
    return;
  }
  const int i = c / nt, j = c - i * nt;
  const bool used = mask[c] == 2 || (i > 0 && mask[c - nt] == 2) || (i + 1 < nr && mask[c + nt] == 2) ||
                    (j > 0 && mask[c - 1] == 2) || (j + 1 < nt && mask[c + 1] == 2);
  if (!used) {
    kR[c] = chip0;
    return;
  }
  double Tc = tally[c] ? T[c] : (red[2] > 0 ? red[1] / red[2] : 1.0);
  Tc = fmax(Tc, 1.0);
  kR[c] = rosseland(lam_e, chip, nlam, Tc);
}

__global__ void k_cond(int nr, int nt, const signed char* mask, const double* rho, const double* kR,
                       const double* hr_in, const double* hr_out, const double* ht_lo, const double* ht_hi, double* D,
                       double* Cr, double* Ct) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt) return;
  const int i = c / nt, j = c - i * nt;
  auto Dof = [&](int k) { return rho[k] > 0 ? 1.0 / (3.0 * rho[k] * kR[k]) : 0.0; };
  const double Dc = Dof(c);
  D[c] = Dc;
  double cr = 0.0, ct = 0.0;
  // faces that carry flux: both cells take part and at least one is a PDA cell
  if (i + 1 < nr && mask[c] && mask[c + nt] && (mask[c] == 2 || mask[c + nt] == 2))
    cr = 1.0 / (hr_out[c] / Dc + hr_in[c + nt] / Dof(c + nt));
  if (j + 1 < nt && mask[c] && mask[c + 1] && (mask[c] == 2 || mask[c + 1] == 2))
    ct = 1.0 / (ht_hi[c] / Dc + ht_lo[c + 1] / Dof(c + 1));
  Cr[c] = cr;
  Ct[c] = ct;
}

// diag on PDA cells (sum of conductances to any dusty neighbour); u initialised: T_MC^4 on
// Dirichlet cells, 0 elsewhere
__global__ void k_diag(int nr, int nt, const signed char* mask, const double* Cr, const double* Ct, const double* T,
                       double* dis, double* u, double* red) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt) return;
  const int i = c / nt, j = c - i * nt;
  const signed char m = mask[c];
  if (m == 1) {
    const double t2 = T[c] * T[c];
    u[c] = t2 * t2;
  } else {
    u[c] = 0.0;
  }
  if (m != 2) {
    dis[c] = 0.0;
    return;
  }
  double d = 0.0;
  if (i > 0 && mask[c - nt]) d += Cr[c - nt];
  if (i + 1 < nr && mask[c + nt]) d += Cr[c];
  if (j > 0 && mask[c - 1]) d += Ct[c - 1];
  if (j + 1 < nt && mask[c + 1]) d += Ct[c];
  if (d > 0) {
    dis[c] = 1.0 / sqrt(d);
  } else {
    dis[c] = 0.0;
    atomicAdd(red + 3, 1.0);  // isolated PDA cell: singular
  }
}

__global__ void k_scaled(int nr, int nt, const signed char* mask, const double* Cr, const double* Ct, const double* dis,
                         float* ar, float* at) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt) return;
  const int i = c / nt, j = c - i * nt;
  float a = 0.f, b = 0.f;
  if (mask[c] == 2) {
    if (i + 1 < nr && mask[c + nt] == 2) a = (float)(-Cr[c] * dis[c] * dis[c + nt]);
    if (j + 1 < nt && mask[c + 1] == 2) b = (float)(-Ct[c] * dis[c] * dis[c + 1]);
  }
  ar[c] = a;
  at[c] = b;
}

// --------------------------------------------------------------------------------------------- FP64
// rs = S (b + sum_f C_f (x_nb - x_c)) on PDA cells; red[slot] += |rs|^2
__global__ void k_resid64(int nr, int nt, const signed char* __restrict__ mask, const double* __restrict__ Cr,
                          const double* __restrict__ Ct, const double* __restrict__ dis, const double* __restrict__ x,
                          const double* __restrict__ b, double* __restrict__ rs, double* red, int slot) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nr * nt; c += gridDim.x * blockDim.x) {
    double v = 0.0;
    if (mask[c] == 2) {
      const int i = c / nt, j = c - i * nt;
      const double xc = x[c];
      double r = b ? b[c] : 0.0;
      if (i > 0 && mask[c - nt]) r += Cr[c - nt] * (x[c - nt] - xc);
      if (i + 1 < nr && mask[c + nt]) r += Cr[c] * (x[c + nt] - xc);
      if (j > 0 && mask[c - 1]) r += Ct[c - 1] * (x[c - 1] - xc);
      if (j + 1 < nt && mask[c + 1]) r += Ct[c] * (x[c + 1] - xc);
      v = dis[c] * r;
    }
    rs[c] = v;
    acc += v * v;
  }
  const double s = block_sum_d(acc, sh);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(red + slot, s);
}

// rhs of the FP32 solve: r = rs / scale, y = 0, all CG vectors zeroed (the iteration kernels only touch
// PDA cells afterwards); sc[0] += |r|^2. Grid-stride over the cells.
__global__ void k_start(int n, const signed char* mask, const double* rs, double inv_scale, float* y, float* r,
                        float* p_old, float* p_new, float* Ap, double* sc) {
  __shared__ float sh[32];
  float v = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const float x = mask[c] == 2 ? (float)(rs[c] * inv_scale) : 0.f;
    r[c] = x;
    y[c] = 0.f;
    p_old[c] = 0.f;
    p_new[c] = 0.f;
    Ap[c] = 0.f;
    v += x * x;
  }
  const float s = block_sum_f(v, sh);
  if (threadIdx.x == 0 && s != 0.f) atomicAdd(sc + 0, (double)s);
}

// scalar layout: sc[0] = rr_0; iteration k: rr_k at 2k (k >= 1 stored at sc[2k]), pAp_k at sc[2k+1]
__device__ __forceinline__ double rr_of(const double* sc, int k) { return sc[2 * k]; }

// The CG iteration kernels sweep "active tiles": runs of 32 consecutive cells (row-major, one warp
// per tile, one lane per cell) that hold at least one PDA cell; `tiles` lists them in increasing
// order (nullptr: every tile of the grid). They read no mask: outside the PDA region the vectors
// are zero and so are the scaled couplings ar, at of every face that is not between two PDA cells,
// including the faces beyond the last radial row / polar column, so the terms of non-PDA
// neighbours vanish and non-PDA cells keep zero. Warp w takes tiles w, w + nw, w + 2 nw, ... (nw
// warps in the grid); lane l fetches the index of the warp's l-th next tile, so one load serves 32
// tiles, and each step handles U tiles with all their loads issued before the arithmetic, so that
// enough bytes are in flight per SM for HBM. The grid is the device's resident block slots, so each
// reduction ends in about a thousand atomics.
constexpr int kUA = 2, kUB = 4;

__device__ __forceinline__ float ld_or0(const float* __restrict__ a, int i, bool ok) { return ok ? __ldg(a + i) : 0.f; }

// first cell of the warp's (s0 + lane)-th tile, or -1 past the end
__device__ __forceinline__ int tile_base(const int* __restrict__ tiles, int ntiles, int w, int nw, int s) {
  const long long t = (long long)w + (long long)s * nw;
  return t < ntiles ? (tiles ? __ldg(tiles + t) : (int)t) * 32 : -1;
}

// kernel A of CG iteration k: p = r + beta p_old and Ap (p recomputed for the four neighbours from r
// and p_old), partial p.Ap
template <int U>
__global__ void __launch_bounds__(256) k_cg_a(int n, int nt, int ntiles, const int* __restrict__ tiles,
                                              const float* __restrict__ ar, const float* __restrict__ at,
                                              const float* __restrict__ r, const float* __restrict__ p_old,
                                              float* __restrict__ p_new, float* __restrict__ Ap, double* sc, const int* kdev, int k, int kmax,
                                              double tol2) {
  __shared__ float sh[32];
  if (kdev) k = *kdev;  // iteration index kept on the device (graph replay)
  if (k >= kmax) return;
  const double rr0 = rr_of(sc, 0), rrk = rr_of(sc, k);
  if (rrk <= tol2 * rr0 || !(rrk == rrk)) return;  // converged (or broken): no-op
  const float beta = k == 0 ? 0.f : (float)(rrk / rr_of(sc, k - 1));
  const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float v = 0.f;
  for (int s0 = 0; w + (long long)s0 * nw < ntiles; s0 += 32) {
    const int base = tile_base(tiles, ntiles, w, nw, s0 + lane);
#pragma unroll 1
    for (int u0 = 0; u0 < 32; u0 += U) {
      int c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int b = __shfl_sync(0xffffffffu, base, u0 + u);
        c[u] = b >= 0 ? b + lane : n;
      }
      if (__shfl_sync(0xffffffffu, base, u0) < 0) break;  // warp-uniform: later tiles are past the end too
      float rc[U], pc[U], aro[U], ato[U], ari[U], ati[U], rn[U][4], pn[U][4];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int cc = c[u];
        const bool in = cc < n, dn = in && cc >= nt, up = in && cc + nt < n, lo = in && cc > 0, hi = in && cc + 1 < n;
        rc[u] = ld_or0(r, cc, in);
        pc[u] = ld_or0(p_old, cc, in);
        aro[u] = ld_or0(ar, cc, in);
        ato[u] = ld_or0(at, cc, in);
        ari[u] = ld_or0(ar, cc - nt, dn);
        ati[u] = ld_or0(at, cc - 1, lo);
        rn[u][0] = ld_or0(r, cc - nt, dn);
        pn[u][0] = ld_or0(p_old, cc - nt, dn);
        rn[u][1] = ld_or0(r, cc + nt, up);
        pn[u][1] = ld_or0(p_old, cc + nt, up);
        rn[u][2] = ld_or0(r, cc - 1, lo);
        pn[u][2] = ld_or0(p_old, cc - 1, lo);
        rn[u][3] = ld_or0(r, cc + 1, hi);
        pn[u][3] = ld_or0(p_old, cc + 1, hi);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c[u] >= n) continue;
        const float p = rc[u] + beta * pc[u];
        float a = p;
        a += ari[u] * (rn[u][0] + beta * pn[u][0]);
        a += aro[u] * (rn[u][1] + beta * pn[u][1]);
        a += ati[u] * (rn[u][2] + beta * pn[u][2]);
        a += ato[u] * (rn[u][3] + beta * pn[u][3]);
        p_new[c[u]] = p;
        Ap[c[u]] = a;
        v += p * a;
      }
    }
  }
  const float s = block_sum_f(v, sh);
  if (threadIdx.x == 0 && s != 0.f) atomicAdd(sc + 2 * k + 1, (double)s);
}

// kernel B of CG iteration k: y += alpha p, r -= alpha Ap, partial r.r
template <int U>
__global__ void __launch_bounds__(256) k_cg_b(int n, int ntiles, const int* __restrict__ tiles,
                                              const float* __restrict__ p_new, const float* __restrict__ Ap,
                                              float* __restrict__ y, float* __restrict__ r, double* sc, const int* kdev, int k, int kmax,
                                              double tol2) {
  __shared__ float sh[32];
  if (kdev) k = *kdev;  // iteration index kept on the device (graph replay)
  if (k >= kmax) return;
  const double rr0 = rr_of(sc, 0), rrk = rr_of(sc, k);
  if (rrk <= tol2 * rr0 || !(rrk == rrk)) return;
  const float alpha = (float)(rrk / sc[2 * k + 1]);
  const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float v = 0.f;
  for (int s0 = 0; w + (long long)s0 * nw < ntiles; s0 += 32) {
    const int base = tile_base(tiles, ntiles, w, nw, s0 + lane);
#pragma unroll 1
    for (int u0 = 0; u0 < 32; u0 += U) {
      int c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int b = __shfl_sync(0xffffffffu, base, u0 + u);
        c[u] = b >= 0 ? b + lane : n;
      }
      if (__shfl_sync(0xffffffffu, base, u0) < 0) break;
      float pv[U], av[U], yv[U], rv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = c[u] < n;
        pv[u] = in ? __ldg(p_new + c[u]) : 0.f;
        av[u] = in ? __ldg(Ap + c[u]) : 0.f;
        yv[u] = in ? y[c[u]] : 0.f;
        rv[u] = in ? r[c[u]] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c[u] >= n) continue;
        y[c[u]] = yv[u] + alpha * pv[u];
        const float rnew = rv[u] - alpha * av[u];
        r[c[u]] = rnew;
        v += rnew * rnew;
      }
    }
  }
  const float s = block_sum_f(v, sh);
  if (threadIdx.x == 0) atomicAdd(sc + 2 * (k + 1), (double)s);
}

// The same two kernels on 128-cell tiles, each lane taking four consecutive cells with 16-byte loads
// and stores (used when ntheta % 4 == 0: a lane's four cells then lie in one polar row, and the rows
// above and below start on 16-byte boundaries). The polar neighbours inside a lane are its own
// cells; those across lanes come by shuffle, at the ends of the tile by single loads.
__device__ __forceinline__ float4 ld4_or0(const float* __restrict__ a, int i, bool ok) {
  return ok ? __ldg(reinterpret_cast<const float4*>(a + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_cg_a4(int n, int nt, int ntiles, const int* __restrict__ tiles,
                                               const float* __restrict__ ar, const float* __restrict__ at,
                                               const float* __restrict__ r, const float* __restrict__ p_old,
                                               float* __restrict__ p_new, float* __restrict__ Ap, double* sc, const int* kdev, int k, int kmax,
                                               double tol2) {
  __shared__ float sh[32];
  if (kdev) k = *kdev;  // iteration index kept on the device (graph replay)
  if (k >= kmax) return;
  const double rr0 = rr_of(sc, 0), rrk = rr_of(sc, k);
  if (rrk <= tol2 * rr0 || !(rrk == rrk)) return;  // converged (or broken): no-op
  const float beta = k == 0 ? 0.f : (float)(rrk / rr_of(sc, k - 1));
  const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const unsigned full = 0xffffffffu;
  float v = 0.f;
  for (int s0 = 0; w + (long long)s0 * nw < ntiles; s0 += 32) {
    const long long tt = (long long)w + (long long)(s0 + lane) * nw;
    const int base = tt < ntiles ? __ldg(tiles + tt) * 128 : -1;
#pragma unroll 1
    for (int u0 = 0; u0 < 32; ++u0) {
      const int b = __shfl_sync(full, base, u0);
      if (b < 0) break;  // warp-uniform
      const int c = b + 4 * lane;
      const bool in = c < n, dn = in && c >= nt, up = in && c + nt < n;
      const float4 rc = ld4_or0(r, c, in), pc = ld4_or0(p_old, c, in);
      const float4 arc = ld4_or0(ar, c, in), atc = ld4_or0(at, c, in);
      const float4 ard = ld4_or0(ar, c - nt, dn);
      const float4 rd = ld4_or0(r, c - nt, dn), pd = ld4_or0(p_old, c - nt, dn);
      const float4 ru = ld4_or0(r, c + nt, up), pu = ld4_or0(p_old, c + nt, up);
      float rl = __shfl_up_sync(full, rc.w, 1), pl = __shfl_up_sync(full, pc.w, 1);
      float atl = __shfl_up_sync(full, atc.w, 1);
      float rr = __shfl_down_sync(full, rc.x, 1), pr = __shfl_down_sync(full, pc.x, 1);
      if (lane == 0) {
        const bool ok = in && c > 0;
        rl = ok ? __ldg(r + c - 1) : 0.f;
        pl = ok ? __ldg(p_old + c - 1) : 0.f;
        atl = ok ? __ldg(at + c - 1) : 0.f;
      }
      if (lane == 31) {
        const bool ok = in && c + 4 < n;
        rr = ok ? __ldg(r + c + 4) : 0.f;
        pr = ok ? __ldg(p_old + c + 4) : 0.f;
      }
      if (!in) continue;
      const float p0 = rc.x + beta * pc.x, p1 = rc.y + beta * pc.y, p2 = rc.z + beta * pc.z, p3 = rc.w + beta * pc.w;
      float4 a;
      a.x = p0 + ard.x * (rd.x + beta * pd.x) + arc.x * (ru.x + beta * pu.x) + atl * (rl + beta * pl) + atc.x * p1;
      a.y = p1 + ard.y * (rd.y + beta * pd.y) + arc.y * (ru.y + beta * pu.y) + atc.x * p0 + atc.y * p2;
      a.z = p2 + ard.z * (rd.z + beta * pd.z) + arc.z * (ru.z + beta * pu.z) + atc.y * p1 + atc.z * p3;
      a.w = p3 + ard.w * (rd.w + beta * pd.w) + arc.w * (ru.w + beta * pu.w) + atc.z * p2 + atc.w * (rr + beta * pr);
      *reinterpret_cast<float4*>(p_new + c) = make_float4(p0, p1, p2, p3);
      *reinterpret_cast<float4*>(Ap + c) = a;
      v += p0 * a.x + p1 * a.y + p2 * a.z + p3 * a.w;
    }
  }
  const float s = block_sum_f(v, sh);
  if (threadIdx.x == 0 && s != 0.f) atomicAdd(sc + 2 * k + 1, (double)s);
}

__global__ void __launch_bounds__(256) k_cg_b4(int n, int ntiles, const int* __restrict__ tiles,
                                               const float* __restrict__ p_new, const float* __restrict__ Ap,
                                               float* __restrict__ y, float* __restrict__ r, double* sc, const int* kdev, int k, int kmax,
                                               double tol2) {
  __shared__ float sh[32];
  if (kdev) k = *kdev;  // iteration index kept on the device (graph replay)
  if (k >= kmax) return;
  const double rr0 = rr_of(sc, 0), rrk = rr_of(sc, k);
  if (rrk <= tol2 * rr0 || !(rrk == rrk)) return;
  const float alpha = (float)(rrk / sc[2 * k + 1]);
  const int lane = threadIdx.x & 31, nw = gridDim.x * (blockDim.x >> 5);
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const unsigned full = 0xffffffffu;
  float v = 0.f;
  for (int s0 = 0; w + (long long)s0 * nw < ntiles; s0 += 32) {
    const long long tt = (long long)w + (long long)(s0 + lane) * nw;
    const int base = tt < ntiles ? __ldg(tiles + tt) * 128 : -1;
#pragma unroll 1
    for (int u0 = 0; u0 < 32; u0 += 2) {
      const int b0 = __shfl_sync(full, base, u0), b1 = __shfl_sync(full, base, u0 + 1);
      if (b0 < 0) break;
      const int c0 = b0 + 4 * lane, c1 = b1 >= 0 ? b1 + 4 * lane : n;
      const bool in0 = c0 < n, in1 = c1 < n;
      const float4 p0 = ld4_or0(p_new, c0, in0), a0 = ld4_or0(Ap, c0, in0);
      const float4 p1 = ld4_or0(p_new, c1, in1), a1 = ld4_or0(Ap, c1, in1);
      float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f), r0 = y0, y1 = y0, r1 = y0;
      if (in0) {
        y0 = *reinterpret_cast<const float4*>(y + c0);
        r0 = *reinterpret_cast<const float4*>(r + c0);
      }
      if (in1) {
        y1 = *reinterpret_cast<const float4*>(y + c1);
        r1 = *reinterpret_cast<const float4*>(r + c1);
      }
      if (in0) {
        const float4 rn = make_float4(r0.x - alpha * a0.x, r0.y - alpha * a0.y, r0.z - alpha * a0.z, r0.w - alpha * a0.w);
        *reinterpret_cast<float4*>(y + c0) =
            make_float4(y0.x + alpha * p0.x, y0.y + alpha * p0.y, y0.z + alpha * p0.z, y0.w + alpha * p0.w);
        *reinterpret_cast<float4*>(r + c0) = rn;
        v += rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w;
      }
      if (in1) {
        const float4 rn = make_float4(r1.x - alpha * a1.x, r1.y - alpha * a1.y, r1.z - alpha * a1.z, r1.w - alpha * a1.w);
        *reinterpret_cast<float4*>(y + c1) =
            make_float4(y1.x + alpha * p1.x, y1.y + alpha * p1.y, y1.z + alpha * p1.z, y1.w + alpha * p1.w);
        *reinterpret_cast<float4*>(r + c1) = rn;
        v += rn.x * rn.x + rn.y * rn.y + rn.z * rn.z + rn.w * rn.w;
      }
    }
  }
  const float s = block_sum_f(v, sh);
  if (threadIdx.x == 0) atomicAdd(sc + 2 * (k + 1), (double)s);
}

__global__ void k_update(int n, const signed char* mask, const double* dis, const float* y, double scale, double* x) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n && mask[c] == 2) x[c] += scale * dis[c] * (double)y[c];
}

__global__ void k_tpda(int n, const signed char* mask, const double* u, const double* Tmc, double* Tp) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  Tp[c] = mask[c] == 2 ? pow(fmax(u[c], 0.0), 0.25) : Tmc[c];
}

// adjoint right-hand side g = w dT/du = w / (4 u^(3/4)) on PDA cells; lam = 0 everywhere
__global__ void k_adj_rhs(int n, const signed char* mask, const double* w, const double* u, double* g, double* lam) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  g[c] = (mask[c] == 2 && u[c] > 0.0) ? w[c] * 0.25 * pow(u[c], -0.75) : 0.0;
  lam[c] = 0.0;
}

// dJ/dD_c = sum over the active faces of c of dJ/dC_f dC_f/dD_c, dJ/dC_f = -(lam_c - lam_n)(u_c - u_n),
// dC_f/dD_c = C_f^2 h_c / D_c^2; then dJ/dlog rho = -D dJ/dD, dJ/dkappa_R = -(D/kappa_R) dJ/dD.
__global__ void k_grad(int nr, int nt, const signed char* mask, const double* Cr, const double* Ct, const double* D,
                       const double* kR, const double* hr_in, const double* hr_out, const double* ht_lo,
                       const double* ht_hi, const double* u, const double* lam, double* g_lr, double* g_kr) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt) return;
  const int i = c / nt, j = c - i * nt;
  double s = 0.0;
  const signed char mc = mask[c];
  if (mc) {
    const double Dc = D[c];
    auto face = [&](int nb, double C, double h) {
      const signed char mn = mask[nb];
      if (!mn || !(C > 0) || (mc != 2 && mn != 2)) return;
      const double dJdC = -(lam[c] - lam[nb]) * (u[c] - u[nb]);
      s += dJdC * C * C * h / (Dc * Dc);
    };
    if (i > 0) face(c - nt, Cr[c - nt], hr_in[c]);
    if (i + 1 < nr) face(c + nt, Cr[c], hr_out[c]);
    if (j > 0) face(c - 1, Ct[c - 1], ht_lo[c]);
    if (j + 1 < nt) face(c + 1, Ct[c], ht_hi[c]);
    if (g_lr) g_lr[c] = s != 0.0 ? -Dc * s : 0.0;
    if (g_kr) g_kr[c] = s != 0.0 ? -Dc / kR[c] * s : 0.0;
  } else {
    if (g_lr) g_lr[c] = 0.0;
    if (g_kr) g_kr[c] = 0.0;
  }
}

}  // namespace mcrt

using namespace mcrt;

#define CK(call, what)                                    \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(d, e_, what); \
  } while (0)

static int nblk(int n) { return (n + 255) / 256; }

// grid of the grid-stride PDA kernels: a few resident blocks per SM, so every reduction ends in about a
// thousand atomics instead of one per 256 cells
static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 128;
  }
  return sms;
}

static int sgrid(int n) { return std::max(1, std::min(nblk(n), sm_count() * 8)); }

// grid of a tile kernel: each resident block slot of the device once (blocks per SM from the
// occupancy calculator), fewer when there are fewer tiles (8 warps, one tile each, per block)
template <class K>
static int tgrid(K kern, int ntiles) {
  static int occ = 0;
  if (!occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ <= 0) occ = 1;
  }
  return std::max(1, std::min((ntiles + 7) / 8, sm_count() * occ));
}

// active tiles of a mask (`width` consecutive cells with at least one PDA cell), in increasing order
static std::vector<int> active_tiles(const std::vector<signed char>& mask, int width) {
  const int n = (int)mask.size();
  std::vector<int> t;
  for (int b = 0; b < n; b += width) {
    const int e = std::min(n, b + width);
    for (int c = b; c < e; ++c)
      if (mask[c] == 2) {
        t.push_back(b / width);
        break;
      }
  }
  return t;
}

static mcrt_status pda_alloc(mcrt_disk* d, int max_inner) {
  PdaState* P = d->pda;
  if (!P) {
    P = new (std::nothrow) PdaState();
    if (!P) return set_error(d, MCRT_ENOMEM, "host allocation");
    d->pda = P;
  }
  const int nr = d->nr, nt = d->nt, n = nr * nt;
  if (P->n != n) {
    P->nr = nr;
    P->nt = nt;
    P->n = n;
    // geometric half-cell resistances
    HalfResistances hr;
    half_resistances(nr, nt, d->rf.data(), d->tf.data(), hr);
    const std::vector<double>&hi_ = hr.hr_in, &ho = hr.hr_out, &tl = hr.ht_lo, &th = hr.ht_hi, &el = hr.ell;
    cudaError_t e = P->hr_in.alloc((size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(P->hr_in.p, hi_.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = P->hr_out.alloc((size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(P->hr_out.p, ho.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = P->ht_lo.alloc((size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(P->ht_lo.p, tl.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = P->ht_hi.alloc((size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(P->ht_hi.p, th.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = P->ell.alloc((size_t)n * 8);
    if (e == cudaSuccess) e = cudaMemcpy(P->ell.p, el.data(), (size_t)n * 8, cudaMemcpyHostToDevice);
    DBuf* d8[] = {&P->kR, &P->D, &P->Cr, &P->Ct, &P->dis, &P->u, &P->lam, &P->b64, &P->rs, &P->w, &P->gl, &P->gk};
    for (DBuf* b : d8)
      if (e == cudaSuccess) e = b->alloc((size_t)n * 8);
    DBuf* d4[] = {&P->ar, &P->at, &P->y, &P->r, &P->p0, &P->p1, &P->Ap};
    for (DBuf* b : d4)
      if (e == cudaSuccess) e = b->alloc((size_t)n * 4);
    if (e == cudaSuccess) e = P->mask.alloc(n);
    if (e == cudaSuccess) e = P->tiles.alloc(((size_t)n + 31) / 32 * sizeof(int));
    if (e == cudaSuccess) e = P->red.alloc(16 * 8);
    if (e == cudaSuccess) e = P->kctr.alloc(16);
    if (e != cudaSuccess) return cuda_fail(d, e, "PDA buffers");
  }
  if (P->max_inner_alloc < max_inner) {
    cudaError_t e = P->sc.alloc(sizeof(double) * (2 * (size_t)max_inner + 8));
    if (e != cudaSuccess) return cuda_fail(d, e, "PDA scalars");
    P->max_inner_alloc = max_inner;
  }
  return MCRT_OK;
}

// Host check that every connected PDA region touches a Dirichlet cell.
static bool components_ok(const mcrt_disk* d, const std::vector<signed char>& mask) {
  const int nr = d->nr, nt = d->nt, n = nr * nt;
  std::vector<int> comp(n, -1), stack;
  for (int s = 0; s < n; ++s) {
    if (mask[s] != 2 || comp[s] >= 0) continue;
    bool dir = false;
    stack.assign(1, s);
    comp[s] = s;
    while (!stack.empty()) {
      const int c = stack.back();
      stack.pop_back();
      const int i = c / nt, j = c % nt;
      const int nb[4] = {i > 0 ? c - nt : -1, i + 1 < nr ? c + nt : -1, j > 0 ? c - 1 : -1, j + 1 < nt ? c + 1 : -1};
      for (int k = 0; k < 4; ++k) {
        const int m = nb[k];
        if (m < 0) continue;
        if (mask[m] == 1) dir = true;
        if (mask[m] == 2 && comp[m] < 0) {
          comp[m] = s;
          stack.push_back(m);
        }
      }
    }
    if (!dir) return false;
  }
  return true;
}

__global__ void k_iter_next(int* k) { ++*k; }

// one CG iteration (kernels A and B) on the active tiles
static void launch_cg_iteration(const PdaState* P, int n, int nt, const int* tiles, float* r, float* pold, float* pnew,
                                float* Ap, float* y, double* sc, const int* kdev, int k, int kmax, double tol2, int ga,
                                int gb, cudaStream_t st) {
  if (P->vec4) {
    k_cg_a4<<<ga, 256, 0, st>>>(n, nt, P->ntiles, tiles, P->ar.as<float>(), P->at.as<float>(), r, pold, pnew, Ap, sc,
                                kdev, k, kmax, tol2);
    k_cg_b4<<<gb, 256, 0, st>>>(n, P->ntiles, tiles, pnew, Ap, y, r, sc, kdev, k, kmax, tol2);
  } else {
    k_cg_a<kUA><<<ga, 256, 0, st>>>(n, nt, P->ntiles, tiles, P->ar.as<float>(), P->at.as<float>(), r, pold, pnew, Ap,
                                    sc, kdev, k, kmax, tol2);
    k_cg_b<kUB><<<gb, 256, 0, st>>>(n, P->ntiles, tiles, pnew, Ap, y, r, sc, kdev, k, kmax, tol2);
  }
}

// an instantiated graph of `count` calls of a launch function captured on a stream; null when the
// stream cannot be captured
struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  template <class F>
  cudaGraphExec_t build(cudaStream_t st, int count, F launch) {
    if (!st || cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int j = 0; j < count; ++j) launch(j);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      exec = nullptr;
    }
    return exec;
  }
  ~ChunkGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

// FP64-refined solve of A x = b on the PDA cells; x holds the Dirichlet values elsewhere.
static mcrt_status refine_solve(mcrt_disk* d, const mcrt_pda_opts* o, double* x, const double* b, int* iters_out) {
  PdaState* P = d->pda;
  const int nr = d->nr, nt = d->nt, n = nr * nt;
  cudaStream_t st = d->stream;
  const signed char* mask = P->mask.as<signed char>();
  const double* Cr = P->Cr.as<double>();
  const double* Ct = P->Ct.as<double>();
  const double* dis = P->dis.as<double>();
  double* red = P->red.as<double>();
  double* sc = P->sc.as<double>();
  float *y = P->y.as<float>(), *r = P->r.as<float>(), *Ap = P->Ap.as<float>();
  float* pb[2] = {P->p0.as<float>(), P->p1.as<float>()};
  const double tol2_in = o->inner_tol * o->inner_tol;
  const int* tiles = P->tiles.as<int>();
  const int ga = P->vec4 ? tgrid(k_cg_a4, P->ntiles) : tgrid(k_cg_a<kUA>, P->ntiles);
  const int gb = P->vec4 ? tgrid(k_cg_b4, P->ntiles) : tgrid(k_cg_b<kUB>, P->ntiles);
  double norm_b = -1.0, best = INFINITY;
  int total_iters = 0, stall = 0;
  constexpr int chunk = 32;
  // the CG iterations of one chunk as a CUDA graph (the index of the iteration lives on the device);
  // without a graph (capture refused, e.g. on the legacy default stream) the kernels launch one by one
  int* kdev = P->kctr.as<int>();
  ChunkGraph cg;
  cudaGraphExec_t chunk_exec = cg.build(st, chunk, [&](int j) {
    launch_cg_iteration(P, n, nt, tiles, r, pb[(j + 1) & 1], pb[j & 1], Ap, y, sc, kdev, 0, o->max_inner, tol2_in, ga,
                        gb, st);
    k_iter_next<<<1, 1, 0, st>>>(kdev);
  });
  for (int outer = 0; outer <= o->max_outer; ++outer) {
    CK(cudaMemsetAsync(red + 4, 0, 8, st), "memset");
    k_resid64<<<sgrid(n), 256, 0, st>>>(nr, nt, mask, Cr, Ct, dis, x, b, P->rs.as<double>(), red, 4);
    d->launches++;
    double rn2 = 0.0;
    CK(cudaMemcpyAsync(&rn2, red + 4, 8, cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaStreamSynchronize(st), "synchronize");
    const double rn = std::sqrt(rn2);
    if (norm_b < 0) norm_b = rn;  // first residual: x = 0 on the PDA cells, so this is |S b_total|
    if (!(rn == rn)) return set_error(d, MCRT_ENOTCONV, "PDA residual is not finite");
    if (rn <= o->tol * norm_b || rn == 0.0) {
      if (iters_out) *iters_out = total_iters;
      return MCRT_OK;
    }
    // FP64 rounding floor of the residual: no halving for three refinement steps below 1e-8
    if (rn < 0.5 * best) {
      best = rn;
      stall = 0;
    } else if (++stall >= 3 && best <= 1e-8 * norm_b) {
      if (iters_out) *iters_out = total_iters;
      return MCRT_OK;
    }
    if (outer == o->max_outer) break;
    // inner FP32 CG on the unit-diagonal system
    CK(cudaMemsetAsync(sc, 0, sizeof(double) * (2 * (size_t)o->max_inner + 8), st), "memset");
    k_start<<<sgrid(n), 256, 0, st>>>(n, mask, P->rs.as<double>(), 1.0 / rn, y, r, pb[1], pb[0], Ap, sc);
    d->launches++;
    int k = 0;
    bool conv = false;
    if (chunk_exec) CK(cudaMemsetAsync(kdev, 0, sizeof(int), st), "memset");
    double h[2 * chunk + 2];
    while (k < o->max_inner && !conv) {
      const int k0 = k;
      const int kend = std::min(k + chunk, o->max_inner);
      if (chunk_exec) {
        // one replay: `chunk` iterations, the iteration index read from the device; iterations at or
        // beyond max_inner do nothing
        CK(cudaGraphLaunch(chunk_exec, st), "graph launch");
        d->launches += 3 * chunk;
        k = kend;
      } else {
        for (; k < kend; ++k) {
          float* pnew = pb[k & 1];
          float* pold = pb[(k + 1) & 1];
          launch_cg_iteration(P, n, nt, tiles, r, pold, pnew, Ap, y, sc, nullptr, k, o->max_inner, tol2_in, ga, gb, st);
          d->launches += 2;
        }
      }
      // rr_0 and rr_{k0..k}
      double rr0 = 0.0;
      CK(cudaMemcpyAsync(&rr0, sc, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
      CK(cudaMemcpyAsync(h, sc + 2 * k0, sizeof(double) * (2 * (size_t)(k - k0) + 1), cudaMemcpyDeviceToHost, st),
         "copy");
      CK(cudaStreamSynchronize(st), "synchronize");
      for (int kk = k0; kk <= k; ++kk) {
        const double v = h[2 * (kk - k0)];
        if (v <= tol2_in * rr0 || !(v == v)) {
          conv = true;
          total_iters += kk;
          break;
        }
      }
    }
    if (!conv) total_iters += k;
    k_update<<<nblk(n), 256, 0, st>>>(n, mask, dis, y, rn, x);
    d->launches++;
    CK(cudaGetLastError(), "PDA kernels");
  }
  if (iters_out) *iters_out = total_iters;
  return set_error(d, MCRT_ENOTCONV, "PDA solve did not reach its tolerance");
}

extern "C" {

void mcrt_default_pda_opts(mcrt_pda_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->min_visits = 30;
  o->max_rel_err = 0.05;
  o->tol = 1e-12;
  o->inner_tol = 1e-5;
  o->max_outer = 50;
  o->max_inner = 20000;
  o->min_cell_tau = 1.0;
  o->kappa_R = nullptr;
  o->rho = nullptr;
}

mcrt_status mcrt_solve_pda(mcrt_disk* d, const mcrt_pda_opts* o, int* out_n, int* out_iters) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!o) return set_error(d, MCRT_EINVAL, "opts is NULL");
  if (!d->has_opacity) return set_error(d, MCRT_ESTATE, "mcrt_set_opacity must come first");
  if (!(o->tol > 0) || !(o->inner_tol > 0 && o->inner_tol < 1) || o->max_outer < 1 || o->max_inner < 1 ||
      o->max_inner > 10000000 || !(o->min_cell_tau >= 0))
    return set_error(d, MCRT_EINVAL, "bad PDA options");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  mcrt_status s = pda_alloc(d, o->max_inner);
  if (s != MCRT_OK) return s;
  if (!d->have_T) {
    s = compute_temperatures(d);
    if (s != MCRT_OK) return s;
  }
  PdaState* P = d->pda;
  const int nr = d->nr, nt = d->nt, n = nr * nt;
  cudaStream_t st = d->stream;
  double* red = P->red.as<double>();
  CK(cudaMemsetAsync(red, 0, 16 * 8, st), "memset");
  const double* rho = d->rho_cgs_d.as<double>();
  double chi_max = 0.0;
  for (int b = 0; b < d->nlam; ++b) chi_max = std::max(chi_max, d->kabs[b] + (1.0 - d->g[b]) * d->ksca[b]);
  k_mask<<<sgrid(n), 256, 0, st>>>(n, rho, P->ell.as<double>(), chi_max, o->min_cell_tau,
                                  d->visits.as<unsigned long long>(), d->relerr.as<double>(),
                                  d->tally.as<unsigned long long>(), o->min_visits, o->max_rel_err,
                                  P->mask.as<signed char>(), red);
  k_bnd_mean<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), d->T_mc.as<double>(), red);
  DBuf over;
  if (o->kappa_R) {
    for (int c = 0; c < n; ++c)
      if (d->rho[c] > 0 && !(o->kappa_R[c] > 0 && std::isfinite(o->kappa_R[c])))
        return set_error(d, MCRT_EINVAL, "kappa_R must be positive where there is dust");
    CK(over.alloc((size_t)n * 8), "cudaMalloc");
    CK(cudaMemcpyAsync(over.p, o->kappa_R, (size_t)n * 8, cudaMemcpyHostToDevice, st), "copy");
  }
  k_kappaR<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), rho, d->tally.as<unsigned long long>(),
                                    d->T_mc.as<double>(), red,
                                    d->gray ? 1 : 0, (double)(d->kabs[0] + (1.0 - d->g[0]) * d->ksca[0]), d->nlam,
                                    d->lam_e_d.as<double>(), d->chip_d.as<double>(), over.as<double>(),
                                    P->kR.as<double>());
  DBuf rho_over;
  const double* rhoD = rho;
  if (o->rho) {
    for (int c = 0; c < n; ++c)
      if (d->rho[c] > 0 && !(o->rho[c] > 0 && std::isfinite(o->rho[c])))
        return set_error(d, MCRT_EINVAL, "rho override must be positive where the disk has dust");
    CK(rho_over.alloc((size_t)n * 8), "cudaMalloc");
    CK(cudaMemcpyAsync(rho_over.p, o->rho, (size_t)n * 8, cudaMemcpyHostToDevice, st), "copy");
    rhoD = rho_over.as<double>();
  }
  k_cond<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), rhoD, P->kR.as<double>(), P->hr_in.as<double>(), P->hr_out.as<double>(),
                                  P->ht_lo.as<double>(), P->ht_hi.as<double>(), P->D.as<double>(), P->Cr.as<double>(),
                                  P->Ct.as<double>());
  k_diag<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), P->Cr.as<double>(), P->Ct.as<double>(),
                                  d->T_mc.as<double>(), P->dis.as<double>(), P->u.as<double>(), red);
  k_scaled<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), P->Cr.as<double>(), P->Ct.as<double>(),
                                    P->dis.as<double>(), P->ar.as<float>(), P->at.as<float>());
  d->launches += 6;
  double hred[4];
  CK(cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st), "copy");
  std::vector<signed char> hmask(n);
  CK(cudaMemcpyAsync(hmask.data(), P->mask.p, n, cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaStreamSynchronize(st), "synchronize");
  CK(cudaGetLastError(), "PDA setup kernels");
  P->n_pda = (int)hred[0];
  if (out_n) *out_n = P->n_pda;
  if (hred[3] > 0 || !components_ok(d, hmask))
    return set_error(d, MCRT_EINVAL, "a PDA region touches no Monte Carlo cell (singular system)");
  P->vec4 = nt % 4 == 0;  // 16-byte kernels on 128-cell tiles
  P->htiles = active_tiles(hmask, P->vec4 ? 128 : 32);
  P->ntiles = (int)P->htiles.size();
  if (P->ntiles > 0)
    CK(cudaMemcpyAsync(P->tiles.p, P->htiles.data(), P->htiles.size() * sizeof(int), cudaMemcpyHostToDevice, st),
       "copy");
  int iters = 0;
  if (P->n_pda > 0) {
    s = refine_solve(d, o, P->u.as<double>(), nullptr, &iters);
    if (s != MCRT_OK) {
      if (out_iters) *out_iters = iters;
      return s;
    }
  }
  if (out_iters) *out_iters = iters;
  k_tpda<<<nblk(n), 256, 0, st>>>(n, P->mask.as<signed char>(), P->u.as<double>(), d->T_mc.as<double>(),
                                  d->T_pda.as<double>());
  d->launches++;
  CK(cudaGetLastError(), "PDA kernels");
  CK(cudaStreamSynchronize(st), "synchronize");
  d->have_pda = true;
  d->T_epoch++;
  return MCRT_OK;
}

mcrt_status mcrt_pda_adjoint_dev(mcrt_disk* d, const double* w_dev, double* g_lr, double* g_kr) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!w_dev) return set_error(d, MCRT_EINVAL, "w is NULL");
  if (!d->have_pda || !d->pda) return set_error(d, MCRT_ESTATE, "mcrt_solve_pda must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  PdaState* P = d->pda;
  const int nr = d->nr, nt = d->nt, n = nr * nt;
  cudaStream_t st = d->stream;
  k_adj_rhs<<<nblk(n), 256, 0, st>>>(n, P->mask.as<signed char>(), w_dev, P->u.as<double>(), P->b64.as<double>(),
                                     P->lam.as<double>());
  d->launches++;
  mcrt_pda_opts o;
  mcrt_default_pda_opts(&o);
  if (P->n_pda > 0) {
    if (P->max_inner_alloc < o.max_inner) {
      mcrt_status s = pda_alloc(d, o.max_inner);
      if (s != MCRT_OK) return s;
    }
    int it = 0;
    mcrt_status s = refine_solve(d, &o, P->lam.as<double>(), P->b64.as<double>(), &it);
    if (s != MCRT_OK) return s;
  }
  k_grad<<<nblk(n), 256, 0, st>>>(nr, nt, P->mask.as<signed char>(), P->Cr.as<double>(), P->Ct.as<double>(),
                                  P->D.as<double>(), P->kR.as<double>(), P->hr_in.as<double>(), P->hr_out.as<double>(),
                                  P->ht_lo.as<double>(), P->ht_hi.as<double>(), P->u.as<double>(), P->lam.as<double>(),
                                  g_lr, g_kr);
  d->launches++;
  CK(cudaGetLastError(), "adjoint kernels");
  return MCRT_OK;
}

mcrt_status mcrt_pda_adjoint(mcrt_disk* d, const double* w, double* g_lr, double* g_kr) {
  if (!d) return set_error(nullptr, MCRT_EINVAL, "disk is NULL");
  if (!w) return set_error(d, MCRT_EINVAL, "w is NULL");
  if (!d->have_pda || !d->pda) return set_error(d, MCRT_ESTATE, "mcrt_solve_pda must come first");
  CK(cudaSetDevice(d->device), "cudaSetDevice");
  PdaState* P = d->pda;
  const size_t n = (size_t)d->nr * d->nt;
  CK(cudaMemcpyAsync(P->w.p, w, n * 8, cudaMemcpyHostToDevice, d->stream), "copy");
  mcrt_status s = mcrt_pda_adjoint_dev(d, P->w.as<double>(), P->gl.as<double>(), P->gk.as<double>());
  if (s != MCRT_OK) return s;
  if (g_lr) CK(cudaMemcpyAsync(g_lr, P->gl.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  if (g_kr) CK(cudaMemcpyAsync(g_kr, P->gk.p, n * 8, cudaMemcpyDeviceToHost, d->stream), "copy");
  CK(cudaStreamSynchronize(d->stream), "synchronize");
  return MCRT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// PDA solve without allocation: the same FP64-refined FP32 CG, on a system the caller supplies in
// its own device buffers, with all working vectors in one file-scope device array. For callers that
// may not allocate device memory after start-up (a host framework that owns every device byte
// through its own pool, or a service that fixes its memory at initialisation), so that no call here
// ever reaches cudaMalloc/cudaFree.
// ------------------------------------------------------------------------------------------------
namespace {
constexpr long long kStaticMaxCells = 131072;  // nr * ntheta limit of mcrt_pda_solve_static
constexpr int kStaticMaxInner = 20000;          // CG iterations per refinement step
constexpr size_t kStaticSc = 2 * (size_t)kStaticMaxInner + 8;
// layout: dis, rs (f64 per cell) | ar, at, y, r, p0, p1, Ap (f32 per cell) | sc, red (f64)
constexpr size_t kStaticBytes = 2 * 8 * kStaticMaxCells + 7 * 4 * kStaticMaxCells + 8 * (kStaticSc + 16);
std::mutex g_static_mu;
void* g_static_addr[64] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_pda_static_scratch[kStaticBytes];

namespace mcrt {
__global__ void k_static_dis(int nr, int nt, const signed char* mask, const double* Cr, const double* Ct, double* dis,
                             double* red) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nr * nt) return;
  const int i = c / nt, j = c - i * nt;
  if (mask[c] != 2) {
    dis[c] = 0.0;
    return;
  }
  double dsum = 0.0;
  if (i > 0 && mask[c - nt]) dsum += Cr[c - nt];
  if (i + 1 < nr && mask[c + nt]) dsum += Cr[c];
  if (j > 0 && mask[c - 1]) dsum += Ct[c - 1];
  if (j + 1 < nt && mask[c + 1]) dsum += Ct[c];
  if (dsum > 0) {
    dis[c] = 1.0 / sqrt(dsum);
  } else {
    dis[c] = 0.0;
    atomicAdd(red + 3, 1.0);
  }
}
// |S b|^2 of the system: the scaled residual with every unknown (mask 2) cell at 0, so that only the fixed
// (mask 1) neighbours contribute; the solve's tolerance is relative to it, as in mcrt_solve_pda
__global__ void k_static_bnorm(int nr, int nt, const signed char* mask, const double* Cr, const double* Ct,
                               const double* dis, const double* u, double* red) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nr * nt; c += gridDim.x * blockDim.x) {
    if (mask[c] != 2) continue;
    const int i = c / nt, j = c - i * nt;
    double r = 0.0;
    if (i > 0 && mask[c - nt] == 1) r += Cr[c - nt] * u[c - nt];
    if (i + 1 < nr && mask[c + nt] == 1) r += Cr[c] * u[c + nt];
    if (j > 0 && mask[c - 1] == 1) r += Ct[c - 1] * u[c - 1];
    if (j + 1 < nt && mask[c + 1] == 1) r += Ct[c] * u[c + 1];
    const double v = dis[c] * r;
    acc += v * v;
  }
  const double s = block_sum_d(acc, sh);
  if (threadIdx.x == 0 && s != 0.0) atomicAdd(red + 5, s);
}
}  // namespace mcrt

namespace {
// makes a device current for the lifetime of the object and restores the caller's current device after
struct CurrentDevice {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit CurrentDevice(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    err = cudaSetDevice(dev);
  }
  ~CurrentDevice() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

extern "C" mcrt_status mcrt_pda_solve_static(int device, int nr, int ntheta, const signed char* mask_dev,
                                             const double* Cr_dev, const double* Ct_dev, double* u_dev,
                                             const mcrt_pda_opts* o, void* cuda_stream, int* out_iters) {
  mcrt_disk* d = nullptr;  // errors go to the thread's last-error message
  if (!mask_dev || !Cr_dev || !Ct_dev || !u_dev || !o) return set_error(nullptr, MCRT_EINVAL, "NULL argument");
  if (nr < 1 || ntheta < 1 || (long long)nr * ntheta > kStaticMaxCells)
    return set_error(nullptr, MCRT_EINVAL,
                     "nr * ntheta must be between 1 and 131072 for mcrt_pda_solve_static (its fixed scratch size)");
  if (!(o->tol > 0) || !(o->inner_tol > 0 && o->inner_tol < 1) || o->max_outer < 1 || o->max_inner < 1)
    return set_error(nullptr, MCRT_EINVAL, "bad PDA options");
  if (o->max_inner > kStaticMaxInner)
    return set_error(nullptr, MCRT_EINVAL, "max_inner must be <= 20000 for mcrt_pda_solve_static");
  if (device < 0 || device >= 64) return set_error(nullptr, MCRT_EINVAL, "device index out of range");
  const CurrentDevice cur(device);  // the caller's current device is restored on every return
  CK(cur.err, "cudaSetDevice");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[device]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_pda_static_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the PDA scratch array");
      g_static_addr[device] = a;
    }
    base = static_cast<unsigned char*>(g_static_addr[device]);
  }
  const int n = nr * ntheta;
  const size_t N = (size_t)kStaticMaxCells;
  double* dis = reinterpret_cast<double*>(base);
  double* rs = dis + N;
  float* ar = reinterpret_cast<float*>(rs + N);
  float* at = ar + N;
  float* y = at + N;
  float* r = y + N;
  float* pb[2] = {r + N, r + 2 * N};
  float* Ap = r + 3 * N;
  double* sc = reinterpret_cast<double*>(Ap + N);
  double* red = sc + kStaticSc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nt = ntheta;
  // scratch keeps the previous call's contents: clear what must start at zero
  CK(cudaMemsetAsync(red, 0, 16 * sizeof(double), st), "memset");
  k_static_dis<<<nblk(n), 256, 0, st>>>(nr, nt, mask_dev, Cr_dev, Ct_dev, dis, red);
  k_scaled<<<nblk(n), 256, 0, st>>>(nr, nt, mask_dev, Cr_dev, Ct_dev, dis, ar, at);
  k_static_bnorm<<<sgrid(n), 256, 0, st>>>(nr, nt, mask_dev, Cr_dev, Ct_dev, dis, u_dev, red);
  double red_h[6] = {0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(red_h, red, sizeof(red_h), cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaStreamSynchronize(st), "synchronize");
  CK(cudaGetLastError(), "PDA kernels");
  if (red_h[3] > 0) return set_error(nullptr, MCRT_EINVAL, "a PDA cell has no conducting face (singular system)");
  const double norm_b = std::sqrt(red_h[5]);  // |S b|: the tolerance does not depend on the starting guess
  const double tol2_in = o->inner_tol * o->inner_tol;
  const int ntiles = (n + 31) / 32;  // every tile of the grid
  const int ga = tgrid(k_cg_a<kUA>, ntiles), gb = tgrid(k_cg_b<kUB>, ntiles);
  double best = INFINITY;
  int total_iters = 0, stall = 0;
  const int chunk = 32;
  double h[2 * chunk + 2];
  for (int outer = 0; outer <= o->max_outer; ++outer) {
    CK(cudaMemsetAsync(red + 4, 0, sizeof(double), st), "memset");
    k_resid64<<<sgrid(n), 256, 0, st>>>(nr, nt, mask_dev, Cr_dev, Ct_dev, dis, u_dev, nullptr, rs, red, 4);
    double rn2 = 0.0;
    CK(cudaMemcpyAsync(&rn2, red + 4, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    CK(cudaStreamSynchronize(st), "synchronize");
    const double rn = std::sqrt(rn2);
    if (!(rn == rn)) return set_error(nullptr, MCRT_ENOTCONV, "PDA residual is not finite");
    if (rn <= o->tol * norm_b || rn == 0.0) {
      if (out_iters) *out_iters = total_iters;
      return MCRT_OK;
    }
    if (rn < 0.5 * best) {
      best = rn;
      stall = 0;
    } else if (++stall >= 3 && best <= 1e-8 * norm_b) {
      if (out_iters) *out_iters = total_iters;
      return MCRT_OK;
    }
    if (outer == o->max_outer) break;
    CK(cudaMemsetAsync(sc, 0, sizeof(double) * kStaticSc, st), "memset");
    k_start<<<sgrid(n), 256, 0, st>>>(n, mask_dev, rs, 1.0 / rn, y, r, pb[1], pb[0], Ap, sc);
    int k = 0;
    bool conv = false;
    while (k < o->max_inner && !conv) {
      const int k0 = k;
      const int kend = std::min(k + chunk, o->max_inner);
      for (; k < kend; ++k) {
        k_cg_a<kUA><<<ga, 256, 0, st>>>(n, nt, ntiles, nullptr, ar, at, r, pb[(k + 1) & 1], pb[k & 1], Ap, sc, nullptr,
                                        k, kStaticMaxInner, tol2_in);
        k_cg_b<kUB><<<gb, 256, 0, st>>>(n, ntiles, nullptr, pb[k & 1], Ap, y, r, sc, nullptr, k, kStaticMaxInner,
                                        tol2_in);
      }
      // rr_0 and rr_{k0..k}
      double rr0 = 0.0;
      CK(cudaMemcpyAsync(&rr0, sc, sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
      CK(cudaMemcpyAsync(h, sc + 2 * k0, sizeof(double) * (2 * (size_t)(k - k0) + 1), cudaMemcpyDeviceToHost, st),
         "copy");
      CK(cudaStreamSynchronize(st), "synchronize");
      for (int kk = k0; kk <= k; ++kk) {
        const double v = h[2 * (kk - k0)];
        if ((kk > 0 || k0 > 0) && (v <= tol2_in * rr0 || !(v == v))) {
          conv = true;
          total_iters += kk;
          break;
        }
      }
    }
    if (!conv) total_iters += k;
    k_update<<<nblk(n), 256, 0, st>>>(n, mask_dev, dis, y, rn, u_dev);
    CK(cudaGetLastError(), "PDA kernels");
  }
  if (out_iters) *out_iters = total_iters;
  return set_error(nullptr, MCRT_ENOTCONV, "PDA solve did not reach its tolerance");
}
