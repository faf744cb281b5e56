// cuda_host_stubs.h -- single-lane host stand-ins for the CUDA builtins that the library's device
// headers name, so that their code can be compiled by the host compiler for CPU tests: one lane (warp
// operations return their own lane's value), atomics as plain read-modify-writes, the fast FP32
// intrinsics as the host's correctly rounded functions, float overloads of the math functions as CUDA
// provides them for device code. threadIdx / blockIdx / blockDim / gridDim are host variables a test may
// set to run a kernel's body lane by lane.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

struct HostIdx {
  unsigned x, y, z;
};
inline HostIdx host_threadIdx{0, 0, 0}, host_blockIdx{0, 0, 0}, host_blockDim{1, 1, 1}, host_gridDim{1, 1, 1};
#define threadIdx host_threadIdx
#define blockIdx host_blockIdx
#define blockDim host_blockDim
#define gridDim host_gridDim
#ifndef __noinline__
#define __noinline__ __attribute__((noinline))
#endif
#define __launch_bounds__(...)
// float overloads of the math functions, as CUDA provides them for device code
using std::acos;
using std::atan2;
using std::cbrt;
using std::cos;
using std::exp;
using std::fabs;
using std::floor;
using std::fmax;
using std::fmin;
using std::isfinite;
using std::log;
using std::pow;
using std::signbit;
using std::sin;
using std::sqrt;
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
inline unsigned long long atomicCAS(unsigned long long* p, unsigned long long cmp, unsigned long long v) {
  const unsigned long long o = *p;
  if (o == cmp) *p = v;
  return o;
}
inline long long __double_as_longlong(double x) {
  long long v;
  std::memcpy(&v, &x, sizeof v);
  return v;
}
template <class T>
inline T __shfl_sync(unsigned, T v, int, int = 32) { return v; }
template <class T>
inline T __shfl_up_sync(unsigned, T v, unsigned, int = 32) { return v; }
template <class T>
inline T __shfl_down_sync(unsigned, T v, unsigned, int = 32) { return v; }
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

