// Host build of the transport kernels' counter-based generator (common.cuh: philox4x32_10), for a CPU
// test against independent implementations.
#include "common.cuh"

extern "C" void philox_host(const unsigned* ctr, const unsigned* key, unsigned* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  mcrt::philox4x32_10(c0, c1, c2, c3, key[0], key[1]);
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}
