// Device helpers shared by the library's kernels: launch bookkeeping,
// the Philox4x32-10 generator, Box-Muller normals and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace afqmc {

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). Round: multiply counter
// words 0 and 2 by two 32-bit constants, keep both product halves, mix with
// words 1 and 3 and the key; the key advances by two Weyl increments.
// ----------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ void mul_hi_lo(uint32_t a, uint32_t b,
                                                   uint32_t& hi, uint32_t& lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hA, lA, hB, lB;
    mul_hi_lo(kMulA, c.x, hA, lA);
    mul_hi_lo(kMulB, c.z, hB, lB);
    U4 n;
    n.x = hB ^ c.y ^ k0;
    n.y = lB;
    n.z = hA ^ c.w ^ k1;
    n.w = lA;
    c = n;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return c;
}

// Word -> (0,1): (r + 1/2) 2^-32, exact in double.
__device__ __forceinline__ double open01(uint32_t r) {
  return ((double)r + 0.5) * 2.3283064365386963e-10;
}

// Box-Muller pair from two words, in double precision.
__device__ __forceinline__ void box_muller(uint32_t ra, uint32_t rb, double& z0,
                                           double& z1) {
  double rad = sqrt(-2.0 * log(open01(ra)));
  double s, c;
  sincospi(2.0 * open01(rb), &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

// The same pair in single precision: u = (r + 1/2) 2^-32 rounded to FP32
// (never 0 or 1 after rounding for r < 2^32 - 128; the top values map to
// 1 - 2^-24 by clamping).
__device__ __forceinline__ void box_muller_f(uint32_t ra, uint32_t rb, float& z0, float& z1) {
  float ua = fminf(((float)ra + 0.5f) * 2.3283064365386963e-10f, 0.99999994f);
  float ub = ((float)rb + 0.5f) * 2.3283064365386963e-10f;
  float rad = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  z0 = rad * c;
  z1 = rad * s;
}

enum { kStreamFields = 0, kStreamComb = 1 };

// ----------------------------------------------------------------------------
// Reductions
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread gets the result. `red` needs
// blockDim.x/32 entries of shared memory.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = 0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

}  // namespace afqmc
