// Per-RHS reductions for kernels whose CTAs are laid out by the FFT passes
// rather than by a vector loop: each CTA reduces its products into one slot of
// a partial-sum table, and the last CTA of a right-hand side to arrive (a
// device-scope counter) sums that RHS's slots in a fixed order.  The scheme and
// the double-float product accumulation are those of the Krylov vector kernels
// (krylov.cu), so fused and unfused iterations reduce alike.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dda_internal.h"

namespace dda {
namespace kred {

// a thread's running sum of float products carried as a double-float pair
// (products split exactly with one FMA, added with the two-sum)
struct AccF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void fma(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(hi, p);
    const float z = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, z)), __fsub_rn(p, z));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
// re + i im += conj(a) b
__device__ __forceinline__ void acc_cdot(AccF& re, AccF& im, float2 a, float2 b) {
  re.fma(a.x, b.x);
  re.fma(a.y, b.y);
  im.fma(a.x, b.y);
  im.fma(-a.y, b.x);
}
__device__ __forceinline__ void acc_nrm(AccF& s, float2 a) {
  s.fma(a.x, a.x);
  s.fma(a.y, a.y);
}

// Block sum of v (all threads call; blockDim.x a multiple of 32, at most 1024); result in out (thread 0 writes).
template <int NS>
__device__ __forceinline__ void block_sum(double (&v)[NS], double* out) {
  __shared__ double red[NS][32];
#pragma unroll
  for (int s = 0; s < NS; ++s)
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_down_sync(0xffffffffu, v[s], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) red[s][w] = v[s];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double x = (threadIdx.x < (blockDim.x >> 5)) ? red[s][threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (threadIdx.x == 0) out[s] = x;
    }
  }
}

// Store this CTA's block sum of acc in slot `slot` of RHS b (nblk slots per RHS, kRedSlots
// doubles each).  Returns true in every thread of the last CTA of b to arrive, with b's totals
// in tot; that CTA also resets b's counter to zero.  All threads of the CTA must call it.
template <int NS>
__device__ __forceinline__ bool last_cta_totals(double (&acc)[NS], double* part, unsigned int* count, int b,
                                                int slot, int nblk, double (&tot)[NS]) {
  double* mine = part + ((int64_t)b * nblk + slot) * kRedSlots;
  block_sum<NS>(acc, mine);
  __shared__ unsigned int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(count + b, 1u) == (unsigned)nblk - 1u) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const double* base = part + (int64_t)b * nblk * kRedSlots;
  double v[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) v[q] = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < NS; ++q) v[q] += __ldcg(base + (int64_t)i * kRedSlots + q);
  __shared__ double res[NS];
  block_sum<NS>(v, res);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NS; ++q) tot[q] = res[q];
  if (threadIdx.x == 0) count[b] = 0;
  return true;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

}  // namespace kred
}  // namespace dda
