// Measurement probe (no counterpart in the guide): one radix-8 DFT stage of the product's FFTs
// computed two ways on the same data, to decide whether tensor cores can replace FP32 butterflies.
//
//  - FP32 butterflies: the product's own Dft<8> (fft.cuh), one 8-point complex vector per thread.
//  - Tensor cores, split TF32: the stage as a real matrix product Y = W X, W the 16 x 16 real form
//    of the unitary 8-point DFT ([[C, S], [-S, C]] / sqrt 8 acting on [Re x; Im x]), X holding 8
//    vectors as columns; mma.sync m16n8k8 TF32 with FP32 accumulation, and each operand split into
//    a TF32 head and a TF32 tail (W X ~ Wh Xh + Wh Xl + Wl Xh, three products) because one TF32
//    product keeps only ~11 significant bits, far from the 1e-5 relative accuracy the product needs.
//    Between repetitions the output fragments are moved back into operand layout with warp shuffles
//    (the exchange an FFT needs between stages).
// Both kernels apply the stage `reps` times to data held in registers (a compute-bound measurement;
// the unitary scaling keeps magnitudes fixed), so the timing is the arithmetic of the stage alone.
#include <cmath>
#include <vector>

#include "dda_internal.h"

namespace dda {
namespace {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// element (r, c) of the 16 x 16 real form of the unitary forward 8-point DFT
__device__ __forceinline__ double wreal(int r, int c) {
  const int k = r & 7, j = c & 7;
  const double ang = 2.0 * 3.14159265358979323846 * (double)((j * k) & 7) / 8.0;
  const double cs = cos(ang) * 0.35355339059327376220, sn = sin(ang) * 0.35355339059327376220;
  const bool out_im = r >= 8, in_im = c >= 8;
  // Re y = C Re x + S Im x ; Im y = -S Re x + C Im x   (y = sum x exp(-i ang))
  if (!out_im) return in_im ? sn : cs;
  return in_im ? cs : -sn;
}

__global__ void k_dft8_fp32(float2* __restrict__ data, int64_t nvec, int reps) {
  const float s = 0.35355339059327376220f;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nvec; v += (int64_t)gridDim.x * blockDim.x) {
    float2 x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = data[v * 8 + j];
    for (int r = 0; r < reps; ++r) {
      Dft<8, -1, float2>::run(x);
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = make_float2(x[j].x * s, x[j].y * s);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) data[v * 8 + j] = x[j];
  }
}

// one warp: 8 vectors (the 8 columns of X) per tile
__global__ void k_dft8_tf32x3(float2* __restrict__ data, int64_t nvec, int reps) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // A fragments (rows g, g+8; cols t, t+4) of both k-steps, head and tail
  uint32_t ah[2][4], al[2][4];
  for (int ks = 0; ks < 2; ++ks) {
    const int cols[4] = {t, t, t + 4, t + 4}, rows[4] = {g, g + 8, g, g + 8};
    for (int q = 0; q < 4; ++q) {
      const float w = (float)wreal(rows[q], ks * 8 + cols[q]);
      ah[ks][q] = to_tf32(w);
      al[ks][q] = to_tf32(w - __uint_as_float(ah[ks][q]));
    }
  }
  const int64_t ntile = nvec / 8;
  const int warps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
  for (int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; tile < ntile; tile += warps) {
    // B operand: X[k][n], k = 0..7 real parts, 8..15 imaginary parts, n = vector; lane holds
    // (k = t, n = g) and (k = t + 4, n = g) of each k-step
    const float2* vg = data + (tile * 8 + g) * 8;
    float xb[2][2] = {{vg[t].x, vg[t + 4].x}, {vg[t].y, vg[t + 4].y}};
    for (int r = 0; r < reps; ++r) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t h0 = to_tf32(xb[ks][0]), h1 = to_tf32(xb[ks][1]);
        const uint32_t l0 = to_tf32(xb[ks][0] - __uint_as_float(h0)), l1 = to_tf32(xb[ks][1] - __uint_as_float(h1));
        mma_tf32(d, al[ks], h0, h1);
        mma_tf32(d, ah[ks], l0, l1);
        mma_tf32(d, ah[ks], h0, h1);
      }
      // D (rows g, g + 8; cols 2t, 2t + 1) -> next B: lane (g, t) needs Y[t][g], Y[t + 4][g] (real)
      // and Y[8 + t][g], Y[12 + t][g] (imaginary); Y[k][n] sits in lane (k mod 8, n / 2), register
      // (k >= 8 ? 2 : 0) + (n & 1)
      const int src0 = t * 4 + (g >> 1), src1 = (t + 4) * 4 + (g >> 1);
      const bool odd = g & 1;
      const float r0a = __shfl_sync(0xffffffffu, d[0], src0), r0b = __shfl_sync(0xffffffffu, d[1], src0);
      const float r1a = __shfl_sync(0xffffffffu, d[0], src1), r1b = __shfl_sync(0xffffffffu, d[1], src1);
      const float i0a = __shfl_sync(0xffffffffu, d[2], src0), i0b = __shfl_sync(0xffffffffu, d[3], src0);
      const float i1a = __shfl_sync(0xffffffffu, d[2], src1), i1b = __shfl_sync(0xffffffffu, d[3], src1);
      xb[0][0] = odd ? r0b : r0a;
      xb[0][1] = odd ? r1b : r1a;
      xb[1][0] = odd ? i0b : i0a;
      xb[1][1] = odd ? i1b : i1a;
    }
    float2* og = data + (tile * 8 + g) * 8;
    og[t] = make_float2(xb[0][0], xb[1][0]);
    og[t + 4] = make_float2(xb[0][1], xb[1][1]);
  }
}

}  // namespace

Err probe_tc_dft(int64_t nvec, int reps, double out[4]) {
  if (nvec < 8 || nvec % 8 || reps < 1) return Err::make(DDA_EINVAL, "nvec must be a positive multiple of 8");
  std::vector<float2> h((size_t)nvec * 8);
  uint64_t st = 0x9e3779b97f4a7c15ull;
  auto rnd = [&]() {
    st ^= st << 13; st ^= st >> 7; st ^= st << 17;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  };
  for (auto& v : h) v = make_float2((float)rnd(), (float)rnd());
  // FP64 reference: the unitary DFT applied reps times to the first 64 vectors
  const int nref = 64;
  std::vector<double> ref((size_t)nref * 16);
  for (int v = 0; v < nref; ++v) {
    double xr[8], xi[8];
    for (int j = 0; j < 8; ++j) { xr[j] = h[v * 8 + j].x; xi[j] = h[v * 8 + j].y; }
    for (int r = 0; r < reps; ++r) {
      double yr[8], yi[8];
      for (int k = 0; k < 8; ++k) {
        yr[k] = yi[k] = 0.0;
        for (int j = 0; j < 8; ++j) {
          const double a = 2.0 * 3.14159265358979323846 * (double)((j * k) & 7) / 8.0;
          yr[k] += xr[j] * std::cos(a) + xi[j] * std::sin(a);
          yi[k] += xi[j] * std::cos(a) - xr[j] * std::sin(a);
        }
      }
      for (int k = 0; k < 8; ++k) { xr[k] = yr[k] / std::sqrt(8.0); xi[k] = yi[k] / std::sqrt(8.0); }
    }
    for (int k = 0; k < 8; ++k) { ref[v * 16 + k] = xr[k]; ref[v * 16 + 8 + k] = xi[k]; }
  }
  float2* d = nullptr;
  DDA_CU(cudaMalloc((void**)&d, sizeof(float2) * h.size()));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  Err err = Err::Ok();
  for (int kind = 0; kind < 2 && err.ok(); ++kind) {
    float ms = 0.f;
    for (int pass = 0; pass < 2 && err.ok(); ++pass) {  // pass 0 warms up
      if (cudaMemcpy(d, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = Err::make(DDA_ECUDA, "probe upload failed");
        break;
      }
      cudaEventRecord(e0);
      if (kind == 0) k_dft8_fp32<<<152 * 8, 256>>>(d, nvec, reps);
      else k_dft8_tf32x3<<<152 * 8, 256>>>(d, nvec, reps);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        err = Err::make(DDA_ECUDA, "probe kernel failed");
      cudaEventElapsedTime(&ms, e0, e1);
    }
    std::vector<float2> got((size_t)nref * 8);
    if (err.ok() && cudaMemcpy(got.data(), d, sizeof(float2) * got.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      err = Err::make(DDA_ECUDA, "probe readback failed");
    double num = 0.0, den = 0.0;
    for (int v = 0; v < nref; ++v)
      for (int k = 0; k < 8; ++k) {
        const double dr = got[v * 8 + k].x - ref[v * 16 + k], di = got[v * 8 + k].y - ref[v * 16 + 8 + k];
        num += dr * dr + di * di;
        den += ref[v * 16 + k] * ref[v * 16 + k] + ref[v * 16 + 8 + k] * ref[v * 16 + 8 + k];
      }
    out[kind] = ms;
    out[2 + kind] = den > 0 ? std::sqrt(num / den) : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  return err;
}

}  // namespace dda
