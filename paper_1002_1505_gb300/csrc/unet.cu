// Learned warm start for the Krylov solve: a small 3-D U-Net trained on the
// solver's own solutions (the guide has no learned component; the solver
// accepts any initial guess, and a better one saves iterations).
//
// Network (channels-last tensors [B][Z][Y][X][C], FP32 in memory):
//   enc1: cin->C1, C1->C1 | pool | enc2: C1->C2, C2->C2 | pool | enc3: C2->C3, C3->C3 | pool
//   bottleneck: C3->C4, C4->C4 | up | dec3: C4+C3->C3, C3->C3 | up | dec2: C3+C2->C2, C2->C2
//   | up | dec1: C2+C1->C1, C1->C1 | head 1x1x1: C1->cout
// 3x3x3 zero-padded convolutions with ReLU, 2x2x2 average pooling, nearest
// x2 upsampling, skips concatenated as [upsampled, skip].
//
// Convolutions are implicit GEMMs on the tensor cores (bfloat16 operands, FP32
// accumulation): the input activation (or incoming gradient) is rounded to
// bfloat16 as it is loaded, weights are kept as an FP32 master copy and repacked
// to bfloat16 tiles after every update.  Two engines: tcgen05 MMAs on TMA-staged
// halo tiles with tensor-memory accumulators, where each of the 27 taps is a
// shifted shared-memory descriptor of the same staged tile (k_conv_tc, the
// default), and mma.sync m16n8k16 with per-thread neighbour gathers (k_conv;
// DDA_UNET_TC=0).  The 1x1x1 head and the weight gradients always use mma.sync.
//   forward     y[v, co]  = sum_{tap, ci} x[v + tap, ci] W[tap, ci, co] + b[co]
//   input grad  gx[v, ci] = sum_{tap, co} g[v - tap, co] W[tap, ci, co]   (same kernel, flipped
//                           taps and transposed weights)
//   weight grad gW[tap, ci, co] = sum_v x[v + tap, ci] g[v, co]            (voxels as the K axis,
//                           per-chunk partials summed in a fixed order: deterministic)
// AdamW (decoupled weight decay) updates the FP32 master parameters.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "bulk.cuh"
#include "dda_internal.h"

namespace dda {
namespace nn {

constexpr int kTaps = 27;
constexpr int kConvThreads = 128;  // 4 warps, 16 voxels each
constexpr int kVoxPerCta = 64;
constexpr int kWgradChunk = 4096;  // voxels reduced by one weight-gradient CTA

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

struct Dims {
  int Z, Y, X;  // per sample
  __host__ __device__ int64_t nvox() const { return (int64_t)Z * Y * X; }
};

__device__ __forceinline__ int64_t neighbour(int64_t v, const Dims& d, int tap, int ntaps, bool flip) {
  if (ntaps == 1) return v;
  int t = flip ? (kTaps - 1 - tap) : tap;
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int64_t nv = d.nvox();
  const int64_t b = v / nv, r = v - b * nv;
  const int x = (int)(r % d.X);
  const int64_t r2 = r / d.X;
  const int y = (int)(r2 % d.Y), z = (int)(r2 / d.Y);
  const int zz = z + dz, yy = y + dy, xx = x + dx;
  if (zz < 0 || zz >= d.Z || yy < 0 || yy >= d.Y || xx < 0 || xx >= d.X) return -1;
  return b * nv + ((int64_t)zz * d.Y + yy) * d.X + xx;
}

// Pack W[tap][ci][co] (FP32, leading dims cin, cout) into mma B fragments
// wp[tap][kc][nt][lane] = {b0, b1}.  transpose: the GEMM reads W^T (input
// gradient): element (k = co, n = ci) of tap t is W[t][ci][co]; the input
// gradient kernel walks the neighbours in the opposite direction instead.
__global__ void k_pack(const float* __restrict__ w, int taps, int cin, int cout, int kc_n, int nt_n, bool transpose,
                       uint2* __restrict__ wp) {
  const int total = taps * kc_n * nt_n * 32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int lane = i % 32;
    int r = i / 32;
    const int nt = r % nt_n;
    r /= nt_n;
    const int kc = r % kc_n, tap = r / kc_n;
    const int g = lane >> 2, t = lane & 3;
    const int n = nt * 8 + g;
    float v[4];
    const int ks[4] = {kc * 16 + 2 * t, kc * 16 + 2 * t + 1, kc * 16 + 2 * t + 8, kc * 16 + 2 * t + 9};
    for (int q = 0; q < 4; ++q) {
      const int k = ks[q];
      float val = 0.f;
      if (!transpose) {
        if (k < cin && n < cout) val = w[((int64_t)tap * cin + k) * cout + n];
      } else {  // K axis = co (0..cout), N axis = ci (0..cin)
        if (k < cout && n < cin) val = w[((int64_t)tap * cin + n) * cout + k];
      }
      v[q] = val;
    }
    wp[i] = make_uint2(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]));
  }
}

// Implicit-GEMM convolution: y[v, 0:cout] = (relu?)(sum_tap x[nb(v, tap), 0:cin] W + bias)
// x has xs channels per voxel (reads channel range [0, cin)); y has ys channels, written at [0, cout).
// flip selects the input-gradient neighbour direction.  grid (ceil(V/64)), block 128.
template <int NT>
__global__ void __launch_bounds__(kConvThreads) k_conv(const float* __restrict__ x, int xs, int cin, int kc_n,
                                                     const uint2* __restrict__ wp, int taps, bool flip,
                                                     const float* __restrict__ bias, float* __restrict__ y, int ys,
                                                     int cout, bool relu, Dims d, int64_t V) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int64_t v0 = (int64_t)blockIdx.x * kVoxPerCta + warp * 16;
  const int64_t r0 = v0 + g, r1 = v0 + g + 8;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  for (int tap = 0; tap < taps; ++tap) {
    const int64_t n0 = (r0 < V) ? neighbour(r0, d, tap, taps, flip) : -1;
    const int64_t n1 = (r1 < V) ? neighbour(r1, d, tap, taps, flip) : -1;
    const float* x0 = n0 >= 0 ? x + n0 * xs : nullptr;
    const float* x1 = n1 >= 0 ? x + n1 * xs : nullptr;
    for (int kc = 0; kc < kc_n; ++kc) {
      const int c0 = kc * 16 + 2 * t;
      auto ld = [&](const float* p, int c) -> float { return (p && c < cin) ? __ldg(p + c) : 0.f; };
      uint32_t a[4];
      a[0] = pack_bf16(ld(x0, c0), ld(x0, c0 + 1));
      a[1] = pack_bf16(ld(x1, c0), ld(x1, c0 + 1));
      a[2] = pack_bf16(ld(x0, c0 + 8), ld(x0, c0 + 9));
      a[3] = pack_bf16(ld(x1, c0 + 8), ld(x1, c0 + 9));
      const uint2* wb = wp + ((int64_t)(tap * kc_n + kc) * NT) * 32 + lane;
#pragma unroll
      for (int n = 0; n < NT; ++n) mma_bf16(acc[n], a, __ldg(wb + n * 32));
    }
  }
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    const int co = n * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t r = h ? r1 : r0;
      if (r >= V) continue;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = co + e;
        if (c >= cout) continue;
        float val = acc[n][2 * h + e] + (bias ? bias[c] : 0.f);
        if (relu) val = fmaxf(val, 0.f);
        y[r * ys + c] = val;
      }
    }
  }
}

// ------------------------------------------------------------------ tcgen05 convolution
// The 3x3x3 implicit GEMM on the fifth-generation tensor cores.  A CTA owns a tile of Tz z planes
// x Ty y rows x all X voxels of one sample.  Per 16-channel chunk, a TMA load brings the tile with
// its one-voxel halo (zero outside the volume: the load starts at coordinate -1) from a bfloat16
// channels-last copy of the input into shared memory, as two 8-channel halves in which staged
// voxel s = (zz * (Ty+2) + yy) * (X+2) + xx sits at byte 16 s.  In that layout the rows of an
// MMA's A operand are 16 bytes apart, so the K-major no-swizzle descriptor with an 8-row stride of
// 128 bytes addresses 128 consecutive staged voxels from any start, and the operand of tap
// (dz, dy, dx) is the output rows' operand moved by dz (Ty+2)(X+2) + dy (X+2) + dx rows: one
// descriptor per tap, no data movement.  The GEMM's M axis runs over consecutive staged positions
// from the first interior voxel, in tiles of 128; positions in the halo columns are computed and
// discarded.  The chunk's weights for all taps come in with one bulk copy.  One thread issues the
// loads and the 27 x (M tiles) MMAs of a chunk (kind::f16, bf16 operands, FP32 accumulators in
// tensor memory, N = output channels rounded to 16); a tcgen05.commit on the chunk's "empty"
// barrier releases its buffer, and two buffers let the next chunk's loads run under the current
// chunk's MMAs.  Every mbarrier wait is bounded (a wait that gives up sets the fault flag and the
// outputs are invalid).  The epilogue reads each M tile with tcgen05.ld (warp w owns rows 32w..),
// adds the bias, applies ReLU and stores the interior voxels in FP32.
namespace tc {
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets, version 1,
// no swizzle
__device__ __forceinline__ uint64_t desc(const void* smem, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (saddr(smem) & 0x3FFFFu) >> 4;
  return a | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// ncol: a power of two in [32, 512]
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncol) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncol)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t tmem, uint32_t ncol) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncol) : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// 5-D tiled TMA load (coordinates innermost first) into shared memory, completion counted on bar
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
      "[%7];" ::"r"(saddr(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
      : "memory");
}
}  // namespace tc

constexpr int kTcThreads = 128;
constexpr uint32_t kTcMaxPolls = 1u << 22;

// tile geometry of the tcgen05 convolution (host-chosen)
struct TcTile {
  int Ty, Tz;          // y rows and z planes per CTA (all X voxels of a row)
  int sx, sy, sz;      // staged extents X+2, Ty+2, Tz+2
  int q_first;         // staged row of the first interior voxel (= the largest tap offset)
  int n_mt;            // 128-row M tiles
  int rows_alloc;      // staged rows per channel half (covers every row an MMA reads), multiple of 8
  int stages;          // 1 or 2 chunk buffers
  uint32_t stage_bytes;
  uint32_t ncol;       // tensor-memory columns allocated (power of two >= n_mt * N, <= 512)
};

__host__ __device__ inline uint32_t tc_act_bytes(const TcTile& t) { return 2u * (uint32_t)t.rows_alloc * 16u; }

// wpk: per (chunk, tap) NP x 16 bf16 in the B-tile layout, chunks outermost
template <int NP>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(const __grid_constant__ CUtensorMap tmap,
                                                        const uint4* __restrict__ wpk, int kc_n, bool flip,
                                                        const float* __restrict__ bias, float* __restrict__ y, int ys,
                                                        int cout, bool relu, Dims d, TcTile tl,
                                                        unsigned int* __restrict__ fault) {
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 128, "N must be a multiple of 16 in [16, 128]");
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_tc);  // [2]: a chunk's loads have landed
  uint64_t* empty = full + 2;                             // [2]: a chunk's MMAs have read its buffer
  uint64_t* done = full + 4;                              // every MMA has finished
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(full + 5);
  unsigned char* buf0 = smem_tc + 1024;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ty0 = blockIdx.x * tl.Ty, tz0 = blockIdx.y * tl.Tz, b = blockIdx.z;
  const uint32_t half_bytes = (uint32_t)tl.rows_alloc * 16u;
  const uint32_t act_bytes = tc_act_bytes(tl);
  const uint32_t w_bytes = (uint32_t)kTaps * NP * 32u;
  const uint32_t box_bytes = 16u * (uint32_t)(tl.sx * tl.sy * tl.sz);
  const int plane = tl.sx * tl.sy;
  if (warp == 0) tc::alloc(tmem_slot, tl.ncol);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) bulk::mbar_init(&full[i], 1);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;
  if (tid == 0) {
    uint32_t fph[2] = {0u, 0u}, eph[2] = {0u, 0u};
    for (int kc = 0; kc < kc_n; ++kc) {
      const int s = (tl.stages == 2) ? (kc & 1) : 0;
      unsigned char* act = buf0 + (size_t)s * tl.stage_bytes;
      unsigned char* wb = act + act_bytes;
      if (kc >= tl.stages) {  // the MMAs of chunk kc - stages have read this buffer
        ok = bulk::mbar_wait(&empty[s], eph[s], kTcMaxPolls, fault) && ok;
        eph[s] ^= 1u;
      }
      bulk::mbar_arrive_expect_tx(&full[s], 2u * box_bytes + w_bytes);
      tc::tma_load_5d(act, &tmap, kc * 16, -1, ty0 - 1, tz0 - 1, b, &full[s]);
      tc::tma_load_5d(act + half_bytes, &tmap, kc * 16 + 8, -1, ty0 - 1, tz0 - 1, b, &full[s]);
      bulk::load_g2s(wb, wpk + (int64_t)kc * kTaps * NP * 2, w_bytes, &full[s]);
      ok = bulk::mbar_wait(&full[s], fph[s], kTcMaxPolls, fault) && ok;
      fph[s] ^= 1u;
      tc::fence_after();
      for (int mt = 0; mt < tl.n_mt; ++mt)
        for (int t = 0; t < kTaps; ++t) {
          const int tt = flip ? (kTaps - 1 - t) : t;
          const int off = (tt / 9 - 1) * plane + ((tt / 3) % 3 - 1) * tl.sx + (tt % 3 - 1);
          const uint32_t row = (uint32_t)(tl.q_first + mt * 128 + off);
          tc::mma(tmem + (uint32_t)(mt * NP), tc::desc(act + (size_t)row * 16u, half_bytes, 128),
                  tc::desc(wb + (size_t)t * NP * 32u, 128, 256), tc::idesc_bf16(NP), (kc > 0 || t > 0) ? 1u : 0u);
        }
      tc::commit(&empty[s]);
    }
    tc::commit(done);
  }
  ok = bulk::mbar_wait(done, 0u, kTcMaxPolls, fault) && ok;
  tc::fence_after();
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int mt = 0; mt < tl.n_mt; ++mt) {
    const int q = tl.q_first + mt * 128 + tid;
    const int zz = q / plane, r = q - zz * plane;
    const int yy = r / tl.sx, xx = r - yy * tl.sx;
    const int z = tz0 + zz - 1, yv = ty0 + yy - 1, x = xx - 1;
    const bool valid = ok && zz >= 1 && zz <= tl.Tz && yy >= 1 && yy <= tl.Ty && xx >= 1 && xx <= d.X && z < d.Z &&
                       yv < d.Y;
    float* yo = y + ((((int64_t)b * d.Z + (valid ? z : 0)) * d.Y + (valid ? yv : 0)) * d.X + (valid ? x : 0)) * ys;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float acc[16];
      tc::ld16(tmem + lane_base + (uint32_t)(mt * NP + c0), acc);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int co = c0 + j;
          if (co < cout) {
            float val = acc[j] + (bias ? bias[co] : 0.f);
            if (relu) val = fmaxf(val, 0.f);
            yo[co] = val;
          }
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, tl.ncol);
}

// bfloat16 channels-last copy of channels [0, cin) of x (xs per voxel), cpad channels (zeros above
// cin): the tcgen05 convolution's TMA source.  One thread per 8 channels of a voxel.
__global__ void k_to_bf16(const float* __restrict__ x, int xs, int cin, int cpad, int64_t V, uint4* __restrict__ out) {
  const int g8 = cpad / 8;
  const int64_t total = V * g8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / g8;
    const int c = (int)(i - v * g8) * 8;
    const float* src = x + v * xs;
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = (c + j < cin) ? __ldg(src + c + j) : 0.f;
    out[i] = make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
  }
}

// pack W[tap][ci][co] (FP32) into the tcgen05 B tiles, blocks ordered (chunk, tap): per block element
// (n, k) at bf16 offset ((n / 8) * 2 + k / 8) * 64 + (n % 8) * 8 + k % 8; forward n = co, k = ci;
// transposed n = ci, k = co
__global__ void k_pack_tc(const float* __restrict__ w, int taps, int cin, int cout, int kc_n, int np, bool transpose,
                          __nv_bfloat16* __restrict__ out) {
  const int64_t total = (int64_t)taps * kc_n * np * 16;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(i % (np * 16));
    const int64_t blk = i / (np * 16);
    const int tap = (int)(blk % taps), kc = (int)(blk / taps);
    const int core = e / 64, in = e % 64;
    const int n = (core / 2) * 8 + in / 8, k = kc * 16 + (core % 2) * 8 + in % 8;
    float val = 0.f;
    if (!transpose) {
      if (k < cin && n < cout) val = w[((int64_t)tap * cin + k) * cout + n];
    } else {
      if (k < cout && n < cin) val = w[((int64_t)tap * cin + n) * cout + k];
    }
    out[i] = __float2bfloat16_rn(val);
  }
}

// Weight gradient partials: part[chunk][tap][kc*16 + row][nt*8 + col] = sum over the chunk's voxels
// of x[nb(v, tap), ci] g[v, co].  grid (nchunk, taps, kc_n), block 128.
template <int NT>
__global__ void __launch_bounds__(kConvThreads) k_wgrad(const float* __restrict__ x, int xs, int cin,
                                                      const float* __restrict__ gy, int gs, int cout, int taps,
                                                      Dims d, int64_t V, float* __restrict__ part, int kc_n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int chunk = blockIdx.x, tap = blockIdx.y, kc = blockIdx.z;
  const int64_t vbeg = (int64_t)chunk * kWgradChunk;
  const int64_t vend = min(V, vbeg + kWgradChunk);
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const int ci_a = kc * 16 + g, ci_b = kc * 16 + g + 8;
  for (int64_t vb = vbeg + warp * 16; vb < vend; vb += 4 * 16) {
    // voxel columns of this k-step: vb + 2t, +1, +8, +9
    const int64_t vc[4] = {vb + 2 * t, vb + 2 * t + 1, vb + 2 * t + 8, vb + 2 * t + 9};
    float xa[4], xb[4];
    int64_t vv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      vv[q] = vc[q] < vend ? vc[q] : -1;
      const int64_t nb = vv[q] >= 0 ? neighbour(vv[q], d, tap, taps, false) : -1;
      xa[q] = (nb >= 0 && ci_a < cin) ? __ldg(x + nb * xs + ci_a) : 0.f;
      xb[q] = (nb >= 0 && ci_b < cin) ? __ldg(x + nb * xs + ci_b) : 0.f;
    }
    uint32_t a[4];
    a[0] = pack_bf16(xa[0], xa[1]);
    a[1] = pack_bf16(xb[0], xb[1]);
    a[2] = pack_bf16(xa[2], xa[3]);
    a[3] = pack_bf16(xb[2], xb[3]);
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int co = n * 8 + g;
      float gv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) gv[q] = (vv[q] >= 0 && co < cout) ? __ldg(gy + vv[q] * gs + co) : 0.f;
      const uint2 b = make_uint2(pack_bf16(gv[0], gv[1]), pack_bf16(gv[2], gv[3]));
      mma_bf16(acc[n], a, b);
    }
  }
  // reduce the 4 warps in shared memory, fixed order
  __shared__ float red[4][16][NT * 8];
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    red[warp][g][n * 8 + 2 * t] = acc[n][0];
    red[warp][g][n * 8 + 2 * t + 1] = acc[n][1];
    red[warp][g + 8][n * 8 + 2 * t] = acc[n][2];
    red[warp][g + 8][n * 8 + 2 * t + 1] = acc[n][3];
  }
  __syncthreads();
  float* out = part + (((int64_t)chunk * taps + tap) * kc_n * 16 + kc * 16) * (NT * 8);
  for (int i = threadIdx.x; i < 16 * NT * 8; i += blockDim.x) {
    const int row = i / (NT * 8), col = i % (NT * 8);
    out[(int64_t)row * (NT * 8) + col] = red[0][row][col] + red[1][row][col] + red[2][row][col] + red[3][row][col];
  }
}

// gw[tap][ci][co] = sum_chunk part[chunk][tap][ci][co] (ci < cin, co < cout)
__global__ void k_wgrad_sum(const float* __restrict__ part, int nchunk, int taps, int cinp, int coutp, int cin,
                            int cout, float* __restrict__ gw) {
  const int total = taps * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int co = i % cout;
    const int r = i / cout;
    const int ci = r % cin, tap = r / cin;
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(((int64_t)c * taps + tap) * cinp + ci) * coutp + co];
    gw[i] = s;
  }
}

// gb[co] = sum_v g[v, co]  (one block per channel, fixed-order tree)
__global__ void k_colsum(const float* __restrict__ g, int gs, int cout, int64_t V, float* __restrict__ gb) {
  const int co = blockIdx.x;
  double s = 0.0;
  for (int64_t v = threadIdx.x; v < V; v += blockDim.x) s += g[v * gs + co];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) gb[co] = (float)red[0];
}

// g *= (out > 0)
__global__ void k_relu_bwd(float* __restrict__ g, const float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(out[i] > 0.f)) g[i] = 0.f;
}

// average pool 2x2x2: y[b, z, y, x, c] = mean of the 8 children; d = output dims
__global__ void k_pool(const float* __restrict__ x, float* __restrict__ y, int C, Dims d, int B) {
  const int64_t total = (int64_t)B * d.nvox() * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t v = i / C;
    const int xx = (int)(v % d.X);
    v /= d.X;
    const int yy = (int)(v % d.Y);
    v /= d.Y;
    const int zz = (int)(v % d.Z);
    const int64_t b = v / d.Z;
    const int X2 = 2 * d.X, Y2 = 2 * d.Y, Z2 = 2 * d.Z;
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int z = 2 * zz + (q >> 2), y2 = 2 * yy + ((q >> 1) & 1), x2 = 2 * xx + (q & 1);
      s += x[(((b * Z2 + z) * Y2 + y2) * X2 + x2) * C + c];
    }
    y[i] = s * 0.125f;
  }
}

// pool backward: gx (fine, C channels) += g (coarse) / 8 ; accumulate selects += vs =
__global__ void k_pool_bwd(const float* __restrict__ g, float* __restrict__ gx, int C, Dims d_fine, int B,
                           bool accumulate) {
  const int64_t total = (int64_t)B * d_fine.nvox() * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t v = i / C;
    const int x = (int)(v % d_fine.X);
    v /= d_fine.X;
    const int y = (int)(v % d_fine.Y);
    v /= d_fine.Y;
    const int z = (int)(v % d_fine.Z);
    const int64_t b = v / d_fine.Z;
    const int Xc = d_fine.X / 2, Yc = d_fine.Y / 2, Zc = d_fine.Z / 2;
    const float val = 0.125f * g[(((b * Zc + z / 2) * Yc + y / 2) * Xc + x / 2) * C + c];
    gx[i] = accumulate ? gx[i] + val : val;
  }
}

// nearest upsample x2 of src (C channels, coarse dims) into channels [0, C) of dst (dst_c channels, fine dims)
__global__ void k_up(const float* __restrict__ src, int C, float* __restrict__ dst, int dst_c, Dims d_fine, int B) {
  const int64_t total = (int64_t)B * d_fine.nvox() * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t v = i / C;
    const int x = (int)(v % d_fine.X);
    v /= d_fine.X;
    const int y = (int)(v % d_fine.Y);
    v /= d_fine.Y;
    const int z = (int)(v % d_fine.Z);
    const int64_t b = v / d_fine.Z;
    const int Xc = d_fine.X / 2, Yc = d_fine.Y / 2, Zc = d_fine.Z / 2;
    const int64_t fine = ((b * d_fine.Z + z) * d_fine.Y + y) * d_fine.X + x;
    dst[fine * dst_c + c] = src[(((b * Zc + z / 2) * Yc + y / 2) * Xc + x / 2) * C + c];
  }
}

// upsample backward: g_src (coarse, C) = sum of the 8 children of channels [0, C) of g (fine, g_c channels)
__global__ void k_up_bwd(const float* __restrict__ g, int g_c, float* __restrict__ gsrc, int C, Dims d_coarse, int B) {
  const int64_t total = (int64_t)B * d_coarse.nvox() * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t v = i / C;
    const int xx = (int)(v % d_coarse.X);
    v /= d_coarse.X;
    const int yy = (int)(v % d_coarse.Y);
    v /= d_coarse.Y;
    const int zz = (int)(v % d_coarse.Z);
    const int64_t b = v / d_coarse.Z;
    const int X2 = 2 * d_coarse.X, Y2 = 2 * d_coarse.Y, Z2 = 2 * d_coarse.Z;
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int z = 2 * zz + (q >> 2), y = 2 * yy + ((q >> 1) & 1), x = 2 * xx + (q & 1);
      s += g[(((b * Z2 + z) * Y2 + y) * X2 + x) * g_c + c];
    }
    gsrc[i] = s;
  }
}

// copy channels: dst[v, doff + c] = src[v, soff + c] for c < C (accumulate: +=)
__global__ void k_copy_ch(const float* __restrict__ src, int sc, int soff, float* __restrict__ dst, int dc, int doff,
                          int C, int64_t V, bool accumulate) {
  const int64_t total = V * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t v = i / C;
    const float val = src[v * sc + soff + c];
    float* o = dst + v * dc + doff + c;
    *o = accumulate ? *o + val : val;
  }
}

// masked MSE: loss partials and gradient g = 2 m (y - t) / (count * C)
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask, int C,
                       int64_t V, double inv_cnt, float* __restrict__ g, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float m = mask[v];
    for (int c = 0; c < C; ++c) {
      const float diff = y[v * C + c] - t[v * C + c];
      s += (double)m * diff * diff;
      g[v * C + c] = (float)(2.0 * m * diff * inv_cnt);
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv_cnt;
}

// AdamW on the flat FP32 parameter vector
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    p[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
  }
}

// Network input per voxel of the box grid (zero outside the target), channels:
// [1, (Re eps - 1)/4, Im eps / 2, Re E_x, Im E_x, Re E_y, Im E_y, Re E_z, Im E_z]
__global__ void k_features(const int32_t* __restrict__ ijk, int64_t n, const uint8_t* __restrict__ comp,
                           const float2* __restrict__ eps, const double2* __restrict__ e, int nrhs, Dims d, int ox,
                           int oy, int oz, float* __restrict__ x) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int xx = ijk[3 * j] + ox, yy = ijk[3 * j + 1] + oy, zz = ijk[3 * j + 2] + oz;
    const int64_t v = (int64_t)b * d.nvox() + ((int64_t)zz * d.Y + yy) * d.X + xx;
    const float2 ep = eps[comp ? comp[3 * j] : 0];  // the x-axis material of the site
    float* o = x + v * 9;
    o[0] = 1.f;
    o[1] = 0.25f * (ep.x - 1.f);
    o[2] = 0.5f * ep.y;
    for (int c = 0; c < 3; ++c) {
      const double2 ev = e[((int64_t)b * 3 + c) * n + j];
      o[3 + 2 * c] = (float)ev.x;
      o[4 + 2 * c] = (float)ev.y;
    }
  }
}

// Training target E_loc = alpha^{-1} P (Re, Im per component), minus E_inc when `e` is given
// (residual mode), and the occupancy mask
__global__ void k_targets(const int32_t* __restrict__ ijk, int64_t n, const uint8_t* __restrict__ comp,
                          const double2* __restrict__ ia, int ncomp, const double2* __restrict__ p,
                          const double2* __restrict__ e, int nrhs, Dims d, int ox, int oy, int oz,
                          float* __restrict__ t, float* __restrict__ mask) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int xx = ijk[3 * j] + ox, yy = ijk[3 * j + 1] + oy, zz = ijk[3 * j + 2] + oz;
    const int64_t v = (int64_t)b * d.nvox() + ((int64_t)zz * d.Y + yy) * d.X + xx;
    for (int c = 0; c < 3; ++c) {
      const int cc = comp ? comp[3 * j + c] : 0;  // composition of axis c
      const double2 a = ia[((int64_t)b * ncomp + cc) * 3 + c];
      const double2 pv = p[((int64_t)b * 3 + c) * n + j];
      double re = a.x * pv.x - a.y * pv.y, im = a.x * pv.y + a.y * pv.x;
      if (e) {
        const double2 ev = e[((int64_t)b * 3 + c) * n + j];
        re -= ev.x;
        im -= ev.y;
      }
      t[v * 6 + 2 * c] = (float)re;
      t[v * 6 + 2 * c + 1] = (float)im;
    }
    mask[v] = 1.f;
  }
}

// Warm start P0 = alpha E_loc = E_loc / alpha^{-1} at the target's sites, E_loc = y (+ E_inc when `e`
// is given: residual mode)
__global__ void k_warm(const int32_t* __restrict__ ijk, int64_t n, const uint8_t* __restrict__ comp,
                       const double2* __restrict__ ia, int ncomp, const float* __restrict__ y,
                       const double2* __restrict__ e, int nrhs, Dims d, int ox, int oy, int oz,
                       double2* __restrict__ p) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int xx = ijk[3 * j] + ox, yy = ijk[3 * j + 1] + oy, zz = ijk[3 * j + 2] + oz;
    const int64_t v = (int64_t)b * d.nvox() + ((int64_t)zz * d.Y + yy) * d.X + xx;
    for (int c = 0; c < 3; ++c) {
      const int cc = comp ? comp[3 * j + c] : 0;  // composition of axis c
      const double2 a = ia[((int64_t)b * ncomp + cc) * 3 + c];
      double er = y[v * 6 + 2 * c], ei = y[v * 6 + 2 * c + 1];
      if (e) {
        const double2 ev = e[((int64_t)b * 3 + c) * n + j];
        er += ev.x;
        ei += ev.y;
      }
      const double den = a.x * a.x + a.y * a.y;
      p[((int64_t)b * 3 + c) * n + j] = make_double2((er * a.x + ei * a.y) / den, (ei * a.x - er * a.y) / den);
    }
  }
}

inline int blocks_for(int64_t n, int th = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + th - 1) / th, 152 * 8)); }

}  // namespace nn
}  // namespace dda

// ============================================================================ network object
struct dda_unet {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int cin = 0, cout = 0, ch[4] = {0, 0, 0, 0};
  struct Layer {
    int taps, cin, cout, kc_n, nt_n, cin_t_kc, cout_t_nt;  // kc/nt for forward; *_t for transposed
    int64_t woff, boff;                                      // offsets into the flat parameter vector
    uint2* wp = nullptr;                                     // forward fragments
    uint2* wt = nullptr;                                     // transposed+flipped fragments (input grad)
    __nv_bfloat16* wtc = nullptr;                            // tcgen05 B tiles, forward (N = cout)
    __nv_bfloat16* wttc = nullptr;                           // tcgen05 B tiles, input gradient (N = cin)
  };
  std::vector<Layer> layers;
  int64_t nparams = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int64_t adam_step = 0;
  // activation workspace (grown on demand)
  float* ws = nullptr;
  size_t ws_bytes = 0;
  float* part = nullptr;
  size_t part_bytes = 0;
  double* lpart = nullptr;
  double* h_loss = nullptr;
  bool use_tc = true;                  // convolutions on tcgen05 (DDA_UNET_TC=0: mma.sync throughout)
  unsigned int* d_fault = nullptr;     // set when a bounded tensor-core wait gave up
  uint4* xb = nullptr;                 // bfloat16 channels-last copy of a tcgen05 convolution's input
  size_t xb_bytes = 0;
};

namespace {

using dda::Err;

dda_status ufail(dda_unet* n, const Err& e) {
  if (n) n->err = e.msg;
  return e.code;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

int np16(int c) { return (c + 15) / 16 * 16; }

Err repack(dda_unet* n) {
  for (auto& L : n->layers) {
    if (n->use_tc) {
      const int64_t t1 = (int64_t)L.taps * L.kc_n * np16(L.cout) * 16;
      dda::nn::k_pack_tc<<<dda::nn::blocks_for(t1), 256, 0, n->stream>>>(n->p + L.woff, L.taps, L.cin, L.cout, L.kc_n,
                                                                          np16(L.cout), false, L.wtc);
      const int64_t t2 = (int64_t)L.taps * L.cin_t_kc * np16(L.cin) * 16;
      dda::nn::k_pack_tc<<<dda::nn::blocks_for(t2), 256, 0, n->stream>>>(n->p + L.woff, L.taps, L.cin, L.cout,
                                                                          L.cin_t_kc, np16(L.cin), true, L.wttc);
      DDA_CU(cudaGetLastError());
      dda::add_launches(2);
    }
    const int tot = L.taps * L.kc_n * L.nt_n * 32;
    dda::nn::k_pack<<<dda::nn::blocks_for(tot), 256, 0, n->stream>>>(n->p + L.woff, L.taps, L.cin, L.cout, L.kc_n,
                                                                       L.nt_n, false, L.wp);
    const int tot2 = L.taps * L.cin_t_kc * L.cout_t_nt * 32;
    dda::nn::k_pack<<<dda::nn::blocks_for(tot2), 256, 0, n->stream>>>(n->p + L.woff, L.taps, L.cin, L.cout,
                                                                        L.cin_t_kc, L.cout_t_nt, true, L.wt);
    DDA_CU(cudaGetLastError());
    dda::add_launches(2);
  }
  return Err::Ok();
}

// Tile of the tcgen05 convolution for a volume d (B samples) and N = np output channels: the (Ty, Tz)
// with the least modelled time per SM, counting for each 16-channel chunk the bytes a CTA loads
// (activation tile with halo, both halves, plus the chunk's weights for 27 taps) and its MMAs
// (27 per 128-row M tile), overlapped when two buffers or two CTAs per SM fit.  false when no tile
// fits (rows longer than 254 voxels): the caller uses the mma.sync kernel.
bool tc_tile(const dda::nn::Dims& d, int B, int np, dda::nn::TcTile* out) {
  constexpr double kSmem = 227.0 * 1024.0, kBytesPerNs = 60.0, kMmaNs = 16.0;
  const int X = d.X;
  if (X + 2 > 256) return false;
  double best = 1e300;
  bool found = false;
  for (int Tz = 1; Tz <= std::min(d.Z, 16); ++Tz)
    for (int Ty = 1; Ty <= std::min(d.Y, 64); ++Ty) {
      dda::nn::TcTile t{};
      t.Ty = Ty;
      t.Tz = Tz;
      t.sx = X + 2;
      t.sy = Ty + 2;
      t.sz = Tz + 2;
      const int plane = t.sx * t.sy;
      t.q_first = plane + t.sx + 1;
      const int q_last = (Tz * t.sy + Ty) * t.sx + X;
      t.n_mt = (q_last - t.q_first + 1 + 127) / 128;
      if (t.n_mt * np > 512) continue;
      t.ncol = 32;
      while ((int)t.ncol < t.n_mt * np) t.ncol *= 2;
      t.rows_alloc = (2 * t.q_first + t.n_mt * 128 + 7) / 8 * 8;
      const double act = 2.0 * t.rows_alloc * 16.0, w = 27.0 * np * 32.0;
      t.stage_bytes = (uint32_t)((act + w + 1023) / 1024) * 1024u;
      if (1024.0 + t.stage_bytes > kSmem) continue;
      t.stages = (1024.0 + 2.0 * t.stage_bytes <= kSmem) ? 2 : 1;
      const int cps = std::max(1, std::min((int)(kSmem / (1024.0 + t.stages * (double)t.stage_bytes)),
                                           (int)(512 / t.ncol)));
      const double load = (2.0 * 16.0 * t.sx * t.sy * t.sz + w) / kBytesPerNs;
      const double mma = t.n_mt * 27.0 * kMmaNs * std::max(1.0, np / 64.0);
      const double per_chunk = (t.stages == 2 || cps >= 2) ? std::max(load, mma) : load + mma;
      const double ctas = (double)B * ((d.Y + Ty - 1) / Ty) * ((d.Z + Tz - 1) / Tz);
      const double waves = std::ceil(ctas / (152.0 * cps));
      const double cost = waves * cps * per_chunk;
      if (cost < best) {
        best = cost;
        *out = t;
        found = true;
      }
    }
  return found;
}

// the driver's tensor-map encoder, looked up once
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 5-D map of the bfloat16 activations [B][Z][Y][X][cpad]: box 8 channels x (X+2) x (Ty+2) x (Tz+2) x 1
Err encode_act_map(CUtensorMap* m, const void* base, int cpad, const dda::nn::Dims& d, int B,
                   const dda::nn::TcTile& t) {
  auto enc = tmap_encoder();
  if (!enc) return Err::make(DDA_ECUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[5] = {(cuuint64_t)cpad, (cuuint64_t)d.X, (cuuint64_t)d.Y, (cuuint64_t)d.Z, (cuuint64_t)B};
  const cuuint64_t strides[4] = {(cuuint64_t)cpad * 2, (cuuint64_t)cpad * 2 * d.X, (cuuint64_t)cpad * 2 * d.X * d.Y,
                                 (cuuint64_t)cpad * 2 * d.X * d.Y * d.Z};
  const cuuint32_t box[5] = {8u, (cuuint32_t)t.sx, (cuuint32_t)t.sy, (cuuint32_t)t.sz, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return Err::make(DDA_ECUDA, "tensor-map encoding failed");
  return Err::Ok();
}

// opt k_conv_tc<NP> in to the full 227 KB of dynamic shared memory (once per instantiation)
template <int NP>
Err tc_smem_optin() {
  static bool done = false;
  if (!done) {
    DDA_CU(cudaFuncSetAttribute(dda::nn::k_conv_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    done = true;
  }
  return Err::Ok();
}

// y = conv(x) for layer L; x has xs channels (uses the first cin), y gets ys channels (writes first cout)
Err conv(dda_unet* n, const dda_unet::Layer& L, const float* x, int xs, float* y, int ys, bool relu, dda::nn::Dims d,
         int B, bool transposed) {
  const int64_t V = (int64_t)B * d.nvox();
  const int blocks = (int)((V + dda::nn::kVoxPerCta - 1) / dda::nn::kVoxPerCta);
  const int kc_n = transposed ? L.cin_t_kc : L.kc_n;
  const int nt_n = transposed ? L.cout_t_nt : L.nt_n;
  const int cin = transposed ? L.cout : L.cin;
  const int cout = transposed ? L.cin : L.cout;
  const uint2* w = transposed ? L.wt : L.wp;
  const float* bias = transposed ? nullptr : n->p + L.boff;
  if (n->use_tc && L.taps == dda::nn::kTaps) {
    const int np = np16(cout);
    dda::nn::TcTile tl;
    if (tc_tile(d, B, np, &tl)) {
      const int cpad = kc_n * 16;
      const size_t need = sizeof(uint16_t) * (size_t)V * cpad;
      if (need > n->xb_bytes) {
        if (n->xb) cudaFree(n->xb);
        n->xb = nullptr;
        n->xb_bytes = 0;
        DDA_CU(cudaMalloc((void**)&n->xb, need));
        n->xb_bytes = need;
      }
      const int64_t items = V * (cpad / 8);
      dda::nn::k_to_bf16<<<dda::nn::blocks_for(items), 256, 0, n->stream>>>(x, xs, cin, cpad, V, n->xb);
      DDA_CU(cudaGetLastError());
      CUtensorMap tmap;
      DDA_TRY(encode_act_map(&tmap, n->xb, cpad, d, B, tl));
      const uint4* wt = reinterpret_cast<const uint4*>(transposed ? L.wttc : L.wtc);
      const dim3 grid((unsigned)((d.Y + tl.Ty - 1) / tl.Ty), (unsigned)((d.Z + tl.Tz - 1) / tl.Tz), (unsigned)B);
      const size_t smem = 1024 + (size_t)tl.stages * tl.stage_bytes;
      switch (np) {
#define CASE(NP)                                                                                                  \
  case NP:                                                                                                        \
    DDA_TRY(tc_smem_optin<NP>());                                                                                 \
    dda::nn::k_conv_tc<NP><<<grid, dda::nn::kTcThreads, smem, n->stream>>>(tmap, wt, kc_n, transposed, bias, y, ys, \
                                                                           cout, relu, d, tl, n->d_fault);        \
    break;
        CASE(16) CASE(32) CASE(48) CASE(64) CASE(80) CASE(96) CASE(112) CASE(128)
#undef CASE
        default: return Err::make(DDA_EUNSUPPORTED, "layer wider than 128 channels");
      }
      DDA_CU(cudaGetLastError());
      dda::add_launches(2);
      return Err::Ok();
    }
  }
  switch (nt_n) {
#define CASE(NT)                                                                                                   \
  case NT:                                                                                                         \
    dda::nn::k_conv<NT><<<blocks, dda::nn::kConvThreads, 0, n->stream>>>(x, xs, cin, kc_n, w, L.taps, transposed, \
                                                                         bias, y, ys, cout, relu, d, V);           \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
    CASE(14) CASE(15) CASE(16)
#undef CASE
    default: return Err::make(DDA_EUNSUPPORTED, "layer wider than 128 channels");
  }
  DDA_CU(cudaGetLastError());
  dda::add_launches(1);
  return Err::Ok();
}

Err grow_ws(dda_unet* n, float** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return Err::Ok();
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  DDA_CU(cudaMalloc((void**)p, bytes));
  *cap = bytes;
  return Err::Ok();
}

// weight and bias gradients of layer L from input x (xs channels) and output gradient gy (gs channels)
Err wgrad(dda_unet* n, const dda_unet::Layer& L, const float* x, int xs, const float* gy, int gs, dda::nn::Dims d,
          int B) {
  const int64_t V = (int64_t)B * d.nvox();
  const int nchunk = (int)((V + dda::nn::kWgradChunk - 1) / dda::nn::kWgradChunk);
  const size_t need = sizeof(float) * (size_t)nchunk * L.taps * L.kc_n * 16 * L.nt_n * 8;
  DDA_TRY(grow_ws(n, &n->part, &n->part_bytes, need));
  dim3 grid(nchunk, L.taps, L.kc_n);
  switch (L.nt_n) {
#define CASE(NT)                                                                                                    \
  case NT:                                                                                                          \
    dda::nn::k_wgrad<NT><<<grid, dda::nn::kConvThreads, 0, n->stream>>>(x, xs, L.cin, gy, gs, L.cout, L.taps, d, V, \
                                                                        n->part, L.kc_n);                           \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return Err::make(DDA_EUNSUPPORTED, "layer wider than 64 channels");
  }
  DDA_CU(cudaGetLastError());
  const int tot = L.taps * L.cin * L.cout;
  dda::nn::k_wgrad_sum<<<dda::nn::blocks_for(tot), 256, 0, n->stream>>>(n->part, nchunk, L.taps, L.kc_n * 16,
                                                                        L.nt_n * 8, L.cin, L.cout, n->g + L.woff);
  dda::nn::k_colsum<<<L.cout, 256, 0, n->stream>>>(gy, gs, L.cout, V, n->g + L.boff);
  DDA_CU(cudaGetLastError());
  dda::add_launches(3);
  return Err::Ok();
}

// Activation buffers of one pass for batch B and base dims d1 (all offsets in floats).
struct Acts {
  float *x, *e1a, *s1, *p1, *e2a, *s2, *p2, *e3a, *s3, *p3, *ba, *bb, *c3, *d3a, *d3b, *c2, *d2a, *d2b, *c1, *d1a,
      *d1b, *y;
  // gradients
  float *g_y, *g_d1b, *g_c1, *g_d2b, *g_c2, *g_d3b, *g_c3, *g_bb, *g_p3, *g_s3, *g_p2, *g_s2, *g_p1, *g_s1, *g_tmp;
};

Err layout(dda_unet* n, int B, dda::nn::Dims d1, bool with_grads, Acts* a) {
  const int64_t V1 = (int64_t)B * d1.nvox(), V2 = V1 / 8, V3 = V2 / 8, V4 = V3 / 8;
  const int c1 = n->ch[0], c2 = n->ch[1], c3 = n->ch[2], c4 = n->ch[3];
  std::vector<std::pair<float**, int64_t>> list = {
      {&a->x, V1 * n->cin}, {&a->e1a, V1 * c1}, {&a->s1, V1 * c1}, {&a->p1, V2 * c1}, {&a->e2a, V2 * c2},
      {&a->s2, V2 * c2}, {&a->p2, V3 * c2}, {&a->e3a, V3 * c3}, {&a->s3, V3 * c3}, {&a->p3, V4 * c3},
      {&a->ba, V4 * c4}, {&a->bb, V4 * c4}, {&a->c3, V3 * (c4 + c3)}, {&a->d3a, V3 * c3}, {&a->d3b, V3 * c3},
      {&a->c2, V2 * (c3 + c2)}, {&a->d2a, V2 * c2}, {&a->d2b, V2 * c2}, {&a->c1, V1 * (c2 + c1)},
      {&a->d1a, V1 * c1}, {&a->d1b, V1 * c1}, {&a->y, V1 * n->cout}};
  if (with_grads) {
    const int64_t cmax = std::max({(int64_t)n->cout, (int64_t)c1 + c2, (int64_t)c4 + c3, (int64_t)c3 + c2});
    std::vector<std::pair<float**, int64_t>> gl = {
        {&a->g_y, V1 * n->cout}, {&a->g_d1b, V1 * c1}, {&a->g_c1, V1 * (c2 + c1)}, {&a->g_d2b, V2 * c2},
        {&a->g_c2, V2 * (c3 + c2)}, {&a->g_d3b, V3 * c3}, {&a->g_c3, V3 * (c4 + c3)}, {&a->g_bb, V4 * c4},
        {&a->g_p3, V4 * c3}, {&a->g_s3, V3 * c3}, {&a->g_p2, V3 * c2}, {&a->g_s2, V2 * c2}, {&a->g_p1, V2 * c1},
        {&a->g_s1, V1 * c1}, {&a->g_tmp, V1 * cmax}};
    list.insert(list.end(), gl.begin(), gl.end());
  }
  int64_t total = 0;
  for (auto& e : list) total += (e.second + 63) / 64 * 64;
  DDA_TRY(grow_ws(n, &n->ws, &n->ws_bytes, sizeof(float) * (size_t)total));
  int64_t off = 0;
  for (auto& e : list) {
    *e.first = n->ws + off;
    off += (e.second + 63) / 64 * 64;
  }
  return Err::Ok();
}

Err forward_pass(dda_unet* n, const Acts& a, int B, dda::nn::Dims d1) {
  const dda::nn::Dims d2{d1.Z / 2, d1.Y / 2, d1.X / 2}, d3{d2.Z / 2, d2.Y / 2, d2.X / 2},
      d4{d3.Z / 2, d3.Y / 2, d3.X / 2};
  const int c1 = n->ch[0], c2 = n->ch[1], c3 = n->ch[2], c4 = n->ch[3];
  auto& L = n->layers;
  cudaStream_t st = n->stream;
  using namespace dda::nn;
  DDA_TRY(conv(n, L[0], a.x, n->cin, a.e1a, c1, true, d1, B, false));
  DDA_TRY(conv(n, L[1], a.e1a, c1, a.s1, c1, true, d1, B, false));
  k_pool<<<blocks_for((int64_t)B * d2.nvox() * c1), 256, 0, st>>>(a.s1, a.p1, c1, d2, B);
  DDA_TRY(conv(n, L[2], a.p1, c1, a.e2a, c2, true, d2, B, false));
  DDA_TRY(conv(n, L[3], a.e2a, c2, a.s2, c2, true, d2, B, false));
  k_pool<<<blocks_for((int64_t)B * d3.nvox() * c2), 256, 0, st>>>(a.s2, a.p2, c2, d3, B);
  DDA_TRY(conv(n, L[4], a.p2, c2, a.e3a, c3, true, d3, B, false));
  DDA_TRY(conv(n, L[5], a.e3a, c3, a.s3, c3, true, d3, B, false));
  k_pool<<<blocks_for((int64_t)B * d4.nvox() * c3), 256, 0, st>>>(a.s3, a.p3, c3, d4, B);
  DDA_TRY(conv(n, L[6], a.p3, c3, a.ba, c4, true, d4, B, false));
  DDA_TRY(conv(n, L[7], a.ba, c4, a.bb, c4, true, d4, B, false));
  k_up<<<blocks_for((int64_t)B * d3.nvox() * c4), 256, 0, st>>>(a.bb, c4, a.c3, c4 + c3, d3, B);
  k_copy_ch<<<blocks_for((int64_t)B * d3.nvox() * c3), 256, 0, st>>>(a.s3, c3, 0, a.c3, c4 + c3, c4, c3,
                                                                      (int64_t)B * d3.nvox(), false);
  DDA_TRY(conv(n, L[8], a.c3, c4 + c3, a.d3a, c3, true, d3, B, false));
  DDA_TRY(conv(n, L[9], a.d3a, c3, a.d3b, c3, true, d3, B, false));
  k_up<<<blocks_for((int64_t)B * d2.nvox() * c3), 256, 0, st>>>(a.d3b, c3, a.c2, c3 + c2, d2, B);
  k_copy_ch<<<blocks_for((int64_t)B * d2.nvox() * c2), 256, 0, st>>>(a.s2, c2, 0, a.c2, c3 + c2, c3, c2,
                                                                      (int64_t)B * d2.nvox(), false);
  DDA_TRY(conv(n, L[10], a.c2, c3 + c2, a.d2a, c2, true, d2, B, false));
  DDA_TRY(conv(n, L[11], a.d2a, c2, a.d2b, c2, true, d2, B, false));
  k_up<<<blocks_for((int64_t)B * d1.nvox() * c2), 256, 0, st>>>(a.d2b, c2, a.c1, c2 + c1, d1, B);
  k_copy_ch<<<blocks_for((int64_t)B * d1.nvox() * c1), 256, 0, st>>>(a.s1, c1, 0, a.c1, c2 + c1, c2, c1,
                                                                      (int64_t)B * d1.nvox(), false);
  DDA_TRY(conv(n, L[12], a.c1, c2 + c1, a.d1a, c1, true, d1, B, false));
  DDA_TRY(conv(n, L[13], a.d1a, c1, a.d1b, c1, true, d1, B, false));
  DDA_TRY(conv(n, L[14], a.d1b, c1, a.y, n->cout, false, d1, B, false));
  DDA_CU(cudaGetLastError());
  dda::add_launches(9);
  return Err::Ok();
}

// conv backward for layer li: output activation `out` (for the ReLU mask), its gradient g_out (gs channels,
// modified in place by the mask), input activation x (xs channels); writes the input gradient to gx (gxs ch.)
Err conv_back(dda_unet* n, int li, const float* x, int xs, const float* out, float* g_out, int gs, float* gx, int gxs,
              dda::nn::Dims d, int B, bool relu) {
  const auto& L = n->layers[li];
  const int64_t V = (int64_t)B * d.nvox();
  if (relu) {
    dda::nn::k_relu_bwd<<<dda::nn::blocks_for(V * gs), 256, 0, n->stream>>>(g_out, out, V * gs);
    dda::add_launches(1);
  }
  DDA_TRY(wgrad(n, L, x, xs, g_out, gs, d, B));
  if (gx) DDA_TRY(conv(n, L, g_out, gs, gx, gxs, false, d, B, true));
  return Err::Ok();
}

Err backward_pass(dda_unet* n, const Acts& a, int B, dda::nn::Dims d1) {
  using namespace dda::nn;
  const Dims d2{d1.Z / 2, d1.Y / 2, d1.X / 2}, d3{d2.Z / 2, d2.Y / 2, d2.X / 2}, d4{d3.Z / 2, d3.Y / 2, d3.X / 2};
  const int c1 = n->ch[0], c2 = n->ch[1], c3 = n->ch[2], c4 = n->ch[3];
  cudaStream_t st = n->stream;
  const int64_t V1 = (int64_t)B * d1.nvox(), V2 = V1 / 8, V3 = V2 / 8, V4 = V3 / 8;
  // head (linear): input d1b
  DDA_TRY(conv_back(n, 14, a.d1b, c1, a.y, a.g_y, n->cout, a.g_d1b, c1, d1, B, false));
  // dec1
  DDA_TRY(conv_back(n, 13, a.d1a, c1, a.d1b, a.g_d1b, c1, a.g_tmp, c1, d1, B, true));
  DDA_TRY(conv_back(n, 12, a.c1, c2 + c1, a.d1a, a.g_tmp, c1, a.g_c1, c2 + c1, d1, B, true));
  k_up_bwd<<<blocks_for(V2 * c2), 256, 0, st>>>(a.g_c1, c2 + c1, a.g_d2b, c2, d2, B);
  k_copy_ch<<<blocks_for(V1 * c1), 256, 0, st>>>(a.g_c1, c2 + c1, c2, a.g_s1, c1, 0, c1, V1, false);
  // dec2
  DDA_TRY(conv_back(n, 11, a.d2a, c2, a.d2b, a.g_d2b, c2, a.g_tmp, c2, d2, B, true));
  DDA_TRY(conv_back(n, 10, a.c2, c3 + c2, a.d2a, a.g_tmp, c2, a.g_c2, c3 + c2, d2, B, true));
  k_up_bwd<<<blocks_for(V3 * c3), 256, 0, st>>>(a.g_c2, c3 + c2, a.g_d3b, c3, d3, B);
  k_copy_ch<<<blocks_for(V2 * c2), 256, 0, st>>>(a.g_c2, c3 + c2, c3, a.g_s2, c2, 0, c2, V2, false);
  // dec3
  DDA_TRY(conv_back(n, 9, a.d3a, c3, a.d3b, a.g_d3b, c3, a.g_tmp, c3, d3, B, true));
  DDA_TRY(conv_back(n, 8, a.c3, c4 + c3, a.d3a, a.g_tmp, c3, a.g_c3, c4 + c3, d3, B, true));
  k_up_bwd<<<blocks_for(V4 * c4), 256, 0, st>>>(a.g_c3, c4 + c3, a.g_bb, c4, d4, B);
  k_copy_ch<<<blocks_for(V3 * c3), 256, 0, st>>>(a.g_c3, c4 + c3, c4, a.g_s3, c3, 0, c3, V3, false);
  // bottleneck
  DDA_TRY(conv_back(n, 7, a.ba, c4, a.bb, a.g_bb, c4, a.g_tmp, c4, d4, B, true));
  DDA_TRY(conv_back(n, 6, a.p3, c3, a.ba, a.g_tmp, c4, a.g_p3, c3, d4, B, true));
  k_pool_bwd<<<blocks_for(V3 * c3), 256, 0, st>>>(a.g_p3, a.g_s3, c3, d3, B, true);
  // enc3
  DDA_TRY(conv_back(n, 5, a.e3a, c3, a.s3, a.g_s3, c3, a.g_tmp, c3, d3, B, true));
  DDA_TRY(conv_back(n, 4, a.p2, c2, a.e3a, a.g_tmp, c3, a.g_p2, c2, d3, B, true));
  k_pool_bwd<<<blocks_for(V2 * c2), 256, 0, st>>>(a.g_p2, a.g_s2, c2, d2, B, true);
  // enc2
  DDA_TRY(conv_back(n, 3, a.e2a, c2, a.s2, a.g_s2, c2, a.g_tmp, c2, d2, B, true));
  DDA_TRY(conv_back(n, 2, a.p1, c1, a.e2a, a.g_tmp, c2, a.g_p1, c1, d2, B, true));
  k_pool_bwd<<<blocks_for(V1 * c1), 256, 0, st>>>(a.g_p1, a.g_s1, c1, d1, B, true);
  // enc1
  DDA_TRY(conv_back(n, 1, a.e1a, c1, a.s1, a.g_s1, c1, a.g_tmp, c1, d1, B, true));
  DDA_TRY(conv_back(n, 0, a.x, n->cin, a.e1a, a.g_tmp, c1, nullptr, 0, d1, B, true));
  DDA_CU(cudaGetLastError());
  dda::add_launches(9);
  return Err::Ok();
}

Err check_dims(const int32_t dims[3]) {
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 8 || dims[k] % 8 != 0) return Err::make(DDA_EINVAL, "network grid dims must be multiples of 8");
  return Err::Ok();
}

}  // namespace

dda_status dda_unet_create(dda_unet** out, int device, void* stream, int cin, int cout, const int32_t ch[4],
                           uint64_t seed) {
  if (!out || !ch || cin < 1 || cout < 1 || cin > 64 || cout > 64) return DDA_EINVAL;
  for (int k = 0; k < 4; ++k)
    if (ch[k] < 1 || ch[k] > 64) return DDA_EINVAL;
  if (ch[3] + ch[2] > 128 || ch[2] + ch[1] > 128 || ch[1] + ch[0] > 128) return DDA_EINVAL;
  *out = nullptr;
  dda_unet* n = new (std::nothrow) dda_unet();
  if (!n) return DDA_ENOMEM;
  n->device = device;
  n->stream = (cudaStream_t)stream;
  n->cin = cin;
  n->cout = cout;
  for (int k = 0; k < 4; ++k) n->ch[k] = ch[k];
  if (cudaSetDevice(device) != cudaSuccess) {
    delete n;
    return DDA_ECUDA;
  }
  const int c1 = ch[0], c2 = ch[1], c3 = ch[2], c4 = ch[3];
  const int convs[15][3] = {{27, cin, c1}, {27, c1, c1},     {27, c1, c2},      {27, c2, c2},      {27, c2, c3},
                            {27, c3, c3},  {27, c3, c4},     {27, c4, c4},      {27, c4 + c3, c3}, {27, c3, c3},
                            {27, c3 + c2, c2}, {27, c2, c2}, {27, c2 + c1, c1}, {27, c1, c1},      {1, c1, cout}};
  int64_t off = 0;
  for (auto& cv : convs) {
    dda_unet::Layer L;
    L.taps = cv[0];
    L.cin = cv[1];
    L.cout = cv[2];
    L.kc_n = ceil_div(L.cin, 16);
    L.nt_n = ceil_div(L.cout, 8);
    L.cin_t_kc = ceil_div(L.cout, 16);
    L.cout_t_nt = ceil_div(L.cin, 8);
    L.woff = off;
    off += (int64_t)L.taps * L.cin * L.cout;
    L.boff = off;
    off += L.cout;
    n->layers.push_back(L);
  }
  n->nparams = off;
  // He-uniform initialization (fan-in = taps * cin), zero biases, deterministic from seed
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  for (auto& L : n->layers) {
    const double bound = std::sqrt(6.0 / (double)(L.taps * L.cin));
    std::uniform_real_distribution<double> U(-bound, bound);
    for (int64_t i = 0; i < (int64_t)L.taps * L.cin * L.cout; ++i) h[L.woff + i] = (float)U(rng);
  }
  bool ok = cudaMalloc((void**)&n->p, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc((void**)&n->g, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc((void**)&n->m, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc((void**)&n->v, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc((void**)&n->lpart, sizeof(double) * 2048) == cudaSuccess &&
            cudaMallocHost((void**)&n->h_loss, sizeof(double) * 2048) == cudaSuccess;
  {
    const char* f = std::getenv("DDA_UNET_TC");
    n->use_tc = !(f && std::atoi(f) == 0);
  }
  ok = ok && cudaMalloc((void**)&n->d_fault, sizeof(unsigned int)) == cudaSuccess &&
       cudaMemset(n->d_fault, 0, sizeof(unsigned int)) == cudaSuccess;
  for (auto& L : n->layers) {
    ok = ok && cudaMalloc((void**)&L.wp, sizeof(uint2) * L.taps * L.kc_n * L.nt_n * 32) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&L.wt, sizeof(uint2) * L.taps * L.cin_t_kc * L.cout_t_nt * 32) == cudaSuccess;
    if (n->use_tc) {
      ok = ok && cudaMalloc((void**)&L.wtc, sizeof(__nv_bfloat16) * L.taps * L.kc_n * np16(L.cout) * 16) == cudaSuccess;
      ok = ok && cudaMalloc((void**)&L.wttc, sizeof(__nv_bfloat16) * L.taps * L.cin_t_kc * np16(L.cin) * 16) ==
                     cudaSuccess;
    }
  }
  if (!ok) {
    dda_unet_destroy(n);
    return DDA_ENOMEM;
  }
  const bool init_ok = cudaMemcpy(n->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) == cudaSuccess &&
                       cudaMemset(n->m, 0, sizeof(float) * off) == cudaSuccess &&
                       cudaMemset(n->v, 0, sizeof(float) * off) == cudaSuccess &&
                       cudaMemset(n->g, 0, sizeof(float) * off) == cudaSuccess;
  Err e = init_ok ? repack(n) : Err::make(DDA_ECUDA, "parameter upload failed");
  if (!e.ok() || cudaStreamSynchronize(n->stream) != cudaSuccess) {
    dda_unet_destroy(n);
    return DDA_ECUDA;
  }
  *out = n;
  return DDA_OK;
}

void dda_unet_destroy(dda_unet* n) {
  if (!n) return;
  cudaSetDevice(n->device);
  if (n->stream) cudaStreamSynchronize(n->stream);
  for (auto& L : n->layers) {
    if (L.wp) cudaFree(L.wp);
    if (L.wt) cudaFree(L.wt);
    if (L.wtc) cudaFree(L.wtc);
    if (L.wttc) cudaFree(L.wttc);
  }
  for (float* q : {n->p, n->g, n->m, n->v, n->ws, n->part})
    if (q) cudaFree(q);
  if (n->lpart) cudaFree(n->lpart);
  if (n->h_loss) cudaFreeHost(n->h_loss);
  if (n->d_fault) cudaFree(n->d_fault);
  if (n->xb) cudaFree(n->xb);
  delete n;
}

// DDA_ECUDA when a tensor-core convolution's bounded wait gave up since the last check (the flag is
// then cleared); call after the stream has been synchronized
dda_status dda_unet_check_fault(dda_unet* n) {
  if (!n || !n->d_fault) return DDA_OK;
  unsigned int h = 0;
  if (cudaMemcpy(&h, n->d_fault, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return DDA_ECUDA;
  if (!h) return DDA_OK;
  cudaMemset(n->d_fault, 0, sizeof(unsigned int));
  n->err = "a tensor-core convolution's bounded wait gave up: results invalid";
  return DDA_ECUDA;
}

const char* dda_unet_last_error(const dda_unet* n) { return n ? n->err.c_str() : "null network"; }

int64_t dda_unet_nparams(const dda_unet* n) { return n ? n->nparams : 0; }

dda_status dda_unet_get_params(dda_unet* n, float* host, int which) {
  if (!n || !host || which < 0 || which > 1) return DDA_EINVAL;
  if (cudaSetDevice(n->device) != cudaSuccess || cudaStreamSynchronize(n->stream) != cudaSuccess)
    return ufail(n, Err::make(DDA_ECUDA, "device sync failed"));
  if (cudaMemcpy(host, which ? n->g : n->p, sizeof(float) * n->nparams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ufail(n, Err::make(DDA_ECUDA, "copy failed"));
  return DDA_OK;
}

dda_status dda_unet_set_params(dda_unet* n, const float* host) {
  if (!n || !host) return DDA_EINVAL;
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  if (cudaMemcpy(n->p, host, sizeof(float) * n->nparams, cudaMemcpyHostToDevice) != cudaSuccess)
    return ufail(n, Err::make(DDA_ECUDA, "copy failed"));
  Err e = repack(n);
  if (!e.ok()) return ufail(n, e);
  return DDA_OK;
}

dda_status dda_unet_forward(dda_unet* n, const float* x_dev, float* y_dev, int batch, const int32_t dims[3]) {
  if (!n || !x_dev || !y_dev || batch < 1 || !dims) return DDA_EINVAL;
  Err e = check_dims(dims);
  if (!e.ok()) return ufail(n, e);
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  const dda::nn::Dims d1{dims[2], dims[1], dims[0]};
  Acts a;
  e = layout(n, batch, d1, false, &a);
  if (e.ok()) {
    const int64_t V1 = (int64_t)batch * d1.nvox();
    if (cudaMemcpyAsync(a.x, x_dev, sizeof(float) * V1 * n->cin, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "input copy failed");
  }
  if (e.ok()) e = forward_pass(n, a, batch, d1);
  if (e.ok()) {
    const int64_t V1 = (int64_t)batch * d1.nvox();
    if (cudaMemcpyAsync(y_dev, a.y, sizeof(float) * V1 * n->cout, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "output copy failed");
  }
  return e.ok() ? DDA_OK : ufail(n, e);
}

dda_status dda_unet_loss_grad(dda_unet* n, const float* x_dev, const float* t_dev, const float* mask_dev, int batch,
                              const int32_t dims[3], double* loss_out) {
  if (!n || !x_dev || !t_dev || !mask_dev || batch < 1 || !dims) return DDA_EINVAL;
  Err e = check_dims(dims);
  if (!e.ok()) return ufail(n, e);
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  const dda::nn::Dims d1{dims[2], dims[1], dims[0]};
  const int64_t V1 = (int64_t)batch * d1.nvox();
  Acts a;
  e = layout(n, batch, d1, true, &a);
  if (e.ok() && cudaMemcpyAsync(a.x, x_dev, sizeof(float) * V1 * n->cin, cudaMemcpyDeviceToDevice, n->stream) !=
                    cudaSuccess)
    e = Err::make(DDA_ECUDA, "input copy failed");
  if (e.ok()) e = forward_pass(n, a, batch, d1);
  // masked-voxel count on the host side of the device: sum the mask once
  double cnt = 0.0;
  if (e.ok()) {
    std::vector<float> hm(V1);
    if (cudaMemcpyAsync(hm.data(), mask_dev, sizeof(float) * V1, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "mask copy failed");
    for (float m : hm) cnt += m;
    if (e.ok() && cnt <= 0) e = Err::make(DDA_EINVAL, "mask selects no voxel");
  }
  const int lb = 512;
  if (e.ok()) {
    dda::nn::k_loss<<<lb, 256, 0, n->stream>>>(a.y, t_dev, mask_dev, n->cout, V1, 1.0 / (cnt * n->cout), a.g_y,
                                                n->lpart);
    dda::add_launches(1);
    e = backward_pass(n, a, batch, d1);
  }
  if (e.ok()) {
    if (cudaMemcpyAsync(n->h_loss, n->lpart, sizeof(double) * lb, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "loss copy failed");
  }
  if (!e.ok()) return ufail(n, e);
  // a tcgen05 convolution whose bounded wait gave up leaves invalid gradients: report it here
  if (n->use_tc && dda_unet_check_fault(n) != DDA_OK) return DDA_ECUDA;
  double L = 0.0;
  for (int i = 0; i < lb; ++i) L += n->h_loss[i];
  if (loss_out) *loss_out = L;
  return DDA_OK;
}

dda_status dda_unet_adamw(dda_unet* n, double lr, double beta1, double beta2, double eps, double wd) {
  if (!n || !(lr > 0)) return DDA_EINVAL;
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  n->adam_step += 1;
  const float c1 = (float)(1.0 - std::pow(beta1, (double)n->adam_step));
  const float c2 = (float)(1.0 - std::pow(beta2, (double)n->adam_step));
  dda::nn::k_adamw<<<dda::nn::blocks_for(n->nparams), 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, n->nparams,
                                                                            (float)lr, (float)beta1, (float)beta2,
                                                                            (float)eps, (float)wd, c1, c2);
  dda::add_launches(1);
  Err e = repack(n);
  if (e.ok() && cudaGetLastError() != cudaSuccess) e = Err::make(DDA_ECUDA, "AdamW launch failed");
  return e.ok() ? DDA_OK : ufail(n, e);
}

namespace dda {
Err unet_features(const int32_t* ijk, int64_t n, const uint8_t* comp, const float2* eps, const double2* e, int nrhs,
                  const int32_t dims[3], const int32_t off[3], float* x, cudaStream_t st) {
  const nn::Dims d{dims[2], dims[1], dims[0]};
  DDA_CU(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)nrhs * d.nvox() * 9, st));
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  nn::k_features<<<dim3(nb, nrhs), 256, 0, st>>>(ijk, n, comp, eps, e, nrhs, d, off[0], off[1], off[2], x);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
Err unet_targets(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const double2* p,
                 const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], float* t, float* mask,
                 cudaStream_t st) {
  const nn::Dims d{dims[2], dims[1], dims[0]};
  DDA_CU(cudaMemsetAsync(t, 0, sizeof(float) * (size_t)nrhs * d.nvox() * 6, st));
  DDA_CU(cudaMemsetAsync(mask, 0, sizeof(float) * (size_t)nrhs * d.nvox(), st));
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  nn::k_targets<<<dim3(nb, nrhs), 256, 0, st>>>(ijk, n, comp, ia, ncomp, p, e, nrhs, d, off[0], off[1], off[2], t,
                                                 mask);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
Err unet_warm(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float* y,
              const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], double2* p, cudaStream_t st) {
  const nn::Dims d{dims[2], dims[1], dims[0]};
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  nn::k_warm<<<dim3(nb, nrhs), 256, 0, st>>>(ijk, n, comp, ia, ncomp, y, e, nrhs, d, off[0], off[1], off[2], p);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
}  // namespace dda

dda_status dda_unet_forward_train(dda_unet* n, const float* x_dev, float* y_dev, int batch, const int32_t dims[3]) {
  if (!n || !x_dev || !y_dev || batch < 1 || !dims) return DDA_EINVAL;
  Err e = check_dims(dims);
  if (!e.ok()) return ufail(n, e);
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  const dda::nn::Dims d1{dims[2], dims[1], dims[0]};
  const int64_t V1 = (int64_t)batch * d1.nvox();
  Acts a;
  e = layout(n, batch, d1, true, &a);
  if (e.ok() && cudaMemcpyAsync(a.x, x_dev, sizeof(float) * V1 * n->cin, cudaMemcpyDeviceToDevice, n->stream) !=
                    cudaSuccess)
    e = Err::make(DDA_ECUDA, "input copy failed");
  if (e.ok()) e = forward_pass(n, a, batch, d1);
  if (e.ok() && cudaMemcpyAsync(y_dev, a.y, sizeof(float) * V1 * n->cout, cudaMemcpyDeviceToDevice, n->stream) !=
                    cudaSuccess)
    e = Err::make(DDA_ECUDA, "output copy failed");
  return e.ok() ? DDA_OK : ufail(n, e);
}

dda_status dda_unet_mse(dda_unet* n, const float* y_dev, const float* t_dev, const float* mask_dev, int batch,
                        const int32_t dims[3], double weight, float* gy_dev, double* loss_out) {
  if (!n || !y_dev || !t_dev || !mask_dev || !gy_dev || batch < 1 || !dims) return DDA_EINVAL;
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  const int64_t V1 = (int64_t)batch * dims[0] * dims[1] * dims[2];
  std::vector<float> hm(V1);
  if (cudaMemcpyAsync(hm.data(), mask_dev, sizeof(float) * V1, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return ufail(n, Err::make(DDA_ECUDA, "mask copy failed"));
  double cnt = 0.0;
  for (float m : hm) cnt += m;
  if (cnt <= 0) return ufail(n, Err::make(DDA_EINVAL, "mask selects no voxel"));
  const int lb = 512;
  dda::nn::k_loss<<<lb, 256, 0, n->stream>>>(y_dev, t_dev, mask_dev, n->cout, V1, weight / (cnt * n->cout), gy_dev,
                                              n->lpart);
  dda::add_launches(1);
  if (cudaMemcpyAsync(n->h_loss, n->lpart, sizeof(double) * lb, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
      cudaStreamSynchronize(n->stream) != cudaSuccess)
    return ufail(n, Err::make(DDA_ECUDA, "loss copy failed"));
  double L = 0.0;
  for (int i = 0; i < lb; ++i) L += n->h_loss[i];
  if (loss_out) *loss_out = L;
  return DDA_OK;
}

dda_status dda_unet_backward(dda_unet* n, const float* gy_dev, int batch, const int32_t dims[3]) {
  if (!n || !gy_dev || batch < 1 || !dims) return DDA_EINVAL;
  Err e = check_dims(dims);
  if (!e.ok()) return ufail(n, e);
  if (cudaSetDevice(n->device) != cudaSuccess) return ufail(n, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
  const dda::nn::Dims d1{dims[2], dims[1], dims[0]};
  const int64_t V1 = (int64_t)batch * d1.nvox();
  Acts a;
  e = layout(n, batch, d1, true, &a);  // same sizes as the preceding dda_unet_forward_train: same buffers
  if (e.ok() && cudaMemcpyAsync(a.g_y, gy_dev, sizeof(float) * V1 * n->cout, cudaMemcpyDeviceToDevice, n->stream) !=
                    cudaSuccess)
    e = Err::make(DDA_ECUDA, "gradient copy failed");
  if (e.ok()) e = backward_pass(n, a, batch, d1);
  return e.ok() ? DDA_OK : ufail(n, e);
}

// --------------------------------------------------------------------- residual loss glue
namespace dda {
namespace nn {
// P0 (complex64) = alpha (E_inc + y) at the target's sites
__global__ void k_guess64(const int32_t* __restrict__ ijk, int64_t n, const uint8_t* __restrict__ comp,
                          const double2* __restrict__ ia, int ncomp, const float* __restrict__ y,
                          const double2* __restrict__ e, int nrhs, Dims d, int ox, int oy, int oz,
                          float2* __restrict__ p) {
  const int b = blockIdx.y;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int xx = ijk[3 * j] + ox, yy = ijk[3 * j + 1] + oy, zz = ijk[3 * j + 2] + oz;
    const int64_t v = (int64_t)b * d.nvox() + ((int64_t)zz * d.Y + yy) * d.X + xx;
    for (int c = 0; c < 3; ++c) {
      const int cc = comp ? comp[3 * j + c] : 0;  // composition of axis c
      const double2 a = ia[((int64_t)b * ncomp + cc) * 3 + c];
      const double2 ev = e[((int64_t)b * 3 + c) * n + j];
      const double er = y[v * 6 + 2 * c] + ev.x, ei = y[v * 6 + 2 * c + 1] + ev.y;
      const double den = a.x * a.x + a.y * a.y;
      p[((int64_t)b * 3 + c) * n + j] = make_float2((float)((er * a.x + ei * a.y) / den),
                                                    (float)((ei * a.x - er * a.y) / den));
    }
  }
}

// r = E - A P0 (complex64) and per-RHS |r|^2, |E|^2 partials
__global__ void k_resid64(const double2* __restrict__ e, float2* __restrict__ r, int64_t n3, double* __restrict__ part,
                          int nblk) {
  const int b = blockIdx.y;
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 ev = e[(int64_t)b * n3 + i];
    const float2 ap = r[(int64_t)b * n3 + i];
    const float rx = (float)ev.x - ap.x, ry = (float)ev.y - ap.y;
    r[(int64_t)b * n3 + i] = make_float2(rx, ry);
    s0 += (double)rx * rx + (double)ry * ry;
    s1 += ev.x * ev.x + ev.y * ev.y;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((int64_t)b * nblk + blockIdx.x) * 2] = red[0][0];
    part[((int64_t)b * nblk + blockIdx.x) * 2 + 1] = red[1][0];
  }
}

// gy += w_b * d|r|^2/dy with g = A^H r:  d/dy_re = -2 Re(conj(g) alpha), d/dy_im = 2 Im(conj(g) alpha)
__global__ void k_resgrad(const int32_t* __restrict__ ijk, int64_t n, const uint8_t* __restrict__ comp,
                          const double2* __restrict__ ia, int ncomp, const float2* __restrict__ g,
                          const double* __restrict__ wb, int nrhs, Dims d, int ox, int oy, int oz,
                          float* __restrict__ gy) {
  const int b = blockIdx.y;
  const double w = wb[b];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int xx = ijk[3 * j] + ox, yy = ijk[3 * j + 1] + oy, zz = ijk[3 * j + 2] + oz;
    const int64_t v = (int64_t)b * d.nvox() + ((int64_t)zz * d.Y + yy) * d.X + xx;
    for (int c = 0; c < 3; ++c) {
      const int cc = comp ? comp[3 * j + c] : 0;  // composition of axis c
      const double2 ai = ia[((int64_t)b * ncomp + cc) * 3 + c];
      const double den = ai.x * ai.x + ai.y * ai.y;
      const double ar = ai.x / den, aim = -ai.y / den;  // alpha = 1 / alpha^{-1}
      const float2 gv = g[((int64_t)b * 3 + c) * n + j];
      // conj(g) alpha
      const double pr = gv.x * ar + gv.y * aim, pim = gv.x * aim - gv.y * ar;
      gy[v * 6 + 2 * c] += (float)(-2.0 * w * pr);
      gy[v * 6 + 2 * c + 1] += (float)(2.0 * w * pim);
    }
  }
}
}  // namespace nn

Err unet_guess64(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float* y,
                 const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], float2* p, cudaStream_t st) {
  const nn::Dims d{dims[2], dims[1], dims[0]};
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  nn::k_guess64<<<dim3(nb, nrhs), 256, 0, st>>>(ijk, n, comp, ia, ncomp, y, e, nrhs, d, off[0], off[1], off[2], p);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
Err unet_resid64(const double2* e, float2* r, int nrhs, int64_t n3, double* part, int nblk, cudaStream_t st) {
  nn::k_resid64<<<dim3(nblk, nrhs), 256, 0, st>>>(e, r, n3, part, nblk);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
Err unet_resgrad(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float2* g,
                 const double* wb, int nrhs, const int32_t dims[3], const int32_t off[3], float* gy, cudaStream_t st) {
  const nn::Dims d{dims[2], dims[1], dims[0]};
  const int nb = (int)std::min<int64_t>((n + 255) / 256, 1024);
  nn::k_resgrad<<<dim3(nb, nrhs), 256, 0, st>>>(ijk, n, comp, ia, ncomp, g, wb, nrhs, d, off[0], off[1], off[2], gy);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
}  // namespace dda
