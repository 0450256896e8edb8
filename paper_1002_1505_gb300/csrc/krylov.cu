// Batched Krylov solvers for A P = E (guide, "Choice of Iterative Algorithm"):
//  - BiCGstab (van der Vorst 1992; the guide's PBCGST option), unpreconditioned,
//    shadow residual = initial residual;
//  - CCG: conjugate gradients on the normal equations A^H A P = A^H E
//    (Petravic & Kuo-Petravic 1979; the guide's PETRKP option);
//  - BiCGstab(2) (Sleijpen & Fokkema 1993), the method family of the guide's
//    PBCGS2 option: two BiCG steps, then a degree-2 minimal-residual step;
//  - COCG (van der Vorst & Melissen 1990), CG with the unconjugated bilinear
//    form for the complex-symmetric A, one product per iteration (the
//    symmetric-Lanczos family of the guide's QMRCCG option).
// Every right-hand side is an independent system solved in lock step: each
// kernel covers all RHS, with per-RHS scalars kept on the device (KState), so
// an iteration needs no host round trip and can be captured in a CUDA graph.
// Vector updates are fused with the reductions that follow them; reductions
// accumulate in FP64 (warp shuffles, then a per-block tree, then one
// deterministic per-RHS pass) whatever the vector precision.
#include <algorithm>

#include "dda_internal.h"

namespace dda {

namespace {

constexpr int kThreads = 256;

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using t = float; };
template <> struct RealOf<double2> { using t = double; };

__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }
template <typename C> __device__ __forceinline__ C from_d(double2 a);
template <> __device__ __forceinline__ float2 from_d<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from_d<double2>(double2 a) { return a; }

// conj(a) * b accumulated in double
__device__ __forceinline__ double2 cdot_acc(double2 acc, double2 a, double2 b) {
  acc.x += a.x * b.x + a.y * b.y;
  acc.y += a.x * b.y - a.y * b.x;
  return acc;
}
__device__ __forceinline__ double nrm_acc(double acc, double2 a) { return acc + a.x * a.x + a.y * a.y; }

// Per-thread accumulator of products.  complex128 vectors: FP64.  complex64
// vectors: a double-float pair (Dekker/Knuth): each product is split exactly
// into p + pe with one FMA, added with the two-sum, so a thread's partial keeps
// about 48 bits using FP32 instructions only (the FP64 pipe of this GPU is too
// slow to keep up with memory); partials are combined in FP64 from the warp up.
template <typename C> struct Acc;
template <> struct Acc<double2> {
  double v = 0.0;
  __device__ __forceinline__ void fma(double a, double b) { v = __fma_rn(a, b, v); }
  __device__ __forceinline__ double get() const { return v; }
};
template <> struct Acc<float2> {
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
template <typename C>
__device__ __forceinline__ void acc_cdot(Acc<C>& re, Acc<C>& im, C a, C b) {
  re.fma(a.x, b.x);
  re.fma(a.y, b.y);
  im.fma(a.x, b.y);
  im.fma(-a.y, b.x);
}
template <typename C>
__device__ __forceinline__ void acc_nrm(Acc<C>& s, C a) {
  s.fma(a.x, a.x);
  s.fma(a.y, a.y);
}

template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* out) {
  __shared__ double red[NS][kThreads / 32];
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

// Sum the per-block partials of one RHS (called by all threads of a block; result in tot, valid in thread 0).
template <int NS>
__device__ __forceinline__ void sum_partials(const double* part, int nblk, double (&tot)[NS]) {
  double v[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) v[s] = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s] += part[i * kRedSlots + s];
  __shared__ double res[NS];
  block_reduce_store<NS>(v, res);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NS; ++s) tot[s] = res[s];
}


// Reduce `acc` over the block into this block's partial slot; the last block of
// RHS b to arrive (device-scope counter) sums all partials of b in a fixed order
// and returns true with the totals in tot (valid in every thread of that block).
// The counter is reset by that last block, so it is zero between kernels.
template <int NS>
__device__ __forceinline__ bool last_block_totals(double (&acc)[NS], const RedBuf& rb, int b, double (&tot)[NS]) {
  double* mine = rb.part + ((int64_t)b * rb.nblk + blockIdx.x) * kRedSlots;
  block_reduce_store<NS>(acc, mine);
  __shared__ unsigned int s_last;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(rb.count + b, 1u) == (unsigned)gridDim.x - 1u) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const double* base = rb.part + (int64_t)b * rb.nblk * kRedSlots;
  double v[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) v[q] = 0.0;
  for (int i = threadIdx.x; i < rb.nblk; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < NS; ++q) v[q] += __ldcg(base + (int64_t)i * kRedSlots + q);
  __shared__ double res[NS];
  block_reduce_store<NS>(v, res);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NS; ++q) tot[q] = res[q];
  if (threadIdx.x == 0) rb.count[b] = 0;
  return true;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// grid-stride bounds for RHS b, block blk
#define VEC_LOOP(n3) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n3); i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ BiCGstab kernels
template <typename C>
__global__ void k_bicg_init(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3, bool have_ax, double tol) {
  const int b = blockIdx.y;
  const int64_t o = (int64_t)b * n3;
  double acc[3] = {0.0, 0.0, 0.0};  // |b|^2, |r|^2
  VEC_LOOP(n3) {
    const double2 bv = to_d(kv.b[o + i]);
    double2 rv = bv;
    if (have_ax) {
      const double2 ax = to_d(kv.r[o + i]);
      rv = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
    const C rc = from_d<C>(rv);
    kv.r[o + i] = rc;
    kv.rhat[o + i] = rc;
    kv.p[o + i] = czero<C>();
    kv.v[o + i] = czero<C>();
    if (!have_ax) kv.x[o + i] = czero<C>();
    acc[0] = nrm_acc(acc[0], bv);
    acc[1] = nrm_acc(acc[1], to_d(rc));
  }
  double t[3];
  if (last_block_totals<3>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    k.bb = t[0];
    k.rr = t[1];
    k.rho = make_double2(t[1], 0.0);
    k.alpha = make_double2(1.0, 0.0);
    k.omega = make_double2(1.0, 0.0);
    k.beta = make_double2(0.0, 0.0);
    k.tol2 = tol * tol * t[0];
    k.it = 0;
    k.mv = 0;
    k.done = (t[0] == 0.0 || t[1] <= k.tol2) ? 1 : 0;
  }
}

// p = r + beta (p - omega v)
template <typename C>
__global__ void k_bicg_p(KrylovVecs<C> kv, const KState* ks, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  using R = typename RealOf<C>::t;
  const C be = mk((R)k.beta.x, (R)k.beta.y), om = mk((R)k.omega.x, (R)k.omega.y);
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    const C pv = kv.p[o + i], vv = kv.v[o + i], rv = kv.r[o + i];
    kv.p[o + i] = cadd(rv, cmul(be, csub(pv, cmul(om, vv))));
  }
}

// partial <rhat, v>
template <typename C>
__global__ void k_bicg_dot_rv(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[2] = {0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im;
    VEC_LOOP(n3) acc_cdot(re, im, kv.rhat[o + i], kv.v[o + i]);
    acc[0] = re.get();
    acc[1] = im.get();
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // v = A p
    const double2 rv = make_double2(t[0], t[1]);
    if (rv.x == 0.0 && rv.y == 0.0) { k.done = 2; return; }
    k.alpha = cdiv(k.rho, rv);
  }
}

// s = r - alpha v ; partial |s|^2
template <typename C>
__global__ void k_bicg_s(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[1] = {0.0};
  if (!k.done) {
    using R = typename RealOf<C>::t;
    const C al = mk((R)k.alpha.x, (R)k.alpha.y);
    const int64_t o = (int64_t)b * n3;
    Acc<C> ss;
    VEC_LOOP(n3) {
      const C s = csub(kv.r[o + i], cmul(al, kv.v[o + i]));
      kv.s[o + i] = s;
      acc_nrm(ss, s);
    }
    acc[0] = ss.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    if (t[0] <= k.tol2) { k.done = 3; k.rr = t[0]; }  // converged on the half step
  }
}

// partial <t, s>, |t|^2
template <typename C>
__global__ void k_bicg_dot_ts(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[3] = {0.0, 0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im, tt;
    VEC_LOOP(n3) {
      const C tv = kv.t[o + i];
      acc_cdot(re, im, tv, kv.s[o + i]);
      acc_nrm(tt, tv);
    }
    acc[0] = re.get();
    acc[1] = im.get();
    acc[2] = tt.get();
  }
  double t[3];
  if (last_block_totals<3>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // t = A s
    k.omega = (t[2] > 0.0) ? make_double2(t[0] / t[2], t[1] / t[2]) : make_double2(0.0, 0.0);
  }
}

// x += alpha p + omega s ; r = s - omega t ; partial <rhat, r>, |r|^2
// (RHS that converged on the half step: x += alpha p, r = s)
template <typename C>
__global__ void k_bicg_xr(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[3] = {0.0, 0.0, 0.0};
  if (k.done == 0 || k.done == 3) {
    using R = typename RealOf<C>::t;
    const C al = mk((R)k.alpha.x, (R)k.alpha.y), om = mk((R)k.omega.x, (R)k.omega.y);
    const bool half = (k.done == 3);
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im, rr;
    VEC_LOOP(n3) {
      const C sv = kv.s[o + i];
      C xv = cadd(kv.x[o + i], cmul(al, kv.p[o + i]));
      C rv = sv;
      if (!half) {
        xv = cadd(xv, cmul(om, sv));
        rv = csub(sv, cmul(om, kv.t[o + i]));
      }
      kv.x[o + i] = xv;
      kv.r[o + i] = rv;
      acc_cdot(re, im, kv.rhat[o + i], rv);
      acc_nrm(rr, rv);
    }
    acc[0] = re.get();
    acc[1] = im.get();
    acc[2] = rr.get();
  }
  double t[3];
  if (last_block_totals<3>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done == 3) { k.done = 1; k.it += 1; return; }
    if (k.done) return;
    k.it += 1;
    k.rr = t[2];
    const double2 rho_new = make_double2(t[0], t[1]);
    if (t[2] <= k.tol2) { k.done = 1; return; }
    if ((k.omega.x == 0.0 && k.omega.y == 0.0) || (rho_new.x == 0.0 && rho_new.y == 0.0)) { k.done = 2; return; }
    k.beta = cmuld(cdiv(rho_new, k.rho), cdiv(k.alpha, k.omega));
    k.rho = rho_new;
  }
}

// ------------------------------------------------------------------ CCG kernels
template <typename C>
__global__ void k_ccg_init(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3, bool have_ax, double tol) {
  const int b = blockIdx.y;
  const int64_t o = (int64_t)b * n3;
  double acc[2] = {0.0, 0.0};
  VEC_LOOP(n3) {
    const double2 bv = to_d(kv.b[o + i]);
    double2 rv = bv;
    if (have_ax) {
      const double2 ax = to_d(kv.r[o + i]);
      rv = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
    const C rc = from_d<C>(rv);
    kv.r[o + i] = rc;
    if (!have_ax) kv.x[o + i] = czero<C>();
    acc[0] = nrm_acc(acc[0], bv);
    acc[1] = nrm_acc(acc[1], to_d(rc));
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    k.bb = t[0];
    k.rr = t[1];
    k.tol2 = tol * tol * t[0];
    k.it = 0;
    k.mv = 0;
    k.done = (t[0] == 0.0 || t[1] <= k.tol2) ? 1 : 0;
  }
}

// p = z (z held in s); partial |z|^2
template <typename C>
__global__ void k_ccg_start(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  const int b = blockIdx.y;
  double acc[1] = {0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> zz;
    VEC_LOOP(n3) {
      const C z = kv.s[o + i];
      kv.p[o + i] = z;
      acc_nrm(zz, z);
    }
    acc[0] = zz.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // z = A^H r
    k.zz = t[0];
    if (t[0] == 0.0) k.done = 2;
  }
}

// partial |w|^2 (w = A p held in v)
template <typename C>
__global__ void k_norm_v(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[1] = {0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> ww;
    VEC_LOOP(n3) acc_nrm(ww, kv.v[o + i]);
    acc[0] = ww.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // w = A p
    if (t[0] == 0.0) { k.done = 2; return; }
    k.alpha = make_double2(k.zz / t[0], 0.0);
  }
}

// x += alpha p ; r -= alpha w ; partial |r|^2
template <typename C>
__global__ void k_ccg_xr(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[1] = {0.0};
  if (!k.done) {
    using R = typename RealOf<C>::t;
    const R al = (R)k.alpha.x;
    const int64_t o = (int64_t)b * n3;
    Acc<C> rr;
    VEC_LOOP(n3) {
      const C pv = kv.p[o + i], wv = kv.v[o + i];
      C xv = kv.x[o + i], rv = kv.r[o + i];
      xv.x += al * pv.x; xv.y += al * pv.y;
      rv.x -= al * wv.x; rv.y -= al * wv.y;
      kv.x[o + i] = xv;
      kv.r[o + i] = rv;
      acc_nrm(rr, rv);
    }
    acc[0] = rr.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.it += 1;
    k.rr = t[0];
    if (t[0] <= k.tol2) k.done = 1;
  }
}

// partial |z|^2 for the new z (in s)
template <typename C>
__global__ void k_norm_s(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[1] = {0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> zz;
    VEC_LOOP(n3) acc_nrm(zz, kv.s[o + i]);
    acc[0] = zz.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // z = A^H r
    k.beta = make_double2(t[0] / k.zz, 0.0);
    k.zz = t[0];
  }
}

// p = z + beta p
template <typename C>
__global__ void k_ccg_p(KrylovVecs<C> kv, const KState* ks, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  using R = typename RealOf<C>::t;
  const R be = (R)k.beta.x;
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    const C z = kv.s[o + i];
    C pv = kv.p[o + i];
    pv.x = z.x + be * pv.x;
    pv.y = z.y + be * pv.y;
    kv.p[o + i] = pv;
  }
}

// ------------------------------------------------------------------ COCG kernels
// Conjugate orthogonal conjugate gradients (van der Vorst & Melissen 1990): CG with the
// unconjugated bilinear form x^T y, valid because A is complex symmetric; one product per
// iteration.  Vectors: x, r, p, q = A p (held in v).  KState: rho = r^T r, alpha, beta.
// re + i im += a^T b (no conjugation)
template <typename C>
__device__ __forceinline__ void acc_bdot(Acc<C>& re, Acc<C>& im, C a, C b) {
  re.fma(a.x, b.x);
  re.fma(-a.y, b.y);
  im.fma(a.x, b.y);
  im.fma(a.y, b.x);
}

template <typename C>
__global__ void k_cocg_init(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3, bool have_ax, double tol) {
  const int b = blockIdx.y;
  const int64_t o = (int64_t)b * n3;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // |b|^2, |r|^2, r^T r
  VEC_LOOP(n3) {
    const double2 bv = to_d(kv.b[o + i]);
    double2 rv = bv;
    if (have_ax) {
      const double2 ax = to_d(kv.r[o + i]);
      rv = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
    const C rc = from_d<C>(rv);
    kv.r[o + i] = rc;
    kv.p[o + i] = rc;
    if (!have_ax) kv.x[o + i] = czero<C>();
    const double2 rd = to_d(rc);
    acc[0] = nrm_acc(acc[0], bv);
    acc[1] = nrm_acc(acc[1], rd);
    acc[2] += rd.x * rd.x - rd.y * rd.y;
    acc[3] += 2.0 * rd.x * rd.y;
  }
  double t[4];
  if (last_block_totals<4>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    k.bb = t[0];
    k.rr = t[1];
    k.rho = make_double2(t[2], t[3]);
    k.alpha = make_double2(0.0, 0.0);
    k.beta = make_double2(0.0, 0.0);
    k.tol2 = tol * tol * t[0];
    k.it = 0;
    k.mv = 0;
    k.done = (t[0] == 0.0 || t[1] <= k.tol2) ? 1 : 0;
  }
}

// partial p^T q (q = A p in v) -> alpha = rho / p^T q
template <typename C>
__global__ void k_cocg_mu(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[2] = {0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im;
    VEC_LOOP(n3) acc_bdot(re, im, kv.p[o + i], kv.v[o + i]);
    acc[0] = re.get();
    acc[1] = im.get();
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // q = A p
    if (t[0] == 0.0 && t[1] == 0.0) { k.done = 2; return; }
    k.alpha = cdiv(k.rho, make_double2(t[0], t[1]));
  }
}

// x += alpha p ; r -= alpha q ; partial |r|^2, r^T r -> convergence, beta
template <typename C>
__global__ void k_cocg_xr(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[3] = {0.0, 0.0, 0.0};
  if (!k.done) {
    const C al = from_d<C>(k.alpha);
    const int64_t o = (int64_t)b * n3;
    Acc<C> rr, re, im;
    VEC_LOOP(n3) {
      const C pv = kv.p[o + i], qv = kv.v[o + i];
      C xv = kv.x[o + i], rv = kv.r[o + i];
      xv = cadd(xv, cmul(al, pv));
      rv = csub(rv, cmul(al, qv));
      kv.x[o + i] = xv;
      kv.r[o + i] = rv;
      acc_nrm(rr, rv);
      acc_bdot(re, im, rv, rv);
    }
    acc[0] = rr.get();
    acc[1] = re.get();
    acc[2] = im.get();
  }
  double t[3];
  if (last_block_totals<3>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& kw = ks[b];
    if (kw.done) return;
    kw.it += 1;
    kw.rr = t[0];
    if (t[0] <= kw.tol2) { kw.done = 1; return; }
    const double2 rho_new = make_double2(t[1], t[2]);
    if (rho_new.x == 0.0 && rho_new.y == 0.0) { kw.done = 2; return; }
    kw.beta = cdiv(rho_new, kw.rho);
    kw.rho = rho_new;
  }
}

// p = r + beta p
template <typename C>
__global__ void k_cocg_p(KrylovVecs<C> kv, const KState* ks, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  const C be = from_d<C>(k.beta);
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) kv.p[o + i] = cadd(kv.r[o + i], cmul(be, kv.p[o + i]));
}

// ------------------------------------------------------------------ QMR, complex symmetric
// Freund's QMR on the symmetric Lanczos process of A (A^T = A): v_1 = r0/|r0|,
// w = A v_n - alpha_n v_n - beta_n v_{n-1} with alpha_n = v_n^T A v_n / v_n^T v_n and
// beta_n = |w_{n-1}| v_n^T v_n / v_{n-1}^T v_{n-1}, v_{n+1} = w / |w|; the tridiagonal columns are
// reduced by complex Givens rotations and x advances along d_n = (v_n - r_{n-1,n} d_{n-1} -
// r_{n-2,n} d_{n-2}) / r_{n,n} by tau_n.

__device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }

// r0 = b - A x0 (A x0 in r when have_ax) into p, v_{n-1} = r = 0, d buffers = 0; |b|^2, |r0|^2
template <typename C>
__global__ void k_qmr_init(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3, bool have_ax, double tol) {
  const int b = blockIdx.y;
  const int64_t o = (int64_t)b * n3;
  double acc[2] = {0.0, 0.0};
  VEC_LOOP(n3) {
    const double2 bv = to_d(kv.b[o + i]);
    double2 rv = bv;
    if (have_ax) {
      const double2 ax = to_d(kv.r[o + i]);
      rv = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
    const C rc = from_d<C>(rv);
    kv.p[o + i] = rc;
    kv.r[o + i] = czero<C>();
    kv.s[o + i] = czero<C>();
    kv.t[o + i] = czero<C>();
    kv.rhat[o + i] = czero<C>();
    if (!have_ax) kv.x[o + i] = czero<C>();
    acc[0] = nrm_acc(acc[0], bv);
    acc[1] = nrm_acc(acc[1], to_d(rc));
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    const double rho = sqrt(t[1]);
    k.bb = t[0];
    k.rr = t[1];
    k.tol2 = tol * tol * t[0];
    k.q_rho = rho;                    // scale of v_1 (beta_1 = 0 makes its use moot)
    k.q_tb = make_double2(rho, 0.0);  // tau_bar_1
    k.q_dp = make_double2(1.0, 0.0);
    k.q_c1 = k.q_c2 = 1.0;
    k.q_s1 = k.q_s2 = make_double2(0.0, 0.0);
    k.it = 0;
    k.mv = 0;
    k.done = (t[0] == 0.0 || t[1] <= k.tol2) ? 1 : 0;
  }
}

// v_1 = r0 / |r0|
template <typename C>
__global__ void k_qmr_scale(KrylovVecs<C> kv, const KState* ks, int64_t n3) {
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  const C f = from_d<C>(make_double2(1.0 / k.q_rho, 0.0));
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) kv.p[o + i] = cmul(f, kv.p[o + i]);
}

// delta = v^T v, v^T q (q = A v in v) -> alpha, beta; v^T v becomes the next step's delta_prev
template <typename C>
__global__ void k_qmr_dots(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> dr, di, gr, gi;
    VEC_LOOP(n3) {
      const C vv = kv.p[o + i], qv = kv.v[o + i];
      acc_bdot(dr, di, vv, vv);
      acc_bdot(gr, gi, vv, qv);
    }
    acc[0] = dr.get();
    acc[1] = di.get();
    acc[2] = gr.get();
    acc[3] = gi.get();
  }
  double t[4];
  if (last_block_totals<4>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // q = A v_n
    const double2 delta = make_double2(t[0], t[1]);
    if (delta.x == 0.0 && delta.y == 0.0) { k.done = 2; return; }  // Lanczos breakdown (no look-ahead)
    k.alpha = cdiv(make_double2(t[2], t[3]), delta);
    k.beta = k.it > 0 ? cdiv(make_double2(k.q_rho * delta.x, k.q_rho * delta.y), k.q_dp) : make_double2(0.0, 0.0);
    k.q_dp = delta;
  }
}

// w = q - alpha v - beta v_{n-1} (into v); |w| -> rotations, tau_n, the column entries
template <typename C>
__global__ void k_qmr_w(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[1] = {0.0};
  if (!k.done) {
    const C al = from_d<C>(k.alpha), be = from_d<C>(k.beta);
    const int64_t o = (int64_t)b * n3;
    Acc<C> ww;
    VEC_LOOP(n3) {
      const C w = csub(csub(kv.v[o + i], cmul(al, kv.p[o + i])), cmul(be, kv.r[o + i]));
      kv.v[o + i] = w;
      acc_nrm(ww, w);
    }
    acc[0] = ww.get();
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& kw = ks[b];
    if (kw.done) return;
    const double rho_next = sqrt(t[0]);
    const double2 alpha = kw.alpha, beta = kw.beta;
    // column n of the tridiagonal (beta, alpha, rho_next) through G_{n-2}, G_{n-1}
    const double2 r2 = cmuld(kw.q_s2, beta);
    const double2 f = make_double2(kw.q_c2 * beta.x, kw.q_c2 * beta.y);
    const double2 s1c = make_double2(kw.q_s1.x, -kw.q_s1.y);
    const double2 sa = cmuld(kw.q_s1, alpha), sf = cmuld(s1c, f);
    const double2 r1 = make_double2(kw.q_c1 * f.x + sa.x, kw.q_c1 * f.y + sa.y);
    const double2 g = make_double2(-sf.x + kw.q_c1 * alpha.x, -sf.y + kw.q_c1 * alpha.y);
    // G_n takes (g, rho_next) to (r_nn, 0): c real, s complex
    double c, rn_abs;
    double2 sn, rn;
    if (rho_next == 0.0) {
      c = 1.0; sn = make_double2(0.0, 0.0); rn = g; rn_abs = cabsd(g);
    } else if (g.x == 0.0 && g.y == 0.0) {
      c = 0.0; sn = make_double2(1.0, 0.0); rn = make_double2(rho_next, 0.0); rn_abs = rho_next;
    } else {
      const double ga = cabsd(g), h = hypot(ga, rho_next);
      const double2 ph = make_double2(g.x / ga, g.y / ga);
      c = ga / h;
      sn = make_double2(ph.x * rho_next / h, ph.y * rho_next / h);  // ph conj(rho_next) / h, rho_next real
      rn = make_double2(ph.x * h, ph.y * h);
      rn_abs = h;
    }
    if (rn_abs == 0.0) { kw.done = 2; return; }
    const double2 tb = kw.q_tb;
    kw.q_tau = make_double2(c * tb.x, c * tb.y);
    const double2 snc = make_double2(-sn.x, sn.y);  // -conj(s)
    kw.q_tb = cmuld(snc, tb);
    kw.q_r1 = r1;
    kw.q_r2 = r2;
    kw.q_rn = rn;
    kw.q_c2 = kw.q_c1;
    kw.q_s2 = kw.q_s1;
    kw.q_c1 = c;
    kw.q_s1 = sn;
    kw.q_rho = rho_next;
    kw.it += 1;
  }
}

// d_n = (v_n - r_{n-1,n} d_{n-1} - r_{n-2,n} d_{n-2}) / r_nn into the oldest d slot, x += tau_n d_n,
// v_{n-1} = v_n, v_{n+1} = w / |w|; the last block tests sqrt(n + 1) |tau_bar| <= tol |b|
template <typename C>
__global__ void k_qmr_dx(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[1] = {0.0};
  if (!k.done) {
    C* dbuf[3] = {kv.s, kv.t, kv.rhat};
    const int n = k.it;
    C* dn = dbuf[n % 3];
    const C* d1 = dbuf[(n + 2) % 3];
    const C* d2 = dbuf[(n + 1) % 3];
    const double2 irn = cdiv(make_double2(1.0, 0.0), k.q_rn);
    const C r1 = from_d<C>(k.q_r1), r2 = from_d<C>(k.q_r2), inv = from_d<C>(irn), tau = from_d<C>(k.q_tau);
    const C sc = from_d<C>(make_double2(k.q_rho > 0.0 ? 1.0 / k.q_rho : 0.0, 0.0));
    const int64_t o = (int64_t)b * n3;
    VEC_LOOP(n3) {
      const C vn = kv.p[o + i];
      const C d = cmul(inv, csub(csub(vn, cmul(r1, d1[o + i])), cmul(r2, d2[o + i])));
      dn[o + i] = d;
      kv.x[o + i] = cadd(kv.x[o + i], cmul(tau, d));
      kv.r[o + i] = vn;
      kv.p[o + i] = cmul(sc, kv.v[o + i]);
    }
  }
  double t[1];
  if (last_block_totals<1>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& kw = ks[b];
    if (kw.done) return;
    const double tb2 = kw.q_tb.x * kw.q_tb.x + kw.q_tb.y * kw.q_tb.y;
    kw.rr = (kw.it + 1) * tb2;  // bound on |r|^2
    if (kw.rr <= kw.tol2) kw.done = 1;
    else if (kw.q_rho == 0.0) kw.done = 2;  // invariant subspace reached without meeting the bound
  }
}

// ------------------------------------------------------------------ Jacobi scaling of site vectors
// v[b][c][j] *= s[b][comp(j, c)][c] (or /= with inv), the diagonal S of the scaled system S A S.
template <typename C>
__global__ void k_scale_sites(C* v, const C* s, const uint8_t* comp, int ncomp, int64_t n, bool inv) {
  const int b = blockIdx.y;
  const int64_t n3 = 3 * n;
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    const int c = (int)(i / n);
    const int64_t j = i - (int64_t)c * n;
    const int cc = comp ? comp[3 * j + c] : 0;
    C f = s[((int64_t)b * ncomp + cc) * 3 + c];
    if (inv) {
      const auto d = f.x * f.x + f.y * f.y;
      f.x = f.x / d;
      f.y = -f.y / d;
    }
    v[o + i] = cmul(v[o + i], f);
  }
}

// ------------------------------------------------------------------ linear combination of two solutions
// dst = c0 src0 + c1 src1 (complex128, length n3): the solution for an incident polarization that is
// a combination of two solved ones (same matrix A)
__global__ void k_combine2(double2* __restrict__ dst, const double2* __restrict__ s0, const double2* __restrict__ s1,
                           double2 c0, double2 c1, int64_t n3) {
  VEC_LOOP(n3) {
    const double2 a = s0[i], b = s1[i];
    dst[i] = make_double2(c0.x * a.x - c0.y * a.y + c1.x * b.x - c1.y * b.y,
                          c0.x * a.y + c0.y * a.x + c1.x * b.y + c1.y * b.x);
  }
}

// ------------------------------------------------------------------ BiCGstab(2) kernels
// r0 = b - A x (or b), shadow = r0, u0 = 0; rho0 = <shadow, r0> (the first BiCG step's rho with beta = 0)
template <typename C>
__global__ void k_b2_init(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3, bool have_ax, double tol) {
  const int b = blockIdx.y;
  const int64_t o = (int64_t)b * n3;
  double acc[2] = {0.0, 0.0};  // |b|^2, |r|^2
  VEC_LOOP(n3) {
    const double2 bv = to_d(kv.b[o + i]);
    double2 rv = bv;
    if (have_ax) {
      const double2 ax = to_d(kv.r[o + i]);
      rv = make_double2(bv.x - ax.x, bv.y - ax.y);
    }
    const C rc = from_d<C>(rv);
    kv.r[o + i] = rc;
    kv.rhat[o + i] = rc;
    kv.p[o + i] = czero<C>();
    if (!have_ax) kv.x[o + i] = czero<C>();
    acc[0] = nrm_acc(acc[0], bv);
    acc[1] = nrm_acc(acc[1], to_d(rc));
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    k.bb = t[0];
    k.rr = t[1];
    k.rho = make_double2(t[1], 0.0);
    k.alpha = make_double2(0.0, 0.0);
    k.omega = make_double2(1.0, 0.0);
    k.beta = make_double2(0.0, 0.0);
    k.tol2 = tol * tol * t[0];
    k.it = 0;
    k.mv = 0;
    k.done = (t[0] == 0.0 || t[1] <= k.tol2) ? 1 : 0;
  }
}

// BiCG step j: u_i = r_i - beta u_i for i <= j (u0 = p, u1 = v; r0 = r, r1 = s)
template <typename C>
__global__ void k_b2_u(KrylovVecs<C> kv, const KState* ks, int j, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  using R = typename RealOf<C>::t;
  const C be = mk((R)k.beta.x, (R)k.beta.y);
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    kv.p[o + i] = csub(kv.r[o + i], cmul(be, kv.p[o + i]));
    if (j == 1) kv.v[o + i] = csub(kv.s[o + i], cmul(be, kv.v[o + i]));
  }
}

// alpha = rho0 / <shadow, u_{j+1}> (u1 = v for j = 0, u2 for j = 1)
template <typename C>
__global__ void k_b2_alpha(KrylovVecs<C> kv, KState* ks, RedBuf rb, int j, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[2] = {0.0, 0.0};
  if (!ks[b].done) {
    const C* u = (j == 0) ? kv.v : kv.u2;
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im;
    VEC_LOOP(n3) acc_cdot(re, im, kv.rhat[o + i], u[o + i]);
    acc[0] = re.get();
    acc[1] = im.get();
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // u_{j+1} = A u_j
    const double2 g = make_double2(t[0], t[1]);
    if (g.x == 0.0 && g.y == 0.0) { k.done = 2; return; }
    k.alpha = cdiv(k.rho, g);
  }
}

// r_i -= alpha u_{i+1} for i <= j; x += alpha u0
template <typename C>
__global__ void k_b2_r(KrylovVecs<C> kv, const KState* ks, int j, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  if (k.done) return;
  using R = typename RealOf<C>::t;
  const C al = mk((R)k.alpha.x, (R)k.alpha.y);
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    kv.r[o + i] = csub(kv.r[o + i], cmul(al, kv.v[o + i]));
    if (j == 1) kv.s[o + i] = csub(kv.s[o + i], cmul(al, kv.u2[o + i]));
    kv.x[o + i] = cadd(kv.x[o + i], cmul(al, kv.p[o + i]));
  }
}

// rho1 = <shadow, r1>; beta = alpha rho1 / rho0; rho0 = rho1
template <typename C>
__global__ void k_b2_beta(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[2] = {0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> re, im;
    VEC_LOOP(n3) acc_cdot(re, im, kv.rhat[o + i], kv.s[o + i]);
    acc[0] = re.get();
    acc[1] = im.get();
  }
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // r1 = A r0
    const double2 rho1 = make_double2(t[0], t[1]);
    if (k.rho.x == 0.0 && k.rho.y == 0.0) { k.done = 2; return; }
    k.beta = cmuld(k.alpha, cdiv(rho1, k.rho));
    k.rho = rho1;
  }
}

// Gram system of the minimal-residual step: |r1|^2, <r1, r2>, |r2|^2, <r1, r0>, <r2, r0>
// (r0 = r, r1 = s, r2 = t); gamma solves [<r1,r1> <r1,r2>; <r2,r1> <r2,r2>] gamma = [<r1,r0>; <r2,r0>]
template <typename C>
__global__ void k_b2_gram(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (!ks[b].done) {
    const int64_t o = (int64_t)b * n3;
    Acc<C> a11, b12r, b12i, a22, c1r, c1i, c2r, c2i;
    VEC_LOOP(n3) {
      const C r0 = kv.r[o + i], r1 = kv.s[o + i], r2 = kv.t[o + i];
      acc_nrm(a11, r1);
      acc_cdot(b12r, b12i, r1, r2);
      acc_nrm(a22, r2);
      acc_cdot(c1r, c1i, r1, r0);
      acc_cdot(c2r, c2i, r2, r0);
    }
    acc[0] = a11.get(); acc[1] = b12r.get(); acc[2] = b12i.get(); acc[3] = a22.get();
    acc[4] = c1r.get(); acc[5] = c1i.get(); acc[6] = c2r.get(); acc[7] = c2i.get();
  }
  double t[8];
  if (last_block_totals<8>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.mv += 1;  // r2 = A r1
    const double a = t[0], d = t[3];
    const double2 bb = make_double2(t[1], t[2]);  // <r1, r2>
    const double2 c1 = make_double2(t[4], t[5]), c2 = make_double2(t[6], t[7]);
    const double det = a * d - (bb.x * bb.x + bb.y * bb.y);
    if (!(det > 0.0)) { k.done = 2; return; }
    // gamma1 = (d c1 - b c2) / det ; gamma2 = (a c2 - conj(b) c1) / det
    const double2 bc2 = cmuld(bb, c2), cbc1 = cmuld(make_double2(bb.x, -bb.y), c1);
    k.g1 = make_double2((d * c1.x - bc2.x) / det, (d * c1.y - bc2.y) / det);
    k.g2 = make_double2((a * c2.x - cbc1.x) / det, (a * c2.y - cbc1.y) / det);
  }
}

// x += g1 r0 + g2 r1 ; r0 -= g1 r1 + g2 r2 ; u0 -= g1 u1 + g2 u2 ; partial |r0|^2, <shadow, r0>,
// then the next cycle's first BiCG coefficients: rho0 <- -omega rho0, beta = alpha <shadow, r0> / rho0
template <typename C>
__global__ void k_b2_mr(KrylovVecs<C> kv, KState* ks, RedBuf rb, int64_t n3) {
  pdl_begin();
  const int b = blockIdx.y;
  const KState k = ks[b];
  double acc[3] = {0.0, 0.0, 0.0};
  if (!k.done) {
    using R = typename RealOf<C>::t;
    const C g1 = mk((R)k.g1.x, (R)k.g1.y), g2 = mk((R)k.g2.x, (R)k.g2.y);
    const int64_t o = (int64_t)b * n3;
    Acc<C> rr, re, im;
    VEC_LOOP(n3) {
      const C r0 = kv.r[o + i], r1 = kv.s[o + i], r2 = kv.t[o + i];
      kv.x[o + i] = cadd(kv.x[o + i], cadd(cmul(g1, r0), cmul(g2, r1)));
      const C rn = csub(r0, cadd(cmul(g1, r1), cmul(g2, r2)));
      kv.r[o + i] = rn;
      kv.p[o + i] = csub(kv.p[o + i], cadd(cmul(g1, kv.v[o + i]), cmul(g2, kv.u2[o + i])));
      acc_nrm(rr, rn);
      acc_cdot(re, im, kv.rhat[o + i], rn);
    }
    acc[0] = rr.get();
    acc[1] = re.get();
    acc[2] = im.get();
  }
  double t[3];
  if (last_block_totals<3>(acc, rb, b, t) && threadIdx.x == 0) {
    KState& k = ks[b];
    if (k.done) return;
    k.it += 2;
    k.rr = t[0];
    if (t[0] <= k.tol2) { k.done = 1; return; }
    k.omega = k.g2;
    const double2 rho0 = cmuld(make_double2(-k.omega.x, -k.omega.y), k.rho);
    const double2 rho1 = make_double2(t[1], t[2]);
    if ((rho0.x == 0.0 && rho0.y == 0.0) || (rho1.x == 0.0 && rho1.y == 0.0)) { k.done = 2; return; }
    k.beta = cmuld(k.alpha, cdiv(rho1, rho0));
    k.rho = rho1;
  }
}

// ------------------------------------------------------------------ refinement helpers
__global__ void k_residual128(const double2* e, const double2* ax, double2* r, double* out2, RedBuf rb, int64_t n3) {
  const int bb = blockIdx.y;
  const int64_t o = (int64_t)bb * n3;
  double acc[2] = {0.0, 0.0};
  VEC_LOOP(n3) {
    const double2 bv = e[o + i], av = ax[o + i];
    const double2 rv = make_double2(bv.x - av.x, bv.y - av.y);
    r[o + i] = rv;
    acc[0] = nrm_acc(acc[0], rv);
    acc[1] = nrm_acc(acc[1], bv);
  }
  const int b = bb;
  double t[2];
  if (last_block_totals<2>(acc, rb, b, t) && threadIdx.x == 0) {
    out2[2 * b] = t[0];
    out2[2 * b + 1] = t[1];
  }
}

template <typename C>
__global__ void k_from128(const double2* src, C* dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = from_d<C>(src[i]);
}

template <typename C>
__global__ void k_add128(double2* dst, const C* src, const int* mask_done, int64_t n3) {
  const int b = blockIdx.y;
  if (mask_done && mask_done[b]) return;
  const int64_t o = (int64_t)b * n3;
  VEC_LOOP(n3) {
    const double2 s = to_d(src[o + i]);
    double2 d = dst[o + i];
    d.x += s.x;
    d.y += s.y;
    dst[o + i] = d;
  }
}

inline dim3 vgrid(const RedBuf& rb, int nrhs) { return dim3(rb.nblk, nrhs); }

}  // namespace

// ------------------------------------------------------------------ host wrappers
#define CHECK_LAUNCH()            \
  do {                            \
    DDA_CU(cudaGetLastError());   \
    add_launches(1);              \
  } while (0)

template <typename C>
Err bicg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol, bool have_ax,
              cudaStream_t st) {
  k_bicg_init<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3, have_ax, tol);
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err bicg_p_update(const KrylovVecs<C>& kv, const KState* ks, int nrhs, int64_t n3, cudaStream_t st) {
  // grid size independent of reductions
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  DDA_CU(launch_k(k_bicg_p<C>, dim3(nb, nrhs), dim3(kThreads), 0, st, kv, ks, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err bicg_alpha(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_bicg_dot_rv<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err bicg_s_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_bicg_s<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err bicg_omega(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_bicg_dot_ts<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err bicg_xr_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_bicg_xr<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err ccg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol, bool have_ax,
             cudaStream_t st) {
  k_ccg_init<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3, have_ax, tol);
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err ccg_start(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  k_ccg_start<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3);
  CHECK_LAUNCH();
  return Err::Ok();
}
// after v = A p: alpha, x/r update, convergence
template <typename C>
Err ccg_alpha_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_norm_v<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  DDA_CU(launch_k(k_ccg_xr<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
// after s = A^H r: beta, p update
template <typename C>
Err ccg_beta_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_norm_s<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  DDA_CU(launch_k(k_ccg_p<C>, dim3(nb, nrhs), dim3(kThreads), 0, st, kv, ks, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err cocg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol, bool have_ax,
              cudaStream_t st) {
  k_cocg_init<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3, have_ax, tol);
  CHECK_LAUNCH();
  return Err::Ok();
}
// after q = A p: alpha, x/r update, convergence and beta, p update
template <typename C>
Err cocg_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_cocg_mu<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  DDA_CU(launch_k(k_cocg_xr<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  DDA_CU(launch_k(k_cocg_p<C>, dim3(nb, nrhs), dim3(kThreads), 0, st, kv, ks, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err qmr_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol, bool have_ax,
             cudaStream_t st) {
  k_qmr_init<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3, have_ax, tol);
  DDA_CU(cudaGetLastError());
  k_qmr_scale<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, n3);
  DDA_CU(cudaGetLastError());
  add_launches(2);
  return Err::Ok();
}

template <typename C>
Err qmr_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_qmr_dots<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  DDA_CU(launch_k(k_qmr_w<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  DDA_CU(launch_k(k_qmr_dx<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}

Err combine2_c128(double2* dst, const double2* s0, const double2* s1, double2 c0, double2 c1, int64_t n3,
                  cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  k_combine2<<<dim3(nb, 1), kThreads, 0, st>>>(dst, s0, s1, c0, c1, n3);
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err scale_sites(C* v, const C* s, const uint8_t* comp, int ncomp, int nrhs, int64_t n, bool inv, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((3 * n + kThreads * 4 - 1) / (kThreads * 4), 1024);
  k_scale_sites<C><<<dim3(nb, nrhs), kThreads, 0, st>>>(v, s, comp, ncomp, n, inv);
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err b2_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol, bool have_ax,
            cudaStream_t st) {
  k_b2_init<C><<<vgrid(rb, nrhs), kThreads, 0, st>>>(kv, ks, rb, n3, have_ax, tol);
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err b2_u_update(const KrylovVecs<C>& kv, const KState* ks, int j, int nrhs, int64_t n3, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  DDA_CU(launch_k(k_b2_u<C>, dim3(nb, nrhs), dim3(kThreads), 0, st, kv, ks, j, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err b2_alpha(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int j, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_b2_alpha<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, j, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err b2_r_update(const KrylovVecs<C>& kv, const KState* ks, int j, int nrhs, int64_t n3, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  DDA_CU(launch_k(k_b2_r<C>, dim3(nb, nrhs), dim3(kThreads), 0, st, kv, ks, j, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err b2_beta(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_b2_beta<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}
template <typename C>
Err b2_mr(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, cudaStream_t st) {
  DDA_CU(launch_k(k_b2_gram<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  DDA_CU(launch_k(k_b2_mr<C>, vgrid(rb, nrhs), dim3(kThreads), 0, st, kv, ks, rb, n3));
  CHECK_LAUNCH();
  return Err::Ok();
}

Err residual_c128(const double2* b, const double2* ax, double2* r, double* out2, RedBuf rb, int nrhs, int64_t n3,
                  cudaStream_t st) {
  k_residual128<<<vgrid(rb, nrhs), kThreads, 0, st>>>(b, ax, r, out2, rb, n3);
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err convert_from_c128(const double2* src, C* dst, int64_t count, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((count + kThreads - 1) / kThreads, 152 * 16);
  k_from128<C><<<nb, kThreads, 0, st>>>(src, dst, count);
  CHECK_LAUNCH();
  return Err::Ok();
}

template <typename C>
Err add_to_c128(double2* dst, const C* src, const int* mask_done, int nrhs, int64_t n3, cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n3 + kThreads * 4 - 1) / (kThreads * 4), 1024);
  k_add128<C><<<dim3(nb, nrhs), kThreads, 0, st>>>(dst, src, mask_done, n3);
  CHECK_LAUNCH();
  return Err::Ok();
}

#define INST(C)                                                                                              \
  template Err bicg_init<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, double, bool, cudaStream_t); \
  template Err bicg_p_update<C>(const KrylovVecs<C>&, const KState*, int, int64_t, cudaStream_t);             \
  template Err bicg_alpha<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);              \
  template Err bicg_s_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);           \
  template Err bicg_omega<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);              \
  template Err bicg_xr_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);          \
  template Err ccg_init<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, double, bool, cudaStream_t);  \
  template Err ccg_start<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);               \
  template Err ccg_alpha_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);        \
  template Err ccg_beta_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);         \
  template Err convert_from_c128<C>(const double2*, C*, int64_t, cudaStream_t);                               \
  template Err add_to_c128<C>(double2*, const C*, const int*, int, int64_t, cudaStream_t);                    \
  template Err b2_init<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, double, bool, cudaStream_t);   \
  template Err b2_u_update<C>(const KrylovVecs<C>&, const KState*, int, int, int64_t, cudaStream_t);          \
  template Err b2_alpha<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int, int64_t, cudaStream_t);           \
  template Err b2_r_update<C>(const KrylovVecs<C>&, const KState*, int, int, int64_t, cudaStream_t);          \
  template Err b2_beta<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);                 \
  template Err b2_mr<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);                  \
  template Err cocg_init<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, double, bool, cudaStream_t); \
  template Err cocg_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);            \
  template Err qmr_init<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, double, bool, cudaStream_t); \
  template Err qmr_update<C>(const KrylovVecs<C>&, KState*, RedBuf, int, int64_t, cudaStream_t);            \
  template Err scale_sites<C>(C*, const C*, const uint8_t*, int, int, int64_t, bool, cudaStream_t);
INST(float2)
INST(double2)

}  // namespace dda
