// Compile-time-length kernels of the FFT-convolution product (same passes and
// workspace layout as matvec.cu, faster engine): every 1-D transform is the
// two-pass register FFT of fft2.cuh, the z-direction pass B is fused with the
// 3x3 Ghat multiply and the inverse pass B in registers, and global loads and
// stores are arranged so that consecutive threads touch consecutive addresses.
//
// Ghat layout: [kx][kz][ky][6] (xx, xy, xz, yy, yz, zz), scaled by 1/M.
// Workspace:   W[b][c][kx][z][ys], ys = ny (3-pass) or py (5-pass).
//
// The templates take the compute type C: float2 (complex64), double2
// (complex128) or dfp::dfc (double-float, df.cuh: complex128 vectors in and
// out, FP32-pair arithmetic inside; Io<C> is the vectors' element type).  The
// x passes are bodies with a compile-time mode so that the complex64 BiCGstab
// iteration can fold its vector updates and dot products into them
// (k_x_fwd_fused / k_x_inv_fused, instantiated in matvec_fused_c64.cu).
#pragma once

#include "bulk.cuh"
#include "dda_internal.h"
#include "df.cuh"
#include "fft2.cuh"
#include "kred.cuh"

namespace dda {
namespace fast {

using f2::Shape;

template <typename C>
__device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }

template <typename C>
__device__ __forceinline__ void load6(const C* __restrict__ gh, C (&g)[6]) {
  if constexpr (sizeof(C) == 8) {  // 48 bytes, 16-byte aligned: three 128-bit loads
    const float4* q = reinterpret_cast<const float4*>(gh);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    g[0] = make_float2(a.x, a.y); g[1] = make_float2(a.z, a.w);
    g[2] = make_float2(b.x, b.y); g[3] = make_float2(b.z, b.w);
    g[4] = make_float2(c.x, c.y); g[5] = make_float2(c.z, c.w);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = gh[i];
  }
}

// u = Ghat v for one voxel: each output component is a 3-term complex dot
// product, written as one FMUL and five FMAs per real part (12 real products
// per output, no separate additions).
template <typename C>
__device__ __forceinline__ C cdot3(C a0, C b0, C a1, C b1, C a2, C b2) {
  C r;
  r.x = fma(a0.x, b0.x, fma(-a0.y, b0.y, fma(a1.x, b1.x, fma(-a1.y, b1.y, fma(a2.x, b2.x, -a2.y * b2.y)))));
  r.y = fma(a0.x, b0.y, fma(a0.y, b0.x, fma(a1.x, b1.y, fma(a1.y, b1.x, fma(a2.x, b2.y, a2.y * b2.x)))));
  return r;
}

template <typename C>
__device__ __forceinline__ void gmul3_r(const C (&gg)[6], C& v0, C& v1, C& v2) {
  const C u0 = cdot3(gg[0], v0, gg[1], v1, gg[2], v2);
  const C u1 = cdot3(gg[1], v0, gg[3], v1, gg[4], v2);
  const C u2 = cdot3(gg[2], v0, gg[4], v1, gg[5], v2);
  v0 = u0;
  v1 = u1;
  v2 = u2;
}

template <typename C>
__device__ __forceinline__ void gmul3(const C* __restrict__ gh, C& v0, C& v1, C& v2) {
  C gg[6];
  load6(gh, gg);
  const C u0 = cdot3(gg[0], v0, gg[1], v1, gg[2], v2);
  const C u1 = cdot3(gg[1], v0, gg[3], v1, gg[4], v2);
  const C u2 = cdot3(gg[2], v0, gg[4], v1, gg[5], v2);
  v0 = u0;
  v1 = u1;
  v2 = u2;
}

// true when RHS b of this launch belongs to a finished solve (whole CTA exits before any barrier)
template <typename C>
__device__ __forceinline__ bool rhs_done(const MvData<C>& d, int b) {
  return d.ks != nullptr && d.ks[b].done != 0;
}

template <typename C>
__device__ __forceinline__ void copy_tw(C* dst, const C* src, int L) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------------------------ BiCGstab updates folded into the x passes
// (complex64, product without conjugation).  The x forward pass visits every (site, component)
// of every RHS exactly once while gathering the product's input, and the x inverse pass while
// scattering its output, so the vector updates and dot products that BiCGstab applies just
// before and after each product can ride on those passes:
//   kFuseP   x forward: p = r + beta (p - omega v) gathered, stored and transformed
//   kFuseS   x forward: s = r - alpha v gathered, stored and transformed; |s|^2 -> half-step test
//   kFuseRV  x inverse: v = A p stored, <rhat, v> -> alpha
//   kFuseTS  x inverse: t = A s stored, <t, s>, |t|^2 -> omega
// with the same per-RHS scalars (KState) and finalisation as the separate vector kernels.
enum FuseMode { kFuseNone = 0, kFuseP = 1, kFuseS = 2, kFuseRV = 3, kFuseTS = 4 };

// this CTA's reduction slot within its RHS, and the CTAs per RHS, of an x-pass grid
// (ceil(ny/TY), nz, nrhs * 3/NC)
template <int NC>
__device__ __forceinline__ int x_slot() {
  return (int)((blockIdx.z % (3 / NC)) * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x);
}
template <int NC>
__device__ __forceinline__ int x_slots() {
  return (int)(gridDim.x * gridDim.y * (3 / NC));
}

// ------------------------------------------------------------------ x forward
// grid (ceil(ny/TY), nz, nrhs * 3/NC): NC components (1 or 3) of TY y rows per CTA.
// smem: tw[PX] | in[NC*TY][ip] | out[NC*PX][TY]
template <typename C, int PX, int TY, int NC, int MODE>
__device__ __forceinline__ void x_fwd_body(const Geom& g, const MvData<C>& d, const typename Io<C>::t* __restrict__ p,
                                           bool conj, int ip, const KrylovVecs<float2>* kf, KState* ksw,
                                           const RedBuf* rbx) {
  constexpr int RA = Shape<PX>::RA, LB = Shape<PX>::LB, H = Shape<PX>::H;
  static_assert(NC == 1 || NC == 3, "one or three components per CTA");
  static_assert(MODE == kFuseNone || (MODE == kFuseP || MODE == kFuseS), "x forward fuses p or s updates");
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* in = tw + PX;
  C* out = in + NC * TY * ip;
  const int y0 = blockIdx.x * TY, z = blockIdx.y;
  const int b = blockIdx.z / (3 / NC), c0 = (blockIdx.z % (3 / NC)) * NC;
  if (rhs_done(d, b)) return;
  copy_tw(tw, d.twx, PX);
  [[maybe_unused]] C k1 = czero<C>(), k2 = czero<C>();  // (beta, omega) or (alpha, -)
  [[maybe_unused]] kred::AccF ss;
  if constexpr (MODE == kFuseP) {
    const KState k = ksw[b];
    k1 = mk((float)k.beta.x, (float)k.beta.y);
    k2 = mk((float)k.omega.x, (float)k.omega.y);
  } else if constexpr (MODE == kFuseS) {
    const KState k = ksw[b];
    k1 = mk((float)k.alpha.x, (float)k.alpha.y);
  }
  // gather: kXU elements per thread per round, their site indices (map) loaded first and their
  // values next, so that a thread has kXU independent loads in flight at each of the two steps;
  // 8 for x lengths of 256 and more (measured 4 % faster on a 256 x 256 x 320 grid), 4 below
  // (8 was slower on 128 x 96 x 64)
  constexpr int kXU = PX >= 256 ? 8 : 4;
  const int nld = NC * TY * g.nx;
  for (int i0 = threadIdx.x; i0 < nld; i0 += kXU * blockDim.x) {
    int32_t idxs[kXU];
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int i = i0 + u * blockDim.x;
      const int x = i % g.nx;
      const int r = i / g.nx;
      const int t = r % TY;
      const int y = y0 + t;
      idxs[u] = (i < nld && y < g.ny) ? __ldg(d.map + ((int64_t)z * g.ny + y) * g.nx + x) : -1;
    }
    C vals[kXU];
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int i = i0 + u * blockDim.x;
      const int cl = (i / g.nx) / TY;
      const int32_t idx = idxs[u];
      C v = czero<C>();
      if (idx >= 0) {
        const int64_t o = ((int64_t)b * 3 + c0 + cl) * g.n + idx;
        if constexpr (MODE == kFuseNone) {
          v = io_get<C>(p[o]);
          if (conj) v = conjc(v);
        } else if constexpr (MODE == kFuseP) {
          v = cadd(kf->r[o], cmul(k1, csub(kf->p[o], cmul(k2, kf->v[o]))));
          kf->p[o] = v;
        } else {
          v = csub(kf->r[o], cmul(k1, kf->v[o]));
          kf->s[o] = v;
          kred::acc_nrm(ss, v);
        }
        if (d.sc) {  // Jacobi scaling: transform s * v
          const int c = c0 + cl;
          v = cmul(v, d.sc[((int64_t)b * g.ncomp + (d.comp ? d.comp[3 * idx + c] : 0)) * 3 + c]);
        }
      }
      vals[u] = v;
    }
#pragma unroll
    for (int u = 0; u < kXU; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < nld) {
        const int x = i % g.nx;
        const int r = i / g.nx;
        in[((r / TY) * TY + r % TY) * ip + x] = vals[u];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NC * TY * LB; i += blockDim.x) {
    const int t = i % TY;
    const int r = i / TY;
    const int n1 = r % LB, cl = r / LB;
    C x[RA], o[2 * RA];
    const C* src = in + (cl * TY + t) * ip;
#pragma unroll
    for (int j = 0; j < RA; ++j) {
      const int xx = n1 + LB * j;
      x[j] = (xx < g.nx) ? src[xx] : czero<C>();
    }
    f2::passA_fwd<PX>(x, n1, tw, o);
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RA; ++k) out[(cl * PX + bb * H + n1 + LB * k) * TY + t] = o[bb * RA + k];
  }
  __syncthreads();
  const int64_t plane = (int64_t)g.nz * g.ys;
  for (int i = threadIdx.x; i < NC * 2 * RA * TY; i += blockDim.x) {
    const int t = i % TY;
    const int r = i / TY;
    const int blk = r % (2 * RA), cl = r / (2 * RA);
    C v[LB];
#pragma unroll
    for (int e = 0; e < LB; ++e) v[e] = out[(cl * PX + blk * LB + e) * TY + t];
    f2::passB_fwd<PX>(v, tw);
    const int y = y0 + t;
    if (y < g.ny) {
      C* dst = d.work + (((int64_t)b * 3 + c0 + cl) * PX + blk * LB) * plane + (int64_t)z * g.ys + y;
#pragma unroll
      for (int e = 0; e < LB; ++e) dst[e * plane] = v[e];
    }
  }
  if constexpr (MODE == kFuseS) {
    double acc[1] = {ss.get()};
    double tot[1];
    if (kred::last_cta_totals<1>(acc, rbx->part, rbx->count, b, x_slot<NC>(), x_slots<NC>(), tot) &&
        threadIdx.x == 0) {
      KState& k = ksw[b];
      if (!k.done && tot[0] <= k.tol2) { k.done = 3; k.rr = tot[0]; }  // converged on the half step
    }
  }
}

template <typename C, int PX, int TY, int NC = 3>
__global__ void __launch_bounds__(256) k_x_fwd(Geom g, MvData<C> d, const typename Io<C>::t* __restrict__ p,
                                               bool conj, int ip) {
  x_fwd_body<C, PX, TY, NC, kFuseNone>(g, d, p, conj, ip, nullptr, nullptr, nullptr);
}

// the x forward pass with the BiCGstab p (MODE = kFuseP) or s (kFuseS) update folded in
template <int PX, int TY, int NC, int MODE>
__global__ void __launch_bounds__(256) k_x_fwd_fused(Geom g, MvData<float2> d, KrylovVecs<float2> kv, KState* ks,
                                                     RedBuf rbx, int ip) {
  x_fwd_body<float2, PX, TY, NC, MODE>(g, d, nullptr, false, ip, &kv, ks, &rbx);
}

// ------------------------------------------------------------------ x inverse + alpha^{-1} P + scatter
// grid and shared memory as k_x_fwd
template <typename C, int PX, int TY, int NC, int MODE>
__device__ __forceinline__ void x_inv_body(const Geom& g, const MvData<C>& d, const typename Io<C>::t* __restrict__ p,
                                           typename Io<C>::t* __restrict__ ap, int rhs0, bool conj, int ip,
                                           const KrylovVecs<float2>* kf, KState* ksw, const RedBuf* rbx) {
  constexpr int RA = Shape<PX>::RA, LB = Shape<PX>::LB, H = Shape<PX>::H;
  static_assert(NC == 1 || NC == 3, "one or three components per CTA");
  static_assert(MODE == kFuseNone || (MODE == kFuseRV || MODE == kFuseTS), "x inverse fuses the dot products");
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* in = tw + PX;
  C* out = in + NC * TY * ip;
  const int y0 = blockIdx.x * TY, z = blockIdx.y;
  const int b = blockIdx.z / (3 / NC), c0 = (blockIdx.z % (3 / NC)) * NC;
  if (rhs_done(d, b)) return;
  copy_tw(tw, d.twx, PX);
  __syncthreads();
  const int64_t plane = (int64_t)g.nz * g.ys;
  for (int i = threadIdx.x; i < NC * 2 * RA * TY; i += blockDim.x) {
    const int t = i % TY;
    const int r = i / TY;
    const int blk = r % (2 * RA), cl = r / (2 * RA);
    const int y = y0 + t;
    C v[LB];
    if (y < g.ny) {
      const C* src = d.work + (((int64_t)b * 3 + c0 + cl) * PX + blk * LB) * plane + (int64_t)z * g.ys + y;
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = src[e * plane];
    } else {
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = czero<C>();
    }
    f2::passB_inv<PX>(v, tw);
#pragma unroll
    for (int e = 0; e < LB; ++e) out[(cl * PX + blk * LB + e) * TY + t] = v[e];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NC * TY * LB; i += blockDim.x) {
    const int t = i % TY;
    const int r = i / TY;
    const int n1 = r % LB, cl = r / LB;
    C v[2 * RA], lo[RA];
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RA; ++k) v[bb * RA + k] = out[(cl * PX + bb * H + n1 + LB * k) * TY + t];
    f2::passA_inv<PX, false>(v, n1, tw, lo, (C*)nullptr);
    C* dst = in + (cl * TY + t) * ip;
#pragma unroll
    for (int j = 0; j < RA; ++j) {
      const int xx = n1 + LB * j;
      if (xx < g.nx) dst[xx] = lo[j];
    }
  }
  __syncthreads();
  const C* ia = d.ia + (int64_t)(rhs0 + b) * g.ncomp * 3;
  const int nst = NC * TY * g.nx;
  [[maybe_unused]] kred::AccF re, im, tt;
  // kXU elements per thread per round, site indices first (independent loads in flight); as in
  // the forward gather, 8 for x lengths of 256 and more, 4 below
  constexpr int kXU = PX >= 256 ? 8 : 4;
  for (int i0 = threadIdx.x; i0 < nst; i0 += kXU * blockDim.x) {
   int32_t idxs[kXU];
#pragma unroll
   for (int u = 0; u < kXU; ++u) {
     const int i = i0 + u * blockDim.x;
     const int y = y0 + (i / g.nx) % TY;
     idxs[u] = (i < nst && y < g.ny) ? __ldg(d.map + ((int64_t)z * g.ny + y) * g.nx + i % g.nx) : -1;
   }
#pragma unroll
   for (int u = 0; u < kXU; ++u) {
    const int i = i0 + u * blockDim.x;
    const int32_t idx = idxs[u];
    if (idx < 0) continue;
    const int x = i % g.nx;
    const int r = i / g.nx;
    const int t = r % TY, cl = r / TY;
    const int c = c0 + cl;
    const int64_t o = ((int64_t)b * 3 + c) * g.n + idx;
    const int cc = d.comp ? d.comp[3 * idx + c] : 0;  // composition of axis c
    C pv = io_get<C>(p[o]);
    if (conj) pv = conjc(pv);
    C res;
    if (d.iat) {  // rotated dielectric frame: row c of the full symmetric alpha^{-1} of this site
      const C* m6 = d.iat + ((int64_t)(rhs0 + b) * g.n + idx) * 6;
      const int64_t oc = ((int64_t)b * 3) * g.n + idx;
      res = in[(cl * TY + t) * ip + x];
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) {
        C q = io_get<C>(p[oc + (int64_t)c2 * g.n]);
        if (conj) q = conjc(q);
        const int lo = c < c2 ? c : c2, hi = c < c2 ? c2 : c;
        res = cadd(res, cmul(m6[lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)], q));
      }
    } else {
      res = d.sc ? cadd(cmul(d.sc[((int64_t)b * g.ncomp + cc) * 3 + c], in[(cl * TY + t) * ip + x]), pv)
                 : cadd(in[(cl * TY + t) * ip + x], cmul(ia[cc * 3 + c], pv));
    }
    ap[o] = io_put<C>(conj ? conjc(res) : res);
    if constexpr (MODE == kFuseRV) {
      kred::acc_cdot(re, im, kf->rhat[o], res);  // <rhat, v>
    } else if constexpr (MODE == kFuseTS) {
      kred::acc_cdot(re, im, res, kf->s[o]);     // <t, s>
      kred::acc_nrm(tt, res);                    // |t|^2
    }
   }
  }
  if constexpr (MODE == kFuseRV) {
    double acc[2] = {re.get(), im.get()};
    double tot[2];
    if (kred::last_cta_totals<2>(acc, rbx->part, rbx->count, b, x_slot<NC>(), x_slots<NC>(), tot) &&
        threadIdx.x == 0) {
      KState& k = ksw[b];
      if (!k.done) {
        k.mv += 1;  // v = A p
        const double2 rv = make_double2(tot[0], tot[1]);
        if (rv.x == 0.0 && rv.y == 0.0) k.done = 2;
        else k.alpha = kred::cdiv(k.rho, rv);
      }
    }
  } else if constexpr (MODE == kFuseTS) {
    double acc[3] = {re.get(), im.get(), tt.get()};
    double tot[3];
    if (kred::last_cta_totals<3>(acc, rbx->part, rbx->count, b, x_slot<NC>(), x_slots<NC>(), tot) &&
        threadIdx.x == 0) {
      KState& k = ksw[b];
      if (!k.done) {
        k.mv += 1;  // t = A s
        k.omega = (tot[2] > 0.0) ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
      }
    }
  }
}

template <typename C, int PX, int TY, int NC = 3>
__global__ void __launch_bounds__(256) k_x_inv(Geom g, MvData<C> d, const typename Io<C>::t* __restrict__ p,
                                               typename Io<C>::t* __restrict__ ap, int rhs0, bool conj, int ip) {
  x_inv_body<C, PX, TY, NC, kFuseNone>(g, d, p, ap, rhs0, conj, ip, nullptr, nullptr, nullptr);
}

// the x inverse pass with the BiCGstab dot products folded in: v = A p and <rhat, v>
// (MODE = kFuseRV), or t = A s with <t, s> and |t|^2 (kFuseTS)
template <int PX, int TY, int NC, int MODE>
__global__ void __launch_bounds__(256) k_x_inv_fused(Geom g, MvData<float2> d, KrylovVecs<float2> kv, KState* ks,
                                                     RedBuf rbx, int ip) {
  const float2* p = MODE == kFuseRV ? kv.p : kv.s;
  float2* ap = MODE == kFuseRV ? kv.v : kv.t;
  x_inv_body<float2, PX, TY, NC, MODE>(g, d, p, ap, 0, false, ip, &kv, ks, &rbx);
}

// ------------------------------------------------------------------ fused y-z plane (3-pass schedule)
// grid (nrhs, px), block NT.  smem: twy[PY] | twz[PZ] | pl[PZ*3][PY+1] (row (z,c) = z*3 + c)
// With BULK, the plane's input and output (three contiguous nz x ny blocks of the
// workspace) move between HBM and shared memory as bulk copies (TMA) when nz*ny is even
// (16-byte granularity), staged in the plane rows z >= nz, which are unused before the
// forward z transform and after the inverse one; otherwise every thread loads and stores
// its own elements.
// shared-memory bytes of the plane pass; the bulk-staged variant keeps its mbarrier after the plane
template <typename C>
__host__ __device__ constexpr size_t plane_bytes(int py, int pz) {
  return sizeof(C) * ((size_t)py + pz + (size_t)pz * 3 * (py + 1));
}

template <typename C, int PY, int PZ, int NT, bool BULK>
__global__ void __launch_bounds__(NT) k_yz_plane(Geom g, MvData<C> d) {
  constexpr int RAy = Shape<PY>::RA, LBy = Shape<PY>::LB, Hy = Shape<PY>::H;
  constexpr int RAz = Shape<PZ>::RA, LBz = Shape<PZ>::LB, Hz = Shape<PZ>::H;
  constexpr int RP = PY + 1;
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  C* twy = reinterpret_cast<C*>(smem_raw);
  C* twz = twy + PY;
  C* pl = twz + PZ;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + ((plane_bytes<C>(PY, PZ) + 15) & ~(size_t)15));
  const int b = blockIdx.x, kx = blockIdx.y;
  if (rhs_done(d, b)) return;
  const int nz = g.nz, ny = g.ny;
  C* wb = d.work + ((int64_t)b * 3 * g.px + kx) * ((int64_t)nz * g.ys);
  const int64_t cstride = (int64_t)g.px * nz * g.ys;
  // staging block [c][z][y] in rows z >= nz, 16-byte aligned
  const bool staged = BULK && ((nz * ny) % 2 == 0) && g.ys == ny;
  C* stage = pl + 3 * nz * RP + ((3 * nz * RP) & 1);
  const uint32_t cbytes = (uint32_t)(sizeof(C) * nz * ny);
  if (staged && threadIdx.x == 0) {
    bulk::mbar_init(bar, 1);
    bulk::mbar_arrive_expect_tx(bar, 3 * cbytes);
    for (int c = 0; c < 3; ++c) bulk::load_g2s(stage + c * nz * ny, wb + c * cstride, cbytes, bar);
  }
  copy_tw(twy, d.twy, PY);
  copy_tw(twz, d.twz, PZ);
  __syncthreads();  // barrier initialised before anyone polls it
  if (staged) bulk::mbar_wait(bar, 0, bulk::kMaxPolls, d.fault);
  // y forward, pass A: staged block (or global) -> registers -> plane
  for (int i = threadIdx.x; i < 3 * nz * LBy; i += blockDim.x) {
    const int n1 = i % LBy;
    const int r = i / LBy;
    const int z = r % nz, c = r / nz;
    const C* src = staged ? stage + (c * nz + z) * ny : wb + c * cstride + (int64_t)z * g.ys;
    C x[RAy], o[2 * RAy];
#pragma unroll
    for (int j = 0; j < RAy; ++j) {
      const int yy = n1 + LBy * j;
      x[j] = (yy < ny) ? src[yy] : czero<C>();
    }
    f2::passA_fwd<PY>(x, n1, twy, o);
    C* row = pl + (z * 3 + c) * RP;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RAy; ++k) row[bb * Hy + n1 + LBy * k] = o[bb * RAy + k];
  }
  __syncthreads();
  // y forward, pass B
  for (int i = threadIdx.x; i < 3 * nz * 2 * RAy; i += blockDim.x) {
    const int rr = i % (3 * nz), blk = i / (3 * nz);
    C* row = pl + rr * RP + blk * LBy;
    C v[LBy];
#pragma unroll
    for (int e = 0; e < LBy; ++e) v[e] = row[e];
    f2::passB_fwd<PY>(v, twy);
#pragma unroll
    for (int e = 0; e < LBy; ++e) row[e] = v[e];
  }
  __syncthreads();
  // z forward, pass A (pencils (c, ky), rows z < nz nonzero)
  for (int i = threadIdx.x; i < 3 * PY * LBz; i += blockDim.x) {
    const int ky = i % PY;
    const int r = i / PY;
    const int c = r % 3, n1 = r / 3;
    C x[RAz], o[2 * RAz];
#pragma unroll
    for (int j = 0; j < RAz; ++j) {
      const int zz = n1 + LBz * j;
      x[j] = (zz < nz) ? pl[(zz * 3 + c) * RP + ky] : czero<C>();
    }
    f2::passA_fwd<PZ>(x, n1, twz, o);
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RAz; ++k) pl[((bb * Hz + n1 + LBz * k) * 3 + c) * RP + ky] = o[bb * RAz + k];
  }
  __syncthreads();
  // z pass B, Ghat, inverse z pass B -- in registers for the three components
  const C* gk = d.ghat + (int64_t)kx * PZ * PY * 6;
  for (int i = threadIdx.x; i < PY * 2 * RAz; i += blockDim.x) {
    const int ky = i % PY, blk = i / PY;
    C v0[LBz], v1[LBz], v2[LBz];
#pragma unroll
    for (int e = 0; e < LBz; ++e) {
      const C* rowp = pl + ((blk * LBz + e) * 3) * RP + ky;
      v0[e] = rowp[0];
      v1[e] = rowp[RP];
      v2[e] = rowp[2 * RP];
    }
    f2::passB_fwd<PZ>(v0, twz);
    f2::passB_fwd<PZ>(v1, twz);
    f2::passB_fwd<PZ>(v2, twz);
#pragma unroll
    for (int e = 0; e < LBz; ++e) gmul3(gk + ((int64_t)(blk * LBz + e) * PY + ky) * 6, v0[e], v1[e], v2[e]);
    f2::passB_inv<PZ>(v0, twz);
    f2::passB_inv<PZ>(v1, twz);
    f2::passB_inv<PZ>(v2, twz);
#pragma unroll
    for (int e = 0; e < LBz; ++e) {
      C* rowp = pl + ((blk * LBz + e) * 3) * RP + ky;
      rowp[0] = v0[e];
      rowp[RP] = v1[e];
      rowp[2 * RP] = v2[e];
    }
  }
  __syncthreads();
  // z inverse, pass A: rows z < nz only
  for (int i = threadIdx.x; i < 3 * PY * LBz; i += blockDim.x) {
    const int ky = i % PY;
    const int r = i / PY;
    const int c = r % 3, n1 = r / 3;
    C v[2 * RAz], lo[RAz];
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RAz; ++k) v[bb * RAz + k] = pl[((bb * Hz + n1 + LBz * k) * 3 + c) * RP + ky];
    f2::passA_inv<PZ, false>(v, n1, twz, lo, (C*)nullptr);
#pragma unroll
    for (int j = 0; j < RAz; ++j) {
      const int zz = n1 + LBz * j;
      if (zz < nz) pl[(zz * 3 + c) * RP + ky] = lo[j];
    }
  }
  __syncthreads();
  // y inverse, pass B
  for (int i = threadIdx.x; i < 3 * nz * 2 * RAy; i += blockDim.x) {
    const int rr = i % (3 * nz), blk = i / (3 * nz);
    C* row = pl + rr * RP + blk * LBy;
    C v[LBy];
#pragma unroll
    for (int e = 0; e < LBy; ++e) v[e] = row[e];
    f2::passB_inv<PY>(v, twy);
#pragma unroll
    for (int e = 0; e < LBy; ++e) row[e] = v[e];
  }
  __syncthreads();
  // y inverse, pass A: plane -> registers -> staged block (or global), y < ny
  for (int i = threadIdx.x; i < 3 * nz * LBy; i += blockDim.x) {
    const int n1 = i % LBy;
    const int r = i / LBy;
    const int z = r % nz, c = r / nz;
    const C* row = pl + (z * 3 + c) * RP;
    C v[2 * RAy], lo[RAy];
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RAy; ++k) v[bb * RAy + k] = row[bb * Hy + n1 + LBy * k];
    f2::passA_inv<PY, false>(v, n1, twy, lo, (C*)nullptr);
    C* dst = staged ? stage + (c * nz + z) * ny : wb + c * cstride + (int64_t)z * g.ys;
#pragma unroll
    for (int j = 0; j < RAy; ++j) {
      const int yy = n1 + LBy * j;
      if (yy < ny) dst[yy] = lo[j];
    }
  }
  if (staged) {
    bulk::fence_smem_to_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int c = 0; c < 3; ++c) bulk::store_s2g(wb + c * cstride, stage + c * nz * ny, cbytes);
      bulk::store_commit();
      bulk::store_wait_read();  // shared memory stays allocated until the copies have read it
    }
  }
}

// ------------------------------------------------------------------ 5-pass: y rows
// rows (b, c, kx, z) of W with ys = PY; RPB rows per CTA.  smem: tw[PY] | s[RPB][PY+1]
template <typename C, int PY, int RPB, bool INV>
__global__ void __launch_bounds__(256) k_y_rows(Geom g, C* __restrict__ work, const C* __restrict__ twg,
                                                int64_t nrows) {
  constexpr int RA = Shape<PY>::RA, LB = Shape<PY>::LB, H = Shape<PY>::H;
  constexpr int RP = PY + 1;
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + PY;
  const int64_t r0 = (int64_t)blockIdx.x * RPB;
  const int nr = (int)min((int64_t)RPB, nrows - r0);
  const int ny = g.ny;
  copy_tw(tw, twg, PY);
  __syncthreads();
  if (!INV) {
    for (int i = threadIdx.x; i < nr * LB; i += blockDim.x) {
      const int n1 = i % LB, r = i / LB;
      const C* src = work + (r0 + r) * PY;
      C x[RA], o[2 * RA];
#pragma unroll
      for (int j = 0; j < RA; ++j) {
        const int yy = n1 + LB * j;
        x[j] = (yy < ny) ? src[yy] : czero<C>();
      }
      f2::passA_fwd<PY>(x, n1, tw, o);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int k = 0; k < RA; ++k) s[r * RP + bb * H + n1 + LB * k] = o[bb * RA + k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * 2 * RA; i += blockDim.x) {
      const int r = i % nr, blk = i / nr;
      C* row = s + r * RP + blk * LB;
      C v[LB];
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = row[e];
      f2::passB_fwd<PY>(v, tw);
#pragma unroll
      for (int e = 0; e < LB; ++e) row[e] = v[e];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * PY; i += blockDim.x) {
      const int r = i / PY, y = i % PY;
      work[(r0 + r) * PY + y] = s[r * RP + y];
    }
  } else {
    // the tile's rows are one contiguous run of nr * PY elements; for a full complex64 tile each
    // thread issues all its loads before its first shared-memory store
    constexpr int kPer = RPB * PY / 256;
    if (sizeof(C) == 8 && nr == RPB && RPB * PY % 256 == 0 && kPer <= 16 && blockDim.x == 256) {
      const C* src = work + r0 * PY;
      C t[kPer > 0 ? kPer : 1];
#pragma unroll
      for (int u = 0; u < kPer; ++u) t[u] = src[threadIdx.x + 256 * u];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int i = threadIdx.x + 256 * u;
        s[(i / PY) * RP + i % PY] = t[u];
      }
    } else {
      for (int i = threadIdx.x; i < nr * PY; i += blockDim.x) {
        const int r = i / PY, y = i % PY;
        s[r * RP + y] = work[(r0 + r) * PY + y];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * 2 * RA; i += blockDim.x) {
      const int r = i % nr, blk = i / nr;
      C* row = s + r * RP + blk * LB;
      C v[LB];
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = row[e];
      f2::passB_inv<PY>(v, tw);
#pragma unroll
      for (int e = 0; e < LB; ++e) row[e] = v[e];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * LB; i += blockDim.x) {
      const int n1 = i % LB, r = i / LB;
      const C* row = s + r * RP;
      C v[2 * RA], lo[RA];
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int k = 0; k < RA; ++k) v[bb * RA + k] = row[bb * H + n1 + LB * k];
      f2::passA_inv<PY, false>(v, n1, tw, lo, (C*)nullptr);
      C* dst = work + (r0 + r) * PY;
#pragma unroll
      for (int j = 0; j < RA; ++j) {
        const int yy = n1 + LB * j;
        if (yy < ny) dst[yy] = lo[j];
      }
    }
  }
}

// ------------------------------------------------------------------ 5-pass: z columns with Ghat
// grid (nrhs, ceil(py/G), px): the right-hand sides of one Ghat tile are
// neighbours in launch order, so a tile is read from HBM once and then hits L2
// for the other right-hand sides.  smem: tw[PZ] | s[PZ*3][G] with zcols_pad() spare elements after
// each pass-B sub-block of LB positions: in pass B a warp touches G consecutive columns of several
// sub-blocks at once, and for complex64 with G = 8 and an even LB the unpadded sub-blocks all start
// on the same shared-memory bank, which doubles the wavefronts of every such warp access.
// RFUSE: pass B, the Ghat multiply and the inverse pass B of all three components in registers
// even for long sub-blocks (one item per thread: NT = G * 2 * RA threads, up to 3 CTAs per SM),
// which halves the shared-memory traffic of the column pass at the cost of occupancy.
template <typename C, int PZ, int G>
constexpr int zcols_pad() {
  // complex64: a warp's column group spans 2G words; when that is under the 32 banks, place
  // consecutive sub-blocks one group width apart (mod 32 words)
  if constexpr (sizeof(C) != 8 || 2 * G >= 32) {
    return 0;
  } else {
    constexpr int gw = 2 * G, stride = (Shape<PZ>::LB * 3 * G * 2) % 32;
    return ((gw - stride + 32) % 32) / 2;
  }
}
template <typename C, int PZ, int G>
constexpr size_t zcols_smem_elems() {
  return (size_t)PZ + (size_t)PZ * 3 * G + (size_t)2 * Shape<PZ>::RA * zcols_pad<C, PZ, G>();
}

// CTAs per SM the register budget is sized for: the fused variants 3; the complex64 kernel whose
// pass B goes through shared memory as many as its shared tile allows (up to 3), so that registers
// do not cap its occupancy below what shared memory permits
template <typename C, int PZ, int G, bool RFUSE>
constexpr int zcols_min_ctas() {
  if constexpr (RFUSE) {
    return 3;
  } else if constexpr (sizeof(C) == 8 && Shape<PZ>::LB * sizeof(C) > 96) {
    constexpr size_t b = sizeof(C) * zcols_smem_elems<C, PZ, G>() + 1024;
    return b * 3 <= 228 * 1024 ? 3 : (b * 2 <= 228 * 1024 ? 2 : 1);
  } else {
    return 1;
  }
}

template <typename C, int PZ, int G, int NT = 256, bool RFUSE = false>
__global__ void __launch_bounds__(NT, (zcols_min_ctas<C, PZ, G, RFUSE>())) k_z_cols(Geom g, MvData<C> d) {
  constexpr int RA = Shape<PZ>::RA, LB = Shape<PZ>::LB, H = Shape<PZ>::H;
  constexpr int P = zcols_pad<C, PZ, G>();  // spare elements after each sub-block
  constexpr bool kFuse = RFUSE || (LB * sizeof(C) <= 96);
  pdl_begin();
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + PZ;
  const int ky0 = blockIdx.y * G, kx = blockIdx.z, b = blockIdx.x;
  if (rhs_done(d, b)) return;
  const int nz = g.nz, py = g.py;
  copy_tw(tw, d.twz, PZ);
  __syncthreads();
  C* wb = d.work + ((int64_t)b * 3 * g.px + kx) * ((int64_t)nz * g.ys);
  const int64_t cstride = (int64_t)g.px * nz * g.ys;
  // forward pass A from global.  The column inputs come from HBM (the y pass wrote them), so for
  // complex64 every load of a thread's items (a compile-time count: blockDim.x == NT) is issued
  // before its first transform and the round trips overlap instead of following one another.
  constexpr int kItemsA = 3 * G * LB;
  constexpr int kItA = (kItemsA + NT - 1) / NT;
  if constexpr (sizeof(C) == 8 && kItA * RA <= 32) {
    C xa[kItA][RA];
#pragma unroll
    for (int it = 0; it < kItA; ++it) {
      const int i = threadIdx.x + it * NT;
      const int gg = i % G, r = i / G;
      const int c = r % 3, n1 = r / 3;
      const bool ok = i < kItemsA && ky0 + gg < py;
#pragma unroll
      for (int j = 0; j < RA; ++j) {
        const int zz = n1 + LB * j;
        xa[it][j] = (ok && zz < nz) ? wb[c * cstride + (int64_t)zz * g.ys + ky0 + gg] : czero<C>();
      }
    }
#pragma unroll
    for (int it = 0; it < kItA; ++it) {
      const int i = threadIdx.x + it * NT;
      if (i < kItemsA) {
        const int gg = i % G, r = i / G;
        const int c = r % 3, n1 = r / 3;
        C o[2 * RA];
        f2::passA_fwd<PZ>(xa[it], n1, tw, o);
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
          for (int k = 0; k < RA; ++k)
            s[((bb * H + n1 + LB * k) * 3 + c) * G + gg + (bb * RA + k) * P] = o[bb * RA + k];
      }
    }
  } else {
    for (int i = threadIdx.x; i < kItemsA; i += blockDim.x) {
      const int gg = i % G;
      const int r = i / G;
      const int c = r % 3, n1 = r / 3;
      const int ky = ky0 + gg;
      C x[RA], o[2 * RA];
#pragma unroll
      for (int j = 0; j < RA; ++j) {
        const int zz = n1 + LB * j;
        x[j] = (zz < nz && ky < py) ? wb[c * cstride + (int64_t)zz * g.ys + ky] : czero<C>();
      }
      f2::passA_fwd<PZ>(x, n1, tw, o);
#pragma unroll
      for (int bb = 0; bb < 2; ++bb)
#pragma unroll
        for (int k = 0; k < RA; ++k) s[((bb * H + n1 + LB * k) * 3 + c) * G + gg + (bb * RA + k) * P] = o[bb * RA + k];
    }
  }
  __syncthreads();
  const C* gk = d.ghat + (int64_t)kx * PZ * py * 6;
  if constexpr (kFuse) {
    for (int i = threadIdx.x; i < G * 2 * RA; i += blockDim.x) {
      const int gg = i % G, blk = i / G;
      const int ky = ky0 + gg;
      C v0[LB], v1[LB], v2[LB];
#pragma unroll
      for (int e = 0; e < LB; ++e) {
        const C* q = s + ((blk * LB + e) * 3) * G + gg + blk * P;
        v0[e] = q[0];
        v1[e] = q[G];
        v2[e] = q[2 * G];
      }
      f2::passB_fwd<PZ>(v0, tw);
      f2::passB_fwd<PZ>(v1, tw);
      f2::passB_fwd<PZ>(v2, tw);
      if (ky < py) {
#pragma unroll
        for (int e = 0; e < LB; ++e) gmul3(gk + ((int64_t)(blk * LB + e) * py + ky) * 6, v0[e], v1[e], v2[e]);
      }
      f2::passB_inv<PZ>(v0, tw);
      f2::passB_inv<PZ>(v1, tw);
      f2::passB_inv<PZ>(v2, tw);
#pragma unroll
      for (int e = 0; e < LB; ++e) {
        C* q = s + ((blk * LB + e) * 3) * G + gg + blk * P;
        q[0] = v0[e];
        q[G] = v1[e];
        q[2 * G] = v2[e];
      }
    }
  } else {
    for (int i = threadIdx.x; i < 3 * G * 2 * RA; i += blockDim.x) {
      const int gg = i % G;
      const int r = i / G;
      const int c = r % 3, blk = r / 3;
      C v[LB];
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = s[((blk * LB + e) * 3 + c) * G + gg + blk * P];
      f2::passB_fwd<PZ>(v, tw);
#pragma unroll
      for (int e = 0; e < LB; ++e) s[((blk * LB + e) * 3 + c) * G + gg + blk * P] = v[e];
    }
    __syncthreads();
    // Ghat multiply: each thread's Ghat records come from L2 (HBM once per batch); the loads of
    // kGBatch items are issued together before their arithmetic so their latencies overlap
    constexpr int kGBatch = 4;
    for (int i0 = threadIdx.x; i0 < PZ * G; i0 += kGBatch * blockDim.x) {
      C gv[kGBatch][6];
      bool ok[kGBatch];
#pragma unroll
      for (int u = 0; u < kGBatch; ++u) {
        const int i = i0 + u * blockDim.x;
        const int gg = i % G, kz = i / G;
        ok[u] = i < PZ * G && ky0 + gg < py;
        if (ok[u]) load6(gk + ((int64_t)kz * py + ky0 + gg) * 6, gv[u]);
      }
#pragma unroll
      for (int u = 0; u < kGBatch; ++u) {
        if (!ok[u]) continue;
        const int i = i0 + u * blockDim.x;
        const int gg = i % G, kz = i / G;
        C* q = s + (kz * 3) * G + gg + (kz / LB) * P;
        C v0 = q[0], v1 = q[G], v2 = q[2 * G];
        gmul3_r(gv[u], v0, v1, v2);
        q[0] = v0;
        q[G] = v1;
        q[2 * G] = v2;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * G * 2 * RA; i += blockDim.x) {
      const int gg = i % G;
      const int r = i / G;
      const int c = r % 3, blk = r / 3;
      C v[LB];
#pragma unroll
      for (int e = 0; e < LB; ++e) v[e] = s[((blk * LB + e) * 3 + c) * G + gg + blk * P];
      f2::passB_inv<PZ>(v, tw);
#pragma unroll
      for (int e = 0; e < LB; ++e) s[((blk * LB + e) * 3 + c) * G + gg + blk * P] = v[e];
    }
  }
  __syncthreads();
  // inverse pass A to global (z < nz)
  for (int i = threadIdx.x; i < 3 * G * LB; i += blockDim.x) {
    const int gg = i % G;
    const int r = i / G;
    const int c = r % 3, n1 = r / 3;
    const int ky = ky0 + gg;
    C v[2 * RA], lo[RA];
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int k = 0; k < RA; ++k) v[bb * RA + k] = s[((bb * H + n1 + LB * k) * 3 + c) * G + gg + (bb * RA + k) * P];
    f2::passA_inv<PZ, false>(v, n1, tw, lo, (C*)nullptr);
    if (ky < py) {
#pragma unroll
      for (int j = 0; j < RA; ++j) {
        const int zz = n1 + LB * j;
        if (zz < nz) wb[c * cstride + (int64_t)zz * g.ys + ky] = lo[j];
      }
    }
  }
}

// ------------------------------------------------------------------ dispatch
#define DDA_FAST_LENGTHS(X) X(16) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(128) X(160) X(192) X(256) X(320)
#define DDA_FAST_PLANES(X)                                                                               \
  X(16, 16) X(24, 24) X(32, 32) X(40, 40) X(48, 48) X(64, 64) X(80, 80) X(96, 96) X(96, 64) X(64, 96) \
  X(96, 48) X(48, 96) X(64, 32) X(32, 64) X(96, 40) X(80, 40) X(48, 32) X(32, 48)

inline bool fast_length(int L) {
  switch (L) {
#define DDA_CASE(L_) case L_:
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    return true;
    default: return false;
  }
}

inline bool fast_plane_pair(int py, int pz) {
#define DDA_CASE(A, B) if (py == A && pz == B) return true;
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
  return false;
}

// y rows per CTA of the x passes: 128-byte row segments where shared memory allows
template <typename C, int PX> constexpr int x_ty() {
  return sizeof(C) == 8 ? (PX <= 128 ? 16 : 8) : (PX <= 128 ? 8 : 4);
}
inline int x_ty_rt(size_t csize, int px) { return csize == 8 ? (px <= 128 ? 16 : 8) : (px <= 128 ? 8 : 4); }
// the tile heights instantiated besides the default (small batches want more, shorter tiles)
inline bool x_ty_valid(size_t csize, int px, int ty) {
  return ty == x_ty_rt(csize, px) || ty == 4 || (ty == 8 && x_ty_rt(csize, px) > 8);
}
// the one-component variant (each CTA transforms one of the three components) has this tile height
template <typename C> constexpr int x_nc1_ty() { return sizeof(C) == 8 ? 16 : 8; }
inline int x_nc1_ty_rt(size_t csize) { return csize == 8 ? 16 : 8; }
inline int x_nc_pick(const MvTune& t) { return t.xnc == 1 ? 1 : 3; }
inline int x_ty_pick(const MvTune& t, size_t csize, int px) {
  if (x_nc_pick(t) == 1) return x_nc1_ty_rt(csize);
  return (t.xty > 0 && x_ty_valid(csize, px, t.xty)) ? t.xty : x_ty_rt(csize, px);
}

// z columns per CTA of the 5-pass z kernel: widest tile under ~110 KB of shared memory
constexpr int zcols_g_rt(size_t csize, int pz) {
  return (size_t)pz * 3 * 32 * csize <= 110 * 1024 ? 32 : ((size_t)pz * 3 * 16 * csize <= 110 * 1024 ? 16 : 8);
}

inline int odd_pitch(int n) { return (n % 2) ? n : n + 1; }

template <typename C>
size_t x_fast_smem(const Geom& g, int TY = 0, int NC = 3) {
  if (TY <= 0) TY = x_ty_rt(sizeof(C), g.px);
  return sizeof(C) * ((size_t)g.px + (size_t)NC * TY * odd_pitch(g.nx) + (size_t)NC * g.px * TY);
}
template <typename C>
size_t plane_fast_smem(const Geom& g) {
  return plane_bytes<C>(g.py, g.pz);
}
// the bulk-staged variant: the plane, then its 8-byte mbarrier at the next 16-byte boundary
template <typename C>
size_t plane_bulk_smem(const Geom& g) {
  return ((plane_bytes<C>(g.py, g.pz) + 15) & ~(size_t)15) + 16;
}
// y rows per CTA of the 5-pass y passes: enough that pass A and pass B give every one of the 256
// threads an item (rows x LB = 256), between 8 and 32 rows
template <int PY>
constexpr int y_rows_per_cta() {
  constexpr int r = 256 / Shape<PY>::LB;
  return r < 8 ? 8 : (r > 32 ? 32 : r);
}
inline int y_rows_per_cta_rt(int py) {
  switch (py) {
#define DDA_CASE(L_) case L_: return y_rows_per_cta<L_>();
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return 8;
  }
}
template <typename C>
size_t yrows_fast_smem(const Geom& g) {
  return sizeof(C) * ((size_t)g.py + (size_t)y_rows_per_cta_rt(g.py) * (g.py + 1));
}
template <typename C>
size_t zcols_fast_smem(const Geom& g) {
  switch (g.pz) {
#define DDA_CASE(L_) case L_: return sizeof(C) * zcols_smem_elems<C, L_, zcols_g_rt(sizeof(C), L_)>();
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return sizeof(C) * ((size_t)g.pz + (size_t)g.pz * 3 * zcols_g_rt(sizeof(C), g.pz));
  }
}

// k_x_fwd / k_x_inv for the variant chosen at run time: three components per CTA with tile
// height TY (the default, 4 or 8), or one component per CTA with the one-component height
template <typename C, int L_, typename F>
Err with_x(int nc, int ty, F&& f) {
  constexpr int D = x_ty<C, L_>();
  using I3 = std::integral_constant<int, 3>;
  if (nc == 1) {
    if (ty == x_nc1_ty<C>()) return f(std::integral_constant<int, x_nc1_ty<C>()>{}, std::integral_constant<int, 1>{});
    return Err::make(DDA_EUNSUPPORTED, "x tile height not instantiated");
  }
  if (ty == D) return f(std::integral_constant<int, D>{}, I3{});
  if constexpr (D != 4) {
    if (ty == 4) return f(std::integral_constant<int, 4>{}, I3{});
  }
  if constexpr (D > 8) {
    if (ty == 8) return f(std::integral_constant<int, 8>{}, I3{});
  }
  return Err::make(DDA_EUNSUPPORTED, "x tile height not instantiated");
}

template <typename C>
Err launch_x_fwd(const Geom& g, const MvData<C>& d, const MvTune& t, const typename Io<C>::t* p, int nrhs, bool conj,
                 cudaStream_t st) {
  const int NC = x_nc_pick(t);
  const int TY = x_ty_pick(t, sizeof(C), g.px);
  const size_t sm = x_fast_smem<C>(g, TY, NC);
  const dim3 grid((g.ny + TY - 1) / TY, g.nz, nrhs * (3 / NC));
  const int ip = odd_pitch(g.nx);
  switch (g.px) {
#define DDA_CASE(L_)                                                                                    \
  case L_:                                                                                              \
    DDA_TRY((with_x<C, L_>(NC, TY, [&](auto tyc, auto ncc) {                                          \
      DDA_CU(launch_k(k_x_fwd<C, L_, decltype(tyc)::value, decltype(ncc)::value>, grid, dim3(256), sm, st, g, \
                      d, p, conj, ip));                                                                \
      return Err::Ok();                                                                                 \
    })));                                                                                               \
    break;
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return Err::make(DDA_EUNSUPPORTED, "no fast x kernel for this length");
  }
  DDA_CU(cudaGetLastError());
  return Err::Ok();
}

template <typename C>
Err launch_x_inv(const Geom& g, const MvData<C>& d, const MvTune& t, const typename Io<C>::t* p,
                 typename Io<C>::t* ap, int nrhs, int rhs0, bool conj, cudaStream_t st) {
  const int NC = x_nc_pick(t);
  const int TY = x_ty_pick(t, sizeof(C), g.px);
  const size_t sm = x_fast_smem<C>(g, TY, NC);
  const dim3 grid((g.ny + TY - 1) / TY, g.nz, nrhs * (3 / NC));
  const int ip = odd_pitch(g.nx);
  switch (g.px) {
#define DDA_CASE(L_)                                                                                         \
  case L_:                                                                                                   \
    DDA_TRY((with_x<C, L_>(NC, TY, [&](auto tyc, auto ncc) {                                               \
      DDA_CU(launch_k(k_x_inv<C, L_, decltype(tyc)::value, decltype(ncc)::value>, grid, dim3(256), sm, st, g, d, \
                      p, ap, rhs0, conj, ip));                                                               \
      return Err::Ok();                                                                                      \
    })));                                                                                                    \
    break;
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return Err::make(DDA_EUNSUPPORTED, "no fast x kernel for this length");
  }
  DDA_CU(cudaGetLastError());
  return Err::Ok();
}

// complex64 only: a complex128 plane does not fit in shared memory at these sizes
template <typename C>
Err launch_plane(const Geom& g, const MvData<C>& d, int nrhs, int nt, cudaStream_t st) {
  if constexpr (sizeof(C) == 8) {
    const size_t sm = plane_fast_smem<C>(g);
    const dim3 grid(nrhs, g.px);
#define DDA_CASE(A, B)                                               \
    if (g.py == A && g.pz == B) {                                    \
      if (nt == 768) DDA_CU(launch_k(k_yz_plane<C, A, B, 768, false>, grid, dim3(768), sm, st, g, d)); \
      else DDA_CU(launch_k(k_yz_plane<C, A, B, 512, false>, grid, dim3(512), sm, st, g, d));             \
      DDA_CU(cudaGetLastError());                                    \
      return Err::Ok();                                              \
    }
    DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
  }
  return Err::make(DDA_EUNSUPPORTED, "no fast plane kernel for this pair");
}

template <typename C>
Err launch_y_rows(const Geom& g, C* work, const C* tw, int64_t nrows, bool inv, cudaStream_t st) {
  const size_t sm = yrows_fast_smem<C>(g);
  const int rpb = y_rows_per_cta_rt(g.py);
  const unsigned nb = (unsigned)((nrows + rpb - 1) / rpb);
  switch (g.py) {
#define DDA_CASE(L_)                                                                            \
  case L_:                                                                                      \
    if (inv) DDA_CU(launch_k(k_y_rows<C, L_, y_rows_per_cta<L_>(), true>, dim3(nb), dim3(256), sm, st, g, work, tw, \
                             nrows));                                                           \
    else DDA_CU(launch_k(k_y_rows<C, L_, y_rows_per_cta<L_>(), false>, dim3(nb), dim3(256), sm, st, g, work, tw,    \
                         nrows));                                                               \
    break;
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return Err::make(DDA_EUNSUPPORTED, "no fast y kernel for this length");
  }
  DDA_CU(cudaGetLastError());
  return Err::Ok();
}

// register-fused z columns (RFUSE): complex64 lengths whose pass-B sub-block is too long for the
// default fused loop; 8 columns per CTA, one (column, sub-block) item per thread
constexpr int kZrG = 8;
template <typename C>
constexpr bool zcols_rfuse_exists(int pz) {
  return sizeof(C) == 8 && (pz == 160 || pz == 320);
}

template <typename C>
Err launch_z_cols(const Geom& g, const MvData<C>& d, int nrhs, cudaStream_t st, bool rfuse = false) {
  if constexpr (sizeof(C) == 8) {
    if (rfuse && zcols_rfuse_exists<C>(g.pz)) {
      const size_t sm = sizeof(C) * (g.pz == 160 ? zcols_smem_elems<C, 160, kZrG>() : zcols_smem_elems<C, 320, kZrG>());
      const dim3 grid(nrhs, (g.py + kZrG - 1) / kZrG, g.px);
      if (g.pz == 160)
        DDA_CU(launch_k(k_z_cols<C, 160, kZrG, kZrG * 2 * Shape<160>::RA, true>, grid,
                        dim3(kZrG * 2 * Shape<160>::RA), sm, st, g, d));
      else
        DDA_CU(launch_k(k_z_cols<C, 320, kZrG, kZrG * 2 * Shape<320>::RA, true>, grid,
                        dim3(kZrG * 2 * Shape<320>::RA), sm, st, g, d));
      DDA_CU(cudaGetLastError());
      return Err::Ok();
    }
  }
  const size_t sm = zcols_fast_smem<C>(g);
  const int G = zcols_g_rt(sizeof(C), g.pz);
  const dim3 grid(nrhs, (g.py + G - 1) / G, g.px);
  switch (g.pz) {
#define DDA_CASE(L_)                                                                      \
  case L_:                                                                                \
    DDA_CU(launch_k(k_z_cols<C, L_, zcols_g_rt(sizeof(C), L_)>, grid, dim3(256), sm, st, g, d)); \
    break;
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return Err::make(DDA_EUNSUPPORTED, "no fast z kernel for this length");
  }
  DDA_CU(cudaGetLastError());
  return Err::Ok();
}

template <typename C, int L_>
void optin_x(int smax) {
  constexpr int D = x_ty<C, L_>();
  optin_smem(k_x_fwd<C, L_, D>, smax);
  optin_smem(k_x_inv<C, L_, D>, smax);
  if constexpr (D != 4) {
    optin_smem(k_x_fwd<C, L_, 4>, smax);
    optin_smem(k_x_inv<C, L_, 4>, smax);
  }
  if constexpr (D > 8) {
    optin_smem(k_x_fwd<C, L_, 8>, smax);
    optin_smem(k_x_inv<C, L_, 8>, smax);
  }
  optin_smem(k_x_fwd<C, L_, x_nc1_ty<C>(), 1>, smax);
  optin_smem(k_x_inv<C, L_, x_nc1_ty<C>(), 1>, smax);
}

// Opt every instantiation of this precision into the device's maximum dynamic shared memory.
template <typename C>
void optin_all(int smax) {
#define DDA_CASE(L_)                                                                                                 \
  optin_x<C, L_>(smax);                                                                                              \
  optin_smem(k_y_rows<C, L_, y_rows_per_cta<L_>(), false>, smax);   \
  optin_smem(k_y_rows<C, L_, y_rows_per_cta<L_>(), true>, smax);    \
  optin_smem(k_z_cols<C, L_, zcols_g_rt(sizeof(C), L_)>, smax);
  DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
  if constexpr (sizeof(C) == 8) {
#define DDA_CASE(A, B)                                                                                    \
  optin_smem(k_yz_plane<C, A, B, 512, false>, smax);     \
  optin_smem(k_yz_plane<C, A, B, 768, false>, smax);
    DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
    optin_smem(k_z_cols<C, 160, kZrG, kZrG * 2 * Shape<160>::RA, true>, smax);
    optin_smem(k_z_cols<C, 320, kZrG, kZrG * 2 * Shape<320>::RA, true>, smax);
  }
}

// The passes between the x passes: the fused y-z plane pass (3-pass schedule, complex64 variants:
// single CTA, cluster-split, bulk-staged), or y rows, z columns, y rows (5-pass).
template <typename C>
Err launch_middle(const Geom& g, const MvData<C>& d, const MvTune& t, int nrhs, cudaStream_t st, int& pass) {
  if (t.plane) {
    if constexpr (sizeof(C) == 8) {
      if (t.clus > 1) {
        DDA_TRY(launch_plane_cluster_c64(g, d, t.clus, nrhs, st));
      } else if (t.bulk) {
        DDA_TRY(launch_plane_bulk_c64(g, d, nrhs, st));
      } else {
        DDA_TRY(launch_plane<C>(g, d, nrhs, t.thr_p, st));
      }
    } else {
      DDA_TRY(launch_plane<C>(g, d, nrhs, t.thr_p, st));
    }
    mark_pass(pass++, st);
    add_launches(3);
  } else {
    const int64_t nrows = (int64_t)nrhs * 3 * g.px * g.nz;
    DDA_TRY(launch_y_rows<C>(g, d.work, d.twy, nrows, false, st));
    mark_pass(pass++, st);
    DDA_TRY(launch_z_cols<C>(g, d, nrhs, st, t.zr != 0));
    mark_pass(pass++, st);
    DDA_TRY(launch_y_rows<C>(g, d.work, d.twy, nrows, true, st));
    mark_pass(pass++, st);
    add_launches(5);
  }
  return Err::Ok();
}

// The whole product on the compile-time-length kernels (3-pass when t.plane, else 5-pass).
template <typename C>
Err launch_matvec_fast(const Geom& g, const MvData<C>& d, const MvTune& t, const typename Io<C>::t* p,
                       typename Io<C>::t* ap, int nrhs, int rhs0, bool conj, cudaStream_t st) {
  int pass = 0;
  mark_pass(pass++, st);
  DDA_TRY(launch_x_fwd<C>(g, d, t, p, nrhs, conj, st));
  mark_pass(pass++, st);
  DDA_TRY(launch_middle<C>(g, d, t, nrhs, st, pass));
  DDA_TRY(launch_x_inv<C>(g, d, t, p, ap, nrhs, rhs0, conj, st));
  mark_pass(pass++, st);
  return Err::Ok();
}

// ------------------------------------------------------------------ BiCGstab half-iterations, folded (complex64)
// x-pass CTAs per RHS of the schedule t (the reduction slots of the folded dot products)
inline int x_ctas_per_rhs(const Geom& g, const MvTune& t) {
  const int NC = x_nc_pick(t);
  const int TY = x_ty_pick(t, sizeof(float2), g.px);
  return ((g.ny + TY - 1) / TY) * g.nz * (3 / NC);
}

template <int MODE, bool FWD>
Err launch_x_fused(const Geom& g, const MvData<float2>& d, const MvTune& t, const KrylovVecs<float2>& kv, KState* ks,
                   const RedBuf& rbx, int nrhs, cudaStream_t st) {
  const int NC = x_nc_pick(t);
  const int TY = x_ty_pick(t, sizeof(float2), g.px);
  const size_t sm = x_fast_smem<float2>(g, TY, NC);
  const dim3 grid((g.ny + TY - 1) / TY, g.nz, nrhs * (3 / NC));
  const int ip = odd_pitch(g.nx);
  switch (g.px) {
#define DDA_CASE(L_)                                                                                      \
  case L_:                                                                                                \
    DDA_TRY((with_x<float2, L_>(NC, TY, [&](auto tyc, auto ncc) {                                        \
      constexpr int TY_ = decltype(tyc)::value, NC_ = decltype(ncc)::value;                               \
      if constexpr (FWD)                                                                                  \
        DDA_CU(launch_k(k_x_fwd_fused<L_, TY_, NC_, MODE>, grid, dim3(256), sm, st, g, d, kv, ks, rbx, ip)); \
      else                                                                                                \
        DDA_CU(launch_k(k_x_inv_fused<L_, TY_, NC_, MODE>, grid, dim3(256), sm, st, g, d, kv, ks, rbx, ip)); \
      return Err::Ok();                                                                                   \
    })));                                                                                                 \
    break;
    DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
    default: return Err::make(DDA_EUNSUPPORTED, "no fast x kernel for this length");
  }
  DDA_CU(cudaGetLastError());
  return Err::Ok();
}

template <int L_>
void optin_x_fused(int smax) {
  constexpr int D = x_ty<float2, L_>();
  auto all_modes = [&](auto tyc, auto ncc) {
    constexpr int TY_ = decltype(tyc)::value, NC_ = decltype(ncc)::value;
    optin_smem(k_x_fwd_fused<L_, TY_, NC_, kFuseP>, smax);
    optin_smem(k_x_fwd_fused<L_, TY_, NC_, kFuseS>, smax);
    optin_smem(k_x_inv_fused<L_, TY_, NC_, kFuseRV>, smax);
    optin_smem(k_x_inv_fused<L_, TY_, NC_, kFuseTS>, smax);
  };
  using I3 = std::integral_constant<int, 3>;
  all_modes(std::integral_constant<int, D>{}, I3{});
  if constexpr (D != 4) all_modes(std::integral_constant<int, 4>{}, I3{});
  if constexpr (D > 8) all_modes(std::integral_constant<int, 8>{}, I3{});
  all_modes(std::integral_constant<int, x_nc1_ty<float2>()>{}, std::integral_constant<int, 1>{});
}

}  // namespace fast
}  // namespace dda
