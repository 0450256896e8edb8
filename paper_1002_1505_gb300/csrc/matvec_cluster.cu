// The fused y-z plane pass of the complex64 product, split over a thread-block
// cluster (3-pass schedule, same workspace layout and results as k_yz_plane).
//
// One kx plane of one right-hand side needs the 3-component y-z spectrum in
// shared memory (3 * PZ * PY complex), which leaves room for a single CTA per
// SM and no overlap between its load, FFT and store phases.  After the first
// two stages of the forward y transform (pass A: radix 2 fused with radix RA)
// the 2*RA pass-B sub-blocks of every row are independent, and so are the z
// transforms, the Ghat multiply and the inverse z transforms of different ky
// columns.  So the plane's spectral columns are divided among the S CTAs of a
// cluster: CTA h owns columns [h*PY/S, (h+1)*PY/S) (2*RA/S whole sub-blocks).
// Only pass A crosses CTAs: the forward pass A scatters each row's outputs to
// the owners' shared memory, and the inverse pass A gathers them back, both
// through distributed shared memory.  Each CTA then holds 1/S of the plane, so
// several CTAs share an SM and their phases overlap.
//
// grid (S, nrhs, px), cluster (S, 1, 1).  smem: twy[PY] | twz[PZ] | pl[PZ*3][RP]
#include <cooperative_groups.h>

#include "matvec_fast.cuh"

namespace dda {
namespace fast {

namespace cg = cooperative_groups;

constexpr int odd_pitch_c(int n) { return (n % 2) ? n : n + 1; }

template <int S> struct ClusterCfg;
template <> struct ClusterCfg<2> { static constexpr int NT = 384, MINB = 2; };
template <> struct ClusterCfg<4> { static constexpr int NT = 256, MINB = 3; };

template <typename C, int PY, int PZ, int S>
__global__ void __launch_bounds__(ClusterCfg<S>::NT, ClusterCfg<S>::MINB) k_yz_cluster(Geom g, MvData<C> d) {
  constexpr int NT = ClusterCfg<S>::NT;
  constexpr int RAy = Shape<PY>::RA, LBy = Shape<PY>::LB;
  constexpr int RAz = Shape<PZ>::RA, LBz = Shape<PZ>::LB, Hz = Shape<PZ>::H;
  static_assert((2 * RAy) % S == 0, "the cluster size must divide the pass-B sub-block count");
  constexpr int SBS = 2 * RAy / S;  // pass-B sub-blocks per CTA
  constexpr int PYS = PY / S;       // spectral columns per CTA
  constexpr int RP = odd_pitch_c(PYS);
  extern __shared__ unsigned char smem_raw[];
  C* twy = reinterpret_cast<C*>(smem_raw);
  C* twz = twy + PY;
  C* pl = twz + PZ;
  const int b = blockIdx.y, kx = blockIdx.z;
  if (rhs_done(d, b)) return;  // every CTA of the cluster has the same b: none waits at a cluster barrier
  cg::cluster_group cl = cg::this_cluster();
  const int h = (int)cl.block_rank();
  const int nz = g.nz, ny = g.ny;
  copy_tw(twy, d.twy, PY);
  copy_tw(twz, d.twz, PZ);
  C* peer[S];
#pragma unroll
  for (int r = 0; r < S; ++r) peer[r] = cl.map_shared_rank(pl, r);
  cl.sync();  // every CTA of the cluster runs (its shared memory exists) and has its twiddles
  C* wb = d.work + ((int64_t)b * 3 * g.px + kx) * ((int64_t)nz * g.ys);
  const int64_t cstride = (int64_t)g.px * nz * g.ys;
  const int R = 3 * nz;  // rows (z, c) with z < nz; row index z*3 + c
  const int r0 = h * R / S, r1 = (h + 1) * R / S;
  // y forward, pass A on this CTA's share of the rows; sub-block s of a row goes to CTA s / SBS
  for (int i = threadIdx.x; i < (r1 - r0) * LBy; i += NT) {
    const int n1 = i % LBy;
    const int r = r0 + i / LBy;
    const int z = r % nz, c = r / nz;
    const C* src = wb + c * cstride + (int64_t)z * g.ys;
    C x[RAy], o[2 * RAy];
#pragma unroll
    for (int j = 0; j < RAy; ++j) {
      const int yy = n1 + LBy * j;
      x[j] = (yy < ny) ? src[yy] : czero<C>();
    }
    f2::passA_fwd<PY>(x, n1, twy, o);
    const int row = (z * 3 + c) * RP + n1;
#pragma unroll
    for (int s = 0; s < 2 * RAy; ++s) peer[s / SBS][row + (s % SBS) * LBy] = o[s];
  }
  cl.sync();
  // y forward, pass B on the local sub-blocks
  for (int i = threadIdx.x; i < R * SBS; i += NT) {
    const int rr = i % R, blk = i / R;
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
  for (int i = threadIdx.x; i < 3 * PYS * LBz; i += NT) {
    const int ky = i % PYS;
    const int r = i / PYS;
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
  // z pass B, Ghat, inverse z pass B in registers for the three components
  const C* gk = d.ghat + (int64_t)kx * PZ * PY * 6 + (int64_t)h * PYS * 6;
  for (int i = threadIdx.x; i < PYS * 2 * RAz; i += NT) {
    const int ky = i % PYS, blk = i / PYS;
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
  for (int i = threadIdx.x; i < 3 * PYS * LBz; i += NT) {
    const int ky = i % PYS;
    const int r = i / PYS;
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
  // y inverse, pass B on the local sub-blocks
  for (int i = threadIdx.x; i < R * SBS; i += NT) {
    const int rr = i % R, blk = i / R;
    C* row = pl + rr * RP + blk * LBy;
    C v[LBy];
#pragma unroll
    for (int e = 0; e < LBy; ++e) v[e] = row[e];
    f2::passB_inv<PY>(v, twy);
#pragma unroll
    for (int e = 0; e < LBy; ++e) row[e] = v[e];
  }
  cl.sync();
  // y inverse, pass A on this CTA's rows, gathering the sub-blocks from their owners
  for (int i = threadIdx.x; i < (r1 - r0) * LBy; i += NT) {
    const int n1 = i % LBy;
    const int r = r0 + i / LBy;
    const int z = r % nz, c = r / nz;
    const int row = (z * 3 + c) * RP + n1;
    C v[2 * RAy], lo[RAy];
#pragma unroll
    for (int s = 0; s < 2 * RAy; ++s) v[s] = peer[s / SBS][row + (s % SBS) * LBy];
    f2::passA_inv<PY, false>(v, n1, twy, lo, (C*)nullptr);
    C* dst = wb + c * cstride + (int64_t)z * g.ys;
#pragma unroll
    for (int j = 0; j < RAy; ++j) {
      const int yy = n1 + LBy * j;
      if (yy < ny) dst[yy] = lo[j];
    }
  }
  cl.sync();  // the other CTAs may still be reading this CTA's shared memory
}

template <int PY, int PZ>
constexpr bool cluster_ok(int S) {
  return (2 * Shape<PY>::RA) % S == 0 && PY % S == 0;
}

size_t cluster_smem(const Geom& g, int S) {
  const int pys = g.py / S;
  return sizeof(float2) * ((size_t)g.py + g.pz + (size_t)g.pz * 3 * odd_pitch_c(pys));
}

template <int PY, int PZ, int S>
Err launch_one(const Geom& g, const MvData<float2>& d, int nrhs, cudaStream_t st) {
  if constexpr (!cluster_ok<PY, PZ>(S)) {
    return Err::make(DDA_EUNSUPPORTED, "cluster size does not divide this plane");
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S, nrhs, g.px);
    cfg.blockDim = dim3(ClusterCfg<S>::NT);
    cfg.dynamicSmemBytes = cluster_smem(g, S);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DDA_CU(cudaLaunchKernelEx(&cfg, k_yz_cluster<float2, PY, PZ, S>, g, d));
    return Err::Ok();
  }
}

template <int PY, int PZ, int S>
int max_clusters(const Geom& g) {
  if constexpr (!cluster_ok<PY, PZ>(S)) {
    return 0;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S, 1, g.px);
    cfg.blockDim = dim3(ClusterCfg<S>::NT);
    cfg.dynamicSmemBytes = cluster_smem(g, S);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_yz_cluster<float2, PY, PZ, S>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }
}

}  // namespace fast

Err launch_plane_cluster_c64(const Geom& g, const MvData<float2>& d, int S, int nrhs, cudaStream_t st) {
#define DDA_CASE(A, B)                                                       \
  if (g.py == A && g.pz == B) {                                              \
    if (S == 2) return fast::launch_one<A, B, 2>(g, d, nrhs, st);           \
    if (S == 4) return fast::launch_one<A, B, 4>(g, d, nrhs, st);           \
  }
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
  return Err::make(DDA_EUNSUPPORTED, "no cluster plane kernel for this pair");
}

int plane_cluster_capacity_c64(const Geom& g, int S, int smax) {
  if (fast::cluster_smem(g, S) > (size_t)smax) return 0;
#define DDA_CASE(A, B)                                                 \
  if (g.py == A && g.pz == B) {                                        \
    if (S == 2) return fast::max_clusters<A, B, 2>(g);                 \
    if (S == 4) return fast::max_clusters<A, B, 4>(g);                 \
  }
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
  return 0;
}

namespace fast {
template <int A, int B>
void optin_pair(int smax) {
  if constexpr (cluster_ok<A, B>(2))
    optin_smem(k_yz_cluster<float2, A, B, 2>, smax);
  if constexpr (cluster_ok<A, B>(4))
    optin_smem(k_yz_cluster<float2, A, B, 4>, smax);
}
}  // namespace fast

void cluster_optin_c64(int smax) {
#define DDA_CASE(A, B) fast::optin_pair<A, B>(smax);
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
}

}  // namespace dda
