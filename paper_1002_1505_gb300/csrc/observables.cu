// Incident field and scattering observables on the device.
//
// E_inc,j = e exp(i k . r_j) (guide, "Incident Polarization State"; plane wave
// along x_LF, expressed in the Target Frame), phase in FP64.
// Efficiency sums (Draine 1988, the formulas behind the guide's Q_ext, Q_abs,
// Q_pha), per RHS, FP64 accumulation, from the cached incident field:
//   S_ext = sum_j Im(E_j^* . P_j),  S_pha = sum_j Re(E_j^* . P_j),
//   S_abs = sum_j sum_a (-Im(alpha^{-1}_aa) - (2/3) k^3) |P_ja|^2
// (the host scales them by 4 pi k, 2 pi k and 4 pi k and divides by pi a_eff^2).
// Far field: F(n) = sum_j P_j exp(-i k n . r_j), from which the host forms
// f_ml = k^3 e_m . F (guide, eq. f_ml_def) and the Mueller matrix.
#include <algorithm>

#include "dda_internal.h"

namespace dda {

namespace {

constexpr int kT = 256;

template <typename C> __device__ __forceinline__ C mkc(double x, double y);
template <> __device__ __forceinline__ float2 mkc<float2>(double x, double y) { return make_float2((float)x, (float)y); }
template <> __device__ __forceinline__ double2 mkc<double2>(double x, double y) { return make_double2(x, y); }

template <typename C>
__global__ void k_einc(const int32_t* ijk, const double* org, const RhsGeom* rg, int64_t n, C* e) {
  const int b = blockIdx.y;
  const RhsGeom g = rg[b];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double rx = ijk[3 * j] + org[0], ry = ijk[3 * j + 1] + org[1], rz = ijk[3 * j + 2] + org[2];
    const double ph = g.k[0] * rx + g.k[1] * ry + g.k[2] * rz;
    double sn, cs;
    sincos(ph, &sn, &cs);
    for (int c = 0; c < 3; ++c) {
      const double er = g.e[2 * c], ei = g.e[2 * c + 1];
      e[((int64_t)b * 3 + c) * n + j] = mkc<C>(er * cs - ei * sn, er * sn + ei * cs);
    }
  }
}

template <int NS>
__device__ __forceinline__ void bred(double (&v)[NS], double* out) {
  __shared__ double red[NS][kT / 32];
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

// efficiency sums from the cached incident field e [nrhs][3][N]
__global__ void k_qsum(const uint8_t* comp, const double2* __restrict__ e, const double2* ia, int ncomp, double kd,
                       const double2* p, int64_t n, double* part) {
  const int b = blockIdx.y;
  const double rr = (2.0 / 3.0) * kd * kd * kd;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const int cc = comp ? comp[3 * j + c] : 0;  // composition of axis c
      const double2 ev = e[((int64_t)b * 3 + c) * n + j];
      const double2 pv = p[((int64_t)b * 3 + c) * n + j];
      // conj(E) * P
      const double re = ev.x * pv.x + ev.y * pv.y, im = ev.x * pv.y - ev.y * pv.x;
      acc[0] += im;
      acc[1] += re;
      const double2 a = ia[((int64_t)b * ncomp + cc) * 3 + c];
      acc[2] += (-a.y - rr) * (pv.x * pv.x + pv.y * pv.y);
    }
  }
  bred<3>(acc, part + ((int64_t)b * gridDim.x + blockIdx.x) * 4);
}

// the same sums for sites with a full symmetric alpha^{-1} (rotated dielectric frames):
// S_abs = sum_j { Im[P_j . (alpha_j^{-1})^* P_j^*] - (2/3) k^3 |P_j|^2 }
__global__ void k_qsum_t(const double2* __restrict__ e, const double2* __restrict__ iat, double kd,
                         const double2* __restrict__ p, int64_t n, double* part) {
  const int b = blockIdx.y;
  const double rr = (2.0 / 3.0) * kd * kd * kd;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double2 P[3];
    for (int c = 0; c < 3; ++c) {
      const double2 ev = e[((int64_t)b * 3 + c) * n + j];
      const double2 pv = p[((int64_t)b * 3 + c) * n + j];
      P[c] = pv;
      acc[0] += ev.x * pv.y - ev.y * pv.x;
      acc[1] += ev.x * pv.x + ev.y * pv.y;
      acc[2] -= rr * (pv.x * pv.x + pv.y * pv.y);
    }
    const double2* m6 = iat + ((int64_t)b * n + j) * 6;
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        const int lo = a < c ? a : c, hi = a < c ? c : a;
        const double2 m = m6[lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)];
        // Im[P_a conj(M_ac) conj(P_c)]
        const double2 t = make_double2(P[a].x * m.x + P[a].y * m.y, P[a].y * m.x - P[a].x * m.y);  // P_a conj(M)
        acc[2] += t.y * P[c].x - t.x * P[c].y;
      }
  }
  bred<3>(acc, part + ((int64_t)b * gridDim.x + blockIdx.x) * 4);
}

__global__ void k_qsum_fin(const double* part, int nblk, double* out3) {
  const int b = blockIdx.x;
  double v[3] = {0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
    for (int s = 0; s < 3; ++s) v[s] += part[((int64_t)b * nblk + i) * 4 + s];
  __shared__ double res[3];
  bred<3>(v, res);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < 3; ++s) out3[3 * b + s] = res[s];
}

// grid (nblk, ndir, nrhs): partial sums of P_j exp(-i k n.r_j) -> part[rhs][dir][blk][6], FP64.
// The phase factorises over the lattice axes, so each CTA first tabulates
// exp(-i k n_a (i + origin_a)) for its direction (box sum entries), then needs two
// complex products per site instead of a sine and cosine.
__global__ void k_far(const int32_t* ijk, const double* org, const double* nhat, double kd, const double2* p,
                      int ndir, int64_t n, int bx, int by, int bz, double* part) {
  extern __shared__ double2 ftab[];
  const int d = blockIdx.y, b = blockIdx.z;
  const double* nh = nhat + ((int64_t)b * ndir + d) * 3;
  const int nt = bx + by + bz;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const int a = i < bx ? 0 : (i < bx + by ? 1 : 2);
    const int ii = a == 0 ? i : (a == 1 ? i - bx : i - bx - by);
    double sn, cs;
    sincos(-kd * nh[a] * ((double)ii + org[a]), &sn, &cs);
    ftab[i] = make_double2(cs, sn);
  }
  __syncthreads();
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double2 tx = ftab[ijk[3 * j]], ty = ftab[bx + ijk[3 * j + 1]], tz = ftab[bx + by + ijk[3 * j + 2]];
    const double2 txy = make_double2(tx.x * ty.x - tx.y * ty.y, tx.x * ty.y + tx.y * ty.x);
    const double cs = txy.x * tz.x - txy.y * tz.y, sn = txy.x * tz.y + txy.y * tz.x;
    for (int c = 0; c < 3; ++c) {
      const double2 pv = p[((int64_t)b * 3 + c) * n + j];
      acc[2 * c] += pv.x * cs - pv.y * sn;
      acc[2 * c + 1] += pv.x * sn + pv.y * cs;
    }
  }
  bred<6>(acc, part + (((int64_t)b * ndir + d) * gridDim.x + blockIdx.x) * 6);
}

__global__ void k_far_fin(const double* part, int nblk, double2* out) {
  const int o = blockIdx.x;  // rhs * ndir + dir
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
    for (int s = 0; s < 6; ++s) v[s] += part[((int64_t)o * nblk + i) * 6 + s];
  __shared__ double res[6];
  bred<6>(v, res);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) out[(int64_t)o * 3 + c] = make_double2(res[2 * c], res[2 * c + 1]);
}

// ------------------------------------------------------------------ many scattering directions
// The far-field phase of a lattice site factorises over the axes:
// exp(-i k n.r) = T_x[i] T_y[j] T_z[l] with T_a[i] = exp(-i k n_a (i + origin_a)); the tables
// are built in FP64 and stored in FP32, one set per (RHS, direction):
// tab[rd * nt + {0 | bx | bx + by} + i], nt = bx + by + bz.
__global__ void k_phase_tables(const double* __restrict__ nhat, int64_t nrd, const double* __restrict__ org, double kd,
                               int bx, int by, int bz, float2* __restrict__ tab) {
  const int nt = bx + by + bz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nrd * nt; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rd = t / nt;
    const int i = (int)(t - rd * nt);
    int a, ii;
    if (i < bx) { a = 0; ii = i; }
    else if (i < bx + by) { a = 1; ii = i - bx; }
    else { a = 2; ii = i - bx - by; }
    double sn, cs;
    sincos(-kd * nhat[rd * 3 + a] * ((double)ii + org[a]), &sn, &cs);
    tab[t] = make_float2((float)cs, (float)sn);
  }
}

// F[rhs][d] = sum_j P_j exp(-i k n_d . r_j) for kDirPerCta directions per CTA: grid (site blocks,
// direction chunks, nrhs); per-thread FP32 sums over its sites, then FP64 across the block.
constexpr int kDirPerCta = 8;
__global__ void __launch_bounds__(kT) k_far_many(const int32_t* __restrict__ ijk, const double2* __restrict__ p,
                                                 int64_t n, int ndir, int bx, int by, int bz,
                                                 const float2* __restrict__ tab, double* __restrict__ part) {
  extern __shared__ float2 stab[];
  const int nt = bx + by + bz;
  const int b = blockIdx.z, d0 = blockIdx.y * kDirPerCta;
  const int nd = min(kDirPerCta, ndir - d0);
  const float2* src = tab + ((int64_t)b * ndir + d0) * nt;
  for (int i = threadIdx.x; i < nd * nt; i += blockDim.x) stab[i] = src[i];
  __syncthreads();
  float acc[kDirPerCta][6];
#pragma unroll
  for (int dd = 0; dd < kDirPerCta; ++dd)
#pragma unroll
    for (int s = 0; s < 6; ++s) acc[dd][s] = 0.f;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int ix = ijk[3 * j], iy = bx + ijk[3 * j + 1], iz = bx + by + ijk[3 * j + 2];
    float2 pv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = p[((int64_t)b * 3 + c) * n + j];
      pv[c] = make_float2((float)v.x, (float)v.y);
    }
#pragma unroll
    for (int dd = 0; dd < kDirPerCta; ++dd) {
      if (dd < nd) {
        const float2* t = stab + dd * nt;
        const float2 tx = t[ix], ty = t[iy], tz = t[iz];
        const float2 txy = make_float2(tx.x * ty.x - tx.y * ty.y, tx.x * ty.y + tx.y * ty.x);
        const float2 ph = make_float2(txy.x * tz.x - txy.y * tz.y, txy.x * tz.y + txy.y * tz.x);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          acc[dd][2 * c] = fmaf(pv[c].x, ph.x, fmaf(-pv[c].y, ph.y, acc[dd][2 * c]));
          acc[dd][2 * c + 1] = fmaf(pv[c].x, ph.y, fmaf(pv[c].y, ph.x, acc[dd][2 * c + 1]));
        }
      }
    }
  }
  double v[kDirPerCta * 6];
#pragma unroll
  for (int dd = 0; dd < kDirPerCta; ++dd)
#pragma unroll
    for (int s = 0; s < 6; ++s) v[dd * 6 + s] = (double)acc[dd][s];
  bred<kDirPerCta * 6>(v, part + (((int64_t)b * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (kDirPerCta * 6));
}

// sum the site-block partials: out[rhs][d][3] (complex)
__global__ void k_far_many_fin(const double* __restrict__ part, int nblk, int nchunk, int ndir,
                               double2* __restrict__ out) {
  const int rc = blockIdx.x;  // rhs * nchunk + chunk
  const int b = rc / nchunk, ch = rc - b * nchunk;
  for (int s = threadIdx.x; s < kDirPerCta * 6; s += blockDim.x) {
    double v = 0.0;
    for (int i = 0; i < nblk; ++i) v += part[((int64_t)rc * nblk + i) * (kDirPerCta * 6) + s];
    const int d = ch * kDirPerCta + s / 6;
    if (d < ndir) {
      const int q = s % 6;
      double* o = reinterpret_cast<double*>(out + ((int64_t)b * ndir + d) * 3);
      o[q] = v;
    }
  }
}

// ------------------------------------------------------------------ radiative force and torque
// Far-field moments for the torque: per (RHS, direction) g = sum_j P_j exp(-i k n.r_j) (3 complex)
// and T[c][a] = sum_j (r_j - r_cm)_c P_ja exp(-i k n.r_j) (9 complex), from the same FP32 phase
// tables; grid (site blocks, direction pairs, nrhs); per-thread FP32 sums, FP64 across the block.
constexpr int kMomDir = 2;
constexpr int kMomVals = 24;  // 12 complex per direction
__global__ void __launch_bounds__(kT) k_far_moments(const int32_t* __restrict__ ijk, const double2* __restrict__ p,
                                                    int64_t n, int ndir, int bx, int by, int bz, float sx, float sy,
                                                    float sz, const float2* __restrict__ tab,
                                                    double* __restrict__ part) {
  extern __shared__ float2 stab[];
  const int nt = bx + by + bz;
  const int b = blockIdx.z, d0 = blockIdx.y * kMomDir;
  const int nd = min(kMomDir, ndir - d0);
  const float2* src = tab + ((int64_t)b * ndir + d0) * nt;
  for (int i = threadIdx.x; i < nd * nt; i += blockDim.x) stab[i] = src[i];
  __syncthreads();
  float acc[kMomDir][kMomVals];
#pragma unroll
  for (int dd = 0; dd < kMomDir; ++dd)
#pragma unroll
    for (int s = 0; s < kMomVals; ++s) acc[dd][s] = 0.f;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = ijk[3 * j], i1 = ijk[3 * j + 1], i2 = ijk[3 * j + 2];
    const float rpos[3] = {(float)i0 + sx, (float)i1 + sy, (float)i2 + sz};
    float2 pv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = p[((int64_t)b * 3 + c) * n + j];
      pv[c] = make_float2((float)v.x, (float)v.y);
    }
#pragma unroll
    for (int dd = 0; dd < kMomDir; ++dd) {
      if (dd < nd) {
        const float2* t = stab + dd * nt;
        const float2 tx = t[i0], ty = t[bx + i1], tz = t[bx + by + i2];
        const float2 txy = make_float2(tx.x * ty.x - tx.y * ty.y, tx.x * ty.y + tx.y * ty.x);
        const float2 ph = make_float2(txy.x * tz.x - txy.y * tz.y, txy.x * tz.y + txy.y * tz.x);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float2 q = make_float2(pv[a].x * ph.x - pv[a].y * ph.y, pv[a].x * ph.y + pv[a].y * ph.x);
          acc[dd][2 * a] += q.x;
          acc[dd][2 * a + 1] += q.y;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[dd][6 + 2 * (3 * c + a)] = fmaf(rpos[c], q.x, acc[dd][6 + 2 * (3 * c + a)]);
            acc[dd][6 + 2 * (3 * c + a) + 1] = fmaf(rpos[c], q.y, acc[dd][6 + 2 * (3 * c + a) + 1]);
          }
        }
      }
    }
  }
  double v[kMomDir * kMomVals];
#pragma unroll
  for (int dd = 0; dd < kMomDir; ++dd)
#pragma unroll
    for (int s = 0; s < kMomVals; ++s) v[dd * kMomVals + s] = (double)acc[dd][s];
  bred<kMomDir * kMomVals>(v, part + (((int64_t)b * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) *
                                         (kMomDir * kMomVals));
}

// sum the site-block partials: out[rhs][d][12] (complex: g_x g_y g_z, then T row-major [c][a])
__global__ void k_far_moments_fin(const double* __restrict__ part, int nblk, int nchunk, int ndir,
                                  double2* __restrict__ out) {
  const int rc = blockIdx.x;  // rhs * nchunk + chunk
  const int b = rc / nchunk, ch = rc - b * nchunk;
  for (int s = threadIdx.x; s < kMomDir * kMomVals; s += blockDim.x) {
    double v = 0.0;
    for (int i = 0; i < nblk; ++i) v += part[((int64_t)rc * nblk + i) * (kMomDir * kMomVals) + s];
    const int d = ch * kMomDir + s / kMomVals;
    if (d < ndir) {
      double* o = reinterpret_cast<double*>(out + ((int64_t)b * ndir + d) * 12);
      o[s % kMomVals] = v;
    }
  }
}

// Incident-field part of the force and torque, per RHS (FP64): out7[b] =
// { sum_j Re(P_j x E_j^*) (3), sum_j (r_j - r_cm) Im(P_j . E_j^*) (3), sum_j Im(P_j . E_j^*) }.
__global__ void k_torque_ext(const int32_t* __restrict__ ijk, const double2* __restrict__ e,
                             const double2* __restrict__ p, int64_t n, double sx, double sy, double sz,
                             double* __restrict__ part) {
  const int b = blockIdx.y;
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double2 P[3], E[3];
    for (int c = 0; c < 3; ++c) {
      P[c] = p[((int64_t)b * 3 + c) * n + j];
      E[c] = e[((int64_t)b * 3 + c) * n + j];
    }
    // P x E^*: component a = P_b E_c^* - P_c E_b^*, real part
    for (int a = 0; a < 3; ++a) {
      const int b1 = (a + 1) % 3, c1 = (a + 2) % 3;
      acc[a] += (P[b1].x * E[c1].x + P[b1].y * E[c1].y) - (P[c1].x * E[b1].x + P[c1].y * E[b1].y);
    }
    double im = 0.0;  // Im(P . E^*)
    for (int c = 0; c < 3; ++c) im += P[c].y * E[c].x - P[c].x * E[c].y;
    acc[3] += ((double)ijk[3 * j] + sx) * im;
    acc[4] += ((double)ijk[3 * j + 1] + sy) * im;
    acc[5] += ((double)ijk[3 * j + 2] + sz) * im;
    acc[6] += im;
  }
  bred<7>(acc, part + ((int64_t)b * gridDim.x + blockIdx.x) * 8);
}

__global__ void k_torque_ext_fin(const double* part, int nblk, double* out7) {
  const int b = blockIdx.x;
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblk; i += blockDim.x)
    for (int s = 0; s < 7; ++s) v[s] += part[((int64_t)b * nblk + i) * 8 + s];
  __shared__ double res[7];
  bred<7>(v, res);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < 7; ++s) out7[7 * b + s] = res[s];
}

// ------------------------------------------------------------------ fields in or near the target
// E and B at kNfPts points per CTA from every dipole (retarded point-dipole fields, FP64), the
// contribution of dipoles closer than one lattice spacing scaled by phi(R) = R^4 (5 - 4 R);
// grid (point chunks, nrhs); out[rhs][point][12] = E (re, im) x 3, then B.
constexpr int kNfPts = 4;

// E and B of the point dipole P (complex 3-vector) at separation (dx, dy, dz) from it, times the
// weight w (the near suppression, and for periodic targets the Bloch phase is in P and the cutoff in
// w), added to acc[0..5] (E) and acc[6..11] (B):
//   E = e^{ikR} { k^2 (n x p) x n / R + [3 n (n.p) - p] (1/R^3 - i k/R^2) },  B = e^{ikR} (n x p) (k^2/R + i k/R^2)
__device__ __forceinline__ void dipole_term(double dx, double dy, double dz, const double2 (&P)[3], double kd, double w,
                                            double* acc) {
  const double R2 = dx * dx + dy * dy + dz * dz;
  const double R = sqrt(R2), iR = 1.0 / R;
  const double nv[3] = {dx * iR, dy * iR, dz * iR};
  const double k2 = kd * kd;
  double sn, cs;
  sincos(kd * R, &sn, &cs);
  double2 nxp[3];
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    nxp[a] = make_double2(nv[a1] * P[a2].x - nv[a2] * P[a1].x, nv[a1] * P[a2].y - nv[a2] * P[a1].y);
  }
  const double2 ndp = make_double2(nv[0] * P[0].x + nv[1] * P[1].x + nv[2] * P[2].x,
                                   nv[0] * P[0].y + nv[1] * P[1].y + nv[2] * P[2].y);
  const double2 f = make_double2(iR * iR * iR, -kd * iR * iR);  // (1/R^3 - i k/R^2)
  const double2 ph = make_double2(cs * w, sn * w);
  const double2 gb = make_double2(k2 * iR, kd * iR * iR);
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    // ((n x p) x n)_a = (nxp)_{a1} n_{a2} - (nxp)_{a2} n_{a1}
    const double2 t1 = make_double2((nxp[a1].x * nv[a2] - nxp[a2].x * nv[a1]) * k2 * iR,
                                    (nxp[a1].y * nv[a2] - nxp[a2].y * nv[a1]) * k2 * iR);
    const double2 u = make_double2(3.0 * nv[a] * ndp.x - P[a].x, 3.0 * nv[a] * ndp.y - P[a].y);
    const double2 t2 = make_double2(u.x * f.x - u.y * f.y, u.x * f.y + u.y * f.x);
    const double2 e = make_double2(t1.x + t2.x, t1.y + t2.y);
    acc[2 * a] += e.x * ph.x - e.y * ph.y;
    acc[2 * a + 1] += e.x * ph.y + e.y * ph.x;
    const double2 bb = make_double2(nxp[a].x * gb.x - nxp[a].y * gb.y, nxp[a].x * gb.y + nxp[a].y * gb.x);
    acc[6 + 2 * a] += bb.x * ph.x - bb.y * ph.y;
    acc[6 + 2 * a + 1] += bb.x * ph.y + bb.y * ph.x;
  }
}

// near suppression of a dipole closer than one lattice spacing: (R/d)^4 (5 - 4 R/d)
__device__ __forceinline__ double near_suppression(double R) { return R < 1.0 ? R * R * R * R * (5.0 - 4.0 * R) : 1.0; }

__global__ void __launch_bounds__(kT) k_near_field(const int32_t* __restrict__ ijk, const double* __restrict__ org,
                                                   const double2* __restrict__ p, int64_t n,
                                                   const double* __restrict__ pts, int64_t npts, double kd,
                                                   double* __restrict__ out) {
  const int b = blockIdx.y;
  const int64_t q0 = (int64_t)blockIdx.x * kNfPts;
  double acc[kNfPts * 12];
#pragma unroll
  for (int i = 0; i < kNfPts * 12; ++i) acc[i] = 0.0;
  double xq[kNfPts][3];
#pragma unroll
  for (int q = 0; q < kNfPts; ++q)
    for (int a = 0; a < 3; ++a) xq[q][a] = (q0 + q < npts) ? pts[(q0 + q) * 3 + a] : 1e300;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double r[3] = {ijk[3 * j] + org[0], ijk[3 * j + 1] + org[1], ijk[3 * j + 2] + org[2]};
    double2 P[3];
    for (int c = 0; c < 3; ++c) P[c] = p[((int64_t)b * 3 + c) * n + j];
#pragma unroll
    for (int q = 0; q < kNfPts; ++q) {
      if (q0 + q >= npts) continue;
      const double dx = xq[q][0] - r[0], dy = xq[q][1] - r[1], dz = xq[q][2] - r[2];
      const double R2 = dx * dx + dy * dy + dz * dz;
      if (R2 == 0.0) continue;
      dipole_term(dx, dy, dz, P, kd, near_suppression(sqrt(R2)), acc + q * 12);
    }
  }
  __shared__ double res[kNfPts * 12];
  bred<kNfPts * 12>(acc, res);
  __syncthreads();
  for (int i = threadIdx.x; i < kNfPts * 12; i += blockDim.x) {
    const int q = i / 12;
    if (q0 + q < npts) out[((int64_t)b * npts + q0 + q) * 12 + (i % 12)] = res[i];
  }
}

// Periodic targets: the replicas R = (0, m P_y, l P_z), |m| <= my, |l| <= mz, of every dipole, with
// moment P e^{i k.R} and weight exp[-(gamma k D)^4] on top of the near suppression, terms with
// (gamma k D)^4 > 40 dropped.  grid (nsplit, point chunks, nrhs): CTA s takes every nsplit-th
// block of the (dipole, replica) pairs; part[(b * nsplit + s) * npts + q][12] partial sums, added
// in a fixed order by k_nf_sum.
__global__ void __launch_bounds__(kT) k_near_field_pbc(const int32_t* __restrict__ ijk, const double* __restrict__ org,
                                                       const double2* __restrict__ p, int64_t n,
                                                       const double* __restrict__ pts, int64_t npts, double kd,
                                                       double ky, double kz, double py, double pz, double gamma, int my,
                                                       int mz, double* __restrict__ part) {
  const int s = blockIdx.x, nsplit = gridDim.x, b = blockIdx.z;
  const int64_t q0 = (int64_t)blockIdx.y * kNfPts;
  double acc[kNfPts * 12];
#pragma unroll
  for (int i = 0; i < kNfPts * 12; ++i) acc[i] = 0.0;
  double xq[kNfPts][3];
#pragma unroll
  for (int q = 0; q < kNfPts; ++q)
    for (int a = 0; a < 3; ++a) xq[q][a] = (q0 + q < npts) ? pts[(q0 + q) * 3 + a] : 1e300;
  const int64_t nrep = (int64_t)(2 * my + 1) * (2 * mz + 1);
  const int64_t pairs = n * nrep;
  const double gk = gamma * kd;
  for (int64_t idx = (int64_t)s * blockDim.x + threadIdx.x; idx < pairs; idx += (int64_t)nsplit * blockDim.x) {
    const int64_t j = idx % n, rep = idx / n;
    const int m = (int)(rep / (2 * mz + 1)) - my, l = (int)(rep % (2 * mz + 1)) - mz;
    const double Ry = m * py, Rz = l * pz;
    double sn, cs;
    sincos(ky * Ry + kz * Rz, &sn, &cs);
    const double r[3] = {ijk[3 * j] + org[0], ijk[3 * j + 1] + org[1] + Ry, ijk[3 * j + 2] + org[2] + Rz};
    double2 P[3];
    for (int c = 0; c < 3; ++c) {
      const double2 v = p[((int64_t)b * 3 + c) * n + j];
      P[c] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
    }
#pragma unroll
    for (int q = 0; q < kNfPts; ++q) {
      if (q0 + q >= npts) continue;
      const double dx = xq[q][0] - r[0], dy = xq[q][1] - r[1], dz = xq[q][2] - r[2];
      const double R2 = dx * dx + dy * dy + dz * dz;
      if (R2 == 0.0) continue;
      const double R = sqrt(R2), t = gk * R, t4 = t * t * t * t;
      if (t4 > 40.0) continue;
      dipole_term(dx, dy, dz, P, kd, near_suppression(R) * exp(-t4), acc + q * 12);
    }
  }
  __shared__ double res[kNfPts * 12];
  bred<kNfPts * 12>(acc, res);
  __syncthreads();
  for (int i = threadIdx.x; i < kNfPts * 12; i += blockDim.x) {
    const int q = i / 12;
    if (q0 + q < npts) part[(((int64_t)b * nsplit + s) * npts + q0 + q) * 12 + (i % 12)] = res[i];
  }
}

// out[b][q][i] = sum over s (in order) of part[b][s][q][i]
__global__ void k_nf_sum(const double* __restrict__ part, int nsplit, int64_t npts, int nrhs, double* __restrict__ out) {
  const int64_t total = (int64_t)nrhs * npts * 12;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / (npts * 12), rem = i - b * npts * 12;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[((b * nsplit + s) * npts) * 12 + rem];
    out[i] = acc;
  }
}

}  // namespace

Err near_field(const int32_t* ijk, const double* origin3, const double2* p, int nrhs, int64_t n, const double* pts,
               int64_t npts, double kd, double* out, cudaStream_t st) {
  const int64_t nchunk = (npts + kNfPts - 1) / kNfPts;
  if (nchunk > 2147483647LL) return Err::make(DDA_EINVAL, "too many field points");
  k_near_field<<<dim3((unsigned)nchunk, nrhs), kT, 0, st>>>(ijk, origin3, p, n, pts, npts, kd, out);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err near_field_pbc(const int32_t* ijk, const double* origin3, const double2* p, int nrhs, int64_t n, const double* pts,
                   int64_t npts, double kd, const double k_tf[3], double py, double pz, double gamma, int my, int mz,
                   double* part, int nsplit, double* out, cudaStream_t st) {
  const int64_t nchunk = (npts + kNfPts - 1) / kNfPts;
  if (nchunk > 65535 || nrhs > 65535 || nsplit < 1) return Err::make(DDA_EINVAL, "too many field points");
  k_near_field_pbc<<<dim3((unsigned)nsplit, (unsigned)nchunk, (unsigned)nrhs), kT, 0, st>>>(
      ijk, origin3, p, n, pts, npts, kd, k_tf[1], k_tf[2], py, pz, gamma, my, mz, part);
  DDA_CU(cudaGetLastError());
  const int64_t total = (int64_t)nrhs * npts * 12;
  k_nf_sum<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((total + kT - 1) / kT, 1216)), kT, 0, st>>>(
      part, nsplit, npts, nrhs, out);
  DDA_CU(cudaGetLastError());
  add_launches(2);
  return Err::Ok();
}

Err farfield_moments(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p,
                     int nrhs, int ndir, int64_t n, const int box[3], const double shift[3], float2* tab, double* part,
                     int nblk, double2* out, cudaStream_t st) {
  const int nt = box[0] + box[1] + box[2];
  const int64_t nrd = (int64_t)nrhs * ndir;
  const int tb = (int)std::min<int64_t>((nrd * nt + kT - 1) / kT, 152 * 32);
  k_phase_tables<<<tb, kT, 0, st>>>(nhat, nrd, origin3, kd, box[0], box[1], box[2], tab);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  const int nchunk = (ndir + kMomDir - 1) / kMomDir;
  const size_t sm = sizeof(float2) * (size_t)kMomDir * nt;
  if (sm > 48 * 1024) return Err::make(DDA_EUNSUPPORTED, "target box too long for the phase tables");
  k_far_moments<<<dim3(nblk, nchunk, nrhs), kT, sm, st>>>(ijk, p, n, ndir, box[0], box[1], box[2], (float)shift[0],
                                                          (float)shift[1], (float)shift[2], tab, part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_far_moments_fin<<<nrhs * nchunk, 64, 0, st>>>(part, nblk, nchunk, ndir, out);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err torque_ext_sums(const int32_t* ijk, const double2* einc, const double2* p, int nrhs, int64_t n,
                    const double shift[3], double* part, int nblk, double* out7, cudaStream_t st) {
  k_torque_ext<<<dim3(nblk, nrhs), kT, 0, st>>>(ijk, einc, p, n, shift[0], shift[1], shift[2], part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_torque_ext_fin<<<nrhs, kT, 0, st>>>(part, nblk, out7);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err farfield_many(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p,
                  int nrhs, int ndir, int64_t n, const int box[3], float2* tab, double* part, int nblk, double2* out,
                  cudaStream_t st) {
  const int nt = box[0] + box[1] + box[2];
  const int64_t nrd = (int64_t)nrhs * ndir;
  const int tb = (int)std::min<int64_t>((nrd * nt + kT - 1) / kT, 152 * 32);
  k_phase_tables<<<tb, kT, 0, st>>>(nhat, nrd, origin3, kd, box[0], box[1], box[2], tab);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  const int nchunk = (ndir + kDirPerCta - 1) / kDirPerCta;
  const size_t sm = sizeof(float2) * (size_t)kDirPerCta * nt;
  if (sm > 48 * 1024) return Err::make(DDA_EUNSUPPORTED, "target box too long for the phase tables");
  k_far_many<<<dim3(nblk, nchunk, nrhs), kT, sm, st>>>(ijk, p, n, ndir, box[0], box[1], box[2], tab, part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_far_many_fin<<<nrhs * nchunk, 64, 0, st>>>(part, nblk, nchunk, ndir, out);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

template <typename C>
Err incident_field(const int32_t* ijk, const double* origin3, const RhsGeom* rg, int nrhs, int64_t n, C* e,
                   cudaStream_t st) {
  const int nb = (int)std::min<int64_t>((n + kT - 1) / kT, 1024);
  k_einc<C><<<dim3(nb, nrhs), kT, 0, st>>>(ijk, origin3, rg, n, e);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}
template Err incident_field<float2>(const int32_t*, const double*, const RhsGeom*, int, int64_t, float2*, cudaStream_t);
template Err incident_field<double2>(const int32_t*, const double*, const RhsGeom*, int, int64_t, double2*,
                                     cudaStream_t);

Err qsums(const uint8_t* comp, const double2* einc, const double2* ia, int ncomp, double kd, const double2* p,
          int nrhs, int64_t n, double* out3, RedBuf rb, cudaStream_t st) {
  k_qsum<<<dim3(rb.nblk, nrhs), kT, 0, st>>>(comp, einc, ia, ncomp, kd, p, n, rb.part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_qsum_fin<<<nrhs, kT, 0, st>>>(rb.part, rb.nblk, out3);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err qsums_tensor(const double2* einc, const double2* iat, double kd, const double2* p, int nrhs, int64_t n,
                 double* out3, RedBuf rb, cudaStream_t st) {
  k_qsum_t<<<dim3(rb.nblk, nrhs), kT, 0, st>>>(einc, iat, kd, p, n, rb.part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_qsum_fin<<<nrhs, kT, 0, st>>>(rb.part, rb.nblk, out3);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err farfield(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p, int nrhs,
             int ndir, int64_t n, const int box[3], double2* out, double2* part, int nblk, cudaStream_t st) {
  double* pd = reinterpret_cast<double*>(part);
  const size_t sm = sizeof(double2) * (size_t)(box[0] + box[1] + box[2]);
  if (sm > 48 * 1024) return Err::make(DDA_EUNSUPPORTED, "target box too long for the far-field phase tables");
  k_far<<<dim3(nblk, ndir, nrhs), kT, sm, st>>>(ijk, origin3, nhat, kd, p, ndir, n, box[0], box[1], box[2], pd);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_far_fin<<<nrhs * ndir, kT, 0, st>>>(pd, nblk, out);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

}  // namespace dda
