// Incident field and scattering observables on the device.
//
// E_inc,j = e exp(i k . r_j) (guide, "Incident Polarization State"; plane wave
// along x_LF, expressed in the Target Frame), phase in FP64.
// Efficiency sums (Draine 1988, the formulas behind the guide's Q_ext, Q_abs,
// Q_pha), per RHS, FP64 accumulation:
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

__global__ void k_qsum(const int32_t* ijk, const uint8_t* comp, const double* org, const RhsGeom* rg,
                       const double2* ia, int ncomp, double kd, const double2* p, int64_t n, double* part) {
  const int b = blockIdx.y;
  const RhsGeom g = rg[b];
  const double rr = (2.0 / 3.0) * kd * kd * kd;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double rx = ijk[3 * j] + org[0], ry = ijk[3 * j + 1] + org[1], rz = ijk[3 * j + 2] + org[2];
    double sn, cs;
    sincos(g.k[0] * rx + g.k[1] * ry + g.k[2] * rz, &sn, &cs);
    const int cc = comp ? comp[j] : 0;
    for (int c = 0; c < 3; ++c) {
      const double er = g.e[2 * c], ei = g.e[2 * c + 1];
      const double Er = er * cs - ei * sn, Ei = er * sn + ei * cs;
      const double2 pv = p[((int64_t)b * 3 + c) * n + j];
      // conj(E) * P
      const double re = Er * pv.x + Ei * pv.y, im = Er * pv.y - Ei * pv.x;
      acc[0] += im;
      acc[1] += re;
      const double2 a = ia[((int64_t)b * ncomp + cc) * 3 + c];
      acc[2] += (-a.y - rr) * (pv.x * pv.x + pv.y * pv.y);
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

// grid (nblk, ndir, nrhs): partial sums of P_j exp(-i k n.r_j) -> part[rhs][dir][blk][6]
__global__ void k_far(const int32_t* ijk, const double* org, const double* nhat, double kd, const double2* p,
                      int ndir, int64_t n, double* part) {
  const int d = blockIdx.y, b = blockIdx.z;
  const double* nh = nhat + ((int64_t)b * ndir + d) * 3;
  const double kx = kd * nh[0], ky = kd * nh[1], kz = kd * nh[2];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double rx = ijk[3 * j] + org[0], ry = ijk[3 * j + 1] + org[1], rz = ijk[3 * j + 2] + org[2];
    double sn, cs;
    sincos(-(kx * rx + ky * ry + kz * rz), &sn, &cs);
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

}  // namespace

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

Err qsums(const int32_t* ijk, const uint8_t* comp, const double* origin3, const RhsGeom* rg, const double2* ia,
          int ncomp, double kd, const double2* p, int nrhs, int64_t n, double* out3, RedBuf rb, cudaStream_t st) {
  k_qsum<<<dim3(rb.nblk, nrhs), kT, 0, st>>>(ijk, comp, origin3, rg, ia, ncomp, kd, p, n, rb.part);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_qsum_fin<<<nrhs, kT, 0, st>>>(rb.part, rb.nblk, out3);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

Err farfield(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p, int nrhs,
             int ndir, int64_t n, double2* out, double2* part, int nblk, cudaStream_t st) {
  double* pd = reinterpret_cast<double*>(part);
  k_far<<<dim3(nblk, ndir, nrhs), kT, 0, st>>>(ijk, origin3, nhat, kd, p, ndir, n, pd);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  k_far_fin<<<nrhs * ndir, kT, 0, st>>>(pd, nblk, out);
  DDA_CU(cudaGetLastError());
  add_launches(1);
  return Err::Ok();
}

}  // namespace dda
