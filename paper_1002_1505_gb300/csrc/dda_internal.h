// Internal declarations of the GB300 DDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "../../include/dda.h"
#include "df.cuh"
#include "fft.cuh"
#ifdef __CUDACC__
#include "pdl.cuh"
#endif

namespace dda {

using cd = std::complex<double>;

// Status with message; every internal helper returns one.
struct Err {
  dda_status code = DDA_OK;
  std::string msg;
  bool ok() const { return code == DDA_OK; }
  static Err Ok() { return Err{}; }
  static Err make(dda_status c, std::string m) { Err e; e.code = c; e.msg = std::move(m); return e; }
};

#define DDA_CU(call)                                                                          \
  do {                                                                                        \
    cudaError_t e__ = (call);                                                                 \
    if (e__ != cudaSuccess)                                                                   \
      return ::dda::Err::make(e__ == cudaErrorMemoryAllocation ? DDA_ENOMEM : DDA_ECUDA,      \
                              std::string(#call) + ": " + cudaGetErrorString(e__));           \
  } while (0)

#define DDA_TRY(expr)                  \
  do {                                 \
    ::dda::Err e__ = (expr);           \
    if (!e__.ok()) return e__;         \
  } while (0)

// ------------------------------------------------------------------ targets (host)
struct HostTarget {
  std::vector<int32_t> ijk;   // N x 3 box-relative lattice indices, x-fastest order
  std::vector<uint8_t> comp;  // N x 3, 0-based composition of each site's x, y, z axis
  int box[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0};
  double a1[3] = {1, 0, 0};
  double a2[3] = {0, 1, 0};
  int ncomp = 1;
  // per-site Dielectric Frame (guide, "Composite Targets with Anisotropic Constituents"): N x 9,
  // row-major R[a][j] = TF component a of the principal axis e_j; empty when every site's
  // dielectric tensor is diagonal in the TF
  std::vector<double> dfrot;
};
Err make_shape_target(int shape, const double* shpar, int nshpar, HostTarget* out);
// df_angles (optional, with per_axis): N x 3 (theta_DF, phi_DF, beta_DF) in radians
Err make_site_target(const int32_t* ixyz, const int32_t* icomp, int64_t n, const double origin[3],
                     const double a1[3], const double a2[3], HostTarget* out, bool per_axis = false,
                     const double* df_angles = nullptr);
// The principal axes e_1, e_2, e_3 of the dielectric tensor in Target-Frame components for the
// guide's rotation angles (theta_DF, phi_DF, beta_DF): R[a][j] = (e_j)_a.
void df_axes(double theta, double phi, double beta, double R[9]);

// ------------------------------------------------------------------ FFT plans (host)
Err make_plan(int L, FftPlan* out);
bool is_smooth235(int v);

// ------------------------------------------------------------------ device geometry
// Everything a matvec kernel needs about the grid, by value.
struct Geom {
  int64_t n;             // occupied sites
  int nx, ny, nz;        // box
  int px, py, pz;        // padded grid
  int ys;                // y stride of the FFT workspace rows (ny: plane path, py: 5-pass path)
  int ncomp;
  FftPlan plx, ply, plz;
};

struct KState;

// Device-resident data shared by matvec kernels of one precision.
template <typename C>
struct MvData {
  const int32_t* map;   // nx*ny*nz box -> site index or -1
  const uint8_t* comp;  // N x 3 compositions (0-based, per site and axis), may be null when ncomp == 1
  const C* ghat;        // [px][py][pz][6] Fourier-space tensor (xx,xy,xz,yy,yz,zz), scaled by 1/M
  const C* ia;          // [nrhs][ncomp][3] diagonal of alpha^{-1}
  const C* twx;         // twiddles exp(-2 pi i j / L), L entries each
  const C* twy;
  const C* twz;
  C* work;              // FFT workspace [nrhs_chunk][3][px][nz][ys]
  // solver state of the RHS of this launch (index = RHS within the launch), or null: the
  // compile-time kernels skip the RHS whose solve has finished (their products are unused)
  const KState* ks = nullptr;
  unsigned int* fault = nullptr;  // set by a kernel whose bounded wait on a bulk copy gave up
  // Jacobi scaling of the product (symmetric diagonal preconditioning of the solve): when set, the
  // product applies S A S instead of A, S = diag(s) with s = alpha^{1/2} per (RHS, composition,
  // axis), layout [nrhs][ncomp][3] counted from the launch's first RHS; then the diagonal term
  // s alpha^{-1} s is the identity.
  const C* sc = nullptr;
  // full symmetric alpha^{-1} per (RHS, site) for targets with rotated dielectric frames:
  // [nrhs][N][6] (xx, xy, xz, yy, yz, zz) from the launch's rhs0 like ia; null = diagonal table
  const C* iat = nullptr;
};

// Launch tuning chosen per grid (autotuner fills it).
struct MvTune {
  int ty = 8;         // y rows per CTA in the x passes
  int g = 8;          // z columns per batch in the z pass
  int thr_x = 256;    // threads, x passes
  int thr_p = 512;    // threads, plane / z passes
  bool plane = true;  // 3-pass schedule (plane fits in shared memory)
  bool fast = false;  // compile-time-length kernels exist for px, py, pz (matvec_fast.cuh)
  bool plane_ok = false;  // the fast 3-pass plane kernel exists and fits for this grid
  int clus = 0;           // plane pass split over a cluster of this many CTAs (0: one CTA per plane)
  int xty = 0;            // y rows per CTA of the compile-time x passes (0: the length's default)
  int xnc = 0;            // components per CTA of the x passes (0 or 3: all three; 1: one)
  bool bulk = false;      // plane pass stages its HBM blocks with bulk copies
  int zr = 0;             // 5-pass z columns with pass B, Ghat and inverse pass B fused in registers
};

// Enqueue ap = A p for nrhs right-hand sides (rhs0 = index of the first one for alpha).
template <typename C>
Err launch_matvec(const Geom& g, const MvData<C>& d, const MvTune& t, const C* p, C* ap, int nrhs, int rhs0,
                  bool conj, cudaStream_t st);
template <typename C>
size_t plane_smem_bytes(const Geom& g, const MvTune& t);
// The product on the compile-time-length kernels (matvec_fast_c64.cu / matvec_fast_c128.cu).
template <typename C>
Err launch_matvec_fast(const Geom& g, const MvData<C>& d, const MvTune& t, const C* p, C* ap, int nrhs, int rhs0,
                       bool conj, cudaStream_t st);
// Opt a kernel into the largest dynamic shared memory the device allows beside the kernel's
// own static shared memory (the attribute is refused when the sum would exceed the limit).
template <typename K>
inline void optin_smem(K kern, int smax) {
  cudaFuncAttributes a{};
  int stat = 0;
  if (cudaFuncGetAttributes(&a, kern) == cudaSuccess) stat = (int)a.sharedSizeBytes;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smax - stat);
}
void fast_optin_c64(int smax);
// Runs the bounded mbarrier wait of the bulk-copy path on a barrier that never completes (a few
// thousand polls) and reports whether it gave up (1) instead of hanging.
Err selftest_bulk_wait(int* gave_up);
// complex64 plane pass split over a thread-block cluster of S CTAs (matvec_cluster.cu)
Err launch_plane_cluster_c64(const Geom& g, const MvData<float2>& d, int S, int nrhs, cudaStream_t st);
int plane_cluster_capacity_c64(const Geom& g, int S, int smax);  // co-resident clusters, 0 = not possible
// complex64 plane pass with its HBM blocks staged by bulk copies (matvec_plane_bulk.cu)
Err launch_plane_bulk_c64(const Geom& g, const MvData<float2>& d, int nrhs, cudaStream_t st);
bool plane_bulk_ok_c64(const Geom& g, int smax);
void plane_bulk_optin_c64(int smax);
void cluster_optin_c64(int smax);
void fast_optin_c128(int smax);
// The product with complex128 vectors in and out and double-float arithmetic (df.cuh) inside:
// the compile-time 5-pass kernels of the complex128 schedule t (matvec_fast_df.cu).  Returns
// DDA_EUNSUPPORTED when t is not a compile-time 5-pass schedule.
Err launch_matvec_df(const Geom& g, const MvData<dfp::dfc>& d, const MvTune& t, const double2* p, double2* ap,
                     int nrhs, int rhs0, bool conj, cudaStream_t st);
void fast_optin_df(int smax);
// Does a fast schedule exist for this grid (all lengths instantiated, tiles fit)?  Sets t.fast and t.plane.
void choose_fast_schedule(const Geom& g, bool c64, int smax, MvTune* t);
// x-pass tile heights (y rows per CTA) of the compile-time kernels: the default for a length, and
// whether a height is instantiated
int x_tile_height_default(size_t csize, int px);
bool x_tile_height_ok(size_t csize, int px, int ty);
int x_tile_height_one_component(size_t csize);
// profiling hook: record the i-th pass event if per-pass events are on
void mark_pass(int i, cudaStream_t st);
size_t x_smem_bytes(const Geom& g, const MvTune& t, size_t csize);

// Profiling and accounting: per-pass events for the next launches on this thread
// (ev[0] before the first pass, ev[i+1] after pass i; null = off), and a global
// count of kernels launched by the library (graph replays included).
void set_pass_events(cudaEvent_t* ev);
unsigned long long launches();
void add_launches(unsigned long long n);
void sub_launches(unsigned long long n);

// Fixed device scratch of dda_matvec_noalloc (bytes) and its per-device address.
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
Err noalloc_scratch(int device, void** out);

// Green tensor: fill + FP64 FFT + pack into ghat128 / ghat64 / ghatdf (double-float, may be null).
// storage <-> natural frequency tables the Green build needs (natx[px] | naty[py] | stx[px/2+1] | sty[py/2+1])
void green_perm_tables(const Geom& g, std::vector<int32_t>* out);
Err build_green(const Geom& g, double kd, const double2* twx, const double2* twy, const double2* twz,
                const int32_t* perm, double2* gw, double2* ghat128, float2* ghat64, dfp::dfc* ghatdf,
                cudaStream_t st);
// The Green tensor of a target periodic along y_TF (period py, 0 = none) and / or z_TF (pz), with
// the Bloch phases of the TF wave vector k_tf and the cutoff exp[-(gamma kd r)^4], transformed over
// the full grid (same output layouts as build_green).
Err build_green_pbc(const Geom& g, double kd, const double k_tf[3], double py, double pz, double gamma,
                    const double2* twx, const double2* twy, const double2* twz, double2* gw, double2* ghat128,
                    float2* ghat64, dfp::dfc* ghatdf, cudaStream_t st);

// Generic batched FFT over rows/strides (used by tests of the engine and the Green build).
template <typename C>
Err fft_rows(C* data, int64_t nrows, int64_t row_stride, const FftPlan& pl, const C* tw, int nin, int nout,
             bool inverse, cudaStream_t st);
template <typename C>
Err fft_strided(C* data, int L, int64_t estride, int64_t ninner, int64_t nouter, int64_t outer_stride,
                const FftPlan& pl, const C* tw, bool inverse, cudaStream_t st);

// ------------------------------------------------------------------ Krylov / BLAS-1 (krylov.cu)
struct RedBuf {
  double* part = nullptr;        // partial sums [nrhs][nblk][kRedSlots]
  unsigned int* count = nullptr; // per-RHS arrival counters (zero between kernels)
  int nblk = 0;
};
constexpr int kRedSlots = 8;

// Per-RHS scalar state of the iterative solvers (device).
struct KState {
  double2 rho, alpha, omega, beta;
  double2 g1, g2; // BiCGstab(2): coefficients of the minimal-residual step
  double bb;      // |b|^2
  double rr;      // |r|^2 (recursive)
  double zz;      // CCG |A^H r|^2
  double tol2;    // (tol)^2 * |b|^2 threshold for this solve
  // QMR (complex symmetric): Givens rotations G_{n-1} = (q_c1, q_s1), G_{n-2} = (q_c2, q_s2), the
  // rotated right-hand side entry q_tb, v_{n-1}^T v_{n-1} (q_dp), |w| of the last step (q_rho), and
  // the current column's entries r_{n-2,n}, r_{n-1,n}, r_{n,n} (q_r2, q_r1, q_rn) and tau_n (q_tau)
  double2 q_s1, q_s2, q_tb, q_dp, q_r1, q_r2, q_rn, q_tau;
  double q_c1, q_c2, q_rho;
  int done;       // 1 = converged, 2 = breakdown
  int it;
  int mv;         // products with A applied to this RHS (products of finished RHS are skipped)
  int pad1;
};

template <typename C> Err k_copy_convert_c128_to(const double2* src, C* dst, int64_t count, cudaStream_t st);
template <typename C> Err k_accumulate_to_c128(double2* dst, const C* src, int64_t count, cudaStream_t st);

template <typename C>
struct KrylovVecs {
  C *x, *r, *rhat, *p, *v, *s, *t, *b;
  C* u2 = nullptr;  // BiCGstab(2) only
};

// BiCGstab / CCG building blocks, all per-RHS batched over nrhs vectors of length n3.
template <typename C> Err bicg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                    double tol, bool have_ax, cudaStream_t st);
template <typename C> Err bicg_p_update(const KrylovVecs<C>& kv, const KState* ks, int nrhs, int64_t n3,
                                        cudaStream_t st);
template <typename C> Err bicg_alpha(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                     cudaStream_t st);
template <typename C> Err bicg_s_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                        cudaStream_t st);
template <typename C> Err bicg_omega(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                     cudaStream_t st);
template <typename C> Err bicg_xr_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                         cudaStream_t st);
// BiCGstab(2) (Sleijpen & Fokkema 1993): vectors r0 = r, r1 = s, r2 = t, u0 = p, u1 = v, u2 = u2,
// shadow = rhat.  init; then per cycle: u_update(0), [u1 = A u0], alpha(1), r_update(0),
// [r1 = A r0], beta(1), u_update(1), [u2 = A u1], alpha(2), r_update(1), [r2 = A r1], mr.
template <typename C> Err b2_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol,
                                  bool have_ax, cudaStream_t st);
template <typename C> Err b2_u_update(const KrylovVecs<C>& kv, const KState* ks, int j, int nrhs, int64_t n3,
                                      cudaStream_t st);
template <typename C> Err b2_alpha(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int j, int nrhs, int64_t n3,
                                   cudaStream_t st);
template <typename C> Err b2_r_update(const KrylovVecs<C>& kv, const KState* ks, int j, int nrhs, int64_t n3,
                                      cudaStream_t st);
template <typename C> Err b2_beta(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                  cudaStream_t st);
template <typename C> Err b2_mr(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                cudaStream_t st);
// COCG (complex-symmetric CG): init; then per iteration [v = A p], update (alpha, x/r, beta, p).
template <typename C> Err cocg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol,
                                    bool have_ax, cudaStream_t st);
// QMR for complex-symmetric A (Freund 1992), no look-ahead: v_n in p, v_{n-1} in r, A v_n / w in v,
// the direction vectors d_n, d_{n-1}, d_{n-2} rotating through s, t, rhat.  Stops when the bound
// sqrt(n + 1) |tau_bar_{n+1}| on the true residual reaches tol |b| (unit-norm Lanczos vectors).
// The solve runs it in complex128 only (near breakdowns of the Lanczos process, see dda_solve).
template <typename C> Err qmr_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3, double tol,
                                   bool have_ax, cudaStream_t st);
template <typename C> Err qmr_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                     cudaStream_t st);
template <typename C> Err cocg_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                      cudaStream_t st);
// dst = c0 s0 + c1 s1 over n3 complex128 elements
Err combine2_c128(double2* dst, const double2* s0, const double2* s1, double2 c0, double2 c1, int64_t n3,
                  cudaStream_t st);
// v[b][c][j] *= s[b][comp(j,c)][c] (inv: divides), the Jacobi scaling of site vectors
template <typename C> Err scale_sites(C* v, const C* s, const uint8_t* comp, int ncomp, int nrhs, int64_t n, bool inv,
                                      cudaStream_t st);
// CCG (CG on the normal equations)
template <typename C> Err ccg_init(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                   double tol, bool have_ax, cudaStream_t st);
template <typename C> Err ccg_start(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                    cudaStream_t st);
template <typename C> Err ccg_alpha_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                           cudaStream_t st);
template <typename C> Err ccg_beta_update(const KrylovVecs<C>& kv, KState* ks, RedBuf rb, int nrhs, int64_t n3,
                                          cudaStream_t st);

// BiCGstab half-iterations of the complex64 solve with the vector updates and dot products folded
// into the x passes of the compile-time product (matvec_fused_c64.cu).  half 0: p = r + beta (p -
// omega v), v = A p, alpha = rho / <rhat, v>; half 1: s = r - alpha v (half-step test on |s|),
// t = A s, omega = <t, s> / |t|^2.  All nrhs RHS of the solve in one launch; d.ks = ks; rbx: a
// reduction table of x_ctas_per_rhs_c64 slots per RHS and zeroed per-RHS counters.
Err launch_bicg_half_c64(const Geom& g, const MvData<float2>& d, const MvTune& t, const KrylovVecs<float2>& kv,
                         KState* ks, const RedBuf& rbx, int nrhs, int half, cudaStream_t st);
int x_ctas_per_rhs_c64(const Geom& g, const MvTune& t);
// the register-fused 5-pass z-column kernel exists for this complex64 grid
bool zcols_rfuse_available_c64(const Geom& g);
// the passes between the x passes of the complex64 product (plane pass or y/z/y), matvec_fast_c64.cu
Err launch_middle_c64(const Geom& g, const MvData<float2>& d, const MvTune& t, int nrhs, cudaStream_t st);
void fused_optin_c64(int smax);

// r = b - ax (c128), returns per-RHS |r|^2 and |b|^2 into out2[2*nrhs] (device)
Err residual_c128(const double2* b, const double2* ax, double2* r, double* out2, RedBuf rb, int nrhs, int64_t n3,
                  cudaStream_t st);
// dst(C) = (C) src(c128)
template <typename C> Err convert_from_c128(const double2* src, C* dst, int64_t count, cudaStream_t st);
// dst(c128) += src(C) for RHS whose mask is 0 (mask may be null)
template <typename C> Err add_to_c128(double2* dst, const C* src, const int* mask_done, int nrhs, int64_t n3,
                                      cudaStream_t st);

// ------------------------------------------------------------------ observables (observables.cu)
struct RhsGeom {     // per RHS, device
  double k[3];       // k vector in TF
  double e[6];       // polarization (re, im) x 3 in TF
};
template <typename C>
Err incident_field(const int32_t* ijk, const double* origin3, const RhsGeom* rg, int nrhs, int64_t n, C* e,
                   cudaStream_t st);
// per RHS: [0] sum Im(E*.P), [1] sum Re(E*.P), [2] sum (-Im ia - 2/3 k^3)|P|^2
Err qsums_tensor(const double2* einc, const double2* iat, double kd, const double2* p, int nrhs, int64_t n,
                 double* out3, RedBuf rb, cudaStream_t st);
Err qsums(const uint8_t* comp, const double2* einc /*[nrhs][3][N]*/, const double2* ia, int ncomp, double kd,
          const double2* p, int nrhs, int64_t n, double* out3, RedBuf rb, cudaStream_t st);
// F[rhs][dir][3] = sum_j P_j exp(-i kd n_dir . r_j); ndirs directions per RHS (nhat given per RHS, TF)
Err farfield(const int32_t* ijk, const double* origin3, const double* nhat /*[nrhs][ndir][3]*/, double kd,
             const double2* p, int nrhs, int ndir, int64_t n, const int box[3], double2* out, double2* part, int nblk,
             cudaStream_t st);
// Far field F = sum_j P_j exp(-i k n.r_j) for many directions (nhat [nrhs][ndir][3] in TF) from
// separable FP32 phase tables (tab: nrhs*ndir*(box sum) float2; part: nrhs*ceil(ndir/8)*nblk*48
// doubles); out [nrhs][ndir][3].
Err farfield_many(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p,
                  int nrhs, int ndir, int64_t n, const int box[3], float2* tab, double* part, int nblk, double2* out,
                  cudaStream_t st);
// Far-field moments for the radiative torque: out[rhs][d][12] = g (3 complex) and
// T[c][a] = sum_j (r_j - r_cm)_c P_ja exp(-i k n.r_j) (9 complex); shift = origin - r_cm.
Err farfield_moments(const int32_t* ijk, const double* origin3, const double* nhat, double kd, const double2* p,
                     int nrhs, int ndir, int64_t n, const int box[3], const double shift[3], float2* tab, double* part,
                     int nblk, double2* out, cudaStream_t st);
// Dipole fields at npts points (host-side incident field not included): out[rhs][pt][12] =
// E then B, (re, im) x 3, FP64; dipoles nearer than one lattice spacing scaled by R^4 (5 - 4R).
Err near_field(const int32_t* ijk, const double* origin3, const double2* p, int nrhs, int64_t n, const double* pts,
               int64_t npts, double kd, double* out, cudaStream_t st);
// The same for a periodic target: replicas (0, m py, l pz), |m| <= my, |l| <= mz, moments times
// e^{i k.R}, each term weighted by exp[-(gamma kd D)^4] (dropped beyond 40 in the exponent); part:
// nrhs * nsplit * npts * 12 doubles of partial sums, added in a fixed order into out.
Err near_field_pbc(const int32_t* ijk, const double* origin3, const double2* p, int nrhs, int64_t n, const double* pts,
                   int64_t npts, double kd, const double k_tf[3], double py, double pz, double gamma, int my, int mz,
                   double* part, int nsplit, double* out, cudaStream_t st);
// Measurement probe: nvec 8-point complex vectors through `reps` unitary DFT-8 stages, on FP32
// butterflies and on split-TF32 tensor-core products; out = {fp32 ms, tensor ms, fp32 error,
// tensor error} (relative L2 against FP64 on the first 64 vectors).
Err probe_tc_dft(int64_t nvec, int reps, double out[4]);
// Incident-field force/torque sums per RHS: out7[b] = {sum Re(P x E^*) (3), sum (r - r_cm) Im(P.E^*) (3),
// sum Im(P.E^*)}; part: nrhs * nblk * 8 doubles.
Err torque_ext_sums(const int32_t* ijk, const double2* einc, const double2* p, int nrhs, int64_t n,
                    const double shift[3], double* part, int nblk, double* out7, cudaStream_t st);

// ------------------------------------------------------------------ learned warm start glue (unet.cu)
Err unet_features(const int32_t* ijk, int64_t n, const uint8_t* comp, const float2* eps, const double2* e, int nrhs,
                  const int32_t dims[3], const int32_t off[3], float* x, cudaStream_t st);
Err unet_targets(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const double2* p,
                 const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], float* t, float* mask,
                 cudaStream_t st);
Err unet_warm(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float* y,
              const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], double2* p, cudaStream_t st);

Err unet_guess64(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float* y,
                 const double2* e, int nrhs, const int32_t dims[3], const int32_t off[3], float2* p, cudaStream_t st);
Err unet_resid64(const double2* e, float2* r, int nrhs, int64_t n3, double* part, int nblk, cudaStream_t st);
Err unet_resgrad(const int32_t* ijk, int64_t n, const uint8_t* comp, const double2* ia, int ncomp, const float2* g,
                 const double* wb, int nrhs, const int32_t dims[3], const int32_t off[3], float* gy, cudaStream_t st);

}  // namespace dda
