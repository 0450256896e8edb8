// C ABI of the GB300 DDA library: context, target/incidence/polarizability
// set-up on the host (FP64), Green-tensor build, product A P, the batched
// Krylov drivers (BiCGstab, CCG; complex64, complex128 or complex64 refined
// against complex128 true residuals) and the observables.
#include <algorithm>
#include <array>
#include <chrono>
#include <thread>
#include <type_traits>
#include <map>
#include <mutex>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dda_internal.h"

using dda::cd;
using dda::Err;

namespace dda {
void init_kernel_attrs();
}

struct dda_ctx {
  int device = 0;
  bool host_only = false;  // device < 0: set-up only, no CUDA calls
  cudaStream_t stream = nullptr;
  std::string err;

  // target
  bool have_target = false;
  dda::HostTarget tgt;
  dda::HostTarget tgt_next;           // scratch for the next dda_setup_target (capacity reused)
  std::vector<int32_t> h_map;         // host box -> site map of the last upload
  int64_t uploaded_n = -1;            // site count and composition use of the last upload
  bool uploaded_comp = false;
  int64_t n = 0;
  int32_t* d_map = nullptr;
  int32_t* d_ijk = nullptr;
  uint8_t* d_comp = nullptr;
  double* d_origin = nullptr;
  int tw_len[3] = {0, 0, 0};          // padded lengths the twiddle tables were built for
  int32_t* d_gperm = nullptr;         // storage <-> natural frequency tables of the Green build
  int gperm_key[2] = {0, 0};          // (px, py) they were built for

  // incident
  bool have_inc = false;
  double kd = 0;
  int n_ori = 0, iorth = 0, nrhs = 0;
  std::vector<double> ori;
  cd e01[3], e02[3];                  // Lab-Frame polarizations
  std::vector<double> axes;           // n_ori x 9: x_LF, y_LF, z_LF in TF
  std::vector<dda::RhsGeom> rg;       // nrhs
  dda::RhsGeom* d_rg = nullptr;
  double2* d_e128 = nullptr;          // cached E_inc [nrhs][3][N]

  // green
  bool have_green = false;
  dda::Geom g64{}, g128{};
  dda::MvTune t64{}, t128{};
  double2* d_ghat128 = nullptr;
  float2* d_ghat64 = nullptr;
  double2* d_tw128[3] = {nullptr, nullptr, nullptr};
  float2* d_tw64[3] = {nullptr, nullptr, nullptr};
  // double-float copies for the FP64-accurate product on FP32 units (built when the
  // complex128 schedule has compile-time kernels)
  dda::dfp::dfc* d_ghatdf = nullptr;
  dda::dfp::dfc* d_twdf[3] = {nullptr, nullptr, nullptr};
  bool ghatdf_valid = false;

  // polarizability
  bool have_alpha = false;
  int presc = 0, ncomp = 1;
  std::vector<cd> ia;                 // nrhs x ncomp x 3
  double2* d_ia128 = nullptr;
  float2* d_ia64 = nullptr;
  dda::dfp::dfc* d_iadf = nullptr;
  std::vector<cd> eps;                // permittivity m^2 per composition
  float2* d_eps = nullptr;
  float2* d_nnv = nullptr;            // residual-loss vectors (three complex64 [nrhs][3][N])
  double* d_nnpart = nullptr;
  double* d_nnw = nullptr;
  // Jacobi scaling s = alpha^{1/2} per (RHS, composition, axis) for preconditioned solves; `jacobi`
  // is set only while a preconditioned solve's Krylov iterations run (true residuals and every
  // other product use the unscaled A)
  double2* d_sc128 = nullptr;
  float2* d_sc64 = nullptr;
  bool jacobi = false;
  // periodic target (unit cell repeated along y_TF and / or z_TF; periods 0 = none)
  double per_y = 0.0, per_z = 0.0, per_gamma = 0.01;
  bool periodic = false;
  // full alpha^{-1} per (RHS, site) for targets with rotated dielectric frames ([nrhs][N][6])
  double2* d_iat128 = nullptr;
  float2* d_iat64 = nullptr;
  bool iat_valid = false;

  // workspaces (grown on demand)
  float2* d_w64 = nullptr;
  unsigned int* d_fault = nullptr;  // set by product kernels whose bounded bulk-copy wait gave up
  int w64_cap = 0;
  double2* d_w128 = nullptr;
  int w128_cap = 0;
  double* d_part = nullptr;
  size_t part_bytes = 0;
  unsigned int* d_count = nullptr;  // per-RHS arrival counters of the fused reductions
  int count_cap = 0;
  void* d_kvec = nullptr;
  size_t kvec_bytes = 0;
  dda::KState* d_ks = nullptr;
  int ks_cap = 0;
  double* d_small = nullptr;
  size_t small_bytes = 0;
  double* h_pinned = nullptr;
  size_t pinned_bytes = 0;
  cudaStream_t own_stream = nullptr;  // used for graph capture when the caller's stream is a default stream
  cudaEvent_t ev = nullptr;
  bool comp_valid = false;            // d_comp holds compositions (ncomp > 1)
  bool einc_valid = false;            // d_e128 holds E_inc for the current incidence
  double2* d_gscratch = nullptr;      // FP64 Green-tensor build scratch
  double2* d_sc = nullptr;            // solve scratch (two complex128 vectors)
  double* d_nh = nullptr;             // far-field directions
  double2* d_F = nullptr;             // far-field sums
  double* d_fpart = nullptr;          // far-field partial sums
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // cached solver graphs (complex64, complex128)
  // A captured iteration graph holds device pointers and launch parameters by value.  `gen`
  // changes whenever a device buffer is (re)allocated or the launch schedule or geometry
  // changes; a graph captured at the same generation for the same solver, iteration count,
  // RHS count and vector length is replayed without a new capture.
  unsigned long long gen = 1;
  bool have_sched = false;  // g64/g128/t64/t128 describe the current grid
  unsigned long long gexec_gen[2] = {0, 0};
  long long gexec_key[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  unsigned long long gexec_kernels[2] = {0, 0};
  int tuned_nrhs[2] = {0, 0};         // RHS count the current schedule was tuned for (c64, c128)
  bool forced_schedule = false;       // DDA_SCHEDULE fixed the schedule: no autotuning
  void* d_tunebuf = nullptr;          // operands of the autotuner's timed products
  // Device buffers grow and are never shrunk while the context lives: set-up
  // calls for a new problem of the same size recompute their results in the
  // same memory instead of freeing and allocating again.
  std::vector<std::pair<void**, size_t>> caps;
};

namespace {

dda_status fail(dda_ctx* c, const Err& e) {
  if (c) c->err = e.msg;
  return e.code;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

Err set_dev(dda_ctx* c) {
  if (c->host_only) return Err::Ok();
  DDA_CU(cudaSetDevice(c->device));
  return Err::Ok();
}

Err need_device(dda_ctx* c) {
  if (c->host_only) return Err::make(DDA_ESTATE, "host-only context (device < 0) cannot run device work");
  return Err::Ok();
}

size_t& cap_of(dda_ctx* c, void** p) {
  for (auto& kv : c->caps)
    if (kv.first == p) return kv.second;
  c->caps.emplace_back(p, 0);
  return c->caps.back().second;
}

// Grow-only device buffer owned by the context (contents are not preserved on growth).
template <typename T>
Err grow(dda_ctx* c, T** p, size_t bytes) {
  size_t& cap = cap_of(c, (void**)p);
  if (*p && bytes <= cap) return Err::Ok();
  if (*p) cudaFree((void*)*p);
  *p = nullptr;
  cap = 0;
  if (bytes == 0) return Err::Ok();
  DDA_CU(cudaMalloc((void**)p, bytes));
  cap = bytes;
  c->gen++;
  return Err::Ok();
}

template <typename T>
Err dalloc(T** p, size_t bytes) {
  if (*p) cudaFree((void*)*p);
  *p = nullptr;
  if (bytes == 0) return Err::Ok();
  DDA_CU(cudaMalloc((void**)p, bytes));
  return Err::Ok();
}

void drop_alpha(dda_ctx* c) {
  c->have_alpha = false;
  c->ia.clear();
  if (c->iat_valid) c->gen++;
  c->iat_valid = false;
}
void drop_green(dda_ctx* c) { c->have_green = false; }
void drop_incident(dda_ctx* c) {
  c->have_inc = false;
  c->einc_valid = false;
  c->rg.clear();
  c->nrhs = 0;
  drop_green(c);
  drop_alpha(c);
}
void drop_target(dda_ctx* c) {
  c->have_target = false;
  c->comp_valid = false;
  c->periodic = false;  // a new target starts finite
  c->per_y = c->per_z = 0.0;
  drop_incident(c);
}

void free_all(dda_ctx* c) {
  for (auto& kv : c->caps) {
    if (*kv.first) cudaFree(*kv.first);
    *kv.first = nullptr;
    kv.second = 0;
  }
  for (auto& g : c->gexec)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

Err upload_target(dda_ctx* c) {
  auto& t = c->tgt;
  const int64_t n = (int64_t)t.comp.size() / 3;
  const int64_t nbox = (int64_t)t.box[0] * t.box[1] * t.box[2];
  std::vector<int32_t>& map = c->h_map;  // kept between calls: no fresh pages per target
  map.assign(nbox, -1);
  for (int64_t j = 0; j < n; ++j) {
    const int64_t b = ((int64_t)t.ijk[3 * j + 2] * t.box[1] + t.ijk[3 * j + 1]) * t.box[0] + t.ijk[3 * j];
    map[b] = (int32_t)j;
  }
  c->n = n;
  if (c->host_only) {
    c->have_target = true;
    return Err::Ok();
  }
  DDA_TRY(grow(c, &c->d_map, sizeof(int32_t) * nbox));
  DDA_TRY(grow(c, &c->d_ijk, sizeof(int32_t) * 3 * n));
  DDA_TRY(grow(c, &c->d_origin, sizeof(double) * 3));
  DDA_CU(cudaMemcpy(c->d_map, map.data(), sizeof(int32_t) * nbox, cudaMemcpyHostToDevice));
  DDA_CU(cudaMemcpy(c->d_ijk, t.ijk.data(), sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice));
  DDA_CU(cudaMemcpy(c->d_origin, t.origin, sizeof(double) * 3, cudaMemcpyHostToDevice));
  c->comp_valid = false;
  if (t.ncomp > 1) {
    DDA_TRY(grow(c, &c->d_comp, 3 * n));
    DDA_CU(cudaMemcpy(c->d_comp, t.comp.data(), 3 * n, cudaMemcpyHostToDevice));
    c->comp_valid = true;
  }
  // captured iteration graphs hold the site count and whether compositions are read
  if (c->uploaded_n != n || c->uploaded_comp != c->comp_valid) c->gen++;
  c->uploaded_n = n;
  c->uploaded_comp = c->comp_valid;
  c->n = n;
  c->have_target = true;
  return Err::Ok();
}

// Lab-Frame unit vectors in the Target Frame for orientation (beta, Theta, Phi)
// (guide, "Orientation of the Target in the Lab Frame", inverse relations).
void lab_axes(const double a1[3], const double a2[3], double beta, double theta, double phi, double out[9]) {
  double a3[3] = {a1[1] * a2[2] - a1[2] * a2[1], a1[2] * a2[0] - a1[0] * a2[2], a1[0] * a2[1] - a1[1] * a2[0]};
  const double ct = std::cos(theta), st = std::sin(theta), cb = std::cos(beta), sb = std::sin(beta);
  const double cp = std::cos(phi), sp = std::sin(phi);
  const double cx[3] = {ct, -st * cb, st * sb};
  const double cy[3] = {st * cp, ct * cb * cp - sb * sp, -(ct * sb * cp + cb * sp)};
  const double cz[3] = {st * sp, ct * cb * sp + sb * cp, -(ct * sb * sp - cb * cp)};
  for (int k = 0; k < 3; ++k) {
    out[k] = cx[0] * a1[k] + cx[1] * a2[k] + cx[2] * a3[k];
    out[3 + k] = cy[0] * a1[k] + cy[1] * a2[k] + cy[2] * a3[k];
    out[6 + k] = cz[0] * a1[k] + cz[1] * a2[k] + cz[2] * a3[k];
  }
}

// diagonal of alpha^{-1} (guide "Dipole Polarizabilities"; CM with radiative
// reaction, LATTDR of Draine & Goodman 1993, GKDLDR of Gutkowicz-Krusin & Draine 2004)
void inv_alpha(int presc, cd m, double kd, const double khat[3], const cd e[3], cd out[3]) {
  const double b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004;
  const cd eps = m * m;
  const double pi = 3.14159265358979323846;
  const cd inv_cm = (4.0 * pi / 3.0) * (eps + 2.0) / (eps - 1.0);
  const cd rr = cd(0.0, -(2.0 / 3.0) * kd * kd * kd);
  if (presc == DDA_CM) {
    for (int a = 0; a < 3; ++a) out[a] = inv_cm + rr;
  } else if (presc == DDA_LATTDR) {
    double s = 0;
    for (int a = 0; a < 3; ++a) s += khat[a] * khat[a] * std::norm(e[a]);
    const cd v = inv_cm + (b1 + eps * b2 + eps * b3 * s) * kd * kd + rr;
    for (int a = 0; a < 3; ++a) out[a] = v;
  } else {
    for (int a = 0; a < 3; ++a) out[a] = inv_cm + (b1 + eps * b2 + eps * b3 * (khat[a] * khat[a])) * kd * kd + rr;
  }
}

Err ensure_part(dda_ctx* c, size_t bytes) {
  if (bytes > c->part_bytes) {
    DDA_TRY(grow(c, &c->d_part, bytes));
    c->part_bytes = bytes;
  }
  // counters for up to 65536 RHS; zeroed once, kept at zero by the kernels that use them
  if (c->count_cap == 0) {
    DDA_TRY(grow(c, &c->d_count, sizeof(unsigned int) * 65536));
    DDA_CU(cudaMemset(c->d_count, 0, sizeof(unsigned int) * 65536));
    c->count_cap = 65536;
  }
  return Err::Ok();
}

Err ensure_small(dda_ctx* c, size_t bytes) {
  if (bytes <= c->small_bytes) return Err::Ok();
  DDA_TRY(grow(c, &c->d_small, bytes));
  c->small_bytes = bytes;
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  c->h_pinned = nullptr;
  DDA_CU(cudaMallocHost((void**)&c->h_pinned, bytes));
  c->pinned_bytes = bytes;
  return Err::Ok();
}

dda::RedBuf redbuf(dda_ctx* c, int nrhs, int64_t n3) {
  dda::RedBuf rb;
  rb.nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n3 + 2047) / 2048, std::max(1, 1216 / std::max(1, nrhs))));
  rb.part = c->d_part;
  rb.count = c->d_count;
  return rb;
}

// Workspace for `want` RHS (capped by a memory budget); returns capacity in RHS.
template <typename C>
Err ensure_work(dda_ctx* c, int want, int* cap_out);

// a CUDA call's status as an Err
inline Err cuda_ok(cudaError_t r, const char* what) {
  return r == cudaSuccess ? Err::Ok() : Err::make(DDA_ECUDA, std::string(what) + ": " + cudaGetErrorString(r));
}

Err ensure_fault_flag(dda_ctx* c) {
  if (c->d_fault) return Err::Ok();
  DDA_TRY(grow(c, &c->d_fault, sizeof(unsigned int) * 4));
  DDA_CU(cudaMemset(c->d_fault, 0, sizeof(unsigned int) * 4));
  return Err::Ok();
}

// A product kernel that gave up waiting for a bulk copy leaves the flag set: report it (once).
Err check_fault(dda_ctx* c) {
  if (!c->d_fault) return Err::Ok();
  unsigned int h = 0;
  DDA_CU(cudaMemcpyAsync(&h, c->d_fault, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  DDA_CU(cudaStreamSynchronize(c->stream));
  if (h == 0) return Err::Ok();
  DDA_CU(cudaMemsetAsync(c->d_fault, 0, sizeof(unsigned int), c->stream));
  return Err::make(DDA_ECUDA, "a product kernel gave up waiting for a bulk copy; the results since the last check are invalid");
}

template <>
Err ensure_work<float2>(dda_ctx* c, int want, int* cap_out) {
  DDA_TRY(ensure_fault_flag(c));
  const dda::Geom& g = c->g64;
  const size_t per = sizeof(float2) * 3ull * g.px * g.nz * g.ys;
  const size_t budget = 24ull << 30;
  int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)want, budget / per));
  DDA_TRY(grow(c, &c->d_w64, per * cap));
  c->w64_cap = (int)std::min<size_t>(cap_of(c, (void**)&c->d_w64) / per, (size_t)1 << 30);
  *cap_out = std::min(c->w64_cap, want);
  return Err::Ok();
}
template <>
Err ensure_work<double2>(dda_ctx* c, int want, int* cap_out) {
  DDA_TRY(ensure_fault_flag(c));
  const dda::Geom& g = c->g128;
  const size_t per = sizeof(double2) * 3ull * g.px * g.nz * g.ys;
  const size_t budget = 24ull << 30;
  int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)want, budget / per));
  DDA_TRY(grow(c, &c->d_w128, per * cap));
  c->w128_cap = (int)std::min<size_t>(cap_of(c, (void**)&c->d_w128) / per, (size_t)1 << 30);
  *cap_out = std::min(c->w128_cap, want);
  return Err::Ok();
}

template <typename C> struct Sel;
template <> struct Sel<float2> {
  static dda::Geom geom(dda_ctx* c) { dda::Geom g = c->g64; g.ncomp = c->ncomp; return g; }
  static const dda::MvTune& tune(dda_ctx* c) { return c->t64; }
  static dda::MvData<float2> data(dda_ctx* c) {
    dda::MvData<float2> d{c->d_map, c->comp_valid ? c->d_comp : nullptr, c->d_ghat64, c->d_ia64, c->d_tw64[0], c->d_tw64[1], c->d_tw64[2], c->d_w64};
    d.fault = c->d_fault;
    d.sc = c->jacobi ? c->d_sc64 : nullptr;
    d.iat = c->iat_valid ? c->d_iat64 : nullptr;
    return d;
  }
};
template <> struct Sel<double2> {
  static dda::Geom geom(dda_ctx* c) { dda::Geom g = c->g128; g.ncomp = c->ncomp; return g; }
  static const dda::MvTune& tune(dda_ctx* c) { return c->t128; }
  static dda::MvData<double2> data(dda_ctx* c) {
    dda::MvData<double2> d{c->d_map, c->comp_valid ? c->d_comp : nullptr, c->d_ghat128, c->d_ia128, c->d_tw128[0], c->d_tw128[1], c->d_tw128[2], c->d_w128};
    d.fault = c->d_fault;
    d.sc = c->jacobi ? c->d_sc128 : nullptr;
    d.iat = c->iat_valid ? c->d_iat128 : nullptr;
    return d;
  }
};

template <typename C> const C* scale_table(dda_ctx* c);
template <> const float2* scale_table<float2>(dda_ctx* c) { return c->d_sc64; }
template <> const double2* scale_table<double2>(dda_ctx* c) { return c->d_sc128; }

// ap = A p over nrhs RHS starting at RHS index rhs0 (chunked by workspace capacity)
// ks (optional): the solver state of RHS rhs0.. ; RHS whose solve has finished are skipped
template <typename C>
Err matvec(dda_ctx* c, const C* p, C* ap, int nrhs, int rhs0, bool conj, const dda::KState* ks = nullptr) {
  int cap = 0;
  DDA_TRY(ensure_work<C>(c, nrhs, &cap));
  const int64_t n3 = 3 * c->n;
  dda::MvData<C> d = Sel<C>::data(c);
  for (int b0 = 0; b0 < nrhs; b0 += cap) {
    const int nb = std::min(cap, nrhs - b0);
    d.ks = ks ? ks + b0 : nullptr;  // indexed by RHS within this launch
    DDA_TRY(dda::launch_matvec<C>(Sel<C>::geom(c), d, Sel<C>::tune(c), p + b0 * n3, ap + b0 * n3, nb,
                                  rhs0 + b0, conj, c->stream));
  }
  return Err::Ok();
}

// The FP64-accurate product in double-float arithmetic (complex128 in and out) on the
// complex128 schedule's compile-time 5-pass kernels; DDA_EUNSUPPORTED where that schedule
// does not exist.
bool df_available(dda_ctx* c) {
  return c->t128.fast && !c->t128.plane && c->ghatdf_valid && c->d_iadf && c->d_twdf[0] && c->d_twdf[1] &&
         c->d_twdf[2] && !c->iat_valid;
}
Err matvec_df(dda_ctx* c, const double2* p, double2* ap, int nrhs, int rhs0, bool conj) {
  if (!df_available(c))
    return Err::make(DDA_EUNSUPPORTED, "no double-float product for this grid (needs the compile-time 5-pass schedule)");
  int cap = 0;
  DDA_TRY(ensure_work<double2>(c, nrhs, &cap));
  const int64_t n3 = 3 * c->n;
  dda::MvData<dda::dfp::dfc> d{c->d_map, c->comp_valid ? c->d_comp : nullptr, c->d_ghatdf, c->d_iadf,
                               c->d_twdf[0], c->d_twdf[1], c->d_twdf[2],
                               reinterpret_cast<dda::dfp::dfc*>(c->d_w128)};
  d.fault = c->d_fault;
  for (int b0 = 0; b0 < nrhs; b0 += cap) {
    const int nb = std::min(cap, nrhs - b0);
    DDA_TRY(dda::launch_matvec_df(Sel<double2>::geom(c), d, c->t128, p + b0 * n3, ap + b0 * n3, nb, rhs0 + b0, conj,
                                  c->stream));
  }
  return Err::Ok();
}
// True residuals of the mixed and complex64 solves use the double-float product when the
// tolerance leaves it a margin of 100 or more (its error is about 1e-12 of |E|) and the grid
// has it; DDA_RESIDUAL=fp64 keeps them on the FP64 units.
bool df_residuals(dda_ctx* c, double tol) {
  if (tol < 1e-10 || !df_available(c)) return false;
  const char* f = std::getenv("DDA_RESIDUAL");
  return !(f && std::string(f) == "fp64");
}

// ------------------------------------------------------------------ autotuner
// The product has several launch schedules for a grid: the fused 3-pass plane
// kernel at 512 or 768 threads, and the 5-pass split (more memory traffic,
// more CTAs; better when few RHS leave SMs idle).  The first product of a
// given (grid, RHS count, precision) times each candidate on the device (one
// warm-up, then three products between CUDA events) and keeps the fastest;
// the choice is cached for the process.
std::mutex g_tune_mu;
std::map<std::array<int, 8>, dda::MvTune> g_tune_cache;

template <typename C>
Err apply_tune(dda_ctx* c, const dda::MvTune& t) {
  dda::MvTune& cur = (sizeof(C) == sizeof(float2)) ? c->t64 : c->t128;
  dda::Geom& g = (sizeof(C) == sizeof(float2)) ? c->g64 : c->g128;
  const int ys = t.plane ? g.ny : g.py;
  if (std::memcmp(&cur, &t, sizeof(t)) != 0 || g.ys != ys) c->gen++;  // a different launch schedule
  cur = t;
  g.ys = ys;
  return Err::Ok();
}

template <typename C>
Err ensure_tuned(dda_ctx* c, int nrhs) {
  const int idx = (sizeof(C) == sizeof(float2)) ? 0 : 1;
  const dda::MvTune base = idx == 0 ? c->t64 : c->t128;
  if (c->forced_schedule || !base.fast || c->tuned_nrhs[idx] == nrhs) return Err::Ok();
  const dda::Geom& g0 = idx == 0 ? c->g64 : c->g128;
  const std::array<int, 8> key = {g0.nx, g0.ny, g0.nz, g0.px, g0.py, g0.pz, nrhs, (int)sizeof(C)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      DDA_TRY(apply_tune<C>(c, it->second));
      c->tuned_nrhs[idx] = nrhs;
      return Err::Ok();
    }
  }
  std::vector<dda::MvTune> cand;
  dda::MvTune t5 = base;
  t5.plane = false;
  if (base.plane_ok) {
    dda::MvTune a = base, b = base;
    a.plane = b.plane = true;
    a.clus = b.clus = 0;
    a.thr_p = 512;
    b.thr_p = 768;
    cand.push_back(a);
    cand.push_back(b);
    if constexpr (sizeof(C) == sizeof(float2)) {
      int smax = 0;
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
      for (int S : {2, 4}) {
        if (dda::plane_cluster_capacity_c64(g0, S, smax) > 0) {
          dda::MvTune t = a;
          t.clus = S;
          cand.push_back(t);
        }
      }
    }
  }
  cand.push_back(t5);
  dda::MvTune best = cand[0];
  {
    const size_t bytes = sizeof(C) * (size_t)nrhs * 3 * c->n;
    DDA_TRY(grow(c, (char**)&c->d_tunebuf, 2 * bytes));
    C* p = (C*)c->d_tunebuf;
    C* ap = p + (size_t)nrhs * 3 * c->n;
    DDA_CU(cudaMemsetAsync(p, 0, bytes, c->stream));
    cudaEvent_t e0, e1;
    DDA_CU(cudaEventCreate(&e0));
    DDA_CU(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    Err err = Err::Ok();
    // one warm-up product, then three timed between events on the context's stream
    auto time_one = [&](const dda::MvTune& t) {
      apply_tune<C>(c, t);
      err = matvec<C>(c, p, ap, nrhs, 0, false);
      if (!err.ok()) return;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 3 && err.ok(); ++r) err = matvec<C>(c, p, ap, nrhs, 0, false);
      cudaEventRecord(e1, c->stream);
      if (!err.ok()) return;
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = t; }
    };
    for (const dda::MvTune& t : cand) {
      time_one(t);
      if (!err.ok()) break;
    }
    // then the x passes' tile height for the chosen schedule (short tiles give small batches more CTAs)
    if (err.ok()) {
      const dda::MvTune chosen = best;
      for (int ty : {4, 8}) {
        if (!dda::x_tile_height_ok(sizeof(C), g0.px, ty) || ty == dda::x_tile_height_default(sizeof(C), g0.px))
          continue;
        dda::MvTune t = chosen;
        t.xty = ty;
        time_one(t);
        if (!err.ok()) break;
      }
    }
    // one component per x-pass CTA (smaller tiles in shared memory, longer rows per store)
    if (err.ok()) {
      dda::MvTune t = best;
      t.xnc = 1;
      t.xty = 0;
      time_one(t);
    }
    // the 5-pass z columns with their middle stages fused in registers (long pass-B sub-blocks)
    if (err.ok() && sizeof(C) == sizeof(float2) && !best.plane && dda::zcols_rfuse_available_c64(g0)) {
      dda::MvTune t = best;
      t.zr = 1;
      time_one(t);
    }
    // and bulk-copy staging of the plane pass's HBM blocks
    int smax_b = 0;
    cudaDeviceGetAttribute(&smax_b, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (err.ok() && sizeof(C) == sizeof(float2) && best.plane && best.clus == 0 &&
        dda::plane_bulk_ok_c64(g0, smax_b)) {
      dda::MvTune t = best;
      t.bulk = true;
      time_one(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DDA_TRY(err);
  }
  DDA_TRY(apply_tune<C>(c, best));
  c->tuned_nrhs[idx] = nrhs;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  return Err::Ok();
}

Err ensure_einc(dda_ctx* c) {
  if (c->einc_valid) return Err::Ok();
  DDA_TRY(grow(c, &c->d_e128, sizeof(double2) * (size_t)c->nrhs * 3 * c->n));
  DDA_TRY(dda::incident_field<double2>(c->d_ijk, c->d_origin, c->d_rg, c->nrhs, c->n, c->d_e128, c->stream));
  c->einc_valid = true;
  return Err::Ok();
}

struct SolveStats {
  std::vector<int> iters, done;
  std::vector<int> mv;  // products with A applied to each RHS
};

// One Krylov solve in precision C over all nrhs RHS. kv.x holds x0 when have_x0.
template <typename C>
Err krylov(dda_ctx* c, const dda_solve_opts& o, const dda::KrylovVecs<C>& kv, double tol, int maxit, bool have_x0,
           SolveStats* stats, std::chrono::steady_clock::time_point t0, bool* timed_out) {
  const int nrhs = c->nrhs;
  const int64_t n3 = 3 * c->n;
  dda::RedBuf rb = redbuf(c, nrhs, n3);
  DDA_TRY(ensure_part(c, sizeof(double) * (size_t)rb.nblk * nrhs * dda::kRedSlots));
  rb.part = c->d_part;
  rb.count = c->d_count;
  DDA_TRY(grow(c, &c->d_ks, sizeof(dda::KState) * nrhs));
  dda::KState* ks = c->d_ks;
  cudaStream_t st = c->stream;
  const bool ccg = (o.solver == DDA_CCG);
  const bool b2 = (o.solver == DDA_BICGSTAB2);
  const bool cocg = (o.solver == DDA_COCG);
  const bool qmr = (o.solver == DDA_QMRCS);
  if (b2 && !kv.u2) return Err::make(DDA_ESTATE, "BiCGstab(2) needs the extra Krylov vector");
  // preconditioned solves iterate on the scaled operator S A S (every product below)
  struct JacobiScope {
    dda_ctx* c;
    bool prev;
    JacobiScope(dda_ctx* cc, bool on) : c(cc), prev(cc->jacobi) { c->jacobi = on; }
    ~JacobiScope() { c->jacobi = prev; }
  } jscope(c, o.precond == DDA_PRECOND_JACOBI);
  if (have_x0) DDA_TRY(matvec<C>(c, kv.x, kv.r, nrhs, 0, false));
  if (cocg) {
    DDA_TRY(dda::cocg_init<C>(kv, ks, rb, nrhs, n3, tol, have_x0, st));
  } else if (qmr) {
    DDA_TRY(dda::qmr_init<C>(kv, ks, rb, nrhs, n3, tol, have_x0, st));
  } else if (ccg) {
    DDA_TRY(dda::ccg_init<C>(kv, ks, rb, nrhs, n3, tol, have_x0, st));
    DDA_TRY(matvec<C>(c, kv.r, kv.s, nrhs, 0, true));
    DDA_TRY(dda::ccg_start<C>(kv, ks, rb, nrhs, n3, st));
  } else if (b2) {
    DDA_TRY(dda::b2_init<C>(kv, ks, rb, nrhs, n3, tol, have_x0, st));
  } else {
    DDA_TRY(dda::bicg_init<C>(kv, ks, rb, nrhs, n3, tol, have_x0, st));
  }
  // BiCGstab in complex64 on the compile-time product with every RHS in one launch folds its
  // vector updates and dot products into the product's x passes: 7 launches per iteration
  // instead of 11 (DDA_FUSE=0 keeps them separate).  Decided below, once the workspace
  // capacity is known.
  bool fused = false;
  dda::RedBuf rbx{};
  // Programmatic dependent launch inside the iteration chain (DDA_PDL=1): every kernel
  // of an iteration may be scheduled behind its predecessor's tail (pdl.cuh).
  const char* pdl_env = std::getenv("DDA_PDL");
  const bool pdl = pdl_env && std::atoi(pdl_env) != 0;
  struct PdlScope {
    bool prev;
    explicit PdlScope(bool on) : prev(dda::pdl_enabled()) { dda::set_pdl(on); }
    ~PdlScope() { dda::set_pdl(prev); }
  };
  // one_iter: one BiCGstab / CCG iteration (2 products), or one BiCGstab(2) cycle (4 products)
  auto one_iter = [&]() -> Err {
    PdlScope scope(pdl);
    if (b2) {
      // r0 = r, r1 = s, r2 = t, u0 = p, u1 = v, u2 = u2
      DDA_TRY(dda::b2_u_update<C>(kv, ks, 0, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.p, kv.v, nrhs, 0, false, ks));
      DDA_TRY(dda::b2_alpha<C>(kv, ks, rb, 0, nrhs, n3, st));
      DDA_TRY(dda::b2_r_update<C>(kv, ks, 0, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.r, kv.s, nrhs, 0, false, ks));
      DDA_TRY(dda::b2_beta<C>(kv, ks, rb, nrhs, n3, st));
      DDA_TRY(dda::b2_u_update<C>(kv, ks, 1, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.v, kv.u2, nrhs, 0, false, ks));
      DDA_TRY(dda::b2_alpha<C>(kv, ks, rb, 1, nrhs, n3, st));
      DDA_TRY(dda::b2_r_update<C>(kv, ks, 1, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.s, kv.t, nrhs, 0, false, ks));
      DDA_TRY(dda::b2_mr<C>(kv, ks, rb, nrhs, n3, st));
    } else if (cocg) {
      DDA_TRY(matvec<C>(c, kv.p, kv.v, nrhs, 0, false, ks));
      DDA_TRY(dda::cocg_update<C>(kv, ks, rb, nrhs, n3, st));
    } else if (qmr) {
      DDA_TRY(matvec<C>(c, kv.p, kv.v, nrhs, 0, false, ks));
      DDA_TRY(dda::qmr_update<C>(kv, ks, rb, nrhs, n3, st));
    } else if (ccg) {
      DDA_TRY(matvec<C>(c, kv.p, kv.v, nrhs, 0, false, ks));
      DDA_TRY(dda::ccg_alpha_update<C>(kv, ks, rb, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.r, kv.s, nrhs, 0, true, ks));
      DDA_TRY(dda::ccg_beta_update<C>(kv, ks, rb, nrhs, n3, st));
    } else if (fused) {
      if constexpr (std::is_same<C, float2>::value) {
        dda::MvData<float2> d = Sel<float2>::data(c);
        d.ks = ks;
        const dda::Geom g = Sel<float2>::geom(c);
        DDA_TRY(dda::launch_bicg_half_c64(g, d, c->t64, kv, ks, rbx, nrhs, 0, st));
        DDA_TRY(dda::launch_bicg_half_c64(g, d, c->t64, kv, ks, rbx, nrhs, 1, st));
        DDA_TRY(dda::bicg_xr_update<C>(kv, ks, rb, nrhs, n3, st));
      }
    } else {
      DDA_TRY(dda::bicg_p_update<C>(kv, ks, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.p, kv.v, nrhs, 0, false, ks));
      DDA_TRY(dda::bicg_alpha<C>(kv, ks, rb, nrhs, n3, st));
      DDA_TRY(dda::bicg_s_update<C>(kv, ks, rb, nrhs, n3, st));
      DDA_TRY(matvec<C>(c, kv.s, kv.t, nrhs, 0, false, ks));
      DDA_TRY(dda::bicg_omega<C>(kv, ks, rb, nrhs, n3, st));
      DDA_TRY(dda::bicg_xr_update<C>(kv, ks, rb, nrhs, n3, st));
    }
    return Err::Ok();
  };
  const int every = o.check_every > 0 ? o.check_every : 8;
  DDA_TRY(ensure_small(c, sizeof(dda::KState) * nrhs));
  {
    int cap = 0;  // no allocation may happen while the stream is being captured
    DDA_TRY(ensure_work<C>(c, nrhs, &cap));
    const char* fe = std::getenv("DDA_FUSE");
    if constexpr (std::is_same<C, float2>::value) {
      fused = !(fe && std::atoi(fe) == 0) && !ccg && !b2 && !cocg && !qmr && c->t64.fast && cap >= nrhs;
      if (fused) {
        // the folded reductions' table follows the vector kernels' table in the same buffer
        const int nx = dda::x_ctas_per_rhs_c64(Sel<float2>::geom(c), c->t64);
        DDA_TRY(ensure_part(c, sizeof(double) * ((size_t)rb.nblk + nx) * nrhs * dda::kRedSlots));
        rb.part = c->d_part;
        rbx.part = c->d_part + (size_t)rb.nblk * nrhs * dda::kRedSlots;
        rbx.count = c->d_count;
        rbx.nblk = nx;
      }
    }
  }
  cudaGraphExec_t gexec = nullptr;
  unsigned long long graph_kernels = 0;
  const int gi = sizeof(C) == sizeof(float2) ? 0 : 1;
  const long long gkey[4] = {o.solver, 8LL * every + (c->jacobi ? 4 : 0) + (fused ? 2 : 0) + (pdl ? 1 : 0), nrhs,
                             (long long)n3};
  const bool reuse = o.use_graph && c->gexec[gi] && c->gexec_gen[gi] == c->gen &&
                     std::equal(gkey, gkey + 4, c->gexec_key[gi]);
  if (reuse) {
    gexec = c->gexec[gi];
    graph_kernels = c->gexec_kernels[gi];
  } else if (o.use_graph) {
    // capture `every` iterations; reuse the context's executable graph when only
    // parameters changed (cudaGraphExecUpdate), instantiate only when the topology did
    const unsigned long long before = dda::launches();
    cudaGraph_t graph = nullptr;
    DDA_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    Err e = Err::Ok();
    for (int k = 0; k < every && e.ok(); ++k) e = one_iter();
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (!e.ok()) { if (graph) cudaGraphDestroy(graph); return e; }
    if (ce != cudaSuccess) return Err::make(DDA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    // captured launches did not run: count them when the graph is replayed
    graph_kernels = dda::launches() - before;
    dda::sub_launches(graph_kernels);
    cudaGraphExec_t& cached = c->gexec[sizeof(C) == sizeof(float2) ? 0 : 1];
    bool updated = false;
    if (cached) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(cached, graph, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        cudaGraphExecDestroy(cached);
        cached = nullptr;
      }
    }
    if (!updated) {
      ce = cudaGraphInstantiate(&cached, graph, 0);
      if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        cached = nullptr;
        return Err::make(DDA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
      }
    }
    cudaGraphDestroy(graph);
    gexec = cached;
    c->gexec_gen[gi] = c->gen;
    std::copy(gkey, gkey + 4, c->gexec_key[gi]);
    c->gexec_kernels[gi] = graph_kernels;
  }
  std::vector<dda::KState> hk(nrhs);
  int it = 0;
  Err res = Err::Ok();
  const int it_per_call = b2 ? 2 : 1;  // iterations (2 products each) per one_iter
  while (true) {
    DDA_CU(cudaMemcpyAsync(c->h_pinned, ks, sizeof(dda::KState) * nrhs, cudaMemcpyDeviceToHost, st));
    DDA_CU(cudaStreamSynchronize(st));
    std::memcpy(hk.data(), c->h_pinned, sizeof(dda::KState) * nrhs);
    bool all = true;
    for (int b = 0; b < nrhs; ++b) all = all && (hk[b].done != 0);
    if (all || it >= maxit) break;
    if (o.timeout_ms > 0) {
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (ms > o.timeout_ms) { *timed_out = true; break; }
    }
    if (gexec) {
      cudaError_t ce = cudaGraphLaunch(gexec, st);
      if (ce != cudaSuccess) { res = Err::make(DDA_ECUDA, std::string("graph launch: ") + cudaGetErrorString(ce)); break; }
      dda::add_launches(graph_kernels);
    } else {
      for (int k = 0; k < every && res.ok(); ++k) res = one_iter();
      if (!res.ok()) break;
    }
    it += every * it_per_call;
  }
  DDA_TRY(res);
  stats->iters.resize(nrhs);
  stats->done.resize(nrhs);
  stats->mv.resize(nrhs);
  for (int b = 0; b < nrhs; ++b) {
    stats->iters[b] = hk[b].it;
    stats->done[b] = hk[b].done;
    stats->mv[b] = hk[b].mv + (have_x0 ? 1 : 0);
  }
  return Err::Ok();
}

}  // namespace

// ============================================================================ C ABI
// (the definitions take C linkage from their declarations in dda.h)

const char* dda_version(void) { return "dda-gb300 0.1 (sm_103a)"; }

dda_status dda_create(dda_ctx** out, int device, void* cuda_stream) {
  if (!out) return DDA_EINVAL;
  *out = nullptr;
  dda_ctx* c = new (std::nothrow) dda_ctx();
  if (!c) return DDA_ENOMEM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (device < 0) {
    c->host_only = true;
    *out = c;
    return DDA_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    delete c;
    return DDA_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return DDA_ECUDA;
  }
  dda::init_kernel_attrs();
  *out = c;
  return DDA_OK;
}

void dda_destroy(dda_ctx* c) {
  if (!c) return;
  if (c->host_only) {
    delete c;
    return;
  }
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_target(c);
  free_all(c);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->ev) cudaEventDestroy(c->ev);
  delete c;
}

const char* dda_last_error(const dda_ctx* c) { return c ? c->err.c_str() : "null context"; }

dda_status dda_set_stream(dda_ctx* c, void* s) {
  if (!c) return DDA_EINVAL;
  c->stream = (cudaStream_t)s;
  return DDA_OK;
}

dda_status dda_setup_shape(dda_ctx* c, int shape, const double* shpar, int nshpar, int64_t* n_out,
                           int32_t box_out[3]) {
  if (!c) return DDA_EINVAL;
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    dda::HostTarget t;
    e = dda::make_shape_target(shape, shpar, nshpar, &t);
    if (!e.ok()) return fail(c, e);
    drop_target(c);
    c->tgt = std::move(t);
    e = upload_target(c);
    if (!e.ok()) return fail(c, e);
    if (n_out) *n_out = c->n;
    if (box_out)
      for (int a = 0; a < 3; ++a) box_out[a] = c->tgt.box[a];
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

static dda_status setup_sites(dda_ctx* c, const int32_t* ixyz, const int32_t* icomp, int64_t n, const double origin[3],
                              const double a1[3], const double a2[3], bool per_axis,
                              const double* df_angles = nullptr) {
  if (!c) return DDA_EINVAL;
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    dda::HostTarget& t = c->tgt_next;  // built in the buffers of the target before last (warm pages)
    e = dda::make_site_target(ixyz, icomp, n, origin, a1, a2, &t, per_axis, df_angles);
    if (!e.ok()) return fail(c, e);
    drop_target(c);
    std::swap(c->tgt, t);
    e = upload_target(c);
    if (!e.ok()) return fail(c, e);
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_setup_target(dda_ctx* c, const int32_t* ixyz, const int32_t* icomp, int64_t n, const double origin[3],
                            const double a1[3], const double a2[3]) {
  return setup_sites(c, ixyz, icomp, n, origin, a1, a2, false);
}

dda_status dda_setup_target_aniso(dda_ctx* c, const int32_t* ixyz, const int32_t* icomp3, int64_t n,
                                  const double origin[3], const double a1[3], const double a2[3]) {
  if (!icomp3)
    return fail(c, Err::make(DDA_EINVAL, "dda_setup_target_aniso: a required pointer is NULL"));
  return setup_sites(c, ixyz, icomp3, n, origin, a1, a2, true);
}

dda_status dda_setup_target_anifrm(dda_ctx* c, const int32_t* ixyz, const int32_t* icomp3, int64_t n,
                                   const double origin[3], const double a1[3], const double a2[3],
                                   const double* df_angles) {
  if (!icomp3 || !df_angles)
    return fail(c, Err::make(DDA_EINVAL, "dda_setup_target_anifrm: a required pointer is NULL"));
  return setup_sites(c, ixyz, icomp3, n, origin, a1, a2, true, df_angles);
}

dda_status dda_get_sites(dda_ctx* c, int32_t* ixyz_out, double origin_out[3]) {
  if (!c) return DDA_EINVAL;
  if (!c->have_target) return fail(c, Err::make(DDA_ESTATE, "no target"));
  if (ixyz_out) std::memcpy(ixyz_out, c->tgt.ijk.data(), sizeof(int32_t) * c->tgt.ijk.size());
  if (origin_out) std::memcpy(origin_out, c->tgt.origin, sizeof(double) * 3);
  return DDA_OK;
}

dda_status dda_get_box(const dda_ctx* c, int64_t* n_out, int32_t box_out[3]) {
  if (!c) return DDA_EINVAL;
  if (!c->have_target) return DDA_ESTATE;
  if (n_out) *n_out = c->n;
  if (box_out)
    for (int a = 0; a < 3; ++a) box_out[a] = c->tgt.box[a];
  return DDA_OK;
}

dda_status dda_set_periodicity(dda_ctx* c, double py, double pz, double gamma) {
  if (!c) return DDA_EINVAL;
  if (!c->have_target) return fail(c, Err::make(DDA_ESTATE, "set a target first"));
  if (!(py >= 0) || !(pz >= 0) || !std::isfinite(py) || !std::isfinite(pz))
    return fail(c, Err::make(DDA_EINVAL, "periods must be >= 0 (0 = not periodic along that axis)"));
  if ((py > 0 && py < c->tgt.box[1]) || (pz > 0 && pz < c->tgt.box[2]))
    return fail(c, Err::make(DDA_EINVAL, "a period shorter than the unit cell's extent would overlap its replicas"));
  const bool per = py > 0 || pz > 0;
  if (per && !(gamma > 0 && gamma < 1)) return fail(c, Err::make(DDA_EINVAL, "gamma must be in (0, 1)"));
  c->per_y = py;
  c->per_z = pz;
  c->per_gamma = per ? gamma : 0.01;
  c->periodic = per;
  drop_green(c);
  return DDA_OK;
}

dda_status dda_kd_from_x(const dda_ctx* c, double x, double* kd_out, double* aeff_out) {
  if (!c || !(x > 0) || !std::isfinite(x)) return DDA_EINVAL;  // const context: status only
  if (!c->have_target || c->n <= 0) return DDA_ESTATE;
  // a_eff = (3 N / 4 pi)^(1/3) d: the radius of a sphere of the target's volume N d^3
  const double aeff = std::cbrt(3.0 * (double)c->n / (4.0 * 3.14159265358979323846));
  if (kd_out) *kd_out = x / aeff;
  if (aeff_out) *aeff_out = aeff;
  return DDA_OK;
}

dda_status dda_set_incident(dda_ctx* c, double kd, const double* ori, int n_ori, const double e01_lf[6], int iorth) {
  if (!c) return DDA_EINVAL;
  if (!c->have_target) return fail(c, Err::make(DDA_ESTATE, "set a target first"));
  if (!(kd > 0) || !std::isfinite(kd)) return fail(c, Err::make(DDA_EINVAL, "kd must be positive"));
  if (!ori || n_ori <= 0 || n_ori > 65535) return fail(c, Err::make(DDA_EINVAL, "need 1..65535 orientations"));
  if (iorth != 1 && iorth != 2) return fail(c, Err::make(DDA_EINVAL, "iorth must be 1 or 2"));
  if (!e01_lf) return fail(c, Err::make(DDA_EINVAL, "e01 missing"));
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    cd e01[3];
    double nrm = 0;
    for (int a = 0; a < 3; ++a) {
      e01[a] = cd(e01_lf[2 * a], e01_lf[2 * a + 1]);
      nrm += std::norm(e01[a]);
    }
    if (!(nrm > 0)) return fail(c, Err::make(DDA_EINVAL, "e01 is zero"));
    nrm = std::sqrt(nrm);
    for (int a = 0; a < 3; ++a) e01[a] /= nrm;
    if (std::abs(e01[0]) > 1e-12) return fail(c, Err::make(DDA_EINVAL, "e01 must be transverse to x_LF"));
    // e02 = x_LF x conj(e01)
    cd e02[3] = {cd(0, 0), -std::conj(e01[2]), std::conj(e01[1])};
    drop_incident(c);
    c->kd = kd;
    c->n_ori = n_ori;
    c->iorth = iorth;
    c->nrhs = n_ori * iorth;
    c->ori.assign(ori, ori + 3 * n_ori);
    for (int a = 0; a < 3; ++a) { c->e01[a] = e01[a]; c->e02[a] = e02[a]; }
    c->axes.resize(9 * n_ori);
    c->rg.resize(c->nrhs);
    for (int o = 0; o < n_ori; ++o) {
      double* ax = &c->axes[9 * o];
      lab_axes(c->tgt.a1, c->tgt.a2, ori[3 * o], ori[3 * o + 1], ori[3 * o + 2], ax);
      for (int l = 0; l < iorth; ++l) {
        dda::RhsGeom& g = c->rg[o * iorth + l];
        const cd* ep = (l == 0) ? e01 : e02;
        for (int k = 0; k < 3; ++k) {
          g.k[k] = kd * ax[k];
          const cd v = ep[0] * ax[k] + ep[1] * ax[3 + k] + ep[2] * ax[6 + k];
          g.e[2 * k] = v.real();
          g.e[2 * k + 1] = v.imag();
        }
      }
    }
    if (!c->host_only) {
      e = grow(c, &c->d_rg, sizeof(dda::RhsGeom) * c->nrhs);
      if (!e.ok()) return fail(c, e);
      if (cudaMemcpy(c->d_rg, c->rg.data(), sizeof(dda::RhsGeom) * c->nrhs, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(c, Err::make(DDA_ECUDA, "copy of incidence failed"));
    }
    c->have_inc = true;
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

int dda_nrhs(const dda_ctx* c) { return (c && c->have_inc) ? c->nrhs : 0; }

dda_status dda_get_incidence(dda_ctx* c, double* k_tf, double* e_tf) {
  if (!c) return DDA_EINVAL;
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the incident beams first"));
  for (int b = 0; b < c->nrhs; ++b) {
    if (k_tf)
      for (int k = 0; k < 3; ++k) k_tf[3 * b + k] = c->rg[b].k[k];
    if (e_tf)
      for (int k = 0; k < 6; ++k) e_tf[6 * b + k] = c->rg[b].e[k];
  }
  return DDA_OK;
}

dda_status dda_incident_field(dda_ctx* c, void* e_dev, int dtype) {
  if (!c) return DDA_EINVAL;
  if (!e_dev)
    return fail(c, Err::make(DDA_EINVAL, "dda_incident_field: a required pointer is NULL"));
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the incident beams first"));
  Err e = need_device(c);
  if (!e.ok()) return fail(c, e);
  e = set_dev(c);
  if (!e.ok()) return fail(c, e);
  if (dtype == DDA_C64)
    e = dda::incident_field<float2>(c->d_ijk, c->d_origin, c->d_rg, c->nrhs, c->n, (float2*)e_dev, c->stream);
  else if (dtype == DDA_C128)
    e = dda::incident_field<double2>(c->d_ijk, c->d_origin, c->d_rg, c->nrhs, c->n, (double2*)e_dev, c->stream);
  else
    return fail(c, Err::make(DDA_EINVAL, "dtype must be DDA_C64 or DDA_C128"));
  return e.ok() ? DDA_OK : fail(c, e);
}

dda_status dda_build_green_fft(dda_ctx* c, const int32_t pad[3]) {
  if (!c) return DDA_EINVAL;
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the incident beams (kd) first"));
  try {
    Err e = need_device(c);
    if (!e.ok()) return fail(c, e);
    e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    int P[3];
    for (int a = 0; a < 3; ++a) {
      if (pad) {
        P[a] = pad[a];
        if (P[a] < 2 * c->tgt.box[a] || (P[a] % 2) || !dda::is_smooth235(P[a]))
          return fail(c, Err::make(DDA_EINVAL, "pad must be even, >= 2 N per axis and 2,3,5-smooth"));
      } else {
        int v = 2 * c->tgt.box[a];
        while (!dda::is_smooth235(v)) v += 2;
        P[a] = v;
      }
    }
    drop_green(c);
    dda::Geom g{};
    g.n = c->n;
    g.nx = c->tgt.box[0]; g.ny = c->tgt.box[1]; g.nz = c->tgt.box[2];
    g.px = P[0]; g.py = P[1]; g.pz = P[2];
    g.ncomp = c->tgt.ncomp;
    e = dda::make_plan(g.px, &g.plx);
    if (e.ok()) e = dda::make_plan(g.py, &g.ply);
    if (e.ok()) e = dda::make_plan(g.pz, &g.plz);
    if (!e.ok()) return fail(c, e);
    // twiddles exp(-2 pi i j / L) in FP64 on the host (kept while the padded lengths stay the same)
    const double pi = 3.14159265358979323846;
    for (int a = 0; a < 3; ++a) {
      const int L = P[a];
      if (c->tw_len[a] == L && c->d_tw128[a] && c->d_tw64[a] && c->d_twdf[a]) continue;
      std::vector<double2> t128(L);
      std::vector<float2> t64(L);
      std::vector<dda::dfp::dfc> tdf(L);
      for (int j = 0; j < L; ++j) {
        const double ang = -2.0 * pi * (double)j / (double)L;
        t128[j] = make_double2(std::cos(ang), std::sin(ang));
        t64[j] = make_float2((float)t128[j].x, (float)t128[j].y);
        tdf[j].x = dda::dfp::df(t128[j].x);
        tdf[j].y = dda::dfp::df(t128[j].y);
      }
      e = grow(c, &c->d_tw128[a], sizeof(double2) * L);
      if (e.ok()) e = grow(c, &c->d_tw64[a], sizeof(float2) * L);
      if (e.ok()) e = grow(c, &c->d_twdf[a], sizeof(dda::dfp::dfc) * L);
      if (!e.ok()) return fail(c, e);
      e = cuda_ok(cudaMemcpy(c->d_tw128[a], t128.data(), sizeof(double2) * L, cudaMemcpyHostToDevice), "twiddle upload");
      if (e.ok()) e = cuda_ok(cudaMemcpy(c->d_tw64[a], t64.data(), sizeof(float2) * L, cudaMemcpyHostToDevice), "twiddle upload");
      if (e.ok())
        e = cuda_ok(cudaMemcpy(c->d_twdf[a], tdf.data(), sizeof(dda::dfp::dfc) * L, cudaMemcpyHostToDevice),
                    "twiddle upload");
      if (!e.ok()) return fail(c, e);
      c->tw_len[a] = L;
    }
    // schedule: 3-pass when the plane fits in the opt-in shared memory
    int smax = 0;
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    dda::MvTune t64{}, t128{};
    t64.g = 8; t128.g = 4;
    dda::Geom g64 = g, g128 = g;
    g64.ys = g.ny; g128.ys = g.ny;
    dda::choose_fast_schedule(g64, true, smax, &t64);
    dda::choose_fast_schedule(g128, false, smax, &t128);
    if (!t64.fast) t64.plane = dda::plane_smem_bytes<float2>(g64, t64) <= (size_t)smax;
    if (!t128.fast) t128.plane = dda::plane_smem_bytes<double2>(g128, t128) <= (size_t)smax;
    // DDA_SCHEDULE pins the schedule instead of autotuning it: "generic" (shared-memory
    // engine of fft.cuh), "fast5" (compile-time kernels, 5 passes), "plane512" / "plane768"
    // (compile-time kernels, fused plane pass where it exists), "cluster2" / "cluster4"
    // (complex64 plane pass split over a cluster of 2 or 4 CTAs where it fits)
    // the same grid as the previous build keeps its tuned schedules (no new tuning, no new graph)
    const bool same_grid = c->have_sched && c->g64.n == g.n && c->g64.nx == g.nx && c->g64.ny == g.ny &&
                           c->g64.nz == g.nz && c->g64.px == g.px && c->g64.py == g.py && c->g64.pz == g.pz &&
                           c->g64.ncomp == g.ncomp;
    const bool prev_forced = c->forced_schedule;
    c->forced_schedule = false;
    if (const char* f = std::getenv("DDA_SCHEDULE")) {
      const std::string sched(f);
      if (sched == "generic") {
        t64.fast = t128.fast = false;
        t64.plane = dda::plane_smem_bytes<float2>(g64, t64) <= (size_t)smax;
        t128.plane = dda::plane_smem_bytes<double2>(g128, t128) <= (size_t)smax;
        c->forced_schedule = true;
      } else if (sched == "fast5") {
        t64.plane = t128.plane = false;
        c->forced_schedule = true;
      } else if (sched == "plane512" || sched == "plane768") {
        t64.thr_p = t128.thr_p = (sched == "plane768") ? 768 : 512;
        c->forced_schedule = true;
      } else if (sched == "cluster2" || sched == "cluster4") {
        const int S = sched == "cluster2" ? 2 : 4;
        if (t64.plane_ok && dda::plane_cluster_capacity_c64(g64, S, smax) > 0) t64.clus = S;
        c->forced_schedule = true;
      }
    }
    // DDA_BULK=1 / 0 pins bulk-copy staging of the plane pass on / off
    if (const char* f = std::getenv("DDA_BULK")) {
      t64.bulk = (std::atoi(f) != 0) && t64.plane_ok && dda::plane_bulk_ok_c64(g64, smax);
      c->forced_schedule = true;
    }
    // DDA_ZFUSE=1 / 0 pins the register-fused 5-pass z columns on / off (complex64, where they exist)
    if (const char* f = std::getenv("DDA_ZFUSE")) {
      t64.zr = (std::atoi(f) != 0 && t64.fast && dda::zcols_rfuse_available_c64(g64)) ? 1 : 0;
      c->forced_schedule = true;
    }
    // DDA_XCOMP=1 runs the x passes with one component per CTA
    if (const char* f = std::getenv("DDA_XCOMP")) {
      if (std::atoi(f) == 1) {
        if (t64.fast) t64.xnc = 1;
        if (t128.fast) t128.xnc = 1;
      }
      c->forced_schedule = true;
    }
    // DDA_XTILE pins the x passes' tile height (y rows per CTA: 4, 8 or 16 where instantiated)
    if (const char* f = std::getenv("DDA_XTILE")) {
      const int ty = std::atoi(f);
      if (t64.fast && dda::x_tile_height_ok(sizeof(float2), g.px, ty)) t64.xty = ty;
      if (t128.fast && dda::x_tile_height_ok(sizeof(double2), g.px, ty)) t128.xty = ty;
      c->forced_schedule = true;
    }
    if (!t64.plane) g64.ys = g.py;
    if (!t128.plane) g128.ys = g.py;
    if (!(same_grid && !prev_forced && !c->forced_schedule)) {
      // a different geometry or schedule invalidates the tuning and the captured iteration graphs
      c->g64 = g64; c->g128 = g128; c->t64 = t64; c->t128 = t128;
      c->tuned_nrhs[0] = c->tuned_nrhs[1] = 0;
      c->gen++;
      c->have_sched = true;
    }
    const int64_t M = (int64_t)g.px * g.py * g.pz;
    e = grow(c, &c->d_ghat128, sizeof(double2) * 6 * M);
    if (e.ok()) e = grow(c, &c->d_ghat64, sizeof(float2) * 6 * M);
    if (e.ok()) e = grow(c, &c->d_gscratch, sizeof(double2) * 6 * M);
    // the double-float copy exists only where the double-float product can run
    c->ghatdf_valid = false;
    const bool want_df = c->t128.fast && !c->t128.plane;
    if (e.ok() && want_df) e = grow(c, &c->d_ghatdf, sizeof(dda::dfp::dfc) * 6 * M);
    if (!e.ok()) return fail(c, e);
    // frequency-order tables of the Green build (kept while px, py stay the same)
    if (e.ok() && (c->gperm_key[0] != g.px || c->gperm_key[1] != g.py || !c->d_gperm)) {
      std::vector<int32_t> tab;
      dda::green_perm_tables(g64, &tab);
      e = grow(c, &c->d_gperm, sizeof(int32_t) * tab.size());
      if (e.ok() && cudaMemcpy(c->d_gperm, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice) !=
                        cudaSuccess)
        e = Err::make(DDA_ECUDA, "Green-table upload failed");
      if (e.ok()) { c->gperm_key[0] = g.px; c->gperm_key[1] = g.py; }
    }
    if (!e.ok()) return fail(c, e);
    if (c->periodic) {
      // the periodic interaction depends on the incidence through the replicas' Bloch phases: every
      // RHS of the context must share one k in the TF (one orientation, or orientations that differ
      // only in Phi)
      for (int b = 1; b < c->nrhs; ++b)
        for (int q = 0; q < 3; ++q)
          if (std::abs(c->rg[b].k[q] - c->rg[0].k[q]) > 1e-12 * c->kd)
            return fail(c, Err::make(DDA_EUNSUPPORTED, "a periodic target needs every RHS to share one incident "
                                                       "direction in the Target Frame"));
      e = dda::build_green_pbc(g64, c->kd, c->rg[0].k, c->per_y, c->per_z, c->per_gamma, c->d_tw128[0],
                               c->d_tw128[1], c->d_tw128[2], c->d_gscratch, c->d_ghat128, c->d_ghat64,
                               want_df ? c->d_ghatdf : nullptr, c->stream);
    } else {
      e = dda::build_green(g64, c->kd, c->d_tw128[0], c->d_tw128[1], c->d_tw128[2], c->d_gperm, c->d_gscratch,
                           c->d_ghat128, c->d_ghat64, want_df ? c->d_ghatdf : nullptr, c->stream);
    }
    if (!e.ok()) return fail(c, e);
    c->ghatdf_valid = want_df;
    c->have_green = true;
    // set-up of dda_matvec_noalloc, once per device with this device current: look up the device
    // address of its fixed scratch array (the array sits in the module of the Green-tensor kernels
    // just launched, so the lookup loads nothing new)
    {
      void* scratch = nullptr;
      e = dda::noalloc_scratch(c->device, &scratch);
      if (!e.ok()) return fail(c, e);
    }
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_set_polarizability(dda_ctx* c, int presc, const double* m_reim, int ncomp) {
  if (!c) return DDA_EINVAL;
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the incident beams (kd) first"));
  if (presc != DDA_CM && presc != DDA_LATTDR && presc != DDA_GKDLDR)
    return fail(c, Err::make(DDA_EINVAL, "unknown prescription"));
  if (!m_reim || ncomp < c->tgt.ncomp || ncomp > 255)
    return fail(c, Err::make(DDA_EINVAL, "need one refractive index per composition"));
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    std::vector<cd> ia((size_t)c->nrhs * ncomp * 3);
    for (int b = 0; b < c->nrhs; ++b) {
      const dda::RhsGeom& g = c->rg[b];
      const double kh[3] = {g.k[0] / c->kd, g.k[1] / c->kd, g.k[2] / c->kd};
      const cd ev[3] = {cd(g.e[0], g.e[1]), cd(g.e[2], g.e[3]), cd(g.e[4], g.e[5])};
      for (int m = 0; m < ncomp; ++m) {
        const cd mm(m_reim[2 * m], m_reim[2 * m + 1]);
        if (!std::isfinite(mm.real()) || !std::isfinite(mm.imag()))
          return fail(c, Err::make(DDA_EINVAL, "refractive index is not finite"));
        if (std::abs(mm * mm - 1.0) == 0.0) return fail(c, Err::make(DDA_EINVAL, "m = 1 has no polarizability"));
        cd* out = &ia[((size_t)b * ncomp + m) * 3];
        inv_alpha(presc, mm, c->kd, kh, ev, out);
        for (int a = 0; a < 3; ++a)
          if (!std::isfinite(out[a].real()) || !std::isfinite(out[a].imag()))
            return fail(c, Err::make(DDA_EINVAL, "1/alpha is not finite for this refractive index"));
      }
    }
    std::vector<double2> h128(ia.size());
    std::vector<float2> h64(ia.size());
    std::vector<dda::dfp::dfc> hdf(ia.size());
    for (size_t i = 0; i < ia.size(); ++i) {
      h128[i] = make_double2(ia[i].real(), ia[i].imag());
      h64[i] = make_float2((float)ia[i].real(), (float)ia[i].imag());
      hdf[i].x = dda::dfp::df(ia[i].real());
      hdf[i].y = dda::dfp::df(ia[i].imag());
    }
    drop_alpha(c);
    if (!c->host_only) {
      e = grow(c, &c->d_ia128, sizeof(double2) * ia.size());
      if (e.ok()) e = grow(c, &c->d_ia64, sizeof(float2) * ia.size());
      if (e.ok()) e = grow(c, &c->d_iadf, sizeof(dda::dfp::dfc) * ia.size());
      if (!e.ok()) return fail(c, e);
      e = cuda_ok(cudaMemcpy(c->d_ia128, h128.data(), sizeof(double2) * ia.size(), cudaMemcpyHostToDevice),
                  "polarizability upload");
      if (e.ok())
        e = cuda_ok(cudaMemcpy(c->d_ia64, h64.data(), sizeof(float2) * ia.size(), cudaMemcpyHostToDevice),
                    "polarizability upload");
      if (e.ok())
        e = cuda_ok(cudaMemcpy(c->d_iadf, hdf.data(), sizeof(dda::dfp::dfc) * ia.size(), cudaMemcpyHostToDevice),
                    "polarizability upload");
      if (!e.ok()) return fail(c, e);
    }
    if (!c->tgt.dfrot.empty()) {
      // rotated dielectric frames: alpha^{-1} = sum_j d_j e_j e_j^T, d_j from the prescription for
      // composition icomp(site, j) with the incidence projected on the principal axes e_j
      const int64_t n = c->n;
      const size_t nt = (size_t)c->nrhs * n * 6;
      std::vector<double2> t128(nt);
      std::vector<float2> t64(nt);
      for (int b = 0; b < c->nrhs; ++b) {
        const dda::RhsGeom& g = c->rg[b];
        const double kh[3] = {g.k[0] / c->kd, g.k[1] / c->kd, g.k[2] / c->kd};
        const cd ev[3] = {cd(g.e[0], g.e[1]), cd(g.e[2], g.e[3]), cd(g.e[4], g.e[5])};
        for (int64_t j = 0; j < n; ++j) {
          const double* R = &c->tgt.dfrot[9 * j];
          double khd[3];
          cd evd[3];
          for (int a = 0; a < 3; ++a) {
            khd[a] = kh[0] * R[a] + kh[1] * R[3 + a] + kh[2] * R[6 + a];
            evd[a] = ev[0] * R[a] + ev[1] * R[3 + a] + ev[2] * R[6 + a];
          }
          cd d[3];
          for (int a = 0; a < 3; ++a) {
            const int cc = c->tgt.comp[3 * j + a];
            cd o3[3];
            inv_alpha(presc, cd(m_reim[2 * cc], m_reim[2 * cc + 1]), c->kd, khd, evd, o3);
            d[a] = o3[a];
          }
          static const int rows[6] = {0, 0, 0, 1, 1, 2}, cols[6] = {0, 1, 2, 1, 2, 2};
          for (int q = 0; q < 6; ++q) {
            cd v(0, 0);
            for (int a = 0; a < 3; ++a) v += d[a] * (R[3 * rows[q] + a] * R[3 * cols[q] + a]);
            const size_t o = ((size_t)b * n + j) * 6 + q;
            t128[o] = make_double2(v.real(), v.imag());
            t64[o] = make_float2((float)v.real(), (float)v.imag());
          }
        }
      }
      if (!c->host_only) {
        e = grow(c, &c->d_iat128, sizeof(double2) * nt);
        if (e.ok()) e = grow(c, &c->d_iat64, sizeof(float2) * nt);
        if (e.ok()) e = cuda_ok(cudaMemcpy(c->d_iat128, t128.data(), sizeof(double2) * nt, cudaMemcpyHostToDevice),
                                "polarizability tensor upload");
        if (e.ok()) e = cuda_ok(cudaMemcpy(c->d_iat64, t64.data(), sizeof(float2) * nt, cudaMemcpyHostToDevice),
                                "polarizability tensor upload");
        if (!e.ok()) return fail(c, e);
      }
      c->iat_valid = true;
      c->gen++;
    }
    c->ia = std::move(ia);
    c->eps.resize(ncomp);
    for (int m = 0; m < ncomp; ++m) {
      const cd mm(m_reim[2 * m], m_reim[2 * m + 1]);
      c->eps[m] = mm * mm;
    }
    c->presc = presc;
    if (c->ncomp != ncomp) c->gen++;
    c->ncomp = ncomp;
    c->have_alpha = true;
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_get_inv_alpha(dda_ctx* c, double* out) {
  if (!c) return DDA_EINVAL;
  if (!out)
    return fail(c, Err::make(DDA_EINVAL, "dda_get_inv_alpha: a required pointer is NULL"));
  if (!c->have_alpha) return fail(c, Err::make(DDA_ESTATE, "no polarizability"));
  for (size_t i = 0; i < c->ia.size(); ++i) {
    out[2 * i] = c->ia[i].real();
    out[2 * i + 1] = c->ia[i].imag();
  }
  return DDA_OK;
}

dda_status dda_matvec(dda_ctx* c, const void* p, void* ap, int nrhs, int dtype) {
  if (!c) return DDA_EINVAL;
  if (!p || !ap)
    return fail(c, Err::make(DDA_EINVAL, "dda_matvec: a required pointer is NULL"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  if (nrhs < 1 || nrhs > c->nrhs) return fail(c, Err::make(DDA_EINVAL, "nrhs out of range"));
  if (p == ap) return fail(c, Err::make(DDA_EINVAL, "p and ap may not alias"));
  Err e = set_dev(c);
  if (!e.ok()) return fail(c, e);
  if (dtype == DDA_C64) {
    e = ensure_tuned<float2>(c, nrhs);
    if (e.ok()) e = matvec<float2>(c, (const float2*)p, (float2*)ap, nrhs, 0, false);
  } else if (dtype == DDA_C128) {
    e = ensure_tuned<double2>(c, nrhs);
    if (e.ok()) e = matvec<double2>(c, (const double2*)p, (double2*)ap, nrhs, 0, false);
  } else if (dtype == DDA_C128DF) {
    e = ensure_tuned<double2>(c, nrhs);
    if (e.ok()) e = matvec_df(c, (const double2*)p, (double2*)ap, nrhs, 0, false);
  } else {
    return fail(c, Err::make(DDA_EINVAL, "dtype must be DDA_C64, DDA_C128 or DDA_C128DF"));
  }
  return e.ok() ? DDA_OK : fail(c, e);
}

namespace {
template <typename C>
Err kvec_alloc(dda_ctx* c, dda::KrylovVecs<C>* kv, int nvec_extra) {
  const size_t one = sizeof(C) * (size_t)c->nrhs * 3 * c->n;
  const size_t need = one * (8 + nvec_extra);
  DDA_TRY(grow(c, &c->d_kvec, need));
  C* base = (C*)c->d_kvec;
  const size_t el = (size_t)c->nrhs * 3 * c->n;
  kv->x = base; kv->r = base + el; kv->rhat = base + 2 * el; kv->p = base + 3 * el;
  kv->v = base + 4 * el; kv->s = base + 5 * el; kv->t = base + 6 * el; kv->b = base + 7 * el;
  kv->u2 = nvec_extra >= 1 ? base + 8 * el : nullptr;
  return Err::Ok();
}

// Jacobi scaling tables s = alpha^{1/2} (principal square root of 1 / alpha^{-1}) per RHS,
// composition and axis, from the host copy of alpha^{-1}; complex128 and complex64 copies.
Err ensure_scale(dda_ctx* c, double* kappa) {
  const size_t nv = (size_t)c->nrhs * c->ncomp * 3;
  if (c->ia.size() != nv) return Err::make(DDA_ESTATE, "polarizabilities missing");
  std::vector<double2> s128(nv);
  std::vector<float2> s64(nv);
  double smax = 0.0, smin = 1e300;
  for (size_t i = 0; i < nv; ++i) {
    const cd s = std::sqrt(1.0 / c->ia[i]);
    smax = std::max(smax, std::abs(s));
    smin = std::min(smin, std::abs(s));
    s128[i] = make_double2(s.real(), s.imag());
    s64[i] = make_float2((float)s.real(), (float)s.imag());
  }
  DDA_TRY(grow(c, &c->d_sc128, sizeof(double2) * nv));
  DDA_TRY(grow(c, &c->d_sc64, sizeof(float2) * nv));
  DDA_CU(cudaMemcpyAsync(c->d_sc128, s128.data(), sizeof(double2) * nv, cudaMemcpyHostToDevice, c->stream));
  DDA_CU(cudaMemcpyAsync(c->d_sc64, s64.data(), sizeof(float2) * nv, cudaMemcpyHostToDevice, c->stream));
  DDA_CU(cudaStreamSynchronize(c->stream));  // the host vectors go out of scope
  *kappa = smin > 0 ? smax / smin : 1.0;
  return Err::Ok();
}

// true residual (FP64 product): |E - A P|^2 and |E|^2 per RHS
// (use_df: the product in double-float arithmetic, matvec_df)
Err true_residual(dda_ctx* c, const double2* p, double2* scratch_ax, double2* scratch_r, std::vector<double>* rel,
                  bool use_df) {
  const int nrhs = c->nrhs;
  const int64_t n3 = 3 * c->n;
  if (use_df) DDA_TRY(matvec_df(c, p, scratch_ax, nrhs, 0, false));
  else DDA_TRY(matvec<double2>(c, p, scratch_ax, nrhs, 0, false));
  dda::RedBuf rb = redbuf(c, nrhs, n3);
  DDA_TRY(ensure_part(c, sizeof(double) * (size_t)rb.nblk * nrhs * dda::kRedSlots));
  rb.part = c->d_part;
  rb.count = c->d_count;
  DDA_TRY(ensure_small(c, sizeof(double) * 2 * nrhs + sizeof(dda::KState) * nrhs));
  DDA_TRY(dda::residual_c128(c->d_e128, scratch_ax, scratch_r, c->d_small, rb, nrhs, n3, c->stream));
  DDA_CU(cudaMemcpyAsync(c->h_pinned, c->d_small, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, c->stream));
  DDA_CU(cudaStreamSynchronize(c->stream));
  rel->resize(nrhs);
  for (int b = 0; b < nrhs; ++b) {
    const double rr = c->h_pinned[2 * b], bb = c->h_pinned[2 * b + 1];
    (*rel)[b] = bb > 0 ? std::sqrt(rr / bb) : 0.0;
  }
  return Err::Ok();
}
}  // namespace

dda_status dda_solve(dda_ctx* c, const dda_solve_opts* opt, void* p_dev, dda_solve_report* rep) {
  if (!c) return DDA_EINVAL;
  if (!opt || !p_dev)
    return fail(c, Err::make(DDA_EINVAL, "dda_solve: a required pointer is NULL"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  dda_solve_opts o = *opt;
  if (o.solver != DDA_BICGSTAB && o.solver != DDA_CCG && o.solver != DDA_BICGSTAB2 && o.solver != DDA_COCG &&
      o.solver != DDA_QMRCS)
    return fail(c, Err::make(DDA_EINVAL, "unknown solver"));
  if (o.precond != DDA_PRECOND_NONE && o.precond != DDA_PRECOND_JACOBI)
    return fail(c, Err::make(DDA_EINVAL, "unknown preconditioner"));
  if (o.precision < DDA_PREC_C64 || o.precision > DDA_PREC_MIXED)
    return fail(c, Err::make(DDA_EINVAL, "unknown precision"));
  if (!(o.tol > 0) || o.maxit < 1) return fail(c, Err::make(DDA_EINVAL, "tol must be > 0 and maxit >= 1"));
  // QMR without look-ahead needs FP64 vectors: a plane-wave start across several wavelengths makes
  // v^T v nearly vanish (near breakdown of the symmetric Lanczos process, |v^T v| ~ 1e-8 |v|^2 on the
  // guide's Au block), and w = A v - alpha v - beta v_prev then cancels beyond complex64's precision
  if (o.solver == DDA_QMRCS && o.precision != DDA_PREC_C128)
    return fail(c, Err::make(DDA_EUNSUPPORTED, "QMR-CS runs in complex128 only (no look-ahead)"));
  // Default streams cannot be captured: run the solve on a context-owned stream
  // ordered after the caller's work (the call is synchronous, so nothing is
  // needed afterwards).
  cudaStream_t user = c->stream;
  struct Restore { dda_ctx* c; cudaStream_t s; ~Restore() { c->stream = s; } } restore{c, user};
  if (o.use_graph && (user == nullptr || user == cudaStreamLegacy || user == cudaStreamPerThread)) {
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, Err::make(DDA_ECUDA, "cudaSetDevice failed"));
    if (!c->own_stream && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, Err::make(DDA_ECUDA, "stream creation failed"));
    if (!c->ev && cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, Err::make(DDA_ECUDA, "event creation failed"));
    cudaEventRecord(c->ev, user);
    cudaStreamWaitEvent(c->own_stream, c->ev, 0);
    c->stream = c->own_stream;
  }
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    const auto t0 = std::chrono::steady_clock::now();
    const int nrhs = c->nrhs;
    const int64_t n3 = 3 * c->n;
    const int64_t el = (int64_t)nrhs * n3;
    double2* P = (double2*)p_dev;
    e = ensure_einc(c);
    if (e.ok()) e = ensure_tuned<double2>(c, nrhs);
    if (e.ok() && o.precision != DDA_PREC_C128) e = ensure_tuned<float2>(c, nrhs);
    if (!e.ok()) return fail(c, e);
    const bool jac = o.precond == DDA_PRECOND_JACOBI;
    if (jac && c->iat_valid)
      return fail(c, Err::make(DDA_EUNSUPPORTED, "Jacobi scaling needs dielectric tensors diagonal in the TF"));
    double kappa = 1.0;  // max |s| / min |s|: the scaled residual test at tol / kappa implies |E - A P| <= tol |E|
    if (jac) e = ensure_scale(c, &kappa);
    if (!e.ok()) return fail(c, e);
    const double ktol = o.tol / kappa;  // Krylov tolerance of the complex64 / complex128 solves
    // Jacobi: the Krylov solver works on S A S y = S b with x = S y (S = diag(alpha^{1/2}))
    const uint8_t* comp = c->comp_valid ? c->d_comp : nullptr;
    auto scale64 = [&](float2* v, bool inv) {
      return jac ? dda::scale_sites<float2>(v, c->d_sc64, comp, c->ncomp, nrhs, c->n, inv, c->stream) : Err::Ok();
    };
    auto scale128 = [&](double2* v, bool inv) {
      return jac ? dda::scale_sites<double2>(v, c->d_sc128, comp, c->ncomp, nrhs, c->n, inv, c->stream) : Err::Ok();
    };
    // Phi reuse: orientations that differ from an earlier one only in Phi see the same k in the TF,
    // so for alpha independent of the polarization (CM, GKDLDR) their two solutions are linear
    // combinations of the earlier orientation's two; those RHS are not iterated on
    std::vector<int> rep_of(c->n_ori, -1);
    bool reuse = o.phi_reuse != 0 && c->iorth == 2 && (c->presc == DDA_CM || c->presc == DDA_GKDLDR);
    if (reuse) {
      bool any = false;
      for (int a = 0; a < c->n_ori; ++a)
        for (int r = 0; r < a && rep_of[a] < 0; ++r)
          if (rep_of[r] < 0 && c->ori[3 * r] == c->ori[3 * a] && c->ori[3 * r + 1] == c->ori[3 * a + 1]) {
            rep_of[a] = r;
            any = true;
          }
      reuse = any;
    }
    std::vector<char> masked(nrhs, 0);
    if (reuse)
      for (int b = 0; b < nrhs; ++b) masked[b] = rep_of[b / 2] >= 0 ? 1 : 0;
    auto zero_masked = [&](void* v, size_t csize) -> Err {
      for (int b = 0; b < nrhs; ++b)
        if (masked[b]) DDA_CU(cudaMemsetAsync((char*)v + csize * (size_t)b * n3, 0, csize * n3, c->stream));
      return Err::Ok();
    };
    std::vector<int> iters(nrhs, 0), outer_n(nrhs, 0);
    std::vector<int> mvb(nrhs, 0);  // products with A applied to each RHS
    auto add_mv = [&](const std::vector<int>& v) {
      for (int b = 0; b < nrhs && b < (int)v.size(); ++b) mvb[b] += v[b];
    };
    auto add_all = [&](int k) {
      for (int b = 0; b < nrhs; ++b) mvb[b] += k;
    };
    bool timed_out = false;
    std::vector<double> rel;
    const bool df_res = o.precision != DDA_PREC_C128 && df_residuals(c, o.tol);
    // scratch c128 pair for true residuals (2 vectors)
    e = grow(c, &c->d_sc, sizeof(double2) * 2 * el);
    if (!e.ok()) return fail(c, e);
    double2* sc = c->d_sc;
    int outer = 0;
    if (o.precision == DDA_PREC_C128) {
      dda::KrylovVecs<double2> kv;
      e = kvec_alloc<double2>(c, &kv, o.solver == DDA_BICGSTAB2 ? 1 : 0);
      if (e.ok()) {
        e = cuda_ok(cudaMemcpyAsync(kv.b, c->d_e128, sizeof(double2) * el, cudaMemcpyDeviceToDevice, c->stream),
                    "right-hand side copy");
        if (e.ok()) e = scale128(kv.b, false);
        if (e.ok() && o.warm_start)
          e = cuda_ok(cudaMemcpyAsync(kv.x, P, sizeof(double2) * el, cudaMemcpyDeviceToDevice, c->stream),
                      "initial guess copy");
        if (e.ok() && o.warm_start) e = scale128(kv.x, true);
        if (e.ok() && reuse) e = zero_masked(kv.b, sizeof(double2));
        if (e.ok() && reuse && o.warm_start) e = zero_masked(kv.x, sizeof(double2));
        SolveStats s;
        if (e.ok()) e = krylov<double2>(c, o, kv, ktol, o.maxit, o.warm_start != 0, &s, t0, &timed_out);
        if (e.ok()) e = scale128(kv.x, false);
        if (e.ok()) e = cuda_ok(cudaMemcpyAsync(P, kv.x, sizeof(double2) * el, cudaMemcpyDeviceToDevice, c->stream),
                                "solution copy");
        if (e.ok()) {
          iters = s.iters;
          add_mv(s.mv);
        }
      }
    } else if (o.precision == DDA_PREC_C64) {
      dda::KrylovVecs<float2> kv;
      e = kvec_alloc<float2>(c, &kv, o.solver == DDA_BICGSTAB2 ? 1 : 0);
      if (e.ok()) e = dda::convert_from_c128<float2>(c->d_e128, kv.b, el, c->stream);
      if (e.ok()) e = scale64(kv.b, false);
      if (e.ok() && o.warm_start) e = dda::convert_from_c128<float2>(P, kv.x, el, c->stream);
      if (e.ok() && o.warm_start) e = scale64(kv.x, true);
      if (e.ok() && reuse) e = zero_masked(kv.b, sizeof(float2));
      if (e.ok() && reuse && o.warm_start) e = zero_masked(kv.x, sizeof(float2));
      SolveStats s;
      if (e.ok()) e = krylov<float2>(c, o, kv, ktol, o.maxit, o.warm_start != 0, &s, t0, &timed_out);
      if (e.ok()) e = scale64(kv.x, false);
      if (e.ok()) {
        e = cuda_ok(cudaMemsetAsync(P, 0, sizeof(double2) * el, c->stream), "solution clear");
        if (e.ok()) e = dda::add_to_c128<float2>(P, kv.x, nullptr, nrhs, n3, c->stream);
        iters = s.iters;
        add_mv(s.mv);
      }
    } else {
      // mixed: inner complex64 solves of A d = r, r from FP64 true residuals
      dda::KrylovVecs<float2> kv;
      e = kvec_alloc<float2>(c, &kv, o.solver == DDA_BICGSTAB2 ? 1 : 0);
      // each inner solve aims straight for tol, but never below the complex64 floor
      const double inner = o.inner_tol > 0 ? o.inner_tol : 5e-6;
      if (e.ok() && !o.warm_start) e = cuda_ok(cudaMemsetAsync(P, 0, sizeof(double2) * el, c->stream), "solution clear");
      int budget = o.maxit;
      while (e.ok()) {
        // r = E - A P (FP64); at P = 0 the residual is E itself
        double2* r128 = sc + el;
        if (outer == 0 && !o.warm_start) {
          e = cuda_ok(cudaMemcpyAsync(r128, c->d_e128, sizeof(double2) * el, cudaMemcpyDeviceToDevice, c->stream),
                      "residual copy");
          if (!e.ok()) break;
          rel.assign(nrhs, 1.0);
        } else {
          e = true_residual(c, P, sc, r128, &rel, df_res);
          add_all(1);
          if (!e.ok()) break;
        }
        bool all = true;
        for (int b = 0; b < nrhs; ++b) all = all && (masked[b] || rel[b] <= o.tol);
        if (all || budget <= 0 || timed_out) break;
        // inner right-hand side: residual of unconverged RHS (converged ones get 0 and stop at once)
        e = dda::convert_from_c128<float2>(r128, kv.b, el, c->stream);
        if (!e.ok()) break;
        for (int b = 0; b < nrhs; ++b)
          if ((masked[b] || rel[b] <= o.tol) && e.ok())
            e = cuda_ok(cudaMemsetAsync(kv.b + (int64_t)b * n3, 0, sizeof(float2) * n3, c->stream),
                        "inner right-hand side clear");
        if (!e.ok()) break;
        e = scale64(kv.b, false);
        if (!e.ok()) break;
        // ask the inner solve for the reduction that reaches 0.8 tol, but at least `inner`: the true
        // residual after an inner complex64 solve stays within a few percent of its recursive one,
        // so 0.8 leaves the margin for one outer pass to end below tol (the true residual decides)
        double worst = 0;
        for (int b = 0; b < nrhs; ++b)
          worst = std::max(worst, (!masked[b] && rel[b] > o.tol) ? o.tol / rel[b] : 0.0);
        const double itol = std::max(inner, 0.8 * worst);
        SolveStats s;
        e = krylov<float2>(c, o, kv, itol, budget, false, &s, t0, &timed_out);
        if (!e.ok()) break;
        for (int b = 0; b < nrhs; ++b) {
          iters[b] += s.iters[b];
          if (!masked[b] && rel[b] > o.tol) outer_n[b] += 1;
        }
        int used = 0;
        for (int b = 0; b < nrhs; ++b) used = std::max(used, s.iters[b]);
        budget -= std::max(used, 1);
        add_mv(s.mv);
        e = scale64(kv.x, false);
        if (!e.ok()) break;
        e = dda::add_to_c128<float2>(P, kv.x, nullptr, nrhs, n3, c->stream);
        ++outer;
      }
    }
    if (!e.ok()) return fail(c, e);
    if (reuse) {
      // P(o, l) = sum_m <e_m(rep), e_l(o)> P(rep, m): the TF polarizations of orientation o are
      // combinations of the representative's two orthonormal ones (same k, same alpha)
      for (int a = 0; a < c->n_ori && e.ok(); ++a) {
        const int r = rep_of[a];
        if (r < 0) continue;
        for (int l = 0; l < 2 && e.ok(); ++l) {
          const dda::RhsGeom& gl = c->rg[2 * a + l];
          cd co[2];
          for (int m = 0; m < 2; ++m) {
            const dda::RhsGeom& gm = c->rg[2 * r + m];
            co[m] = cd(0, 0);
            for (int q = 0; q < 3; ++q)
              co[m] += std::conj(cd(gm.e[2 * q], gm.e[2 * q + 1])) * cd(gl.e[2 * q], gl.e[2 * q + 1]);
          }
          e = dda::combine2_c128(P + (int64_t)(2 * a + l) * n3, P + (int64_t)(2 * r) * n3,
                                 P + (int64_t)(2 * r + 1) * n3, make_double2(co[0].real(), co[0].imag()),
                                 make_double2(co[1].real(), co[1].imag()), n3, c->stream);
        }
      }
      if (!e.ok()) return fail(c, e);
      rel.clear();  // the reconstructed RHS get their own FP64 true residual below
    }
    // final true residual in FP64 (for MIXED it was computed by the loop's last pass)
    if (o.precision != DDA_PREC_MIXED || rel.empty()) {
      e = true_residual(c, P, sc, sc + el, &rel, df_res);
      add_all(1);
      if (!e.ok()) return fail(c, e);
    }
    std::vector<double> ner(nrhs, NAN);
    if (o.normal_eq) {
      // |A^H (A P - E)| / |A^H E| with FP64 products (guide, eq. err_tol)
      double2* r128 = sc + el;  // holds E - A P from true_residual
      e = matvec<double2>(c, r128, sc, nrhs, 0, true);
      dda::RedBuf rb = redbuf(c, nrhs, n3);
      std::vector<double> num(nrhs), den(nrhs);
      if (e.ok()) {
        // reuse residual kernel: |0 - x|^2 gives |x|^2
        e = dda::residual_c128(sc, sc, r128, c->d_small, rb, nrhs, n3, c->stream);  // r128 = 0, second slot |sc|^2
      }
      if (e.ok()) {
        e = cuda_ok(cudaMemcpyAsync(c->h_pinned, c->d_small, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost,
                                    c->stream), "norm readback");
        if (e.ok()) e = cuda_ok(cudaStreamSynchronize(c->stream), "norm readback");
        for (int b = 0; b < nrhs; ++b) num[b] = c->h_pinned[2 * b + 1];
        if (e.ok()) e = matvec<double2>(c, c->d_e128, sc, nrhs, 0, true);
        add_all(2);
      }
      if (e.ok()) e = dda::residual_c128(sc, sc, r128, c->d_small, rb, nrhs, n3, c->stream);
      if (e.ok()) {
        e = cuda_ok(cudaMemcpyAsync(c->h_pinned, c->d_small, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost,
                                    c->stream), "norm readback");
        if (e.ok()) e = cuda_ok(cudaStreamSynchronize(c->stream), "norm readback");
        for (int b = 0; b < nrhs; ++b) {
          den[b] = c->h_pinned[2 * b + 1];
          ner[b] = den[b] > 0 ? std::sqrt(num[b] / den[b]) : 0.0;
        }
      }
      if (!e.ok()) return fail(c, e);
    }
    {
      const Err fe = check_fault(c);
      if (!fe.ok()) return fail(c, fe);
    }
    bool all = true;
    for (int b = 0; b < nrhs; ++b) {
      const bool conv = rel[b] <= o.tol;
      all = all && conv;
      if (rep) {
        rep[b].iters = iters[b];
        rep[b].matvecs = mvb[b];
        rep[b].outer = (o.precision == DDA_PREC_MIXED) ? outer_n[b] : 0;
        rep[b].converged = conv ? 1 : 0;
        rep[b].true_rel_resid = rel[b];
        rep[b].normal_eq_ratio = ner[b];
      }
    }
    if (timed_out && !all) return fail(c, Err::make(DDA_ETIMEOUT, "solve exceeded timeout_ms"));
    if (!all) return fail(c, Err::make(DDA_ENOCONV, "some right-hand side did not reach tol within maxit"));
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

namespace {

// 4 x 4 Mueller matrix (row-major) from the far-field amplitudes f[m][l] (m: theta-hat / phi-hat
// component, l: incident polarization e01 / e02) at scattering azimuth phi: the amplitude matrix
// S_1..S_4 by the guide's GETMUELLER relations (a, b, c, d = conj of the y and z Lab-Frame components
// of e01 and e02), then the Bohren & Huffman relations
void mueller_from_f(const cd f[2][2], cd A, cd B, cd Cc, cd D, double phs, double* m) {
  const double cp = std::cos(phs), sp = std::sin(phs);
  const cd I(0, 1);
  const cd S1 = -I * (f[1][0] * (B * cp - A * sp) + f[1][1] * (D * cp - Cc * sp));
  const cd S2 = -I * (f[0][0] * (A * cp + B * sp) + f[0][1] * (Cc * cp + D * sp));
  const cd S3 = I * (f[0][0] * (B * cp - A * sp) + f[0][1] * (D * cp - Cc * sp));
  const cd S4 = I * (f[1][0] * (A * cp + B * sp) + f[1][1] * (Cc * cp + D * sp));
  auto cj = [](cd z) { return std::conj(z); };
  m[0] = 0.5 * (std::norm(S1) + std::norm(S2) + std::norm(S3) + std::norm(S4));
  m[1] = 0.5 * (std::norm(S2) - std::norm(S1) + std::norm(S4) - std::norm(S3));
  m[2] = (S2 * cj(S3) + S1 * cj(S4)).real();
  m[3] = (S2 * cj(S3) - S1 * cj(S4)).imag();
  m[4] = 0.5 * (std::norm(S2) - std::norm(S1) + std::norm(S3) - std::norm(S4));
  m[5] = 0.5 * (std::norm(S1) + std::norm(S2) - std::norm(S3) - std::norm(S4));
  m[6] = (S2 * cj(S3) - S1 * cj(S4)).real();
  m[7] = (S2 * cj(S3) + S1 * cj(S4)).imag();
  m[8] = (S2 * cj(S4) + S1 * cj(S3)).real();
  m[9] = (S2 * cj(S4) - S1 * cj(S3)).real();
  m[10] = (S1 * cj(S2) + S3 * cj(S4)).real();
  m[11] = (S2 * cj(S1) + S4 * cj(S3)).imag();
  m[12] = (S4 * cj(S2) + S1 * cj(S3)).imag();
  m[13] = (S4 * cj(S2) - S1 * cj(S3)).imag();
  m[14] = (S1 * cj(S2) - S3 * cj(S4)).imag();
  m[15] = (S1 * cj(S2) - S3 * cj(S4)).real();
}

}  // namespace

dda_status dda_cross_sections(dda_ctx* c, const void* p_dev, double* q_out, const double* dirs, int ndir,
                              double* mueller_out) {
  if (!c) return DDA_EINVAL;
  if (!p_dev)
    return fail(c, Err::make(DDA_EINVAL, "dda_cross_sections: a required pointer is NULL"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  if (ndir < 0 || (ndir > 0 && (!dirs || !mueller_out))) return fail(c, Err::make(DDA_EINVAL, "bad directions"));
  if (ndir > 0 && c->periodic)
    return fail(c, Err::make(DDA_EUNSUPPORTED, "Mueller matrices of periodic targets are not available"));
  if (ndir > 0 && c->iorth != 2) return fail(c, Err::make(DDA_EINVAL, "Mueller matrices need iorth = 2"));
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    const int nrhs = c->nrhs;
    const double2* P = (const double2*)p_dev;
    const double pi = 3.14159265358979323846;
    const double aeff = std::cbrt(3.0 * (double)c->n / (4.0 * pi));
    const double geo = pi * aeff * aeff, k = c->kd;
    if (q_out) {
      dda::RedBuf rb;
      rb.nblk = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 1023) / 1024, 1216 / std::max(1, nrhs)));
      e = ensure_part(c, sizeof(double) * (size_t)rb.nblk * nrhs * 4);
      if (!e.ok()) return fail(c, e);
      rb.part = c->d_part;
      e = ensure_small(c, sizeof(double) * 3 * nrhs);
      if (!e.ok()) return fail(c, e);
      e = ensure_einc(c);
      if (e.ok() && c->iat_valid)
        e = dda::qsums_tensor(c->d_e128, c->d_iat128, k, P, nrhs, c->n, c->d_small, rb, c->stream);
      else if (e.ok())
        e = dda::qsums(c->comp_valid ? c->d_comp : nullptr, c->d_e128, c->d_ia128, c->ncomp, k, P, nrhs, c->n,
                       c->d_small, rb, c->stream);
      if (!e.ok()) return fail(c, e);
      if (cudaMemcpyAsync(c->h_pinned, c->d_small, sizeof(double) * 3 * nrhs, cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fail(c, Err::make(DDA_ECUDA, "q sums failed"));
      for (int b = 0; b < nrhs; ++b) {
        const double cext = 4 * pi * k * c->h_pinned[3 * b], cpha = 2 * pi * k * c->h_pinned[3 * b + 1];
        const double cabs = 4 * pi * k * c->h_pinned[3 * b + 2];
        q_out[4 * b] = cext / geo;
        q_out[4 * b + 1] = cabs / geo;
        q_out[4 * b + 2] = (cext - cabs) / geo;
        q_out[4 * b + 3] = cpha / geo;
      }
    }
    if (ndir > 0) {
      // scattering directions (LFRAME) per orientation, in TF
      std::vector<double> nh((size_t)nrhs * ndir * 3);
      std::vector<double> th((size_t)c->n_ori * ndir * 3), ph((size_t)c->n_ori * ndir * 3);
      for (int o = 0; o < c->n_ori; ++o) {
        const double* ax = &c->axes[9 * o];
        for (int d = 0; d < ndir; ++d) {
          const double t = dirs[2 * d], f = dirs[2 * d + 1];
          const double nl[3] = {std::cos(t), std::sin(t) * std::cos(f), std::sin(t) * std::sin(f)};
          const double tl[3] = {-std::sin(t), std::cos(t) * std::cos(f), std::cos(t) * std::sin(f)};
          const double pl[3] = {0.0, -std::sin(f), std::cos(f)};
          for (int kk = 0; kk < 3; ++kk) {
            const double nt = nl[0] * ax[kk] + nl[1] * ax[3 + kk] + nl[2] * ax[6 + kk];
            th[((size_t)o * ndir + d) * 3 + kk] = tl[0] * ax[kk] + tl[1] * ax[3 + kk] + tl[2] * ax[6 + kk];
            ph[((size_t)o * ndir + d) * 3 + kk] = pl[0] * ax[kk] + pl[1] * ax[3 + kk] + pl[2] * ax[6 + kk];
            for (int l = 0; l < c->iorth; ++l) nh[(((size_t)(o * c->iorth + l)) * ndir + d) * 3 + kk] = nt;
          }
        }
      }
      const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 2047) / 2048, 64));
      e = grow(c, &c->d_nh, sizeof(double) * nh.size());
      if (e.ok()) e = grow(c, &c->d_F, sizeof(double2) * (size_t)nrhs * ndir * 3);
      if (e.ok()) e = grow(c, &c->d_fpart, sizeof(double) * 6 * (size_t)nrhs * ndir * nblk);
      double2* d_F = c->d_F;
      if (e.ok()) {
        e = cuda_ok(cudaMemcpy(c->d_nh, nh.data(), sizeof(double) * nh.size(), cudaMemcpyHostToDevice),
                    "direction upload");
        const int box[3] = {c->tgt.box[0], c->tgt.box[1], c->tgt.box[2]};
        if (e.ok())
          e = dda::farfield(c->d_ijk, c->d_origin, c->d_nh, k, P, nrhs, ndir, c->n, box, d_F, (double2*)c->d_fpart,
                            nblk, c->stream);
      }
      std::vector<double2> F((size_t)nrhs * ndir * 3);
      if (e.ok()) {
        e = cuda_ok(cudaMemcpyAsync(F.data(), d_F, sizeof(double2) * F.size(), cudaMemcpyDeviceToHost, c->stream),
                    "far-field readback");
        if (e.ok() && cudaStreamSynchronize(c->stream) != cudaSuccess) e = Err::make(DDA_ECUDA, "far field failed");
      }
      if (!e.ok()) return fail(c, e);
      const double k3 = k * k * k;
      // a, b, c, d of the guide's GETMUELLER relations (Lab-Frame e01, e02)
      const cd A = std::conj(c->e01[1]), B = std::conj(c->e01[2]), Cc = std::conj(c->e02[1]), D = std::conj(c->e02[2]);
      for (int o = 0; o < c->n_ori; ++o)
        for (int d = 0; d < ndir; ++d) {
          cd f[2][2];
          for (int l = 0; l < 2; ++l) {
            const double2* Fv = &F[(((size_t)(o * 2 + l)) * ndir + d) * 3];
            const double* e1 = &th[((size_t)o * ndir + d) * 3];
            const double* e2 = &ph[((size_t)o * ndir + d) * 3];
            cd s1(0, 0), s2(0, 0);
            for (int kk = 0; kk < 3; ++kk) {
              const cd fv(Fv[kk].x, Fv[kk].y);
              s1 += e1[kk] * fv;
              s2 += e2[kk] * fv;
            }
            f[0][l] = k3 * s1;
            f[1][l] = k3 * s2;
          }
          mueller_from_f(f, A, B, Cc, D, dirs[2 * d + 1], mueller_out + ((size_t)o * ndir + d) * 16);
        }
    }
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}


dda_status dda_periodic_scattering(dda_ctx* c, const void* p_dev, int n_spec, const double* spec, double* dirs_out,
                                   double* mueller_out, double* tr_out) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || n_spec < 1 || !spec)
    return fail(c, Err::make(DDA_EINVAL, "dda_periodic_scattering: a required pointer is NULL or a size is out of range"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  if (!c->periodic) return fail(c, Err::make(DDA_EUNSUPPORTED, "the target is not periodic (dda_set_periodicity)"));
  const bool two_d = c->per_y > 0 && c->per_z > 0;
  if (mueller_out && c->iorth != 2) return fail(c, Err::make(DDA_EINVAL, "Mueller matrices need iorth = 2"));
  if (tr_out && !two_d)
    return fail(c, Err::make(DDA_EINVAL, "transmission and reflection coefficients need a doubly periodic target"));
  try {
    Err e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    const double pi = 3.14159265358979323846, k = c->kd;
    const double* k0 = c->rg[0].k;  // every RHS of a periodic context shares its TF incidence
    const int per_spec = two_d ? 2 : 1;
    const int ndir = n_spec * per_spec;
    // directions (TF unit vectors) of the orders: doubly periodic (M, N) on the transmission and the
    // reflection side; singly periodic the cone of order M at azimuth zeta around the axis
    std::vector<double> nd((size_t)ndir * 3, 0.0);
    for (int sp = 0; sp < n_spec; ++sp) {
      const double M = spec[2 * sp], N = spec[2 * sp + 1];
      if (two_d) {
        if (M != std::floor(M) || N != std::floor(N))
          return fail(c, Err::make(DDA_EINVAL, "diffraction orders (M, N) must be integers"));
        const double ky = k0[1] + 2.0 * pi * M / c->per_y, kz = k0[2] + 2.0 * pi * N / c->per_z;
        const double kx2 = k * k - ky * ky - kz * kz;
        if (!(kx2 > 0.0)) return fail(c, Err::make(DDA_EINVAL, "diffraction order (M, N) is not allowed here"));
        const double sx = k0[0] >= 0.0 ? 1.0 : -1.0;
        for (int side = 0; side < 2; ++side) {
          double* n = &nd[((size_t)sp * 2 + side) * 3];
          n[0] = (side == 0 ? sx : -sx) * std::sqrt(kx2) / k;
          n[1] = ky / k;
          n[2] = kz / k;
        }
      } else {
        if (M != std::floor(M)) return fail(c, Err::make(DDA_EINVAL, "the cone order M must be an integer"));
        const bool ax_y = c->per_y > 0;
        const double ka = ax_y ? k0[1] + 2.0 * pi * M / c->per_y : k0[2] + 2.0 * pi * M / c->per_z;
        const double kp2 = k * k - ka * ka;
        if (!(kp2 > 0.0)) return fail(c, Err::make(DDA_EINVAL, "cone order M is not allowed here"));
        const double kp = std::sqrt(kp2);
        double* n = &nd[(size_t)sp * 3];
        n[0] = kp * std::cos(N) / k;
        n[1] = ax_y ? ka / k : kp * std::sin(N) / k;
        n[2] = ax_y ? kp * std::sin(N) / k : ka / k;
      }
    }
    if (dirs_out) {
      for (int sp = 0; sp < n_spec; ++sp)
        for (int side = 0; side < 2; ++side)
          for (int q = 0; q < 3; ++q)
            dirs_out[((size_t)sp * 2 + side) * 3 + q] = side < per_spec ? nd[((size_t)sp * per_spec + side) * 3 + q] : 0.0;
    }
    if (!mueller_out && !tr_out) return DDA_OK;
    // F = sum_j P_j exp(-i k n.r_j) of every RHS in every direction (FP64, the finite targets' kernel)
    const int nrhs = c->nrhs;
    const double2* P = (const double2*)p_dev;
    std::vector<double> nh((size_t)nrhs * ndir * 3);
    for (int b = 0; b < nrhs; ++b) std::copy(nd.begin(), nd.end(), nh.begin() + (size_t)b * ndir * 3);
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 2047) / 2048, 64));
    e = grow(c, &c->d_nh, sizeof(double) * nh.size());
    if (e.ok()) e = grow(c, &c->d_F, sizeof(double2) * (size_t)nrhs * ndir * 3);
    if (e.ok()) e = grow(c, &c->d_fpart, sizeof(double) * 6 * (size_t)nrhs * ndir * nblk);
    if (e.ok())
      e = cuda_ok(cudaMemcpy(c->d_nh, nh.data(), sizeof(double) * nh.size(), cudaMemcpyHostToDevice),
                  "direction upload");
    const int box[3] = {c->tgt.box[0], c->tgt.box[1], c->tgt.box[2]};
    if (e.ok())
      e = dda::farfield(c->d_ijk, c->d_origin, c->d_nh, k, P, nrhs, ndir, c->n, box, c->d_F, (double2*)c->d_fpart,
                        nblk, c->stream);
    std::vector<double2> F((size_t)nrhs * ndir * 3);
    if (e.ok()) {
      e = cuda_ok(cudaMemcpyAsync(F.data(), c->d_F, sizeof(double2) * F.size(), cudaMemcpyDeviceToHost, c->stream),
                  "far-field readback");
      if (e.ok() && cudaStreamSynchronize(c->stream) != cudaSuccess) e = Err::make(DDA_ECUDA, "far field failed");
    }
    if (!e.ok()) return fail(c, e);
    auto Fv = [&](int b, int d, int q) {
      const double2 v = F[((size_t)b * ndir + d) * 3 + q];
      return cd(v.x, v.y);
    };
    if (tr_out) {
      // E_s = (2 pi i k^2 / (A k |n_x|)) (I - n n).F; powers per unit area relative to the incident
      const double area = c->per_y * c->per_z, n0x = std::abs(k0[0]) / k;
      for (int b = 0; b < nrhs; ++b)
        for (int sp = 0; sp < n_spec; ++sp)
          for (int side = 0; side < 2; ++side) {
            const int d = sp * 2 + side;
            const double* n = &nd[(size_t)d * 3];
            const cd f[3] = {Fv(b, d, 0), Fv(b, d, 1), Fv(b, d, 2)};
            const cd nf = n[0] * f[0] + n[1] * f[1] + n[2] * f[2];
            const cd pre = cd(0.0, 2.0 * pi * k * k / (area * k * std::abs(n[0])));
            double pw = 0.0;
            for (int q = 0; q < 3; ++q) {
              cd Eq = pre * (f[q] - n[q] * nf);
              if (side == 0 && spec[2 * sp] == 0.0 && spec[2 * sp + 1] == 0.0)
                Eq += cd(c->rg[b].e[2 * q], c->rg[b].e[2 * q + 1]);
              pw += std::norm(Eq);
            }
            tr_out[((size_t)b * n_spec + sp) * 2 + side] = pw * std::abs(n[0]) / n0x;
          }
    }
    if (mueller_out) {
      // the finite-target Mueller matrix of the same amplitudes, scaled from 1/(k r)^2 to the plane
      // waves' (2 pi / (A k k_x))^2 or the cones' 2 pi / (k k_perp L^2) (guide's S^(2d), S^(1d))
      const double k3 = k * k * k;
      const cd A = std::conj(c->e01[1]), B = std::conj(c->e01[2]), Cc = std::conj(c->e02[1]), D = std::conj(c->e02[2]);
      for (int o = 0; o < c->n_ori; ++o) {
        const double* ax = &c->axes[9 * o];
        for (int sp = 0; sp < n_spec; ++sp)
          for (int side = 0; side < 2; ++side) {
            double* m = mueller_out + (((size_t)o * n_spec + sp) * 2 + side) * 16;
            if (side >= per_spec) {
              std::fill(m, m + 16, 0.0);
              continue;
            }
            const int d = sp * per_spec + side;
            const double* n = &nd[(size_t)d * 3];
            const double nl[3] = {n[0] * ax[0] + n[1] * ax[1] + n[2] * ax[2], n[0] * ax[3] + n[1] * ax[4] + n[2] * ax[5],
                                  n[0] * ax[6] + n[1] * ax[7] + n[2] * ax[8]};
            const double th = std::acos(std::max(-1.0, std::min(1.0, nl[0])));
            // along +-x_LF (the (0, 0) orders) the scattering plane is undefined: azimuth 0 there
            const double ph = std::hypot(nl[1], nl[2]) > 1e-9 ? std::atan2(nl[2], nl[1]) : 0.0;
            const double tl[3] = {-std::sin(th), std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph)};
            const double pl[3] = {0.0, -std::sin(ph), std::cos(ph)};
            double e1[3], e2[3];
            for (int q = 0; q < 3; ++q) {
              e1[q] = tl[0] * ax[q] + tl[1] * ax[3 + q] + tl[2] * ax[6 + q];
              e2[q] = pl[0] * ax[q] + pl[1] * ax[3 + q] + pl[2] * ax[6 + q];
            }
            cd f[2][2];
            for (int l = 0; l < 2; ++l) {
              cd s1(0, 0), s2(0, 0);
              for (int q = 0; q < 3; ++q) {
                s1 += e1[q] * Fv(o * 2 + l, d, q);
                s2 += e2[q] * Fv(o * 2 + l, d, q);
              }
              f[0][l] = k3 * s1;
              f[1][l] = k3 * s2;
            }
            mueller_from_f(f, A, B, Cc, D, ph, m);
            double scale;
            if (two_d) {
              const double g = 2.0 * pi / (c->per_y * c->per_z * k * k * std::abs(n[0]));
              scale = g * g;
            } else {
              const double L = c->per_y > 0 ? c->per_y : c->per_z;
              const double na = c->per_y > 0 ? n[1] : n[2];
              scale = 2.0 * pi / (k * k * std::sqrt(std::max(0.0, 1.0 - na * na)) * L * L);
            }
            for (int q = 0; q < 16; ++q) m[q] *= scale;
          }
      }
    }
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

unsigned long long dda_kernel_launches(void) { return dda::launches(); }

namespace {
template <typename C>
Err matvec_fixed_scratch(dda_ctx* c, const C* p, C* ap, int nrhs) {
  const dda::Geom g = Sel<C>::geom(c);
  const size_t need = sizeof(C) * 3ull * g.px * g.nz * g.ys * (size_t)nrhs;
  if (need > dda::kNoAllocScratchBytes)
    return Err::make(DDA_EINVAL, "dda_matvec_noalloc: this grid needs " + std::to_string(need) +
                                     " bytes of FFT scratch for " + std::to_string(nrhs) +
                                     " RHS, above the fixed limit of " + std::to_string(dda::kNoAllocScratchBytes) +
                                     " bytes; pass fewer RHS or use dda_matvec");
  void* scratch = nullptr;
  DDA_TRY(dda::noalloc_scratch(c->device, &scratch));
  dda::MvData<C> d = Sel<C>::data(c);
  d.work = (C*)scratch;
  dda::MvTune t = Sel<C>::tune(c);
  // a bulk-staged plane pass reports a bounded wait that gave up through the context's fault
  // flag; without that flag (no earlier allocating call made it) run the plane pass unstaged
  if (!d.fault) t.bulk = false;
  return dda::launch_matvec<C>(g, d, t, p, ap, nrhs, 0, false, c->stream);
}
}  // namespace

dda_status dda_matvec_noalloc(dda_ctx* c, const void* p, void* ap, int nrhs, int dtype) {
  if (!c) return DDA_EINVAL;
  if (!p || !ap)
    return fail(c, Err::make(DDA_EINVAL, "dda_matvec_noalloc: a required pointer is NULL"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  if (nrhs < 1 || nrhs > c->nrhs) return fail(c, Err::make(DDA_EINVAL, "nrhs out of range"));
  if (p == ap) return fail(c, Err::make(DDA_EINVAL, "p and ap may not alias"));
  Err e = set_dev(c);
  if (!e.ok()) return fail(c, e);
  if (dtype == DDA_C64) e = matvec_fixed_scratch<float2>(c, (const float2*)p, (float2*)ap, nrhs);
  else if (dtype == DDA_C128) e = matvec_fixed_scratch<double2>(c, (const double2*)p, (double2*)ap, nrhs);
  else return fail(c, Err::make(DDA_EINVAL, "dtype must be DDA_C64 or DDA_C128"));
  return e.ok() ? DDA_OK : fail(c, e);
}

dda_status dda_profile_matvec(dda_ctx* c, int nrhs, int dtype, int iters, double* ms_per_pass, int* npass) {
  if (!c) return DDA_EINVAL;
  if (!ms_per_pass || !npass || iters < 1)
    return fail(c, Err::make(DDA_EINVAL, "dda_profile_matvec: a required pointer is NULL or iters < 1"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  if (nrhs < 1 || nrhs > c->nrhs) return fail(c, Err::make(DDA_EINVAL, "nrhs out of range"));
  if (dtype != DDA_C64 && dtype != DDA_C128 && dtype != DDA_C128DF) return fail(c, Err::make(DDA_EINVAL, "bad dtype"));
  Err e = set_dev(c);
  if (!e.ok()) return fail(c, e);
  e = (dtype == DDA_C64) ? ensure_tuned<float2>(c, nrhs) : ensure_tuned<double2>(c, nrhs);
  if (!e.ok()) return fail(c, e);
  const bool plane = (dtype == DDA_C64) ? c->t64.plane : c->t128.plane;
  const int np = plane ? 3 : 5;
  const size_t cs = dtype == DDA_C64 ? sizeof(float2) : sizeof(double2);
  const size_t bytes = cs * (size_t)nrhs * 3 * c->n;
  void *p = nullptr, *ap = nullptr;
  cudaEvent_t ev[6] = {};
  std::vector<double> acc(np, 0.0);
  e = dalloc((char**)&p, bytes);
  if (e.ok()) e = dalloc((char**)&ap, bytes);
  if (e.ok() && cudaMemsetAsync(p, 0, bytes, c->stream) != cudaSuccess) e = Err::make(DDA_ECUDA, "memset failed");
  for (int i = 0; i <= np && e.ok(); ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) e = Err::make(DDA_ECUDA, "event creation failed");
  if (e.ok()) e = (dtype == DDA_C64) ? ensure_tuned<float2>(c, nrhs) : ensure_tuned<double2>(c, nrhs);
  for (int it = 0; it < iters && e.ok(); ++it) {
    dda::set_pass_events(ev);
    if (dtype == DDA_C64) e = matvec<float2>(c, (const float2*)p, (float2*)ap, nrhs, 0, false);
    else if (dtype == DDA_C128DF) e = matvec_df(c, (const double2*)p, (double2*)ap, nrhs, 0, false);
    else e = matvec<double2>(c, (const double2*)p, (double2*)ap, nrhs, 0, false);
    dda::set_pass_events(nullptr);
    if (!e.ok()) break;
    if (cudaEventSynchronize(ev[np]) != cudaSuccess) { e = Err::make(DDA_ECUDA, "profile sync failed"); break; }
    for (int i = 0; i < np; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      acc[i] += ms;
    }
  }
  dda::set_pass_events(nullptr);
  for (int i = 0; i <= np; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  dfree(p);
  dfree(ap);
  if (e.ok()) e = check_fault(c);
  if (!e.ok()) return fail(c, e);
  for (int i = 0; i < np; ++i) ms_per_pass[i] = acc[i] / iters;
  *npass = np;
  return DDA_OK;
}

// ------------------------------------------------------------------ angular averages
// Scattering directions and solid-angle weights (guide, "Averaging over Scattering
// Directions"): theta_j equally spaced in s(theta) = theta + theta/(theta + theta0),
// theta0 = 2 pi/(1 + x), N_theta from eta rounded to the nearest integer, N_phi(j) rings of
// phi_{j,k} = 2 pi (k - 1)/N_phi(j), one direction at theta = 0 and at theta = pi.
struct ScaDir {
  double theta, phi, w;
};
std::vector<ScaDir> scattering_directions(double x, double eta) {
  const double pi = 3.14159265358979323846;
  const double th0 = 2.0 * pi / (1.0 + x);
  const double nreal = 1.0 + 2.0 * (3.0 + x) / eta * (1.0 + 1.0 / (pi + th0)) / (1.0 + th0 / ((pi + th0) * (pi + th0)));
  const int nth = std::max(3, (int)std::nearbyint(nreal));
  std::vector<double> th(nth);
  const double ds = pi * (1.0 + 1.0 / (pi + th0)) / (nth - 1);
  for (int j = 0; j < nth; ++j) {
    const double sj = j * ds;
    th[j] = ((sj - 1.0 - th0) + std::sqrt((1.0 + th0 - sj) * (1.0 + th0 - sj) + 4.0 * th0 * sj)) / 2.0;
  }
  th[0] = 0.0;
  th[nth - 1] = pi;
  std::vector<ScaDir> out;
  for (int j = 0; j < nth; ++j) {
    const bool pole = (j == 0 || j == nth - 1);
    const int nphi = pole ? 1 : std::max(3, (int)std::nearbyint(4.0 * pi * std::sin(th[j]) / (th[j + 1] - th[j - 1])));
    double w;
    if (j == 0) w = 2.0 * pi / nphi * (1.0 - (std::cos(th[0]) + std::cos(th[1])) / 2.0);
    else if (j == nth - 1) w = 2.0 * pi / nphi * ((std::cos(th[nth - 2]) + std::cos(th[nth - 1])) / 2.0 + 1.0);
    else w = pi / nphi * (std::cos(th[j - 1]) - std::cos(th[j + 1]));
    for (int k = 0; k < nphi; ++k) out.push_back({th[j], 2.0 * pi * k / nphi, w});
  }
  return out;
}

dda_status dda_angular_averages(dda_ctx* c, const void* p_dev, double eta, double* out, int32_t* ndir_out) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || !out || !(eta > 0.0))
    return fail(c, Err::make(DDA_EINVAL, "dda_angular_averages: a required pointer is NULL or eta is not positive"));
  if (c->periodic)
    return fail(c, Err::make(DDA_EUNSUPPORTED, "not available for periodic targets (scattering goes into diffraction orders)"));
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the target and the incident beams first"));
  try {
    Err e = need_device(c);
    if (e.ok()) e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    const double pi = 3.14159265358979323846;
    const int nrhs = c->nrhs;
    const double k = c->kd;
    const double aeff = std::cbrt(3.0 * (double)c->n / (4.0 * pi));
    const std::vector<ScaDir> dirs = scattering_directions(k * aeff, eta);
    const int ndir = (int)dirs.size();
    const int box[3] = {c->tgt.box[0], c->tgt.box[1], c->tgt.box[2]};
    const int nt = box[0] + box[1] + box[2];
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 2047) / 2048, 64));
    const int nchunk = (ndir + 7) / 8;
    // RHS per pass: phase tables under ~256 MB
    const int per = (int)std::max<int64_t>(1, std::min<int64_t>(nrhs, (256ll << 20) / ((int64_t)ndir * nt * 8)));
    std::vector<double> nl((size_t)ndir * 3);
    for (int d = 0; d < ndir; ++d) {
      const double t = dirs[d].theta, f = dirs[d].phi;
      nl[3 * d] = std::cos(t);
      nl[3 * d + 1] = std::sin(t) * std::cos(f);
      nl[3 * d + 2] = std::sin(t) * std::sin(f);
    }
    float2* d_tab = nullptr;
    double* d_part = nullptr;
    double* d_nh = nullptr;
    double2* d_F = nullptr;
    e = dalloc((char**)&d_tab, sizeof(float2) * (size_t)per * ndir * nt);
    if (e.ok()) e = dalloc((char**)&d_part, sizeof(double) * (size_t)per * nchunk * nblk * 48);
    if (e.ok()) e = dalloc((char**)&d_nh, sizeof(double) * (size_t)per * ndir * 3);
    if (e.ok()) e = dalloc((char**)&d_F, sizeof(double2) * (size_t)per * ndir * 3);
    std::vector<double> nh((size_t)per * ndir * 3);
    std::vector<double2> F((size_t)per * ndir * 3);
    for (int b0 = 0; b0 < nrhs && e.ok(); b0 += per) {
      const int nb = std::min(per, nrhs - b0);
      // directions in the Target Frame of each RHS's orientation
      for (int bb = 0; bb < nb; ++bb) {
        const double* ax = &c->axes[9 * ((b0 + bb) / c->iorth)];
        for (int d = 0; d < ndir; ++d)
          for (int q = 0; q < 3; ++q)
            nh[((size_t)bb * ndir + d) * 3 + q] = nl[3 * d] * ax[q] + nl[3 * d + 1] * ax[3 + q] + nl[3 * d + 2] * ax[6 + q];
      }
      if (cudaMemcpyAsync(d_nh, nh.data(), sizeof(double) * (size_t)nb * ndir * 3, cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess) {
        e = Err::make(DDA_ECUDA, "direction upload failed");
        break;
      }
      const double2* P = (const double2*)p_dev + (size_t)b0 * 3 * c->n;
      e = dda::farfield_many(c->d_ijk, c->d_origin, d_nh, k, P, nb, ndir, c->n, box, d_tab, d_part, nblk, d_F,
                             c->stream);
      if (!e.ok()) break;
      if (cudaMemcpyAsync(F.data(), d_F, sizeof(double2) * (size_t)nb * ndir * 3, cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        e = Err::make(DDA_ECUDA, "far-field sums failed");
        break;
      }
      // dC_sca/dOmega = k^4 |F - n (n . F)|^2, summed with the solid-angle weights
      const double k4 = k * k * k * k;
      for (int bb = 0; bb < nb; ++bb) {
        double csum = 0, g1 = 0, g2 = 0, gv[3] = {0, 0, 0};
        for (int d = 0; d < ndir; ++d) {
          const double* n = &nh[((size_t)bb * ndir + d) * 3];
          const double2* Fv = &F[((size_t)bb * ndir + d) * 3];
          cd f[3], nf(0, 0);
          for (int q = 0; q < 3; ++q) {
            f[q] = cd(Fv[q].x, Fv[q].y);
            nf += n[q] * f[q];
          }
          double i2 = 0;
          for (int q = 0; q < 3; ++q) i2 += std::norm(f[q] - n[q] * nf);
          const double dc = k4 * i2 * dirs[d].w;
          const double ct = std::cos(dirs[d].theta);
          csum += dc;
          g1 += dc * ct;
          g2 += dc * ct * ct;
          for (int q = 0; q < 3; ++q) gv[q] += dc * nl[3 * d + q];
        }
        double* o = out + 6 * (size_t)(b0 + bb);
        o[0] = csum / (pi * aeff * aeff);
        o[1] = csum > 0 ? g1 / csum : 0.0;
        o[2] = csum > 0 ? g2 / csum : 0.0;
        for (int q = 0; q < 3; ++q) o[3 + q] = csum > 0 ? gv[q] / csum : 0.0;
      }
    }
    dfree(d_tab);
    dfree(d_part);
    dfree(d_nh);
    dfree(d_F);
    if (!e.ok()) return fail(c, e);
    if (ndir_out) *ndir_out = ndir;
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_force_torque(dda_ctx* c, const void* p_dev, double eta, double* out, int32_t* ndir_out) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || !out || !(eta > 0.0))
    return fail(c, Err::make(DDA_EINVAL, "dda_force_torque: a required pointer is NULL or eta is not positive"));
  if (c->periodic)
    return fail(c, Err::make(DDA_EUNSUPPORTED, "not available for periodic targets (scattering goes into diffraction orders)"));
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the target and the incident beams first"));
  try {
    Err e = need_device(c);
    if (e.ok()) e = set_dev(c);
    if (e.ok()) e = ensure_einc(c);
    if (!e.ok()) return fail(c, e);
    const double pi = 3.14159265358979323846;
    const int nrhs = c->nrhs;
    const double k = c->kd;
    const double aeff = std::cbrt(3.0 * (double)c->n / (4.0 * pi));
    const std::vector<ScaDir> dirs = scattering_directions(k * aeff, eta);
    const int ndir = (int)dirs.size();
    const int box[3] = {c->tgt.box[0], c->tgt.box[1], c->tgt.box[2]};
    const int nt = box[0] + box[1] + box[2];
    // torque about the centroid of the sites: lever arms r_j - r_cm = ijk_j + (origin - r_cm)
    double cm[3] = {0, 0, 0};
    for (int64_t j = 0; j < c->n; ++j)
      for (int q = 0; q < 3; ++q) cm[q] += (double)c->tgt.ijk[3 * j + q];
    double shift[3];
    for (int q = 0; q < 3; ++q) shift[q] = -cm[q] / (double)c->n;  // origin - r_cm in box-index units
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((c->n + 2047) / 2048, 64));
    const int nchunk = (ndir + 1) / 2;
    const int per = (int)std::max<int64_t>(1, std::min<int64_t>(nrhs, (256ll << 20) / ((int64_t)ndir * nt * 8)));
    std::vector<double> nl((size_t)ndir * 3);
    for (int d = 0; d < ndir; ++d) {
      const double t = dirs[d].theta, f = dirs[d].phi;
      nl[3 * d] = std::cos(t);
      nl[3 * d + 1] = std::sin(t) * std::cos(f);
      nl[3 * d + 2] = std::sin(t) * std::sin(f);
    }
    float2* d_tab = nullptr;
    double* d_part = nullptr;
    double* d_nh = nullptr;
    double2* d_M = nullptr;
    double* d_ext = nullptr;
    const size_t part_doubles = std::max<size_t>((size_t)per * nchunk * nblk * 48, (size_t)nrhs * nblk * 8);
    e = dalloc((char**)&d_tab, sizeof(float2) * (size_t)per * ndir * nt);
    if (e.ok()) e = dalloc((char**)&d_part, sizeof(double) * part_doubles);
    if (e.ok()) e = dalloc((char**)&d_nh, sizeof(double) * (size_t)per * ndir * 3);
    if (e.ok()) e = dalloc((char**)&d_M, sizeof(double2) * (size_t)per * ndir * 12);
    if (e.ok()) e = dalloc((char**)&d_ext, sizeof(double) * 7 * (size_t)nrhs);
    // incident part, all RHS at once
    std::vector<double> ext(7 * (size_t)nrhs);
    if (e.ok()) e = dda::torque_ext_sums(c->d_ijk, c->d_e128, (const double2*)p_dev, nrhs, c->n, shift, d_part, nblk,
                                         d_ext, c->stream);
    if (e.ok() && (cudaMemcpyAsync(ext.data(), d_ext, sizeof(double) * 7 * nrhs, cudaMemcpyDeviceToHost, c->stream) !=
                       cudaSuccess ||
                   cudaStreamSynchronize(c->stream) != cudaSuccess))
      e = Err::make(DDA_ECUDA, "incident force sums failed");
    std::vector<double> nh((size_t)per * ndir * 3);
    std::vector<double2> M((size_t)per * ndir * 12);
    const double k3 = k * k * k / (8.0 * pi), k4 = k * k * k * k / (8.0 * pi);
    for (int b0 = 0; b0 < nrhs && e.ok(); b0 += per) {
      const int nb = std::min(per, nrhs - b0);
      for (int bb = 0; bb < nb; ++bb) {
        const double* ax = &c->axes[9 * ((b0 + bb) / c->iorth)];
        for (int d = 0; d < ndir; ++d)
          for (int q = 0; q < 3; ++q)
            nh[((size_t)bb * ndir + d) * 3 + q] = nl[3 * d] * ax[q] + nl[3 * d + 1] * ax[3 + q] + nl[3 * d + 2] * ax[6 + q];
      }
      if (cudaMemcpyAsync(d_nh, nh.data(), sizeof(double) * (size_t)nb * ndir * 3, cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess) {
        e = Err::make(DDA_ECUDA, "direction upload failed");
        break;
      }
      const double2* P = (const double2*)p_dev + (size_t)b0 * 3 * c->n;
      e = dda::farfield_moments(c->d_ijk, c->d_origin, d_nh, k, P, nb, ndir, c->n, box, shift, d_tab, d_part, nblk,
                                d_M, c->stream);
      if (!e.ok()) break;
      if (cudaMemcpyAsync(M.data(), d_M, sizeof(double2) * (size_t)nb * ndir * 12, cudaMemcpyDeviceToHost, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        e = Err::make(DDA_ECUDA, "far-field moments failed");
        break;
      }
      for (int bb = 0; bb < nb; ++bb) {
        const int b = b0 + bb;
        double kh[3];
        for (int q = 0; q < 3; ++q) kh[q] = c->rg[b].k[q] / k;
        const double* s7 = &ext[7 * (size_t)b];
        // incident part: F = (k/2) sum Im(P.E^*) khat; Gamma = 1/2 sum Re(P x E^*) + (k/2) (sum r Im(P.E^*)) x khat
        double F[3], G[3];
        for (int q = 0; q < 3; ++q) {
          F[q] = 0.5 * k * s7[6] * kh[q];
          const int q1 = (q + 1) % 3, q2 = (q + 2) % 3;
          G[q] = 0.5 * s7[q] + 0.5 * k * (s7[3 + q1] * kh[q2] - s7[3 + q2] * kh[q1]);
        }
        // the array's own field, as far-field integrals over the guide's directions
        for (int d = 0; d < ndir; ++d) {
          const double* n = &nh[((size_t)bb * ndir + d) * 3];
          const double2* Mv = &M[((size_t)bb * ndir + d) * 12];
          const double w = dirs[d].w;
          cd g[3], f[3], ng(0, 0);
          for (int q = 0; q < 3; ++q) {
            g[q] = cd(Mv[q].x, Mv[q].y);
            ng += n[q] * g[q];
          }
          double ff = 0;
          for (int q = 0; q < 3; ++q) {
            f[q] = g[q] - n[q] * ng;
            ff += std::norm(f[q]);
          }
          double rh[3];  // Re h, h_c = sum_a T[c][a] conj(f_a)
          for (int cc = 0; cc < 3; ++cc) {
            cd h(0, 0);
            for (int a = 0; a < 3; ++a) h += cd(Mv[3 + 3 * cc + a].x, Mv[3 + 3 * cc + a].y) * std::conj(f[a]);
            rh[cc] = h.real();
          }
          for (int q = 0; q < 3; ++q) {
            const int q1 = (q + 1) % 3, q2 = (q + 2) % 3;
            F[q] -= k4 * w * ff * n[q];
            G[q] += k3 * w * (g[q1] * std::conj(f[q2]) - g[q2] * std::conj(f[q1])).imag();
            G[q] -= k4 * w * (rh[q1] * n[q2] - rh[q2] * n[q1]);
          }
        }
        const double sc = 8.0 / (aeff * aeff);
        for (int q = 0; q < 3; ++q) {
          out[6 * (size_t)b + q] = sc * F[q];
          out[6 * (size_t)b + 3 + q] = sc * k * G[q];
        }
      }
    }
    dfree(d_tab);
    dfree(d_part);
    dfree(d_nh);
    dfree(d_M);
    dfree(d_ext);
    if (!e.ok()) return fail(c, e);
    if (ndir_out) *ndir_out = ndir;
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_near_field(dda_ctx* c, const void* p_dev, const double* pts, int64_t npts, double* e_out,
                          double* b_out) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || !pts || !e_out || npts < 1)
    return fail(c, Err::make(DDA_EINVAL, "dda_near_field: a required pointer is NULL or a size is out of range"));
  if (!c->have_inc) return fail(c, Err::make(DDA_ESTATE, "set the target and the incident beams first"));
  try {
    Err e = need_device(c);
    if (e.ok()) e = set_dev(c);
    if (!e.ok()) return fail(c, e);
    for (int64_t i = 0; i < 3 * npts; ++i)
      if (!std::isfinite(pts[i])) return fail(c, Err::make(DDA_EINVAL, "field points must be finite"));
    const int nrhs = c->nrhs;
    double* d_pts = nullptr;
    double* d_out = nullptr;
    e = dalloc((char**)&d_pts, sizeof(double) * 3 * (size_t)npts);
    if (e.ok()) e = dalloc((char**)&d_out, sizeof(double) * 12 * (size_t)npts * nrhs);
    std::vector<double> h((size_t)12 * npts * nrhs);
    if (e.ok()) e = cuda_ok(cudaMemcpyAsync(d_pts, pts, sizeof(double) * 3 * npts, cudaMemcpyHostToDevice, c->stream),
                            "point upload");
    double* d_part = nullptr;
    if (e.ok() && !c->periodic) {
      e = dda::near_field(c->d_ijk, c->d_origin, (const double2*)p_dev, nrhs, c->n, d_pts, npts, c->kd, d_out,
                          c->stream);
    } else if (e.ok()) {
      // replicas far enough that every term within the cutoff radius 40^(1/4) / (gamma kd) of any
      // point is included: the radius plus the points' and sites' extent along y and z
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t j = 0; j < c->n; ++j)
        for (int a = 1; a < 3; ++a) {
          const double v = c->tgt.ijk[3 * j + a] + c->tgt.origin[a];
          lo[a] = std::min(lo[a], v);
          hi[a] = std::max(hi[a], v);
        }
      double plo[3] = {1e300, 1e300, 1e300}, phi[3] = {-1e300, -1e300, -1e300};
      for (int64_t i = 0; i < npts; ++i)
        for (int a = 1; a < 3; ++a) {
          plo[a] = std::min(plo[a], pts[3 * i + a]);
          phi[a] = std::max(phi[a], pts[3 * i + a]);
        }
      const double rcut = std::pow(40.0, 0.25) / (c->per_gamma * c->kd);
      int mrange[3] = {0, 0, 0};
      const double per[3] = {0.0, c->per_y, c->per_z};
      for (int a = 1; a < 3; ++a) {
        if (per[a] <= 0) continue;
        const double ext = std::max(std::abs(phi[a] - lo[a]), std::abs(hi[a] - plo[a]));
        const double mr = std::ceil((rcut + ext) / per[a]);
        if (mr > 1e6) e = Err::make(DDA_EINVAL, "interaction cutoff too small for the periods (too many replicas)");
        mrange[a] = (int)std::min(mr, 1e6);
      }
      const int64_t nchunk = (npts + 3) / 4;
      const int64_t pairs = c->n * (int64_t)(2 * mrange[1] + 1) * (2 * mrange[2] + 1);
      // bound the work (each term is ~150 FP64 operations): 2e11 terms take seconds
      if (e.ok() && (double)pairs * (double)npts * nrhs > 2e11)
        e = Err::make(DDA_EINVAL, "too many replica terms for the near field (raise gamma or pass fewer points)");
      const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((pairs + 4095) / 4096,
                                                                      std::max<int64_t>(1, 1216 / std::max<int64_t>(1, nchunk * nrhs))));
      if (e.ok()) e = dalloc((char**)&d_part, sizeof(double) * 12 * (size_t)npts * nrhs * nsplit);
      if (e.ok())
        e = dda::near_field_pbc(c->d_ijk, c->d_origin, (const double2*)p_dev, nrhs, c->n, d_pts, npts, c->kd,
                                c->rg[0].k, c->per_y, c->per_z, c->per_gamma, mrange[1], mrange[2], d_part, nsplit,
                                d_out, c->stream);
    }
    if (e.ok()) e = cuda_ok(cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                                            c->stream), "field readback");
    if (e.ok()) e = cuda_ok(cudaStreamSynchronize(c->stream), "field readback");
    dfree(d_pts);
    dfree(d_out);
    if (d_part) dfree(d_part);
    if (!e.ok()) return fail(c, e);
    // add the incident plane wave E = e exp(i k.x), B = khat x E (FP64 on the host)
    for (int b = 0; b < nrhs; ++b) {
      const dda::RhsGeom& g = c->rg[b];
      const double kh[3] = {g.k[0] / c->kd, g.k[1] / c->kd, g.k[2] / c->kd};
      for (int64_t i = 0; i < npts; ++i) {
        const double* x = pts + 3 * i;
        const cd ph = std::exp(cd(0.0, g.k[0] * x[0] + g.k[1] * x[1] + g.k[2] * x[2]));
        cd E[3], B[3];
        const double* f = &h[((size_t)b * npts + i) * 12];
        for (int a = 0; a < 3; ++a) E[a] = cd(g.e[2 * a], g.e[2 * a + 1]) * ph;
        for (int a = 0; a < 3; ++a) B[a] = kh[(a + 1) % 3] * E[(a + 2) % 3] - kh[(a + 2) % 3] * E[(a + 1) % 3];
        double* eo = e_out + ((size_t)b * npts + i) * 6;
        for (int a = 0; a < 3; ++a) {
          eo[2 * a] = f[2 * a] + E[a].real();
          eo[2 * a + 1] = f[2 * a + 1] + E[a].imag();
        }
        if (b_out) {
          double* bo = b_out + ((size_t)b * npts + i) * 6;
          for (int a = 0; a < 3; ++a) {
            bo[2 * a] = f[6 + 2 * a] + B[a].real();
            bo[2 * a + 1] = f[6 + 2 * a + 1] + B[a].imag();
          }
        }
      }
    }
    return DDA_OK;
  } catch (const std::bad_alloc&) {
    return fail(c, Err::make(DDA_ENOMEM, "host allocation failed"));
  }
}

dda_status dda_orientation_grid(const double beta_deg[2], int nbeta, const double theta_deg[2], int ntheta,
                                const double phi_deg[2], int nphi, double* ori_out, double* w_out) {
  if (!beta_deg || !theta_deg || !phi_deg || !ori_out || !w_out || nbeta < 1 || ntheta < 1 || nphi < 1)
    return DDA_EINVAL;
  const double rad = 3.14159265358979323846 / 180.0;
  // beta and Phi: midpoints of equal intervals; cos(Theta): Simpson nodes (odd) or midpoints (even)
  std::vector<double> cth(ntheta), wth(ntheta);
  const double c0 = std::cos(theta_deg[0] * rad), c1 = std::cos(theta_deg[1] * rad);
  if (ntheta == 1) {
    cth[0] = c0;
    wth[0] = 1.0;
  } else if (ntheta % 2 == 1) {
    for (int i = 0; i < ntheta; ++i) {
      cth[i] = c0 + (c1 - c0) * (double)i / (ntheta - 1);
      const double s = (i == 0 || i == ntheta - 1) ? 1.0 : (i % 2 ? 4.0 : 2.0);
      wth[i] = s / 3.0 / (ntheta - 1);
    }
  } else {
    for (int i = 0; i < ntheta; ++i) {
      cth[i] = c0 + (c1 - c0) * (i + 0.5) / ntheta;
      wth[i] = 1.0 / ntheta;
    }
  }
  int64_t o = 0;
  for (int ib = 0; ib < nbeta; ++ib) {
    const double beta = (beta_deg[0] + (beta_deg[1] - beta_deg[0]) * (ib + 0.5) / nbeta) * rad;
    for (int it = 0; it < ntheta; ++it) {
      const double th = std::acos(std::max(-1.0, std::min(1.0, cth[it])));
      for (int ip = 0; ip < nphi; ++ip, ++o) {
        ori_out[3 * o] = beta;
        ori_out[3 * o + 1] = th;
        ori_out[3 * o + 2] = (phi_deg[0] + (phi_deg[1] - phi_deg[0]) * (ip + 0.5) / nphi) * rad;
        w_out[o] = wth[it] / ((double)nbeta * nphi);
      }
    }
  }
  return DDA_OK;
}

dda_status dda_orientation_average(const double* w, int n_ori, int iorth, const double* vals, int64_t nval,
                                   double* out) {
  if (!w || !vals || !out || n_ori < 1 || (iorth != 1 && iorth != 2) || nval < 1) return DDA_EINVAL;
  for (int o = 0; o < n_ori; ++o)
    if (!std::isfinite(w[o])) return DDA_EINVAL;
  // out[pol][k] = sum_o w_o vals[o][pol][k], summed in orientation order in FP64
  for (int l = 0; l < iorth; ++l)
    for (int64_t k = 0; k < nval; ++k) {
      double acc = 0.0;
      for (int o = 0; o < n_ori; ++o) acc += w[o] * vals[((int64_t)o * iorth + l) * nval + k];
      out[(int64_t)l * nval + k] = acc;
    }
  return DDA_OK;
}

dda_status dda_probe_tc_dft(int device, int64_t nvec, int reps, double out[4]) {
  if (!out) return DDA_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return DDA_ECUDA;
  const Err e = dda::probe_tc_dft(nvec, reps, out);
  return e.ok() ? DDA_OK : e.code;
}

dda_status dda_selftest_bulk_wait(int device, int32_t* gave_up) {
  if (!gave_up) return DDA_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return DDA_ECUDA;
  int v = -1;
  const Err e = dda::selftest_bulk_wait(&v);
  if (!e.ok()) return e.code;
  *gave_up = v;
  return DDA_OK;
}

dda_status dda_schedule_info(dda_ctx* c, int dtype, int32_t info[12]) {
  if (!c) return DDA_EINVAL;
  if (!info)
    return fail(c, Err::make(DDA_EINVAL, "dda_schedule_info: a required pointer is NULL"));
  for (int i = 0; i < 12; ++i) info[i] = 0;
  if (!c->have_green) return fail(c, Err::make(DDA_ESTATE, "build the Green tensor first"));
  if (dtype != DDA_C64 && dtype != DDA_C128 && dtype != DDA_C128DF) return fail(c, Err::make(DDA_EINVAL, "bad dtype"));
  const dda::MvTune& t = dtype == DDA_C64 ? c->t64 : c->t128;
  info[0] = t.plane ? 3 : 5;
  info[1] = t.fast ? 1 : 0;
  info[2] = t.plane ? (t.clus == 2 ? 384 : t.clus == 4 ? 256 : t.thr_p) : 0;
  info[3] = c->tuned_nrhs[dtype == DDA_C64 ? 0 : 1];
  info[4] = t.plane && t.clus > 1 ? t.clus : 1;
  info[6] = t.plane && t.bulk ? 1 : 0;
  info[8] = !t.plane && t.zr ? 1 : 0;
  {
    const dda::Geom& g = dtype == DDA_C64 ? c->g64 : c->g128;
    const size_t cs = dtype == DDA_C64 ? sizeof(float2) : sizeof(double2);
    info[5] = !t.fast ? 0
              : t.xnc == 1 ? dda::x_tile_height_one_component(cs)
                           : (t.xty > 0 && dda::x_tile_height_ok(cs, g.px, t.xty) ? t.xty
                                                                                  : dda::x_tile_height_default(cs, g.px));
    info[7] = !t.fast ? 0 : (t.xnc == 1 ? 1 : 3);
  }
  return DDA_OK;
}

dda_status dda_solve_batch(dda_ctx* const* ctxs, int nctx, const dda_solve_opts* opt, void* const* p_devs,
                           dda_solve_report* const* reps, dda_status* statuses) {
  if (!ctxs || nctx < 1 || !opt || !p_devs) return DDA_EINVAL;
  for (int i = 0; i < nctx; ++i) {
    if (!ctxs[i] || !p_devs[i]) return DDA_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], Err::make(DDA_EINVAL, "a context appears twice in the batch"));
  }
  // tune every target's product schedules alone first (timings free of contention)
  for (int i = 0; i < nctx; ++i) {
    dda_ctx* c = ctxs[i];
    if (!c->have_alpha || !c->have_green)
      return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
    Err e = set_dev(c);
    if (e.ok()) e = ensure_tuned<double2>(c, c->nrhs);
    if (e.ok() && opt->precision != DDA_PREC_C128) e = ensure_tuned<float2>(c, c->nrhs);
    if (e.ok() && c->stream && cudaStreamSynchronize(c->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "stream synchronize failed");
    if (!e.ok()) return fail(c, e);
  }
  // each target gets a stream of its own for the concurrent part (ordered after its caller's stream)
  std::vector<cudaStream_t> user(nctx);
  for (int i = 0; i < nctx; ++i) {
    dda_ctx* c = ctxs[i];
    user[i] = c->stream;
    if (!c->own_stream && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, Err::make(DDA_ECUDA, "stream creation failed"));
    if (!c->ev && cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, Err::make(DDA_ECUDA, "event creation failed"));
    cudaEventRecord(c->ev, user[i]);
    cudaStreamWaitEvent(c->own_stream, c->ev, 0);
    c->stream = c->own_stream;
  }
  std::vector<dda_status> st(nctx, DDA_OK);
  std::vector<std::thread> pool;
  pool.reserve(nctx);
  for (int i = 0; i < nctx; ++i) {
    pool.emplace_back([&, i]() {
      dda_solve_opts o = *opt;
      o.use_graph = 1;
      st[i] = dda_solve(ctxs[i], &o, p_devs[i], reps ? reps[i] : nullptr);
    });
  }
  for (auto& t : pool) t.join();
  for (int i = 0; i < nctx; ++i) ctxs[i]->stream = user[i];
  dda_status first = DDA_OK;
  for (int i = 0; i < nctx; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == DDA_OK && st[i] != DDA_OK) first = st[i];
  }
  return first;
}

// ------------------------------------------------------------------ learned warm start: context side
namespace {
Err grid_place(dda_ctx* c, const int32_t dims[3], const int32_t off_in[3], int32_t off[3]) {
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < c->tgt.box[a] || dims[a] % 8)
      return Err::make(DDA_EINVAL, "network grid must cover the box and be a multiple of 8 per axis");
    off[a] = off_in ? off_in[a] : (dims[a] - c->tgt.box[a]) / 2;
    if (off[a] < 0 || off[a] + c->tgt.box[a] > dims[a]) return Err::make(DDA_EINVAL, "box does not fit at offset");
  }
  return Err::Ok();
}
}  // namespace

dda_status dda_unet_features(dda_ctx* c, float* x_dev, const int32_t dims[3], const int32_t offset[3]) {
  if (!c) return DDA_EINVAL;
  if (!x_dev || !dims)
    return fail(c, Err::make(DDA_EINVAL, "dda_unet_features: a required pointer is NULL"));
  if (!c->have_alpha) return fail(c, Err::make(DDA_ESTATE, "set target, incidence and alpha first"));
  int32_t off[3];
  Err e = grid_place(c, dims, offset, off);
  if (e.ok()) e = need_device(c);
  if (e.ok()) e = set_dev(c);
  if (e.ok()) e = ensure_einc(c);
  std::vector<float2> eps(c->ncomp);
  for (int m = 0; m < c->ncomp; ++m) eps[m] = make_float2((float)c->eps[m].real(), (float)c->eps[m].imag());
  if (e.ok()) e = grow(c, &c->d_eps, sizeof(float2) * c->ncomp);
  if (e.ok() && cudaMemcpy(c->d_eps, eps.data(), sizeof(float2) * c->ncomp, cudaMemcpyHostToDevice) != cudaSuccess)
    e = Err::make(DDA_ECUDA, "copy failed");
  if (e.ok())
    e = dda::unet_features(c->d_ijk, c->n, c->comp_valid ? c->d_comp : nullptr, c->d_eps, c->d_e128, c->nrhs, dims,
                           off, x_dev, c->stream);
  return e.ok() ? DDA_OK : fail(c, e);
}

dda_status dda_unet_targets(dda_ctx* c, const void* p_dev, float* t_dev, float* mask_dev, const int32_t dims[3],
                            const int32_t offset[3], int residual) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || !t_dev || !mask_dev || !dims)
    return fail(c, Err::make(DDA_EINVAL, "dda_unet_targets: a required pointer is NULL"));
  if (!c->have_alpha) return fail(c, Err::make(DDA_ESTATE, "set target, incidence and alpha first"));
  int32_t off[3];
  Err e = grid_place(c, dims, offset, off);
  if (e.ok()) e = need_device(c);
  if (e.ok()) e = set_dev(c);
  if (e.ok() && residual) e = ensure_einc(c);
  if (e.ok())
    e = dda::unet_targets(c->d_ijk, c->n, c->comp_valid ? c->d_comp : nullptr, c->d_ia128, c->ncomp,
                          (const double2*)p_dev, residual ? c->d_e128 : nullptr, c->nrhs, dims, off, t_dev, mask_dev,
                          c->stream);
  return e.ok() ? DDA_OK : fail(c, e);
}

dda_status dda_unet_warm_start(dda_ctx* c, const float* y_dev, const int32_t dims[3], const int32_t offset[3],
                               int residual, void* p_dev) {
  if (!c) return DDA_EINVAL;
  if (!p_dev || !y_dev || !dims)
    return fail(c, Err::make(DDA_EINVAL, "dda_unet_warm_start: a required pointer is NULL"));
  if (!c->have_alpha) return fail(c, Err::make(DDA_ESTATE, "set target, incidence and alpha first"));
  int32_t off[3];
  Err e = grid_place(c, dims, offset, off);
  if (e.ok()) e = need_device(c);
  if (e.ok()) e = set_dev(c);
  if (e.ok() && residual) e = ensure_einc(c);
  if (e.ok())
    e = dda::unet_warm(c->d_ijk, c->n, c->comp_valid ? c->d_comp : nullptr, c->d_ia128, c->ncomp, y_dev,
                       residual ? c->d_e128 : nullptr, c->nrhs, dims, off, (double2*)p_dev, c->stream);
  return e.ok() ? DDA_OK : fail(c, e);
}

dda_status dda_unet_residual_grad(dda_ctx* c, const float* y_dev, const int32_t dims[3], const int32_t offset[3],
                                  double weight, float* gy_dev, double* loss_out) {
  if (!c) return DDA_EINVAL;
  if (!y_dev || !gy_dev || !dims)
    return fail(c, Err::make(DDA_EINVAL, "dda_unet_residual_grad: a required pointer is NULL"));
  if (!c->have_alpha || !c->have_green)
    return fail(c, Err::make(DDA_ESTATE, "set target, incidence, Green tensor and alpha first"));
  int32_t off[3];
  Err e = grid_place(c, dims, offset, off);
  if (e.ok()) e = need_device(c);
  if (e.ok()) e = set_dev(c);
  if (e.ok()) e = ensure_einc(c);
  const int nrhs = c->nrhs;
  const int64_t n3 = 3 * c->n, el = (int64_t)nrhs * n3;
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((n3 + 2047) / 2048, 256));
  if (e.ok()) e = grow(c, &c->d_nnv, sizeof(float2) * 3 * el);
  if (e.ok()) e = grow(c, &c->d_nnpart, sizeof(double) * 2 * nblk * nrhs);
  if (e.ok()) e = grow(c, &c->d_nnw, sizeof(double) * nrhs);
  if (e.ok()) e = ensure_tuned<float2>(c, nrhs);
  if (!e.ok()) return fail(c, e);
  float2 *p0 = c->d_nnv, *r = c->d_nnv + el, *g = c->d_nnv + 2 * el;
  const uint8_t* comp = c->comp_valid ? c->d_comp : nullptr;
  e = dda::unet_guess64(c->d_ijk, c->n, comp, c->d_ia128, c->ncomp, y_dev, c->d_e128, nrhs, dims, off, p0, c->stream);
  if (e.ok()) e = matvec<float2>(c, p0, r, nrhs, 0, false);
  if (e.ok()) e = dda::unet_resid64(c->d_e128, r, nrhs, n3, c->d_nnpart, nblk, c->stream);
  if (e.ok()) e = matvec<float2>(c, r, g, nrhs, 0, true);
  std::vector<double> part(2 * (size_t)nblk * nrhs), w(nrhs);
  if (e.ok()) {
    if (cudaMemcpyAsync(part.data(), c->d_nnpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      e = Err::make(DDA_ECUDA, "residual copy failed");
  }
  if (!e.ok()) return fail(c, e);
  double L = 0.0;
  for (int b = 0; b < nrhs; ++b) {
    double rr = 0, ee = 0;
    for (int k = 0; k < nblk; ++k) {
      rr += part[((size_t)b * nblk + k) * 2];
      ee += part[((size_t)b * nblk + k) * 2 + 1];
    }
    w[b] = ee > 0 ? weight / ee : 0.0;  // loss term weight * |r_b|^2 / |E_b|^2
    L += w[b] * rr;
  }
  if (cudaMemcpyAsync(c->d_nnw, w.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return fail(c, Err::make(DDA_ECUDA, "weight copy failed"));
  e = dda::unet_resgrad(c->d_ijk, c->n, comp, c->d_ia128, c->ncomp, g, c->d_nnw, nrhs, dims, off, gy_dev, c->stream);
  if (e.ok() && cudaStreamSynchronize(c->stream) != cudaSuccess) e = Err::make(DDA_ECUDA, "sync failed");
  if (!e.ok()) return fail(c, e);
  if (loss_out) *loss_out = L;
  return DDA_OK;
}
