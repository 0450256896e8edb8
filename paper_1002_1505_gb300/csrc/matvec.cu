// FFT-convolution product A P of the discrete dipole approximation and the
// FP64 Fourier-space Green tensor it uses.
//
// (A P)_j = alpha_j^{-1} P_j + sum_{k != j} A(r_j - r_k) P_k  (guide, eq. AP=E;
// A_jk of Draine 1988).  The sum is a discrete convolution over lattice
// offsets (Goodman, Draine & Flatau 1991), evaluated on a zero-padded grid
// Px x Py x Pz >= 2 Nx x 2 Ny x 2 Nz:  conv = IFFT3( Ghat . FFT3(P) ), with the
// symmetric 3x3 Ghat (6 complex components) applied pointwise.
//
// Pass schedule (per right-hand side b, all three components together):
//   X   gather P from the compact site list into box rows, forward FFT along x
//       (input pruned to Nx), store the spectrum transposed as W[b][c][kx][z][y];
//   YZ  per kx plane: forward FFT along y (pruned to Ny), then per batch of ky
//       columns forward FFT along z (pruned to Nz), 3x3 Ghat multiply, inverse
//       FFT along z (only z < Nz kept), then inverse FFT along y (only y < Ny
//       kept); all in shared memory when a plane of 3 x Nz x Py fits (3-pass
//       schedule), else as three separate launches (5-pass schedule);
//   X^-1 inverse FFT along x (only x < Nx kept), add alpha^{-1} P, scatter back
//       to the compact site list.
// Spectral positions stay in the engine's digit-reversed order throughout.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "dda_internal.h"

namespace dda {

namespace {

template <typename C> struct Real;
template <> struct Real<float2> { using t = float; };
template <> struct Real<double2> { using t = double; };

template <typename C>
__device__ __forceinline__ void load_tw(C* dst, const C* src, int L) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) dst[i] = src[i];
}

// u = Ghat v, Ghat symmetric with components (xx, xy, xz, yy, yz, zz)
template <typename C>
__device__ __forceinline__ void gmul(const C* gh, C& v0, C& v1, C& v2) {
  const C g0 = gh[0], g1 = gh[1], g2 = gh[2], g3 = gh[3], g4 = gh[4], g5 = gh[5];
  C u0 = cadd(cadd(cmul(g0, v0), cmul(g1, v1)), cmul(g2, v2));
  C u1 = cadd(cadd(cmul(g1, v0), cmul(g3, v1)), cmul(g4, v2));
  C u2 = cadd(cadd(cmul(g2, v0), cmul(g4, v1)), cmul(g5, v2));
  v0 = u0;
  v1 = u1;
  v2 = u2;
}

template <typename C>
__device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }

// ------------------------------------------------------------------ X forward
// grid (ceil(ny/ty), nz, nrhs); smem: tw[px] + s[3*ty][px+1]
template <typename C>
__global__ void k_xfwd(Geom g, MvData<C> d, const C* __restrict__ p, int ty, bool conj) {
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + g.px;
  const int ps = g.px + 1;
  const int y0 = blockIdx.x * ty, z = blockIdx.y, b = blockIdx.z;
  load_tw(tw, d.twx, g.px);
  const int nld = 3 * ty * g.nx;
  for (int i = threadIdx.x; i < nld; i += blockDim.x) {
    const int x = i % g.nx;
    const int rest = i / g.nx;
    const int t = rest % ty, c = rest / ty;
    const int y = y0 + t;
    C v = czero<C>();
    if (y < g.ny) {
      const int32_t idx = d.map[((int64_t)z * g.ny + y) * g.nx + x];
      if (idx >= 0) {
        v = p[((int64_t)b * 3 + c) * g.n + idx];
        if (conj) v = conjc(v);
        if (d.sc) v = cmul(v, d.sc[((int64_t)b * g.ncomp + (d.comp ? d.comp[3 * idx + c] : 0)) * 3 + c]);
      }
    }
    s[(c * ty + t) * ps + x] = v;
  }
  __syncthreads();
  fft_forward(s, Batch{3 * ty, ps, 1, false}, g.plx, g.nx, tw);
  const int nst = 3 * g.px * ty;
  const int64_t plane = (int64_t)g.nz * g.ys;
  for (int i = threadIdx.x; i < nst; i += blockDim.x) {
    const int t = i % ty;
    const int rest = i / ty;
    const int kx = rest % g.px, c = rest / g.px;
    const int y = y0 + t;
    if (y < g.ny)
      d.work[(((int64_t)b * 3 + c) * g.px + kx) * plane + (int64_t)z * g.ys + y] = s[(c * ty + t) * ps + kx];
  }
}

// ------------------------------------------------------------------ X inverse + diagonal + scatter
template <typename C>
__global__ void k_xinv(Geom g, MvData<C> d, const C* __restrict__ p, C* __restrict__ ap, int ty, int rhs0,
                       bool conj) {
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + g.px;
  const int ps = g.px + 1;
  const int y0 = blockIdx.x * ty, z = blockIdx.y, b = blockIdx.z;
  load_tw(tw, d.twx, g.px);
  const int nld = 3 * g.px * ty;
  const int64_t plane = (int64_t)g.nz * g.ys;
  for (int i = threadIdx.x; i < nld; i += blockDim.x) {
    const int t = i % ty;
    const int rest = i / ty;
    const int kx = rest % g.px, c = rest / g.px;
    const int y = y0 + t;
    C v = czero<C>();
    if (y < g.ny) v = d.work[(((int64_t)b * 3 + c) * g.px + kx) * plane + (int64_t)z * g.ys + y];
    s[(c * ty + t) * ps + kx] = v;
  }
  __syncthreads();
  fft_inverse(s, Batch{3 * ty, ps, 1, false}, g.plx, g.nx, tw);
  const int nst = 3 * ty * g.nx;
  const C* ia = d.ia + (int64_t)(rhs0 + b) * g.ncomp * 3;
  for (int i = threadIdx.x; i < nst; i += blockDim.x) {
    const int x = i % g.nx;
    const int rest = i / g.nx;
    const int t = rest % ty, c = rest / ty;
    const int y = y0 + t;
    if (y >= g.ny) continue;
    const int32_t idx = d.map[((int64_t)z * g.ny + y) * g.nx + x];
    if (idx < 0) continue;
    const int64_t o = ((int64_t)b * 3 + c) * g.n + idx;
    const int cc = d.comp ? d.comp[3 * idx + c] : 0;  // composition of axis c
    C pv = p[o];
    if (conj) pv = conjc(pv);
    C out;
    if (d.iat) {  // rotated dielectric frame: row c of the full symmetric alpha^{-1} of this site
      const C* m6 = d.iat + ((int64_t)(rhs0 + b) * g.n + idx) * 6;
      out = s[(c * ty + t) * ps + x];
      for (int c2 = 0; c2 < 3; ++c2) {
        C q = p[((int64_t)b * 3 + c2) * g.n + idx];
        if (conj) q = conjc(q);
        const int lo = c < c2 ? c : c2, hi = c < c2 ? c2 : c;
        out = cadd(out, cmul(m6[lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)], q));
      }
    } else {
      out = d.sc ? cadd(cmul(d.sc[((int64_t)b * g.ncomp + cc) * 3 + c], s[(c * ty + t) * ps + x]), pv)
                 : cadd(s[(c * ty + t) * ps + x], cmul(ia[cc * 3 + c], pv));
    }
    ap[o] = conj ? conjc(out) : out;
  }
}

// ------------------------------------------------------------------ z columns: FFT, Ghat, IFFT
// col layout [pz][3][G]; columns ky0..ky0+G-1 of plane kx. Caller loaded z < nz.
template <typename C>
__device__ __forceinline__ void zcol_process(C* col, const Geom& g, const MvData<C>& d, const C* twz, int kx,
                                             int ky0, int G) {
  const Batch bz{3 * G, 1, 3 * G, true};
  fft_forward(col, bz, g.plz, g.nz, twz);
  const int npt = g.pz * G;
  for (int i = threadIdx.x; i < npt; i += blockDim.x) {
    const int gg = i % G, kz = i / G;
    const int ky = ky0 + gg;
    if (ky >= g.py) continue;
    const C* gh = d.ghat + (((int64_t)kx * g.pz + kz) * g.py + ky) * 6;
    C* e = col + (kz * 3) * G + gg;
    C v0 = e[0], v1 = e[G], v2 = e[2 * G];
    gmul(gh, v0, v1, v2);
    e[0] = v0;
    e[G] = v1;
    e[2 * G] = v2;
  }
  __syncthreads();
  fft_inverse(col, bz, g.plz, g.nz, twz);
}

// ------------------------------------------------------------------ fused YZ plane (3-pass schedule)
// grid (nrhs, px) -- consecutive blocks share kx so the Ghat plane is reused from L2.
// smem: twy[py] twz[pz] plane[3*nz][py] col[pz][3][G]
template <typename C>
__global__ void k_yzplane(Geom g, MvData<C> d, int G) {
  extern __shared__ unsigned char smem_raw[];
  C* twy = reinterpret_cast<C*>(smem_raw);
  C* twz = twy + g.py;
  C* pl = twz + g.pz;
  C* col = pl + 3 * g.nz * g.py;
  const int b = blockIdx.x, kx = blockIdx.y;
  load_tw(twy, d.twy, g.py);
  load_tw(twz, d.twz, g.pz);
  C* wb = d.work + (((int64_t)b * 3) * g.px + kx) * ((int64_t)g.nz * g.ys);
  const int64_t cstride = (int64_t)g.px * g.nz * g.ys;
  const int nld = 3 * g.nz * g.ny;
  for (int i = threadIdx.x; i < nld; i += blockDim.x) {
    const int y = i % g.ny;
    const int rest = i / g.ny;
    const int z = rest % g.nz, c = rest / g.nz;
    pl[(c * g.nz + z) * g.py + y] = wb[c * cstride + (int64_t)z * g.ys + y];
  }
  __syncthreads();
  const Batch by{3 * g.nz, g.py, 1, false};
  fft_forward(pl, by, g.ply, g.ny, twy);
  for (int ky0 = 0; ky0 < g.py; ky0 += G) {
    const int ncl = 3 * g.nz * G;
    for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
      const int gg = i % G;
      const int rest = i / G;
      const int z = rest % g.nz, c = rest / g.nz;
      const int ky = ky0 + gg;
      col[(z * 3 + c) * G + gg] = (ky < g.py) ? pl[(c * g.nz + z) * g.py + ky] : czero<C>();
    }
    __syncthreads();
    zcol_process(col, g, d, twz, kx, ky0, G);
    for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
      const int gg = i % G;
      const int rest = i / G;
      const int z = rest % g.nz, c = rest / g.nz;
      const int ky = ky0 + gg;
      if (ky < g.py) pl[(c * g.nz + z) * g.py + ky] = col[(z * 3 + c) * G + gg];
    }
    __syncthreads();
  }
  fft_inverse(pl, by, g.ply, g.ny, twy);
  for (int i = threadIdx.x; i < nld; i += blockDim.x) {
    const int y = i % g.ny;
    const int rest = i / g.ny;
    const int z = rest % g.nz, c = rest / g.nz;
    wb[c * cstride + (int64_t)z * g.ys + y] = pl[(c * g.nz + z) * g.py + y];
  }
}

// ------------------------------------------------------------------ 5-pass pieces
// z pass alone: grid (nrhs, ceil(py/G), px)
template <typename C>
__global__ void k_zconv(Geom g, MvData<C> d, int G) {
  extern __shared__ unsigned char smem_raw[];
  C* twz = reinterpret_cast<C*>(smem_raw);
  C* col = twz + g.pz;
  const int ky0 = blockIdx.y * G, kx = blockIdx.z, b = blockIdx.x;  // RHS fastest: Ghat tiles reused from L2
  load_tw(twz, d.twz, g.pz);
  C* wb = d.work + (((int64_t)b * 3) * g.px + kx) * ((int64_t)g.nz * g.ys);
  const int64_t cstride = (int64_t)g.px * g.nz * g.ys;
  const int ncl = 3 * g.nz * G;
  for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
    const int gg = i % G;
    const int rest = i / G;
    const int z = rest % g.nz, c = rest / g.nz;
    const int ky = ky0 + gg;
    col[(z * 3 + c) * G + gg] = (ky < g.py) ? wb[c * cstride + (int64_t)z * g.ys + ky] : czero<C>();
  }
  __syncthreads();
  zcol_process(col, g, d, twz, kx, ky0, G);
  for (int i = threadIdx.x; i < ncl; i += blockDim.x) {
    const int gg = i % G;
    const int rest = i / G;
    const int z = rest % g.nz, c = rest / g.nz;
    const int ky = ky0 + gg;
    if (ky < g.py) wb[c * cstride + (int64_t)z * g.ys + ky] = col[(z * 3 + c) * G + gg];
  }
}

// contiguous rows of length L (row r at data + r*row_stride): rows_per_block rows per CTA
template <typename C>
__global__ void k_fft_rows(C* data, int64_t nrows, int64_t row_stride, FftPlan pl, const C* twg, int nin,
                           int nout, int rpb, bool inverse) {
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + pl.L;
  const int L = pl.L, ps = L + 1;
  load_tw(tw, twg, L);
  const int64_t r0 = (int64_t)blockIdx.x * rpb;
  const int nr = (int)min((int64_t)rpb, nrows - r0);
  const int lim_in = inverse ? L : nin;
  for (int i = threadIdx.x; i < nr * lim_in; i += blockDim.x) {
    const int r = i / lim_in, e = i % lim_in;
    s[r * ps + e] = data[(r0 + r) * row_stride + e];
  }
  __syncthreads();
  const Batch bt{nr, ps, 1, false};
  if (inverse) fft_inverse(s, bt, pl, nout, tw);
  else fft_forward(s, bt, pl, nin, tw);
  const int lim_out = inverse ? nout : L;
  for (int i = threadIdx.x; i < nr * lim_out; i += blockDim.x) {
    const int r = i / lim_out, e = i % lim_out;
    data[(r0 + r) * row_stride + e] = s[r * ps + e];
  }
}

// strided pencils: element e of pencil (o, i) at data[o*outer_stride + i + e*estride];
// grid (ceil(ninner/ti), nouter); smem tw[L] + s[L][ti]
template <typename C>
__global__ void k_fft_strided(C* data, int64_t estride, int64_t ninner, int64_t outer_stride, FftPlan pl,
                              const C* twg, int ti, bool inverse) {
  extern __shared__ unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s = tw + pl.L;
  const int L = pl.L;
  load_tw(tw, twg, L);
  const int64_t i0 = (int64_t)blockIdx.x * ti;
  const int ni = (int)min((int64_t)ti, ninner - i0);
  C* base = data + (int64_t)blockIdx.y * outer_stride + i0;
  for (int i = threadIdx.x; i < L * ti; i += blockDim.x) {
    const int ii = i % ti, e = i / ti;
    s[e * ti + ii] = (ii < ni) ? base[e * estride + ii] : czero<C>();
  }
  __syncthreads();
  const Batch bt{ti, 1, ti, true};
  if (inverse) fft_inverse(s, bt, pl, L, tw);
  else fft_forward(s, bt, pl, L, tw);
  for (int i = threadIdx.x; i < L * ti; i += blockDim.x) {
    const int ii = i % ti, e = i / ti;
    if (ii < ni) base[e * estride + ii] = s[e * ti + ii];
  }
}

// ------------------------------------------------------------------ Green tensor
// A_ab(n) = exp(ikr)/r [k^2 (rh_a rh_b - d_ab) + (ikr - 1)/r^2 (3 rh_a rh_b - d_ab)] for offset n != 0
// reachable by two sites (|n_x| < Nx ...), else 0.  Output Gw[6][pz][py][px].
// The interaction tensor of a lattice offset n, component c (xx, xy, xz, yy, yz, zz), is even
// or odd in each of n_x, n_y, n_z: xy is odd in x and y, xz in x and z, yz in y and z, the
// diagonal components even in all three.  Its zero-padded DFT inherits the same parity per
// axis, so the FP64 build fills and transforms only what the parities do not determine:
// the x transforms run on the rows with y <= Py/2, z <= Pz/2, the y transforms on the
// planes z <= Pz/2 for natural kx <= Px/2, the z transforms on natural kx <= Px/2,
// ky <= Py/2, and the missing parts are mirrored in between and in the final pack (1/4 of
// the FFT work and of the fill of a plain 3-D transform).
__device__ __forceinline__ bool odd_in(int c, int axis) {
  // bit a of the mask = odd in axis a (0 = x, 1 = y, 2 = z)
  const int mask[6] = {0, 3, 5, 0, 6, 0};
  return (mask[c] >> axis) & 1;
}

// q[c][zq][yq][x] for zq <= Pz/2, yq <= Py/2 and all x (offsets wrapped along x)
__global__ void k_green_fill_q(Geom g, double kd, double2* q) {
  const int hy1 = g.py / 2 + 1, hz1 = g.pz / 2 + 1;
  const int64_t Q = (int64_t)g.px * hy1 * hz1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Q; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.px);
    const int64_t rest = i / g.px;
    const int y = (int)(rest % hy1), z = (int)(rest / hy1);
    int ox = 0;
    bool ok = y < g.ny && z < g.nz;
    if (x < g.nx) ox = x; else if (x > g.px - g.nx) ox = x - g.px; else ok = false;
    if (ox == 0 && y == 0 && z == 0) ok = false;
    double2 out[6];
    for (int c = 0; c < 6; ++c) out[c] = make_double2(0.0, 0.0);
    if (ok) {
      const double rx = ox, ry = y, rz = z;
      const double r2 = rx * rx + ry * ry + rz * rz;
      const double r = sqrt(r2);
      const double inv_r = 1.0 / r;
      const double h[3] = {rx * inv_r, ry * inv_r, rz * inv_r};
      double sn, cs;
      sincos(kd * r, &sn, &cs);
      // pref = exp(ikr)/r ; t2 = (ikr - 1)/r^2
      const double2 pref = make_double2(cs * inv_r, sn * inv_r);
      const double2 t2 = make_double2(-1.0 / r2, kd * r / r2);
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
      for (int c = 0; c < 6; ++c) {
        const double hh = h[ia[c]] * h[ib[c]];
        const double dl = (ia[c] == ib[c]) ? 1.0 : 0.0;
        const double a = kd * kd * (hh - dl);
        const double bq = 3.0 * hh - dl;
        const double2 inner = make_double2(a + t2.x * bq, t2.y * bq);
        out[c] = make_double2(pref.x * inner.x - pref.y * inner.y, pref.x * inner.y + pref.y * inner.x);
      }
    }
    for (int c = 0; c < 6; ++c) q[(int64_t)c * Q + i] = out[c];
  }
}

// After the x transform only the natural frequencies kx <= Px/2 are carried on (the others
// follow by the x parity); the spectra are in the engine's digit-reversed storage order, so
// the host passes the storage position stx[k] of natural frequency k and, for the final
// pack, the natural frequency natx[s] of storage position s (likewise for y).
// t[c][zq][y][k] (all y, k <= Px/2) from q[c][zq][yq][stx[k]]: rows y > Py/2 mirror Py - y
__global__ void k_green_expand_y(Geom g, const int32_t* __restrict__ stx, const double2* __restrict__ q,
                                 double2* __restrict__ t) {
  const int hx1 = g.px / 2 + 1, hy1 = g.py / 2 + 1, hz1 = g.pz / 2 + 1;
  const int64_t Q = (int64_t)g.px * hy1 * hz1, T = (int64_t)hx1 * g.py * hz1;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < 6 * T; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o / T);
    const int64_t i = o - c * T;
    const int k = (int)(i % hx1);
    const int64_t rest = i / hx1;
    const int y = (int)(rest % g.py), z = (int)(rest / g.py);
    const bool mir = y > g.py / 2;
    const int ys = mir ? g.py - y : y;
    double2 v = q[(int64_t)c * Q + ((int64_t)z * hy1 + ys) * g.px + stx[k]];
    if (mir && odd_in(c, 1)) v = make_double2(-v.x, -v.y);
    t[o] = v;
  }
}

// f[c][z][ky][kx] (all z; natural ky <= Py/2, kx <= Px/2) from t[c][zq][sty[ky]][kx]:
// planes z > Pz/2 mirror Pz - z with the z parity
__global__ void k_green_expand_z(Geom g, const int32_t* __restrict__ sty, const double2* __restrict__ t,
                                 double2* __restrict__ f) {
  const int hx1 = g.px / 2 + 1, hy1 = g.py / 2 + 1, hz1 = g.pz / 2 + 1;
  const int64_t T = (int64_t)hx1 * g.py * hz1, P = (int64_t)hx1 * hy1, F = P * g.pz;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < 6 * F; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o / F);
    const int64_t i = o - c * F;
    const int z = (int)(i / P);
    const int64_t r = i - (int64_t)z * P;
    const int ky = (int)(r / hx1), kx = (int)(r - (int64_t)ky * hx1);
    const bool mir = z > g.pz / 2;
    const int zs = mir ? g.pz - z : z;
    double2 v = t[(int64_t)c * T + ((int64_t)zs * g.py + sty[ky]) * hx1 + kx];
    if (mir && odd_in(c, 2)) v = make_double2(-v.x, -v.y);
    f[o] = v;
  }
}

// ghat[kx][kz][ky][6] (storage positions) = f[c][kz][ky'][kx'] / M, with kx', ky' the natural
// frequencies folded into [0, P/2] and the sign of the parities of the folds
__global__ void k_green_pack(Geom g, const int32_t* __restrict__ natx, const int32_t* __restrict__ naty,
                             const double2* __restrict__ f, double2* __restrict__ g128, float2* __restrict__ g64,
                             dfp::dfc* __restrict__ gdf) {
  const int64_t M = (int64_t)g.px * g.py * g.pz;
  const int hx1 = g.px / 2 + 1, hy1 = g.py / 2 + 1;
  const int64_t P = (int64_t)hx1 * hy1, F = P * g.pz;
  const double inv = 1.0 / (double)M;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < 6 * M; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o % 6);
    const int64_t pt = o / 6;
    const int ky = (int)(pt % g.py);
    const int64_t rest = pt / g.py;
    const int kz = (int)(rest % g.pz), kx = (int)(rest / g.pz);
    int nx = natx[kx], ny = naty[ky];
    const bool fx = nx > g.px / 2, fy = ny > g.py / 2;
    if (fx) nx = g.px - nx;
    if (fy) ny = g.py - ny;
    double2 v = f[(int64_t)c * F + (int64_t)kz * P + (int64_t)ny * hx1 + nx];
    const bool neg = (fx && odd_in(c, 0)) != (fy && odd_in(c, 1));
    const double sc = neg ? -inv : inv;
    const double2 w = make_double2(v.x * sc, v.y * sc);
    g128[o] = w;
    g64[o] = make_float2((float)w.x, (float)w.y);
    if (gdf) gdf[o] = dfp::from_c128(w);
  }
}

// natural frequency of storage position p of an in-place DIF transform with this plan:
// a radix-R stage on length L leaves frequency residue k at offset k (L/R) of the next sub-transform
int natural_index(const FftPlan& pl, int p) {
  int L = pl.L, nat = 0, mult = 1;
  for (int s = 0; s < pl.nst && L > 1; ++s) {
    const int R = pl.radix[s], m = L / R;
    nat += mult * (p / m);
    mult *= R;
    p %= m;
    L = m;
  }
  return nat;
}

int g_smem_optin = 0;
std::atomic<unsigned long long> g_launches{0};

// Dynamic shared memory above 48 KB needs the per-kernel opt-in attribute; it is
// set once to the device maximum (init_kernel_attrs), so launches made while a
// stream is being captured need no attribute calls.
Err set_smem(size_t bytes) {
  if (g_smem_optin == 0) return Err::make(DDA_ESTATE, "kernel attributes not initialized");
  if (bytes > (size_t)g_smem_optin)
    return Err::make(DDA_EUNSUPPORTED, "FFT tile needs " + std::to_string(bytes) + " B of shared memory, device allows " +
                                           std::to_string(g_smem_optin));
  return Err::Ok();
}

template <typename K>
void optin(K kern) {
  optin_smem(kern, g_smem_optin);
}

}  // namespace

size_t x_smem_bytes(const Geom& g, const MvTune& t, size_t csize) {
  return csize * ((size_t)g.px + (size_t)3 * t.ty * (g.px + 1));
}

template <typename C>
size_t plane_smem_bytes(const Geom& g, const MvTune& t) {
  return sizeof(C) * ((size_t)g.py + g.pz + (size_t)3 * g.nz * g.py + (size_t)g.pz * 3 * t.g);
}


// optional per-pass events (profiling): ev[0] before the first pass, ev[i+1] after pass i
thread_local cudaEvent_t* t_pass_events = nullptr;
inline void mark(int i, cudaStream_t st) {
  if (t_pass_events) cudaEventRecord(t_pass_events[i], st);
}
void mark_pass(int i, cudaStream_t st) { mark(i, st); }

template <typename C>
Err launch_matvec(const Geom& g, const MvData<C>& d, const MvTune& t, const C* p, C* ap, int nrhs, int rhs0,
                  bool conj, cudaStream_t st) {
  if (nrhs <= 0) return Err::Ok();
  if (d.sc && rhs0 != 0) {  // the scale table is indexed from the launch's first RHS
    MvData<C> dd = d;
    dd.sc += (int64_t)rhs0 * g.ncomp * 3;
    return launch_matvec<C>(g, dd, t, p, ap, nrhs, 0, conj, st);  // the alpha table is unused when scaled
  }
  if (t.fast) return launch_matvec_fast<C>(g, d, t, p, ap, nrhs, rhs0, conj, st);
  int pass = 0;
  mark(pass++, st);
  const size_t sx = x_smem_bytes(g, t, sizeof(C));
  DDA_TRY(set_smem(sx));
  dim3 gx((g.ny + t.ty - 1) / t.ty, g.nz, nrhs);
  k_xfwd<C><<<gx, t.thr_x, sx, st>>>(g, d, p, t.ty, conj);
  DDA_CU(cudaGetLastError());
  mark(pass++, st);
  if (t.plane) {
    const size_t sp = plane_smem_bytes<C>(g, t);
    DDA_TRY(set_smem(sp));
    k_yzplane<C><<<dim3(nrhs, g.px), t.thr_p, sp, st>>>(g, d, t.g);
    DDA_CU(cudaGetLastError());
    mark(pass++, st);
    g_launches += 3;
  } else {
    // 5-pass: Y forward rows, Z columns, Y inverse rows
    const int64_t nrows = (int64_t)nrhs * 3 * g.px * g.nz;
    const int rpb = 4;
    const size_t sr = sizeof(C) * ((size_t)g.py + (size_t)rpb * (g.py + 1));
    DDA_TRY(set_smem(sr));
    const unsigned nb = (unsigned)((nrows + rpb - 1) / rpb);
    k_fft_rows<C><<<nb, t.thr_x, sr, st>>>(d.work, nrows, g.ys, g.ply, d.twy, g.ny, g.py, rpb, false);
    DDA_CU(cudaGetLastError());
    mark(pass++, st);
    const size_t sz = sizeof(C) * ((size_t)g.pz + (size_t)g.pz * 3 * t.g);
    DDA_TRY(set_smem(sz));
    k_zconv<C><<<dim3(nrhs, (g.py + t.g - 1) / t.g, g.px), t.thr_p, sz, st>>>(g, d, t.g);
    DDA_CU(cudaGetLastError());
    mark(pass++, st);
    k_fft_rows<C><<<nb, t.thr_x, sr, st>>>(d.work, nrows, g.ys, g.ply, d.twy, g.py, g.ny, rpb, true);
    DDA_CU(cudaGetLastError());
    mark(pass++, st);
    g_launches += 5;
  }
  k_xinv<C><<<gx, t.thr_x, sx, st>>>(g, d, p, ap, t.ty, rhs0, conj);
  DDA_CU(cudaGetLastError());
  mark(pass++, st);
  return Err::Ok();
}

// ------------------------------------------------------------------ fixed scratch for dda_matvec_noalloc
// The FFT workspace of the product for callers that cannot allocate device
// memory.  It is part of the module image: every GPU that loads the library
// holds these bytes until the process exits.  All calls share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// Device address of the fixed scratch on `device`.  The first call for a device
// makes that device current and asks the runtime for the symbol's address
// (host code only holds a stand-in for the array, never its device address);
// later calls return the cached pointer.
Err noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return Err::make(DDA_EINVAL, "device index out of range for the fixed scratch");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    int prev = 0;
    DDA_CU(cudaGetDevice(&prev));
    DDA_CU(cudaSetDevice(device));
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess || ptr == nullptr)
      return Err::make(DDA_ECUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") +
                                      cudaGetErrorString(e));
    g_noalloc_addr[device] = ptr;
  }
  *out = g_noalloc_addr[device];
  return Err::Ok();
}

void set_pass_events(cudaEvent_t* ev) { t_pass_events = ev; }
namespace {
thread_local bool t_pdl = false;
}
bool pdl_enabled() { return t_pdl; }
void set_pdl(bool on) { t_pdl = on; }
unsigned long long launches() { return g_launches.load(); }
void add_launches(unsigned long long n) { g_launches += n; }
void sub_launches(unsigned long long n) { g_launches -= n; }

template <typename C>
Err fft_rows(C* data, int64_t nrows, int64_t row_stride, const FftPlan& pl, const C* tw, int nin, int nout,
             bool inverse, cudaStream_t st) {
  const int rpb = 4;
  const size_t sr = sizeof(C) * ((size_t)pl.L + (size_t)rpb * (pl.L + 1));
  DDA_TRY(set_smem(sr));
  const unsigned nb = (unsigned)((nrows + rpb - 1) / rpb);
  k_fft_rows<C><<<nb, 256, sr, st>>>(data, nrows, row_stride, pl, tw, nin, nout, rpb, inverse);
  DDA_CU(cudaGetLastError());
  g_launches += 1;
  return Err::Ok();
}

template <typename C>
Err fft_strided(C* data, int L, int64_t estride, int64_t ninner, int64_t nouter, int64_t outer_stride,
                const FftPlan& pl, const C* tw, bool inverse, cudaStream_t st) {
  const int ti = 16;
  const size_t sm = sizeof(C) * ((size_t)L + (size_t)L * ti);
  DDA_TRY(set_smem(sm));
  dim3 grid((unsigned)((ninner + ti - 1) / ti), (unsigned)nouter);
  k_fft_strided<C><<<grid, 256, sm, st>>>(data, estride, ninner, outer_stride, pl, tw, ti, inverse);
  DDA_CU(cudaGetLastError());
  g_launches += 1;
  return Err::Ok();
}

void init_kernel_attrs() {
  if (g_smem_optin) return;
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  g_smem_optin = v;
  optin(k_xfwd<float2>); optin(k_xfwd<double2>);
  optin(k_xinv<float2>); optin(k_xinv<double2>);
  optin(k_yzplane<float2>); optin(k_yzplane<double2>);
  optin(k_zconv<float2>); optin(k_zconv<double2>);
  optin(k_fft_rows<float2>); optin(k_fft_rows<double2>);
  optin(k_fft_strided<float2>); optin(k_fft_strided<double2>);
  fast_optin_c64(v);
  cluster_optin_c64(v);
  plane_bulk_optin_c64(v);
  fast_optin_c128(v);
  fast_optin_df(v);
  fused_optin_c64(v);
}

void green_perm_tables(const Geom& g, std::vector<int32_t>* out) {
  const int hx1 = g.px / 2 + 1, hy1 = g.py / 2 + 1;
  out->assign((size_t)g.px + g.py + hx1 + hy1, 0);
  int32_t* natx = out->data();
  int32_t* naty = natx + g.px;
  int32_t* stx = naty + g.py;
  int32_t* sty = stx + hx1;
  for (int p = 0; p < g.px; ++p) {
    natx[p] = natural_index(g.plx, p);
    if (natx[p] <= g.px / 2) stx[natx[p]] = p;
  }
  for (int p = 0; p < g.py; ++p) {
    naty[p] = natural_index(g.ply, p);
    if (naty[p] <= g.py / 2) sty[naty[p]] = p;
  }
}

Err build_green(const Geom& g, double kd, const double2* twx, const double2* twy, const double2* twz,
                const int32_t* perm, double2* gw, double2* ghat128, float2* ghat64, dfp::dfc* ghatdf,
                cudaStream_t st) {
  const int64_t M = (int64_t)g.px * g.py * g.pz;
  const int hx1 = g.px / 2 + 1, hy1 = g.py / 2 + 1, hz1 = g.pz / 2 + 1;
  const int64_t Q = (int64_t)g.px * hy1 * hz1, T = (int64_t)hx1 * g.py * hz1, F = (int64_t)hx1 * hy1 * g.pz;
  auto nblk = [](int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); };
  Err e = Err::Ok();
  // perm (green_perm_tables): natx[px] | naty[py] | stx[hx1] | sty[hy1]
  const int32_t* d_natx = perm;
  const int32_t* d_naty = d_natx + g.px;
  const int32_t* d_stx = d_naty + g.py;
  const int32_t* d_sty = d_stx + hx1;
  // q (in gw): the quarter y <= Py/2, z <= Pz/2 of the wrapped tensor; x rows transformed in place
  double2* q = gw;
  if (e.ok()) {
    k_green_fill_q<<<nblk(Q), 256, 0, st>>>(g, kd, q);
    if (cudaGetLastError() != cudaSuccess) e = Err::make(DDA_ECUDA, "Green fill failed");
  }
  if (e.ok()) e = fft_rows<double2>(q, 6 * (int64_t)hy1 * hz1, g.px, g.plx, twx, g.px, g.px, false, st);
  // t (in the ghat128 buffer, free until the pack): planes z <= Pz/2, all y, natural kx <= Px/2
  double2* t = ghat128;
  if (e.ok()) {
    k_green_expand_y<<<nblk(6 * T), 256, 0, st>>>(g, d_stx, q, t);
    if (cudaGetLastError() != cudaSuccess) e = Err::make(DDA_ECUDA, "Green expand (y) failed");
  }
  if (e.ok()) e = fft_strided<double2>(t, g.py, hx1, hx1, 6 * (int64_t)hz1, (int64_t)hx1 * g.py, g.ply, twy, false, st);
  // f (in gw): all z, natural ky <= Py/2, kx <= Px/2; z columns transformed
  if (e.ok()) {
    k_green_expand_z<<<nblk(6 * F), 256, 0, st>>>(g, d_sty, t, gw);
    if (cudaGetLastError() != cudaSuccess) e = Err::make(DDA_ECUDA, "Green expand (z) failed");
  }
  if (e.ok())
    e = fft_strided<double2>(gw, g.pz, (int64_t)hx1 * hy1, (int64_t)hx1 * hy1, 6, F, g.plz, twz, false, st);
  if (e.ok()) {
    k_green_pack<<<nblk(6 * M), 256, 0, st>>>(g, d_natx, d_naty, gw, ghat128, ghat64, ghatdf);
    if (cudaGetLastError() != cudaSuccess) e = Err::make(DDA_ECUDA, "Green pack failed");
  }
  g_launches += 4;
  return e;
}

// ------------------------------------------------------------------ periodic targets
// The interaction of a target unit cell repeated with periods (py, pz) along y_TF, z_TF under a
// plane wave of TF wave vector k: A^per(r) = sum_R exp(i k.R) A(r - R) exp[-(gamma kd |r - R|)^4]
// over the replica offsets R = (0, m py, n pz) (the term r - R = 0 omitted), kept wherever the
// cutoff factor is above exp(-40).  It is not even in r for oblique incidence, so every offset of
// the wrapped grid is filled and transformed (no parity shortcut).  One CTA per grid point; its
// threads stride over the replicas and sum in FP64, then a fixed-order block reduction.
namespace {
constexpr int kPbcT = 256;
__global__ void __launch_bounds__(kPbcT) k_green_fill_pbc(Geom g, double kd, double k1, double k2, double py,
                                                          double pz, double gamma, int my, int mz, double rmax,
                                                          double2* __restrict__ gw) {
  const int64_t M = (int64_t)g.px * g.py * g.pz;
  const int64_t i = blockIdx.x;
  const int x = (int)(i % g.px);
  const int64_t rest = i / g.px;
  const int y = (int)(rest % g.py), z = (int)(rest / g.py);
  int o[3];
  const int xs[3] = {x, y, z}, ns[3] = {g.nx, g.ny, g.nz}, ps[3] = {g.px, g.py, g.pz};
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    if (xs[a] < ns[a]) o[a] = xs[a];
    else if (xs[a] > ps[a] - ns[a]) o[a] = xs[a] - ps[a];
    else ok = false;
  }
  double acc[12];
  for (int q = 0; q < 12; ++q) acc[q] = 0.0;
  if (ok) {
    const int nm = 2 * my + 1, nn = 2 * mz + 1;
    const int64_t nrep = (int64_t)nm * nn;
    const double gk = gamma * kd;
    for (int64_t t = threadIdx.x; t < nrep; t += kPbcT) {
      const int m = (int)(t / nn) - my, n = (int)(t % nn) - mz;
      const double Ry = m * py, Rz = n * pz;
      const double rx = o[0], ry = o[1] - Ry, rz = o[2] - Rz;
      const double r2 = rx * rx + ry * ry + rz * rz;
      if (r2 == 0.0 || r2 > rmax * rmax) continue;
      const double r = sqrt(r2), inv_r = 1.0 / r;
      const double u = gk * r, u2 = u * u;
      const double cut = exp(-u2 * u2);
      double sb, cb;
      sincos(k1 * Ry + k2 * Rz, &sb, &cb);   // Bloch phase exp(i k.R)
      double sn, cs;
      sincos(kd * r, &sn, &cs);
      // pref = exp(ikr)/r * phase * cut ; t2 = (ikr - 1)/r^2
      const double2 e1 = make_double2(cs * inv_r * cut, sn * inv_r * cut);
      const double2 pref = make_double2(e1.x * cb - e1.y * sb, e1.x * sb + e1.y * cb);
      const double2 t2 = make_double2(-1.0 / r2, kd * r / r2);
      const double h[3] = {rx * inv_r, ry * inv_r, rz * inv_r};
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
      for (int c = 0; c < 6; ++c) {
        const double hh = h[ia[c]] * h[ib[c]];
        const double dl = (ia[c] == ib[c]) ? 1.0 : 0.0;
        const double2 inner = make_double2(kd * kd * (hh - dl) + t2.x * (3.0 * hh - dl), t2.y * (3.0 * hh - dl));
        acc[2 * c] += pref.x * inner.x - pref.y * inner.y;
        acc[2 * c + 1] += pref.x * inner.y + pref.y * inner.x;
      }
    }
  }
  __shared__ double red[12][kPbcT / 32];
  for (int q = 0; q < 12; ++q)
    for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < 12; ++q) red[q][w] = acc[q];
  __syncthreads();
  if (threadIdx.x < 12) {
    double v = 0.0;
    for (int k = 0; k < kPbcT / 32; ++k) v += red[threadIdx.x][k];
    const int c = threadIdx.x / 2;
    double* dst = reinterpret_cast<double*>(gw + (int64_t)c * M + i);
    dst[threadIdx.x % 2] = v;
  }
}

// ghat[kx][kz][ky][6] (storage positions) = gw[c][kz][ky][kx] / M after the full transform
__global__ void k_green_pack_full(Geom g, const double2* __restrict__ f, double2* __restrict__ g128,
                                  float2* __restrict__ g64, dfp::dfc* __restrict__ gdf) {
  const int64_t M = (int64_t)g.px * g.py * g.pz;
  const double inv = 1.0 / (double)M;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < 6 * M; o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o % 6);
    const int64_t pt = o / 6;
    const int ky = (int)(pt % g.py);
    const int64_t rest = pt / g.py;
    const int kz = (int)(rest % g.pz), kx = (int)(rest / g.pz);
    const double2 v = f[(int64_t)c * M + ((int64_t)kz * g.py + ky) * g.px + kx];
    const double2 w = make_double2(v.x * inv, v.y * inv);
    g128[o] = w;
    g64[o] = make_float2((float)w.x, (float)w.y);
    if (gdf) gdf[o] = dfp::from_c128(w);
  }
}
}  // namespace

Err build_green_pbc(const Geom& g, double kd, const double k_tf[3], double py, double pz, double gamma,
                    const double2* twx, const double2* twy, const double2* twz, double2* gw, double2* ghat128,
                    float2* ghat64, dfp::dfc* ghatdf, cudaStream_t st) {
  const int64_t M = (int64_t)g.px * g.py * g.pz;
  if (M > 2147483647LL) return Err::make(DDA_EUNSUPPORTED, "periodic Green grid too large");
  // replicas within rmax + the longest offset; (gamma kd r)^4 <= 40
  const double reach = std::sqrt((double)g.nx * g.nx + (double)g.ny * g.ny + (double)g.nz * g.nz);
  const double rmax = std::pow(40.0, 0.25) / (gamma * kd);
  const int my = py > 0 ? (int)std::ceil((rmax + reach) / py) : 0;
  const int mz = pz > 0 ? (int)std::ceil((rmax + reach) / pz) : 0;
  if ((double)(2 * my + 1) * (2 * mz + 1) > 4.0e8)
    return Err::make(DDA_EUNSUPPORTED, "too many periodic replicas for this gamma and period (raise gamma)");
  k_green_fill_pbc<<<(unsigned)M, kPbcT, 0, st>>>(g, kd, k_tf[1], k_tf[2], py, pz, gamma, my, mz, rmax, gw);
  if (cudaGetLastError() != cudaSuccess) return Err::make(DDA_ECUDA, "periodic Green fill failed");
  DDA_TRY(fft_rows<double2>(gw, 6 * (int64_t)g.py * g.pz, g.px, g.plx, twx, g.px, g.px, false, st));
  DDA_TRY(fft_strided<double2>(gw, g.py, g.px, g.px, 6 * (int64_t)g.pz, (int64_t)g.px * g.py, g.ply, twy, false, st));
  DDA_TRY(fft_strided<double2>(gw, g.pz, (int64_t)g.px * g.py, (int64_t)g.px * g.py, 6, M, g.plz, twz, false, st));
  const int nb = (int)std::min<int64_t>((6 * M + 255) / 256, 152 * 16);
  k_green_pack_full<<<nb, 256, 0, st>>>(g, gw, ghat128, ghat64, ghatdf);
  if (cudaGetLastError() != cudaSuccess) return Err::make(DDA_ECUDA, "periodic Green pack failed");
  g_launches += 2;
  return Err::Ok();
}

template Err launch_matvec<float2>(const Geom&, const MvData<float2>&, const MvTune&, const float2*, float2*, int,
                                   int, bool, cudaStream_t);
template Err launch_matvec<double2>(const Geom&, const MvData<double2>&, const MvTune&, const double2*, double2*,
                                    int, int, bool, cudaStream_t);
template size_t plane_smem_bytes<float2>(const Geom&, const MvTune&);
template size_t plane_smem_bytes<double2>(const Geom&, const MvTune&);
template Err fft_rows<float2>(float2*, int64_t, int64_t, const FftPlan&, const float2*, int, int, bool, cudaStream_t);
template Err fft_rows<double2>(double2*, int64_t, int64_t, const FftPlan&, const double2*, int, int, bool,
                               cudaStream_t);
template Err fft_strided<float2>(float2*, int, int64_t, int64_t, int64_t, int64_t, const FftPlan&, const float2*,
                                 bool, cudaStream_t);
template Err fft_strided<double2>(double2*, int, int64_t, int64_t, int64_t, int64_t, const FftPlan&, const double2*,
                                  bool, cudaStream_t);

}  // namespace dda
