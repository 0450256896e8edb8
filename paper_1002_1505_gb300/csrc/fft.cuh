// In-place mixed-radix FFT engine on shared memory, used by every FFT pass of
// the DDA convolution (Goodman, Draine & Flatau 1991: the off-diagonal part of
// A P is a discrete convolution evaluated with zero-padded 3-D FFTs).
//
// Forward transforms are decimation-in-frequency (Gentleman-Sande) and leave
// the spectrum in mixed-radix digit-reversed order; inverse transforms are the
// exact reverse (decimation-in-time) and take that order back to natural
// order.  The convolution never needs the spectrum in natural order: the
// Fourier-space Green tensor is produced by the same forward plans, so both
// operands share one permutation and no reordering pass exists anywhere.
//
// Pruning for the zero-padded lengths L = 2n: the plan always begins with a
// radix-2 stage when L is even.  A forward transform whose input has only
// `nin` <= L/2 nonzero entries skips the upper-half loads of that stage
// (y0 = x, y1 = x w^n), and an inverse transform whose output is needed only
// for indices < `nout` <= L/2 computes only the lower half of its last stage.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

// ------------------------------------------------------------------ plans
constexpr int kMaxStages = 12;

struct FftPlan {
  int L;                  // transform length
  int nst;                // number of stages
  int radix[kMaxStages];  // radix of each DIF stage (stage 0 = outermost)
  int len[kMaxStages];    // sub-transform length entering each DIF stage
};

#ifdef __CUDACC__
// ------------------------------------------------------------------ complex helpers
template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by i*s (s = +1 or -1)
template <typename C> __device__ __forceinline__ C cmuli(C a, int s) { C r; r.x = -s * a.y; r.y = s * a.x; return r; }
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }

// ------------------------------------------------------------------ small DFTs
// y_k = sum_j x_j exp(S * 2 pi i j k / R), S = -1 forward, +1 inverse.
template <int R, int S, typename C> struct Dft;

template <int S, typename C> struct Dft<2, S, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int S, typename C> struct Dft<3, S, C> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(v[0].x);
    const R h = (R)(S * 0.86602540378443864676);  // S sin(2 pi / 3)
    const C s = cadd(v[1], v[2]);
    const C d = csub(v[1], v[2]);
    C m;  // x0 - s/2
    m.x = fma((R)-0.5, s.x, v[0].x);
    m.y = fma((R)-0.5, s.y, v[0].y);
    v[0] = cadd(v[0], s);
    // outputs m +- i h d, one FMA per real part
    v[1] = mk(fma(-h, d.y, m.x), fma(h, d.x, m.y));
    v[2] = mk(fma(h, d.y, m.x), fma(-h, d.x, m.y));
  }
};

template <int S, typename C> struct Dft<4, S, C> {
  static __device__ __forceinline__ void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmuli(csub(v[1], v[3]), S);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <int S, typename C> struct Dft<5, S, C> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(v[0].x);
    const R c1 = (R)0.30901699437494742410;   // cos(2 pi/5)
    const R c2 = (R)-0.80901699437494742410;  // cos(4 pi/5)
    const R s1 = (R)0.95105651629515357212;   // sin(2 pi/5)
    const R s2 = (R)0.58778525229247312917;   // sin(4 pi/5)
    C p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    C p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    C x0 = v[0];
    C a1 = cadd(x0, cadd(cscale(p1, c1), cscale(p2, c2)));
    C a2 = cadd(x0, cadd(cscale(p1, c2), cscale(p2, c1)));
    C b1 = cmuli(cadd(cscale(m1, s1), cscale(m2, s2)), S);
    C b2 = cmuli(csub(cscale(m1, s2), cscale(m2, s1)), S);
    v[0] = cadd(x0, cadd(p1, p2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

template <int S, typename C> struct Dft<8, S, C> {
  static __device__ __forceinline__ void run(C* v) {
    using R = decltype(v[0].x);
    const R r2 = (R)0.70710678118654752440;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, S, C>::run(e);
    Dft<4, S, C>::run(o);
    // w8^k = exp(S 2 pi i k / 8): k=1 -> (1 + iS)/sqrt2, k=2 -> iS, k=3 -> (-1 + iS)/sqrt2.
    // The 1/sqrt2 factor is folded into the butterflies' FMAs.
    const C a1 = mk(o[1].x - S * o[1].y, o[1].y + S * o[1].x);  // (1 + iS) o1
    const C a3 = mk(-o[3].x - S * o[3].y, S * o[3].x - o[3].y);  // (-1 + iS) o3
    const C o2 = cmuli(o[2], S);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = mk(fma(r2, a1.x, e[1].x), fma(r2, a1.y, e[1].y));
    v[5] = mk(fma(-r2, a1.x, e[1].x), fma(-r2, a1.y, e[1].y));
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = mk(fma(r2, a3.x, e[3].x), fma(r2, a3.y, e[3].y));
    v[7] = mk(fma(-r2, a3.x, e[3].x), fma(-r2, a3.y, e[3].y));
  }
};

// ------------------------------------------------------------------ stages
// Layout of a batch of pencils in shared memory: element e of pencil p sits at
// s[p * pstride + e * estride].  `pfast` selects the thread decode: pencils
// fastest (strided pencils, pstride == 1) or elements fastest (contiguous).
struct Batch {
  int np;       // number of pencils
  int pstride;  // distance between pencils
  int estride;  // distance between elements of one pencil
  bool pfast;
};

__device__ __forceinline__ void decode(const Batch& b, int t, int per, int& p, int& q) {
  if (b.pfast) { p = t % b.np; q = t / b.np; }
  else { p = t / per; q = t - p * per; }
}

// One DIF stage of radix R on sub-blocks of length Ls (forward, twiddles after).
template <int R, typename C>
__device__ __forceinline__ void dif_stage(C* s, const Batch& b, int L, int Ls, const C* tw, int tid,
                                          int nth) {
  const int per = L / R;
  const int m = Ls / R;
  const int tws = L / Ls;
  const int total = b.np * per;
  for (int t = tid; t < total; t += nth) {
    int p, q;
    decode(b, t, per, p, q);
    int blk = q / m, n1 = q - blk * m;
    C* base = s + p * b.pstride + (blk * Ls + n1) * b.estride;
    C v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = base[j * m * b.estride];
    Dft<R, -1, C>::run(v);
    base[0] = v[0];
#pragma unroll
    for (int k = 1; k < R; ++k) base[k * m * b.estride] = cmul(v[k], tw[n1 * k * tws]);
  }
}

// One DIT stage of radix R (inverse, conjugate twiddles before the butterfly).
template <int R, typename C>
__device__ __forceinline__ void dit_stage(C* s, const Batch& b, int L, int Ls, const C* tw, int tid,
                                          int nth) {
  const int per = L / R;
  const int m = Ls / R;
  const int tws = L / Ls;
  const int total = b.np * per;
  for (int t = tid; t < total; t += nth) {
    int p, q;
    decode(b, t, per, p, q);
    int blk = q / m, n1 = q - blk * m;
    C* base = s + p * b.pstride + (blk * Ls + n1) * b.estride;
    C v[R];
    v[0] = base[0];
#pragma unroll
    for (int k = 1; k < R; ++k) v[k] = cmulc(base[k * m * b.estride], tw[n1 * k * tws]);
    Dft<R, 1, C>::run(v);
#pragma unroll
    for (int j = 0; j < R; ++j) base[j * m * b.estride] = v[j];
  }
}

// First forward stage when the plan starts with radix 2: only the first `nin`
// inputs can be nonzero.  Elements at or beyond nin are read as zero.
template <typename C>
__device__ __forceinline__ void dif_first2(C* s, const Batch& b, int L, int nin, const C* tw, int tid,
                                           int nth) {
  const int h = L / 2;
  const int total = b.np * h;
  for (int t = tid; t < total; t += nth) {
    int p, n1;
    decode(b, t, h, p, n1);
    C* base = s + p * b.pstride + n1 * b.estride;
    C x0 = (n1 < nin) ? base[0] : czero<C>();
    C x1 = (n1 + h < nin) ? base[h * b.estride] : czero<C>();
    C y0 = cadd(x0, x1);
    C y1 = cmul(csub(x0, x1), tw[n1]);
    base[0] = y0;
    base[h * b.estride] = y1;
  }
}

// Last inverse stage for a plan starting with radix 2; writes outputs < nout only.
template <typename C>
__device__ __forceinline__ void dit_last2(C* s, const Batch& b, int L, int nout, const C* tw, int tid,
                                          int nth) {
  const int h = L / 2;
  const int total = b.np * h;
  for (int t = tid; t < total; t += nth) {
    int p, n1;
    decode(b, t, h, p, n1);
    C* base = s + p * b.pstride + n1 * b.estride;
    C v0 = base[0];
    C v1 = cmulc(base[h * b.estride], tw[n1]);
    if (n1 < nout) base[0] = cadd(v0, v1);
    if (n1 + h < nout) base[h * b.estride] = csub(v0, v1);
  }
}

template <typename C>
__device__ __forceinline__ void run_dif(int R, C* s, const Batch& b, int L, int Ls, const C* tw, int tid,
                                        int nth) {
  switch (R) {
    case 2: dif_stage<2>(s, b, L, Ls, tw, tid, nth); break;
    case 3: dif_stage<3>(s, b, L, Ls, tw, tid, nth); break;
    case 4: dif_stage<4>(s, b, L, Ls, tw, tid, nth); break;
    case 5: dif_stage<5>(s, b, L, Ls, tw, tid, nth); break;
    default: dif_stage<8>(s, b, L, Ls, tw, tid, nth); break;
  }
}

template <typename C>
__device__ __forceinline__ void run_dit(int R, C* s, const Batch& b, int L, int Ls, const C* tw, int tid,
                                        int nth) {
  switch (R) {
    case 2: dit_stage<2>(s, b, L, Ls, tw, tid, nth); break;
    case 3: dit_stage<3>(s, b, L, Ls, tw, tid, nth); break;
    case 4: dit_stage<4>(s, b, L, Ls, tw, tid, nth); break;
    case 5: dit_stage<5>(s, b, L, Ls, tw, tid, nth); break;
    default: dit_stage<8>(s, b, L, Ls, tw, tid, nth); break;
  }
}

// Forward transform of a batch (all threads of the block call it).  Inputs at
// element index >= nin are treated as zero when the plan starts with radix 2;
// otherwise the caller must have zeroed them.  Ends with a barrier.
template <typename C>
__device__ void fft_forward(C* s, const Batch& b, const FftPlan& pl, int nin, const C* tw) {
  const int tid = threadIdx.x, nth = blockDim.x;
  int st = 0;
  if (pl.radix[0] == 2) {
    dif_first2(s, b, pl.L, nin, tw, tid, nth);
    st = 1;
    __syncthreads();
  }
  for (; st < pl.nst; ++st) {
    run_dif(pl.radix[st], s, b, pl.L, pl.len[st], tw, tid, nth);
    __syncthreads();
  }
}

// Inverse (unnormalized) transform of a batch from digit-reversed order back to
// natural order; outputs at index >= nout are not produced when the plan
// starts with radix 2.  Ends with a barrier.
template <typename C>
__device__ void fft_inverse(C* s, const Batch& b, const FftPlan& pl, int nout, const C* tw) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int stop = (pl.radix[0] == 2) ? 1 : 0;
  for (int st = pl.nst - 1; st >= stop; --st) {
    run_dit(pl.radix[st], s, b, pl.L, pl.len[st], tw, tid, nth);
    __syncthreads();
  }
  if (stop) {
    dit_last2(s, b, pl.L, nout, tw, tid, nth);
    __syncthreads();
  }
}

#endif  // __CUDACC__

}  // namespace dda
