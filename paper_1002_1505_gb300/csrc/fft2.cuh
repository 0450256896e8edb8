// Two-pass register FFTs for the zero-padded lengths of the DDA convolution.
//
// A length L = 2 * RA * LB transform (the same stage list as make_plan: a
// radix-2 stage, then the plan's radices) is split into two passes, each done
// in registers by one thread:
//   pass A  stage 0 (radix 2) fused with stage 1 (radix RA).  Thread n1 in
//           [0, LB) reads the RA inputs at n1 + LB*j and writes 2*RA outputs
//           at b*L/2 + n1 + LB*k (b = 0, 1).  Forward, the upper half of the
//           input is zero (zero padding), so stage 0 is y0 = x, y1 = x w^n.
//   pass B  the remaining stages on one contiguous sub-block of LB elements.
// Forward passes are decimation in frequency and leave the spectrum in the
// same digit-reversed order as the generic engine (fft.cuh); inverse passes
// undo them exactly (decimation in time, conjugate twiddles, unnormalized),
// and inverse pass A produces only the lower half of the output (pruning)
// unless asked for both.  One shared-memory exchange separates the passes.
// Pass A's twiddles (which depend on the thread) come from a table
// tw[i] = exp(-2 pi i i/L), i < L; pass B's are compile-time constants.
#pragma once

#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace dda {
namespace f2 {

struct CPlan {
  int nst;
  int r[kMaxStages];
};

// Compile-time copy of make_plan's stage list (targets.cpp): 2, then radix-8
// stages for the remaining power of two with one radix 4 or 2 for the
// remainder, then 3s and 5s.
constexpr CPlan cplan(int L) {
  CPlan p{};
  int k = 0;
  int rest = L / 2;
  p.r[k++] = 2;
  int a = 0;
  while (rest % 2 == 0) { rest /= 2; ++a; }
  int r2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int n2 = 0;
  while (a >= 3) { r2[n2++] = 8; a -= 3; }
  if (a == 2) r2[n2++] = 4;
  else if (a == 1) r2[n2++] = 2;
  for (int i = 0; i < n2; ++i) p.r[k++] = r2[i];
  while (rest % 3 == 0) { rest /= 3; p.r[k++] = 3; }
  while (rest % 5 == 0) { rest /= 5; p.r[k++] = 5; }
  p.nst = k;
  return p;
}

template <int L>
struct Shape {
  static constexpr CPlan P = cplan(L);
  static constexpr int RA = P.nst > 1 ? P.r[1] : 1;  // radix fused with the radix-2 stage
  static constexpr int LB = L / (2 * RA);             // sub-block length handled by pass B
  static constexpr int H = L / 2;
  static_assert(L % 2 == 0, "even lengths only");
};

// a + b * conj(w) as four FMAs (the last DIT stage when only one output half is kept)
template <typename C>
__device__ __forceinline__ C addmulc(C a, C b, C w) {
  C r;
  r.x = fma(b.x, w.x, fma(b.y, w.y, a.x));
  r.y = fma(b.y, w.x, fma(-b.x, w.y, a.y));
  return r;
}

// ------------------------------------------------------------------ pass A
// x[j] = input at n1 + LB*j (upper half of the input is zero); out[b*RA+k] goes to b*H + n1 + LB*k.
template <int L, typename C>
__device__ __forceinline__ void passA_fwd(C* x, int n1, const C* tw, C* out) {
  constexpr int RA = Shape<L>::RA, LB = Shape<L>::LB;
  if constexpr (RA == 1) {
    out[0] = x[0];
    out[1] = cmul(x[0], tw[n1]);
  } else {
    C y[RA];
#pragma unroll
    for (int j = 0; j < RA; ++j) y[j] = cmul(x[j], tw[n1 + LB * j]);
    Dft<RA, -1, C>::run(x);
    Dft<RA, -1, C>::run(y);
    out[0] = x[0];
    out[RA] = y[0];
#pragma unroll
    for (int k = 1; k < RA; ++k) {
      const C w = tw[2 * n1 * k];
      out[k] = cmul(x[k], w);
      out[RA + k] = cmul(y[k], w);
    }
  }
}

// in[b*RA+k] from b*H + n1 + LB*k; lo[j] = output at n1 + LB*j, hi[j] at H + n1 + LB*j (if HI).
template <int L, bool HI, typename C>
__device__ __forceinline__ void passA_inv(C* in, int n1, const C* tw, C* lo, C* hi) {
  constexpr int RA = Shape<L>::RA, LB = Shape<L>::LB;
  if constexpr (RA == 1) {
    if constexpr (HI) {
      const C t = cmulc(in[1], tw[n1]);
      lo[0] = cadd(in[0], t);
      hi[0] = csub(in[0], t);
    } else {
      lo[0] = addmulc(in[0], in[1], tw[n1]);
    }
  } else {
    C u0[RA], u1[RA];
    u0[0] = in[0];
    u1[0] = in[RA];
#pragma unroll
    for (int k = 1; k < RA; ++k) {
      const C w = tw[2 * n1 * k];
      u0[k] = cmulc(in[k], w);
      u1[k] = cmulc(in[RA + k], w);
    }
    Dft<RA, 1, C>::run(u0);
    Dft<RA, 1, C>::run(u1);
#pragma unroll
    for (int j = 0; j < RA; ++j) {
      if constexpr (HI) {
        const C t = cmulc(u1[j], tw[n1 + LB * j]);
        lo[j] = cadd(u0[j], t);
        hi[j] = csub(u0[j], t);
      } else {
        lo[j] = addmulc(u0[j], u1[j], tw[n1 + LB * j]);  // pruned: the upper half is never needed
      }
    }
  }
}

// ------------------------------------------------------------------ compile-time twiddles
// Pass B's twiddle indices are all compile-time constants, so its twiddles are
// folded into the instructions: exp(2 pi i m / L) is evaluated at compile time
// (octant reduction on the integer m, then Taylor series of sin and cos on
// [0, pi/4]), and the trivial factors 1, -1, +-i cost no multiply at all.
namespace ct {
constexpr double kQuarterPi = 0.78539816339744830962;
constexpr double sin_t(double t) {  // t in [0, pi/4]
  double term = t, s = t;
  for (int n = 1; n < 12; ++n) {
    term *= -t * t / ((2.0 * n) * (2.0 * n + 1.0));
    s += term;
  }
  return s;
}
constexpr double cos_t(double t) {
  double term = 1.0, s = 1.0;
  for (int n = 1; n < 12; ++n) {
    term *= -t * t / ((2.0 * n - 1.0) * (2.0 * n));
    s += term;
  }
  return s;
}
// cos and sin of 2 pi m / L: the angle is (pi/4) (o + r/L) with o = floor(8m/L)
constexpr double cs2pi(int m, int L, bool want_sin) {
  m %= L;
  if (m < 0) m += L;
  const long q = 8L * m;
  const int o = (int)(q / L);
  const long r = q - (long)o * L;
  const double a = kQuarterPi * (double)r / (double)L;        // (pi/4) r/L
  const double b = kQuarterPi * (double)(L - r) / (double)L;  // pi/4 - a
  double c = 0, s = 0;
  switch (o) {
    case 0: c = cos_t(a); s = sin_t(a); break;
    case 1: c = sin_t(b); s = cos_t(b); break;
    case 2: c = -sin_t(a); s = cos_t(a); break;
    case 3: c = -cos_t(b); s = sin_t(b); break;
    case 4: c = -cos_t(a); s = -sin_t(a); break;
    case 5: c = -sin_t(b); s = -cos_t(b); break;
    case 6: c = sin_t(a); s = -cos_t(a); break;
    default: c = cos_t(b); s = -sin_t(b); break;
  }
  return want_sin ? s : c;
}
}  // namespace ct

// a * exp(S 2 pi i M / L) with M, S compile-time (S = -1: forward twiddle, +1: its conjugate)
template <int L, int M, int S, typename C>
__device__ __forceinline__ C twc(C a) {
  constexpr int m = ((M % L) + L) % L;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == L) {
    return mk(-a.x, -a.y);
  } else if constexpr (4 * m == L) {
    return cmuli(a, S);
  } else if constexpr (4 * m == 3 * L) {
    return cmuli(a, -S);
  } else {
    using R = decltype(a.x);
    constexpr R c = (R)ct::cs2pi(m, L, false);
    constexpr R s = (R)(S * ct::cs2pi(m, L, true));
    return mk(fma(a.x, c, -a.y * s), fma(a.x, s, a.y * c));
  }
}

// compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1
template <typename F, int... Is>
__device__ __forceinline__ void sfor_(F& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_(f, std::make_integer_sequence<int, N>{});
}

template <int L, int S>
constexpr int stage_len() {  // sub-transform length entering stage S
  int ls = L;
  for (int s = 0; s < S; ++s) ls /= Shape<L>::P.r[s];
  return ls;
}

// ------------------------------------------------------------------ pass B
// DIF stage S of the plan applied to one sub-block v[LB] (all indices compile-time).
template <int L, int S, typename C>
__device__ __forceinline__ void passB_fwd_stage(C* v) {
  constexpr CPlan P = Shape<L>::P;
  if constexpr (S < P.nst) {
    constexpr int LB = Shape<L>::LB;
    constexpr int R = P.r[S];
    constexpr int Ls = stage_len<L, S>();
    constexpr int m = Ls / R;
    constexpr int tws = L / Ls;
    sfor<LB / Ls>([&](auto sbc) {
      constexpr int base = decltype(sbc)::value * Ls;
      sfor<m>([&](auto n1c) {
        constexpr int n1 = decltype(n1c)::value;
        C t[R];
#pragma unroll
        for (int j = 0; j < R; ++j) t[j] = v[base + n1 + m * j];
        Dft<R, -1, C>::run(t);
        v[base + n1] = t[0];
        sfor<R - 1>([&](auto kc) {
          constexpr int k = decltype(kc)::value + 1;
          v[base + n1 + m * k] = twc<L, n1 * k * tws, -1>(t[k]);
        });
      });
    });
    passB_fwd_stage<L, S + 1>(v);
  }
}

template <int L, int S, typename C>
__device__ __forceinline__ void passB_inv_stage(C* v) {
  constexpr CPlan P = Shape<L>::P;
  if constexpr (S < P.nst) {
    passB_inv_stage<L, S + 1>(v);  // inverse runs the stages backwards
    constexpr int LB = Shape<L>::LB;
    constexpr int R = P.r[S];
    constexpr int Ls = stage_len<L, S>();
    constexpr int m = Ls / R;
    constexpr int tws = L / Ls;
    sfor<LB / Ls>([&](auto sbc) {
      constexpr int base = decltype(sbc)::value * Ls;
      sfor<m>([&](auto n1c) {
        constexpr int n1 = decltype(n1c)::value;
        C t[R];
        t[0] = v[base + n1];
        sfor<R - 1>([&](auto kc) {
          constexpr int k = decltype(kc)::value + 1;
          t[k] = twc<L, n1 * k * tws, 1>(v[base + n1 + m * k]);
        });
        Dft<R, 1, C>::run(t);
#pragma unroll
        for (int j = 0; j < R; ++j) v[base + n1 + m * j] = t[j];
      });
    });
  }
}

template <int L, typename C>
__device__ __forceinline__ void passB_fwd(C* v, const C* /*tw: unused, twiddles are compile-time*/) {
  passB_fwd_stage<L, 2>(v);
}
template <int L, typename C>
__device__ __forceinline__ void passB_inv(C* v, const C* /*tw*/) {
  passB_inv_stage<L, 2>(v);
}

}  // namespace f2
}  // namespace dda
