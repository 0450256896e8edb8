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
// Twiddles come from a table tw[i] = exp(-2 pi i i/L), i < L.
#pragma once

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
    const C t = cmulc(in[1], tw[n1]);
    lo[0] = cadd(in[0], t);
    if constexpr (HI) hi[0] = csub(in[0], t);
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
      const C t = cmulc(u1[j], tw[n1 + LB * j]);
      lo[j] = cadd(u0[j], t);
      if constexpr (HI) hi[j] = csub(u0[j], t);
    }
  }
}

// ------------------------------------------------------------------ pass B
// DIF stage S of the plan applied to one sub-block v[LB] (all indices compile-time).
template <int L, int S, typename C>
__device__ __forceinline__ void passB_fwd_stage(C* v, const C* tw) {
  constexpr CPlan P = Shape<L>::P;
  if constexpr (S < P.nst) {
    constexpr int LB = Shape<L>::LB;
    constexpr int R = P.r[S];
    // sub-transform length entering stage S
    constexpr int Ls = [] {
      int ls = L;
      for (int s = 0; s < S; ++s) ls /= Shape<L>::P.r[s];
      return ls;
    }();
    constexpr int m = Ls / R;
    constexpr int tws = L / Ls;
#pragma unroll
    for (int sb = 0; sb < LB / Ls; ++sb) {
#pragma unroll
      for (int n1 = 0; n1 < m; ++n1) {
        C t[R];
#pragma unroll
        for (int j = 0; j < R; ++j) t[j] = v[sb * Ls + n1 + m * j];
        Dft<R, -1, C>::run(t);
        v[sb * Ls + n1] = t[0];
#pragma unroll
        for (int k = 1; k < R; ++k) v[sb * Ls + n1 + m * k] = cmul(t[k], tw[n1 * k * tws]);
      }
    }
    passB_fwd_stage<L, S + 1>(v, tw);
  }
}

template <int L, int S, typename C>
__device__ __forceinline__ void passB_inv_stage(C* v, const C* tw) {
  constexpr CPlan P = Shape<L>::P;
  if constexpr (S < P.nst) {
    passB_inv_stage<L, S + 1>(v, tw);  // inverse runs the stages backwards
    constexpr int LB = Shape<L>::LB;
    constexpr int R = P.r[S];
    constexpr int Ls = [] {
      int ls = L;
      for (int s = 0; s < S; ++s) ls /= Shape<L>::P.r[s];
      return ls;
    }();
    constexpr int m = Ls / R;
    constexpr int tws = L / Ls;
#pragma unroll
    for (int sb = 0; sb < LB / Ls; ++sb) {
#pragma unroll
      for (int n1 = 0; n1 < m; ++n1) {
        C t[R];
        t[0] = v[sb * Ls + n1];
#pragma unroll
        for (int k = 1; k < R; ++k) t[k] = cmulc(v[sb * Ls + n1 + m * k], tw[n1 * k * tws]);
        Dft<R, 1, C>::run(t);
#pragma unroll
        for (int j = 0; j < R; ++j) v[sb * Ls + n1 + m * j] = t[j];
      }
    }
  }
}

template <int L, typename C>
__device__ __forceinline__ void passB_fwd(C* v, const C* tw) {
  passB_fwd_stage<L, 2>(v, tw);
}
template <int L, typename C>
__device__ __forceinline__ void passB_inv(C* v, const C* tw) {
  passB_inv_stage<L, 2>(v, tw);
}

}  // namespace f2
}  // namespace dda
