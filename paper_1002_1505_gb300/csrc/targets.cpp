// Host-side lattice targets (guide, "Target Generation"): ELLIPSOID, RCTGLPRSM,
// CYLINDER1 and HEX_PRISM, plus explicit site lists (the FROM_FILE route).
//
// Sites sit at cell centres: along an axis with L candidate sites, site i has
// Target-Frame coordinate i + 1/2 - L/2 (centroid origin); RCTGLPRSM puts the
// origin at the centre of its upper x face (x from -SHPAR_1 to 0).  Every
// inclusion test runs in exact 64-bit integer arithmetic on doubled
// coordinates u = 2x, with surface ties counted as inside.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dda_internal.h"

namespace dda {

namespace {

Err positive_int(double v, const char* what, int64_t* out) {
  double r = std::nearbyint(v);
  if (!(std::fabs(v - r) < 1e-9) || r < 1 || r > 4096)
    return Err::make(DDA_EINVAL, std::string(what) + " must be an integer number of lattice spacings in 1..4096");
  *out = (int64_t)r;
  return Err::Ok();
}

// doubled coordinate of candidate i on an axis of L centred cells
inline int64_t centred(int64_t i, int64_t L) { return 2 * i + 1 - L; }

// Collect the occupied candidates of an L0 x L1 x L2 grid (doubled coords via
// ux/uy/uz) into a cropped target; inside(ux,uy,uz) decides membership.
template <typename F>
Err collect(int64_t L0, int64_t L1, int64_t L2, const std::vector<int64_t>& ux, const std::vector<int64_t>& uy,
            const std::vector<int64_t>& uz, F inside, const double a1[3], const double a2[3], HostTarget* out) {
  int64_t lo[3] = {L0, L1, L2}, hi[3] = {-1, -1, -1};
  std::vector<int32_t> tmp;
  for (int64_t k = 0; k < L2; ++k)
    for (int64_t j = 0; j < L1; ++j)
      for (int64_t i = 0; i < L0; ++i)
        if (inside(ux[i], uy[j], uz[k])) {
          tmp.push_back((int32_t)i);
          tmp.push_back((int32_t)j);
          tmp.push_back((int32_t)k);
          lo[0] = std::min(lo[0], i); hi[0] = std::max(hi[0], i);
          lo[1] = std::min(lo[1], j); hi[1] = std::max(hi[1], j);
          lo[2] = std::min(lo[2], k); hi[2] = std::max(hi[2], k);
        }
  if (tmp.empty()) return Err::make(DDA_EINVAL, "target has no occupied sites");
  out->ijk.resize(tmp.size());
  for (size_t s = 0; s < tmp.size(); s += 3) {
    out->ijk[s] = tmp[s] - (int32_t)lo[0];
    out->ijk[s + 1] = tmp[s + 1] - (int32_t)lo[1];
    out->ijk[s + 2] = tmp[s + 2] - (int32_t)lo[2];
  }
  for (int a = 0; a < 3; ++a) out->box[a] = (int)(hi[a] - lo[a] + 1);
  out->origin[0] = 0.5 * (double)ux[lo[0]];
  out->origin[1] = 0.5 * (double)uy[lo[1]];
  out->origin[2] = 0.5 * (double)uz[lo[2]];
  std::memcpy(out->a1, a1, sizeof(double) * 3);
  std::memcpy(out->a2, a2, sizeof(double) * 3);
  out->comp.assign(tmp.size(), 0);  // N x 3
  out->ncomp = 1;
  return Err::Ok();
}

std::vector<int64_t> centred_axis(int64_t L) {
  std::vector<int64_t> u(L);
  for (int64_t i = 0; i < L; ++i) u[i] = centred(i, L);
  return u;
}

}  // namespace

Err make_shape_target(int shape, const double* shpar, int nshpar, HostTarget* out) {
  if (!shpar || nshpar < 3) return Err::make(DDA_EINVAL, "shape needs 3 SHPAR values");
  static const double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0}, ez[3] = {0, 0, 1};
  if (shape == DDA_ELLIPSOID) {
    int64_t s1, s2, s3;
    DDA_TRY(positive_int(shpar[0], "SHPAR_1", &s1));
    DDA_TRY(positive_int(shpar[1], "SHPAR_2", &s2));
    DDA_TRY(positive_int(shpar[2], "SHPAR_3", &s3));
    // (x/S1)^2 + (y/S2)^2 + (z/S3)^2 <= 1/4 with u = 2x, times (S1 S2 S3)^2
    const int64_t w1 = (s2 * s3) * (s2 * s3), w2 = (s1 * s3) * (s1 * s3), w3 = (s1 * s2) * (s1 * s2);
    const int64_t rhs = (s1 * s2 * s3) * (s1 * s2 * s3);
    auto in = [&](int64_t u, int64_t v, int64_t w) { return u * u * w1 + v * v * w2 + w * w * w3 <= rhs; };
    return collect(s1, s2, s3, centred_axis(s1), centred_axis(s2), centred_axis(s3), in, ex, ey, out);
  }
  if (shape == DDA_RCTGLPRSM) {
    int64_t s1, s2, s3;
    DDA_TRY(positive_int(shpar[0], "SHPAR_1", &s1));
    DDA_TRY(positive_int(shpar[1], "SHPAR_2", &s2));
    DDA_TRY(positive_int(shpar[2], "SHPAR_3", &s3));
    std::vector<int64_t> ux(s1);
    for (int64_t i = 0; i < s1; ++i) ux[i] = 2 * i + 1 - 2 * s1;  // x in [-S1, 0]
    auto in = [](int64_t, int64_t, int64_t) { return true; };
    return collect(s1, s2, s3, ux, centred_axis(s2), centred_axis(s3), in, ex, ey, out);
  }
  if (shape == DDA_CYLINDER1) {
    int64_t len, dia;
    DDA_TRY(positive_int(shpar[0], "SHPAR_1", &len));
    DDA_TRY(positive_int(shpar[1], "SHPAR_2", &dia));
    int ax = (int)std::nearbyint(shpar[2]);
    if (ax < 1 || ax > 3) return Err::make(DDA_EINVAL, "CYLINDER1 SHPAR_3 must be 1, 2 or 3");
    --ax;
    int64_t L[3] = {dia, dia, dia};
    L[ax] = len;
    const double* a1 = ax == 0 ? ex : (ax == 1 ? ey : ez);
    const double* a2 = ax == 0 ? ey : (ax == 1 ? ez : ex);
    auto in = [&](int64_t u, int64_t v, int64_t w) {
      int64_t c[3] = {u, v, w};
      int64_t s = 0;
      for (int a = 0; a < 3; ++a)
        if (a != ax) s += c[a] * c[a];
      return s <= dia * dia;  // radial^2 <= (S2/2)^2 in doubled coordinates
    };
    return collect(L[0], L[1], L[2], centred_axis(L[0]), centred_axis(L[1]), centred_axis(L[2]), in, a1, a2, out);
  }
  if (shape == DDA_HEX_PRISM) {
    int64_t len, vv;
    DDA_TRY(positive_int(shpar[0], "SHPAR_1", &len));
    DDA_TRY(positive_int(shpar[1], "SHPAR_2", &vv));
    int sel = (int)std::nearbyint(shpar[2]);
    static const int axes[6][2] = {{0, 1}, {0, 2}, {1, 0}, {1, 2}, {2, 0}, {2, 1}};
    if (sel < 1 || sel > 6) return Err::make(DDA_EINVAL, "HEX_PRISM SHPAR_3 must be 1..6");
    const int ax1 = axes[sel - 1][0], ax2 = axes[sel - 1][1], ax3 = 3 - ax1 - ax2;
    int64_t L[3] = {vv, vv, vv};
    L[ax1] = len;
    double a1[3] = {0, 0, 0}, a2[3] = {0, 0, 0};
    a1[ax1] = 1;
    a2[ax2] = 1;
    const int64_t v2 = vv * vv;
    // p along the face normal a2, q along a3 (vertex direction), doubled:
    // 4p^2 <= 3 S2^2, and 2 sqrt3 |p q| <= a = 3 S2^2 - p^2 - 3 q^2  <=>  a >= 0 && 12 p^2 q^2 <= a^2
    auto in = [&](int64_t u, int64_t v, int64_t w) {
      int64_t c[3] = {u, v, w};
      const int64_t p = c[ax2], q = c[ax3];
      if (4 * p * p > 3 * v2) return false;
      const int64_t a = 3 * v2 - p * p - 3 * q * q;
      if (a < 0) return false;
      const int64_t pq = p * q;
      return 12 * pq * pq <= a * a;
    };
    return collect(L[0], L[1], L[2], centred_axis(L[0]), centred_axis(L[1]), centred_axis(L[2]), in, a1, a2, out);
  }
  return Err::make(DDA_EINVAL, "unknown shape id");
}

void df_axes(double th, double ph, double be, double R[9]) {
  const double ct = std::cos(th), st = std::sin(th), cp = std::cos(ph), sp = std::sin(ph), cb = std::cos(be),
               sb = std::sin(be);
  const double e1[3] = {ct, st * cp, st * sp};
  const double e2[3] = {-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp};
  const double e3[3] = {st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)};
  for (int a = 0; a < 3; ++a) {
    R[3 * a + 0] = e1[a];
    R[3 * a + 1] = e2[a];
    R[3 * a + 2] = e3[a];
  }
}

Err make_site_target(const int32_t* ixyz, const int32_t* icomp, int64_t n, const double origin[3],
                     const double a1[3], const double a2[3], HostTarget* out, bool per_axis,
                     const double* df_angles) {
  if (!ixyz || n <= 0) return Err::make(DDA_EINVAL, "site list is empty");
  if (n > (int64_t)1 << 30) return Err::make(DDA_EINVAL, "too many sites");
  int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
  for (int64_t j = 0; j < n; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], ixyz[3 * j + a]);
      hi[a] = std::max(hi[a], ixyz[3 * j + a]);
    }
  for (int a = 0; a < 3; ++a)
    if ((int64_t)hi[a] - lo[a] + 1 > 4096) return Err::make(DDA_EINVAL, "site list spans more than 4096 cells");
  // x-fastest order by the box key; a list already in that order (as dda_get_sites returns it)
  // is taken as is (strictly increasing keys: sorted and free of duplicates)
  auto key = [&](int64_t j) {
    return (((int64_t)(ixyz[3 * j + 2] - lo[2]) * 4096 + (ixyz[3 * j + 1] - lo[1])) * 4096) + (ixyz[3 * j] - lo[0]);
  };
  bool sorted = true;
  for (int64_t j = 1, prev = key(0); j < n && sorted; ++j) {
    const int64_t k = key(j);
    sorted = k > prev;
    prev = k;
  }
  std::vector<int64_t> order;
  if (!sorted) {
    std::vector<int64_t> keys(n);
    for (int64_t j = 0; j < n; ++j) keys[j] = key(j);
    order.resize(n);
    for (int64_t j = 0; j < n; ++j) order[j] = j;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return keys[a] < keys[b]; });
    for (int64_t j = 1; j < n; ++j)
      if (keys[order[j]] == keys[order[j - 1]]) return Err::make(DDA_EINVAL, "duplicate site in list");
  }
  out->ijk.resize(3 * n);
  out->comp.resize(3 * n);
  out->dfrot.clear();
  if (df_angles) {
    out->dfrot.resize(9 * n);
    for (int64_t s = 0; s < n; ++s) {
      const int64_t j = sorted ? s : order[s];
      const double* an = df_angles + 3 * j;
      if (!std::isfinite(an[0]) || !std::isfinite(an[1]) || !std::isfinite(an[2]))
        return Err::make(DDA_EINVAL, "dielectric-frame angles must be finite");
      df_axes(an[0], an[1], an[2], &out->dfrot[9 * s]);
    }
  }
  int maxc = 1;
  if (sorted && !icomp) {  // the common case: one material, list in order
    for (int64_t s = 0; s < n; ++s)
      for (int a = 0; a < 3; ++a) out->ijk[3 * s + a] = ixyz[3 * s + a] - lo[a];
    std::fill(out->comp.begin(), out->comp.end(), (uint8_t)0);
  } else {
    for (int64_t s = 0; s < n; ++s) {
      const int64_t j = sorted ? s : order[s];
      for (int a = 0; a < 3; ++a) out->ijk[3 * s + a] = ixyz[3 * j + a] - lo[a];
      for (int a = 0; a < 3; ++a) {
        const int c = icomp ? icomp[per_axis ? 3 * j + a : j] : 1;
        if (c < 1 || c > 255) return Err::make(DDA_EINVAL, "composition index must be in 1..255");
        out->comp[3 * s + a] = (uint8_t)(c - 1);
        maxc = std::max(maxc, c);
      }
    }
  }
  for (int a = 0; a < 3; ++a) {
    out->box[a] = hi[a] - lo[a] + 1;
    out->origin[a] = (origin ? origin[a] : 0.0) + lo[a];
  }
  static const double ex[3] = {1, 0, 0}, ey[3] = {0, 1, 0};
  std::memcpy(out->a1, a1 ? a1 : ex, sizeof(double) * 3);
  std::memcpy(out->a2, a2 ? a2 : ey, sizeof(double) * 3);
  out->ncomp = maxc;
  return Err::Ok();
}

// ------------------------------------------------------------------ FFT plans
bool is_smooth235(int v) {
  if (v < 1) return false;
  for (int f : {2, 3, 5})
    while (v % f == 0) v /= f;
  return v == 1;
}

// Stage list: a leading radix 2 (pruned stage for zero-padded data), then the
// remaining power of two as radix-8 stages with one radix-4 or radix-2 stage
// for the remainder (a radix 8 right after the leading radix 2 keeps the
// register sub-blocks of the second pass short), then radix 3 and 5 stages.
Err make_plan(int L, FftPlan* out) {
  if (L < 2 || (L % 2) != 0 || !is_smooth235(L))
    return Err::make(DDA_EINVAL, "FFT length must be even and a product of 2, 3 and 5");
  FftPlan p{};
  p.L = L;
  int k = 0;
  int rest = L / 2;
  p.radix[k++] = 2;
  int a = 0;
  while (rest % 2 == 0) { rest /= 2; ++a; }
  std::vector<int> r2;
  while (a >= 3) { r2.push_back(8); a -= 3; }
  if (a == 2) r2.push_back(4);
  else if (a == 1) r2.push_back(2);
  for (int r : r2) p.radix[k++] = r;
  while (rest % 3 == 0) { rest /= 3; p.radix[k++] = 3; }
  while (rest % 5 == 0) { rest /= 5; p.radix[k++] = 5; }
  if (k > kMaxStages) return Err::make(DDA_EINVAL, "FFT length needs too many stages");
  p.nst = k;
  int len = L;
  for (int s = 0; s < k; ++s) {
    p.len[s] = len;
    len /= p.radix[s];
  }
  *out = p;
  return Err::Ok();
}

}  // namespace dda
