// BiCGstab half-iterations of the complex64 inner solve with the vector updates
// and dot products folded into the x passes of the compile-time product
// (matvec_fast.cuh, kFuseP / kFuseS / kFuseRV / kFuseTS): 3 + 3 launches per
// iteration plus the x/r update, instead of 3 + 3 product launches and four
// separate vector kernels.
#include "matvec_fast.cuh"

namespace dda {
// half 0: p = r + beta (p - omega v), v = A p, <rhat, v> -> alpha
// half 1: s = r - alpha v (|s|^2 half-step test), t = A s, <t, s>, |t|^2 -> omega
Err launch_bicg_half_c64(const Geom& g, const MvData<float2>& d, const MvTune& t, const KrylovVecs<float2>& kv,
                         KState* ks, const RedBuf& rbx, int nrhs, int half, cudaStream_t st) {
  using namespace fast;
  if (!t.fast) return Err::make(DDA_EUNSUPPORTED, "folded BiCGstab updates need the compile-time kernels");
  if (half == 0) DDA_TRY((launch_x_fused<kFuseP, true>(g, d, t, kv, ks, rbx, nrhs, st)));
  else DDA_TRY((launch_x_fused<kFuseS, true>(g, d, t, kv, ks, rbx, nrhs, st)));
  DDA_TRY(launch_middle_c64(g, d, t, nrhs, st));  // compiled with the complex64 product kernels
  if (half == 0) DDA_TRY((launch_x_fused<kFuseRV, false>(g, d, t, kv, ks, rbx, nrhs, st)));
  else DDA_TRY((launch_x_fused<kFuseTS, false>(g, d, t, kv, ks, rbx, nrhs, st)));
  return Err::Ok();  // launch_middle_c64 counted the 3 (or 5) launches of the product
}
int x_ctas_per_rhs_c64(const Geom& g, const MvTune& t) { return fast::x_ctas_per_rhs(g, t); }
bool zcols_rfuse_available_c64(const Geom& g) { return fast::zcols_rfuse_exists<float2>(g.pz); }
void fused_optin_c64(int smax) {
#define DDA_CASE(L_) fast::optin_x_fused<L_>(smax);
  DDA_FAST_LENGTHS(DDA_CASE)
#undef DDA_CASE
}
}  // namespace dda
