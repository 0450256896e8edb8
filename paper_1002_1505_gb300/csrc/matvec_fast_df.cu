// Double-float instantiations of the compile-time-length product kernels: the
// complex128 product computed in pairs of FP32 numbers (df.cuh), which runs on
// GB300's FP32 units instead of its FP64 units (1/64 of the FP32 rate).  Input
// and output vectors stay complex128; the Green tensor, the twiddle tables and
// alpha^{-1} are double-float copies of their FP64 values.
#include "matvec_fast.cuh"

namespace dda {
Err launch_matvec_df(const Geom& g, const MvData<dfp::dfc>& d, const MvTune& t, const double2* p, double2* ap,
                     int nrhs, int rhs0, bool conj, cudaStream_t st) {
  if (!t.fast || t.plane) return Err::make(DDA_EUNSUPPORTED, "the double-float product needs the compile-time 5-pass schedule");
  return fast::launch_matvec_fast<dfp::dfc>(g, d, t, p, ap, nrhs, rhs0, conj, st);
}
void fast_optin_df(int smax) { fast::optin_all<dfp::dfc>(smax); }
}  // namespace dda
