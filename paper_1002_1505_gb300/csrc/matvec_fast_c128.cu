// complex128 instantiations of the compile-time-length product kernels.
#include "matvec_fast.cuh"

namespace dda {
template <>
Err launch_matvec_fast<double2>(const Geom& g, const MvData<double2>& d, const MvTune& t, const double2* p,
                                double2* ap, int nrhs, int rhs0, bool conj, cudaStream_t st) {
  return fast::launch_matvec_fast<double2>(g, d, t, p, ap, nrhs, rhs0, conj, st);
}
void fast_optin_c128(int smax) { fast::optin_all<double2>(smax); }
}  // namespace dda
