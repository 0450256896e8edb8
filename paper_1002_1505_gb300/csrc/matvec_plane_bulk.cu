// The complex64 plane pass with its HBM input and output blocks staged by bulk
// copies (TMA; see k_yz_plane), compiled apart from the other plane variants.
#include "matvec_fast.cuh"

namespace dda {

bool plane_bulk_ok_c64(const Geom& g, int smax) {
  return fast::fast_plane_pair(g.py, g.pz) && (g.nz * g.ny) % 2 == 0 &&
         fast::plane_bulk_smem<float2>(g) <= (size_t)smax;
}

Err launch_plane_bulk_c64(const Geom& g, const MvData<float2>& d, int nrhs, cudaStream_t st) {
  const size_t sm = fast::plane_bulk_smem<float2>(g);
  const dim3 grid(nrhs, g.px);
#define DDA_CASE(A, B)                                                                  \
  if (g.py == A && g.pz == B) {                                                         \
    DDA_CU(launch_k(fast::k_yz_plane<float2, A, B, 512, true>, grid, dim3(512), sm, st, g, d)); \
    DDA_CU(cudaGetLastError());                                                         \
    return Err::Ok();                                                                   \
  }
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
  return Err::make(DDA_EUNSUPPORTED, "no bulk-staged plane kernel for this pair");
}

void plane_bulk_optin_c64(int smax) {
#define DDA_CASE(A, B) optin_smem(fast::k_yz_plane<float2, A, B, 512, true>, smax);
  DDA_FAST_PLANES(DDA_CASE)
#undef DDA_CASE
}

}  // namespace dda
