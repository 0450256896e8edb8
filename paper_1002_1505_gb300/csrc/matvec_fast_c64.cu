// complex64 instantiations of the compile-time-length product kernels.
#include "matvec_fast.cuh"

namespace dda {
template <>
Err launch_matvec_fast<float2>(const Geom& g, const MvData<float2>& d, const MvTune& t, const float2* p, float2* ap,
                               int nrhs, int rhs0, bool conj, cudaStream_t st) {
  return fast::launch_matvec_fast<float2>(g, d, t, p, ap, nrhs, rhs0, conj, st);
}
void fast_optin_c64(int smax) { fast::optin_all<float2>(smax); }
Err launch_middle_c64(const Geom& g, const MvData<float2>& d, const MvTune& t, int nrhs, cudaStream_t st) {
  int pass = 0;
  return fast::launch_middle<float2>(g, d, t, nrhs, st, pass);
}

namespace {
// one CTA: a barrier expecting one arrival and 16 bytes that nobody sends
__global__ void k_selftest_bulk_wait(unsigned int* flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) bulk::mbar_init(&bar, 1);
  __syncthreads();
  bulk::mbar_wait(&bar, 0, 4096, flag);
}
}  // namespace

Err selftest_bulk_wait(int* gave_up) {
  unsigned int* d = nullptr;
  DDA_CU(cudaMalloc(&d, sizeof(unsigned int)));
  cudaError_t ce = cudaMemset(d, 0, sizeof(unsigned int));
  if (ce == cudaSuccess) {
    k_selftest_bulk_wait<<<1, 32>>>(d);
    ce = cudaGetLastError();
  }
  unsigned int h = 0;
  if (ce == cudaSuccess) ce = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (ce != cudaSuccess) return Err::make(DDA_ECUDA, cudaGetErrorString(ce));
  *gave_up = h ? 1 : 0;
  return Err::Ok();
}

int x_tile_height_default(size_t csize, int px) { return fast::x_ty_rt(csize, px); }
bool x_tile_height_ok(size_t csize, int px, int ty) { return fast::x_ty_valid(csize, px, ty); }
int x_tile_height_one_component(size_t csize) { return fast::x_nc1_ty_rt(csize); }

void choose_fast_schedule(const Geom& g, bool c64, int smax, MvTune* t) {
  t->fast = fast::fast_length(g.px) && fast::fast_length(g.py) && fast::fast_length(g.pz);
  if (!t->fast) return;
  const size_t cs = c64 ? sizeof(float2) : sizeof(double2);
  const size_t xs = c64 ? fast::x_fast_smem<float2>(g) : fast::x_fast_smem<double2>(g);
  const size_t ys = c64 ? fast::yrows_fast_smem<float2>(g) : fast::yrows_fast_smem<double2>(g);
  const size_t zs = c64 ? fast::zcols_fast_smem<float2>(g) : fast::zcols_fast_smem<double2>(g);
  if (xs > (size_t)smax || ys > (size_t)smax || zs > (size_t)smax) {
    t->fast = false;
    return;
  }
  (void)cs;
  t->plane = c64 && fast::fast_plane_pair(g.py, g.pz) && fast::plane_fast_smem<float2>(g) <= (size_t)smax;
  t->plane_ok = t->plane;
}
}  // namespace dda
