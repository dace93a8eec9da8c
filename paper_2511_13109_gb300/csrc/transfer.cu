// Interpolation between Kuhn grids and its transpose (Sec. 2.1): one thread
// per coarse (restriction) or fine (prolongation) vertex; the per-point
// formulas are restrict_point / prolong_point in device_ops.cuh.
#include <stdlib.h>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

template <typename T>
__global__ void restrict_kernel(int nf, int ncomp, bool mask, T scale, const T* __restrict__ rf, T* __restrict__ rc) {
  grid_dep_entry();
  const int nvf = nf + 1, nvc = nf / 2 + 1;
  const int Vc = nvc * nvc * nvc, Vf = nvf * nvf * nvf;  // 32-bit: grids are limited on the host
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Vc) return;
  const int t = id / nvc, I = id - t * nvc, K = t / nvc, J = t - K * nvc;
  for (int c = 0; c < ncomp; ++c) rc[c * Vc + id] = restrict_point<T>(nf, mask, scale, rf + c * Vf, I, J, K);
}

template <typename T, bool ADD>
__global__ void prolong_kernel(int nf, int ncomp, bool mask, const T* __restrict__ ec, T* __restrict__ xf) {
  grid_dep_entry();
  const int nvf = nf + 1, nvc = nf / 2 + 1;
  const int Vc = nvc * nvc * nvc, Vf = nvf * nvf * nvf;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Vf) return;
  const int t = id / nvf, i = id - t * nvf, k = t / nvf, j = t - k * nvf;
  for (int c = 0; c < ncomp; ++c) {
    const T v = prolong_point<T>(nf, mask, ec + c * Vc, i, j, k);
    if (ADD)
      xf[c * Vf + id] = add_rn(xf[c * Vf + id], v);
    else
      xf[c * Vf + id] = v;
  }
}

}  // namespace

bool pdl_enabled(cudaStream_t s) {
  static const bool on = [] {
    const char* v = getenv("AGCA_PDL");
    return !(v && v[0] == '0');
  }();
  return on && s != nullptr && s != cudaStreamLegacy;
}

template <typename T>
cudaError_t launch_restrict(int nf, int ncomp, bool mask, T scale, const T* rf, T* rc, cudaStream_t s) {
  const int64_t Vc = nverts(nf / 2);
  const int bs = 256;
  KL(launch_k(restrict_kernel<T>, dim3((unsigned)((Vc + bs - 1) / bs)), dim3(bs), 0, s,
     nf, ncomp, mask, scale, rf, rc));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(int nf, int ncomp, bool mask, bool add, const T* ec, T* xf, cudaStream_t s) {
  const int64_t Vf = nverts(nf);
  const int bs = 256;
  const unsigned g = (unsigned)((Vf + bs - 1) / bs);
  if (add)
    KL(launch_k(prolong_kernel<T, true>, dim3(g), dim3(bs), 0, s, nf, ncomp, mask, ec, xf));
  else
    KL(launch_k(prolong_kernel<T, false>, dim3(g), dim3(bs), 0, s, nf, ncomp, mask, ec, xf));
  return cudaGetLastError();
}

template cudaError_t launch_restrict<float>(int, int, bool, float, const float*, float*, cudaStream_t);
template cudaError_t launch_restrict<double>(int, int, bool, double, const double*, double*, cudaStream_t);
template cudaError_t launch_prolong<float>(int, int, bool, bool, const float*, float*, cudaStream_t);
template cudaError_t launch_prolong<double>(int, int, bool, bool, const double*, double*, cudaStream_t);

}  // namespace agca
