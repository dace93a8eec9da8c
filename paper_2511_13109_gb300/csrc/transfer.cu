// Linear interpolation between Kuhn grids and its transpose (Sec. 2.1).
//
// On the refined grid every fine vertex is either 2i (a coarse vertex) or the
// midpoint 2i + d of the coarse Kuhn edge (i, i + d), d in {0,1}^3 \ {0}
// (the Kuhn edges of a cube join corners whose difference has entries of one
// sign).  Hence
//   (P e)(2i) = e(i),  (P e)(2i + d) = (e(i) + e(i + d)) / 2,
//   (P^T r)(i) = r(2i) + 1/2 sum_d [ r(2i + d) + r(2i - d) ].
// The weights are known a priori and never stored.
#include <stdlib.h>

#include "agca_internal.cuh"

namespace agca {

namespace {

template <typename T>
__global__ void restrict_kernel(int nf, int ncomp, bool mask, T scale, const T* __restrict__ rf, T* __restrict__ rc) {
  grid_dep_entry();
  const int nc = nf / 2;
  const int nvf = nf + 1, nvc = nc + 1;
  const int64_t Vc = (int64_t)nvc * nvc * nvc, Vf = (int64_t)nvf * nvf * nvf;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= Vc) return;
  const int I = (int)(id % nvc), J = (int)((id / nvc) % nvc), K = (int)(id / ((int64_t)nvc * nvc));
  const bool bd = I == 0 || J == 0 || K == 0 || I == nc || J == nc || K == nc;
  for (int c = 0; c < ncomp; ++c) {
    T out = T(0);
    if (!(mask && bd)) {
      const T* r = rf + c * Vf;
      const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
      T acc = T(0);
#pragma unroll
      for (int d = 1; d < 8; ++d) {
        const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
        if (fi + dx <= nf && fj + dy <= nf && fk + dz <= nf)
          acc += r[(fi + dx) + (int64_t)nvf * ((fj + dy) + (int64_t)nvf * (fk + dz))];
        if (fi - dx >= 0 && fj - dy >= 0 && fk - dz >= 0)
          acc += r[(fi - dx) + (int64_t)nvf * ((fj - dy) + (int64_t)nvf * (fk - dz))];
      }
      out = scale * (r[fi + (int64_t)nvf * (fj + (int64_t)nvf * fk)] + T(0.5) * acc);
    }
    rc[c * Vc + id] = out;
  }
}

template <typename T, bool ADD>
__global__ void prolong_kernel(int nf, int ncomp, bool mask, const T* __restrict__ ec, T* __restrict__ xf) {
  grid_dep_entry();
  const int nc = nf / 2;
  const int nvf = nf + 1, nvc = nc + 1;
  const int64_t Vc = (int64_t)nvc * nvc * nvc, Vf = (int64_t)nvf * nvf * nvf;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= Vf) return;
  const int i = (int)(id % nvf), j = (int)((id / nvf) % nvf), k = (int)(id / ((int64_t)nvf * nvf));
  const bool bd = i == 0 || j == 0 || k == 0 || i == nf || j == nf || k == nf;
  const int I = i >> 1, J = j >> 1, K = k >> 1, dx = i & 1, dy = j & 1, dz = k & 1;
  const int64_t c0 = I + (int64_t)nvc * (J + (int64_t)nvc * K);
  const int64_t c1 = (I + dx) + (int64_t)nvc * ((J + dy) + (int64_t)nvc * (K + dz));
  const bool odd = dx | dy | dz;
  for (int c = 0; c < ncomp; ++c) {
    const T* e = ec + c * Vc;
    T v = odd ? T(0.5) * (e[c0] + e[c1]) : e[c0];
    if (mask && bd) v = T(0);
    if (ADD)
      xf[c * Vf + id] += v;
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
