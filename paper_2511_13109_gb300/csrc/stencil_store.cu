// Stencil storage of the stored-Galerkin part of the coarse AGCA operators
// (Remark 5, Eq. 5.8): per vertex touched by a flagged element, 15 blocks of
// 3 x 3 couplings (the vertex and its 14 Kuhn neighbours) holding the sum of
// the flagged elements' local Galerkin matrices, instead of 144 values per
// flagged element.  The unflagged elements stay matrix-free (DCA); a coarse
// apply adds sum_o S_v[o] x(v + o) at each touched vertex.
//
// Set-up, per coarse level: mark the vertices of flagged elements, compact
// them (ascending vertex id), and assemble each touched vertex's stencil from
// the element matrices of the flagged tetrahedra around it (fixed order: the
// 8 cubes sharing the vertex, then the tetrahedron type, then the element's
// local vertices), in FP64; the mixed-precision store keeps S / s_v in FP32
// with s_v the largest |entry| of the vertex's stencil.
#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

// the tetrahedra of the 8 cubes around vertex (i, j, k): cube origin (i - ox,
// j - oy, k - oz) for corner q = ox + 2 oy + 4 oz of that cube; tetrahedron t
// contains the vertex iff corner_local(t, q) >= 0
template <typename F>
__device__ __forceinline__ void for_tets_around(int n, int i, int j, int k, F f) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ox = q & 1, oy = (q >> 1) & 1, oz = (q >> 2) & 1;
    const int ci = i - ox, cj = j - oy, ck = k - oz;
    if (ci < 0 || cj < 0 || ck < 0 || ci >= n || cj >= n || ck >= n) continue;
    const int64_t cube = ci + (int64_t)n * (cj + (int64_t)n * ck);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int a = corner_local(t, q);
      if (a >= 0) f(6 * cube + t, t, q, a);
    }
  }
}

__global__ void mark_vertices_kernel(const int n, const uint8_t* __restrict__ flags, uint8_t* __restrict__ mark) {
  grid_dep_entry();
  const int nv = n + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  uint8_t m = 0;
  for_tets_around(n, i, j, k, [&](int64_t e, int, int, int) { m |= flags[e]; });
  mark[v] = m ? 1 : 0;
}

// one thread per (touched vertex, component row c)
__global__ void stencil_assemble_kernel(const int n, const int64_t n_sv, const int32_t* __restrict__ slist,
                                        const int32_t* __restrict__ fidx, const double* __restrict__ gca,
                                        double* __restrict__ sten) {
  grid_dep_entry();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n_sv * 3) return;
  const int64_t s = id / 3;
  const int c = (int)(id - s * 3);
  const int nv = n + 1;
  const int v = slist[s];
  const int i = v % nv, j = (v / nv) % nv, k = v / (nv * nv);
  double acc[15][3];
#pragma unroll
  for (int o = 0; o < 15; ++o)
#pragma unroll
    for (int d = 0; d < 3; ++d) acc[o][d] = 0.0;
  for_tets_around(n, i, j, k, [&](int64_t e, int t, int qv, int a) {
    const int f = fidx[e];
    if (f < 0) return;
    const double* M = gca + (int64_t)f * 144 + (c * 4 + a) * 12;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int qb = tet_corner(t, b);
      const int o = kuhn_offset_index((qb & 1) - (qv & 1), ((qb >> 1) & 1) - ((qv >> 1) & 1),
                                      ((qb >> 2) & 1) - ((qv >> 2) & 1));
#pragma unroll
      for (int oo = 0; oo < 15; ++oo) {
        if (oo != o) continue;  // constant register indexing
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[oo][d] += M[d * 4 + b];
      }
    }
  });
  double* out = sten + s * 135;
#pragma unroll
  for (int o = 0; o < 15; ++o)
#pragma unroll
    for (int d = 0; d < 3; ++d) out[o * 9 + c * 3 + d] = acc[o][d];
}

__global__ void stencil_to_f32_kernel(const int64_t n_sv, const double* __restrict__ s64, float* __restrict__ s32,
                                      float* __restrict__ scale) {
  grid_dep_entry();
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n_sv) return;
  const double* in = s64 + s * 135;
  double mx = 0.0;
  for (int q = 0; q < 135; ++q) mx = fmax(mx, fabs(in[q]));
  const double sc = mx > 0.0 ? mx : 1.0;
  for (int q = 0; q < 135; ++q) s32[s * 135 + q] = (float)(in[q] / sc);
  scale[s] = (float)sc;
}

// DCA coefficient with the flagged elements zeroed (their part is in the stencils)
__global__ void masked_coef_kernel(const int64_t E, const double* __restrict__ mean, const int32_t* __restrict__ fidx,
                                   double* __restrict__ coefm) {
  grid_dep_entry();
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  coefm[e] = fidx[e] >= 0 ? 0.0 : mean[e];
}

unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_mark_vertices(int n, const uint8_t* flags, uint8_t* mark, cudaStream_t s) {
  const int64_t V = nverts(n);
  KL(launch_k(mark_vertices_kernel, dim3(nblocks(V, 256)), dim3(256), 0, s, n, flags, mark));
  return cudaGetLastError();
}

cudaError_t launch_stencil_assemble(int n, int64_t n_sv, const int32_t* slist, const int32_t* fidx, const double* gca,
                                    double* sten, cudaStream_t s) {
  if (n_sv == 0) return cudaSuccess;
  KL(launch_k(stencil_assemble_kernel, dim3(nblocks(3 * n_sv, 128)), dim3(128), 0, s, n, n_sv, slist, fidx, gca,
              sten));
  return cudaGetLastError();
}

cudaError_t launch_stencil_to_f32(int64_t n_sv, const double* s64, float* s32, float* scale, cudaStream_t s) {
  if (n_sv == 0) return cudaSuccess;
  KL(launch_k(stencil_to_f32_kernel, dim3(nblocks(n_sv, 128)), dim3(128), 0, s, n_sv, s64, s32, scale));
  return cudaGetLastError();
}

cudaError_t launch_masked_coef(int64_t E, const double* mean, const int32_t* fidx, double* coefm, cudaStream_t s) {
  KL(launch_k(masked_coef_kernel, dim3(nblocks(E, 256)), dim3(256), 0, s, E, mean, fidx, coefm));
  return cudaGetLastError();
}

}  // namespace agca
