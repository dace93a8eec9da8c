// Batched element-wise kernels: many independent problems per launch.
// Grid (chunks, problems): block row y serves problem y, blocks past the end
// of a smaller problem exit at once.  A problem whose MINRES has converged
// (sc[MS_DONE] != 0) is skipped.  Used by the batched solve of
// agca_batch_solve (persistent stencil launches live in stencil.cu).
#include <math.h>

#include <algorithm>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

constexpr int kBT = 256;
constexpr int kDotBlocks = 64;  // per problem: fixed, so the reductions are deterministic

__device__ __forceinline__ bool skip(const double* sc) { return sc && sc[MS_DONE] != 0.0; }

template <typename T>
__global__ void restrict_batch_kernel(const XferTask* __restrict__ tasks) {
  grid_dep_entry();
  const XferTask tk = tasks[blockIdx.y];
  if (skip(tk.sc)) return;
  const int nf = tk.nf, nvf = nf + 1, nvc = nf / 2 + 1;
  const int Vc = nvc * nvc * nvc, Vf = nvf * nvf * nvf;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Vc) return;
  const T* rf = static_cast<const T*>(tk.src);
  T* rc = static_cast<T*>(tk.dst);
  const int t = id / nvc, I = id - t * nvc, K = t / nvc, J = t - K * nvc;
  for (int c = 0; c < tk.ncomp; ++c)
    rc[c * Vc + id] = restrict_point<T>(nf, tk.mask, (T)tk.scale, rf + c * Vf, I, J, K);
}

template <typename T, bool ADD>
__global__ void prolong_batch_kernel(const XferTask* __restrict__ tasks) {
  grid_dep_entry();
  const XferTask tk = tasks[blockIdx.y];
  if (skip(tk.sc)) return;
  const int nf = tk.nf, nvf = nf + 1, nvc = nf / 2 + 1;
  const int Vc = nvc * nvc * nvc, Vf = nvf * nvf * nvf;
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= Vf) return;
  const T* ec = static_cast<const T*>(tk.src);
  T* xf = static_cast<T*>(tk.dst);
  const int t = id / nvf, i = id - t * nvf, k = t / nvf, j = t - k * nvf;
  for (int c = 0; c < tk.ncomp; ++c) {
    const T v = prolong_point<T>(nf, tk.mask, ec + c * Vc, i, j, k);
    if (ADD)
      xf[c * Vf + id] = add_rn(xf[c * Vf + id], v);
    else
      xf[c * Vf + id] = v;
  }
}

template <typename TI, typename TO>
__global__ void convert_batch_kernel(const XferTask* __restrict__ tasks) {
  grid_dep_entry();
  const XferTask tk = tasks[blockIdx.y];
  if (skip(tk.sc)) return;
  const TI* in = static_cast<const TI*>(tk.src);
  TO* out = static_cast<TO*>(tk.dst);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tk.count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// coarsest solves, one block per problem
template <typename T>
__global__ void coarse_solve_batch_kernel(const XferTask* __restrict__ tasks) {
  grid_dep_entry();
  extern __shared__ double sm[];
  const XferTask tk = tasks[blockIdx.x];
  if (skip(tk.sc)) return;
  coarse_solve_block<T>(tk.nf, tk.m1, tk.m2, static_cast<const T*>(tk.src), static_cast<T*>(tk.dst), sm);
}

// ------------------------------------------------------------------ Krylov
template <int OP>
__global__ void __launch_bounds__(kBT) reduce_batch_kernel(const KTask* __restrict__ tasks, double* partials) {
  grid_dep_entry();
  const KTask tk = tasks[blockIdx.y];
  double acc = 0.0;
  if (!skip(tk.sc)) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tk.n; i += (int64_t)gridDim.x * blockDim.x)
      acc = (OP == KB_DOT) ? fma(tk.a[i], tk.b[i], acc) : acc + tk.a[i];
  }
  __shared__ double red[kBT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kBT / 32; ++w) v += red[w];
    partials[blockIdx.y * kDotBlocks + blockIdx.x] = v;
  }
}

__global__ void reduce_batch_final_kernel(const KTask* __restrict__ tasks, const double* partials) {
  grid_dep_entry();
  const KTask tk = tasks[blockIdx.x];
  if (skip(tk.sc)) return;
  __shared__ double red[kDotBlocks];
  red[threadIdx.x] = partials[blockIdx.x * kDotBlocks + threadIdx.x];
  __syncthreads();
  for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) tk.sc[tk.slot] = tk.scale * red[0];
}

__global__ void vec_batch_kernel(const KTask* __restrict__ tasks, int op) {
  grid_dep_entry();
  const KTask tk = tasks[blockIdx.y];
  if (op == KB_UPDATE ? tk.sc[MS_UPD_SKIP] != 0.0 : skip(tk.sc)) return;
  const double* sc = tk.sc;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  if (op == KB_LANCZOS) {  // c <- a/g - (delta/g) b - (g/g_old) c   (a = Kz, b = v, c = v_old)
    const double g = sc[MS_GAMMA], go = sc[MS_GAMMA_OLD];
    const double ig = 1.0 / g;
    const double delta = sc[MS_DOT_KZZ] * ig * ig;
    const double al = delta * ig, be = g / go;
    for (int64_t i = i0; i < tk.n; i += st) tk.c[i] = tk.a[i] * ig - al * tk.b[i] - be * tk.c[i];
  } else if (op == KB_UPDATE) {  // c <- (a/g_prev - a3 c - a2 b)/a1 ; d += xcoef c   (a = z, b = w, c = w_old, d = x)
    const double ig = sc[MS_INV_GAMMA_PREV], a1 = sc[MS_A1], a2 = sc[MS_A2], a3 = sc[MS_A3], xc = sc[MS_XCOEF];
    const double ia1 = 1.0 / a1;
    for (int64_t i = i0; i < tk.n; i += st) {
      const double wn = (tk.a[i] * ig - a3 * tk.c[i] - a2 * tk.b[i]) * ia1;
      tk.c[i] = wn;
      tk.d[i] = fma(xc, wn, tk.d[i]);
    }
  } else if (op == KB_PDIV) {  // c <- (a - sc[slot]) * b
    const double m = sc[tk.slot];
    for (int64_t i = i0; i < tk.n; i += st) tk.c[i] = (tk.a[i] - m) * tk.b[i];
  } else if (op == KB_SUBS) {  // c <- a - sc[slot]
    const double m = sc[tk.slot];
    for (int64_t i = i0; i < tk.n; i += st) tk.c[i] = tk.a[i] - m;
  }
}

// MINRES scalar recurrence, one thread per problem (as minres_scalar_kernel)
__device__ void scalars_one(double* sc) {
  if (sc[MS_DONE] != 0.0) {
    sc[MS_UPD_SKIP] = 1.0;
    return;
  }
  const double g = sc[MS_GAMMA];
  const double delta = sc[MS_DOT_KZZ] / (g * g);
  const double gn2 = sc[MS_DOT_ZV];
  const double gn = gn2 > 0.0 ? sqrt(gn2) : 0.0;
  const double c = sc[MS_C], co = sc[MS_C_OLD], s = sc[MS_S], so = sc[MS_S_OLD];
  const double a0 = c * delta - co * s * g;
  const double a1 = sqrt(a0 * a0 + gn * gn);
  const double a2 = s * delta + co * c * g;
  const double a3 = so * g;
  const double eta = sc[MS_ETA];
  if (!(a1 > 0.0) || !isfinite(a1)) {
    sc[MS_DONE] = 2.0;
    sc[MS_UPD_SKIP] = 1.0;
    return;
  }
  const double cn = a0 / a1, sn = gn / a1;
  sc[MS_A1] = a1;
  sc[MS_A2] = a2;
  sc[MS_A3] = a3;
  sc[MS_XCOEF] = cn * eta;
  sc[MS_INV_GAMMA_PREV] = 1.0 / g;
  sc[MS_UPD_SKIP] = 0.0;
  sc[MS_ETA] = -sn * eta;
  sc[MS_C_OLD] = c;
  sc[MS_C] = cn;
  sc[MS_S_OLD] = s;
  sc[MS_S] = sn;
  sc[MS_GAMMA_OLD] = g;
  sc[MS_GAMMA] = gn;
  sc[MS_ITERS] += 1.0;
  if (fabs(sc[MS_ETA]) <= sc[MS_TOL_ABS] || !(gn > 0.0)) sc[MS_DONE] = 1.0;
}

__global__ void scalars_batch_kernel(const KTask* __restrict__ tasks, int ntasks) {
  grid_dep_entry();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ntasks) return;
  double* sc = tasks[p].sc;
  scalars_one(sc);
  if (tasks[p].c) tasks[p].c[0] = sc[MS_DONE];  // contiguous copy of the done flags for the host
}


inline unsigned chunks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

template <typename T>
cudaError_t launch_xfer_batch(int kind, const XferTask* tasks, int ntasks, int64_t max_count, int max_m,
                              cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const dim3 g(chunks(max_count, kBT), (unsigned)ntasks);
  const dim3 gc(std::min<unsigned>(g.x, 1216u), (unsigned)ntasks);
  switch (kind) {
    case XK_RESTRICT: KL(launch_k(restrict_batch_kernel<T>, g, dim3(kBT), 0, s, tasks)); break;
    case XK_PROLONG_ADD: KL(launch_k(prolong_batch_kernel<T, true>, g, dim3(kBT), 0, s, tasks)); break;
    case XK_PROLONG: KL(launch_k(prolong_batch_kernel<T, false>, g, dim3(kBT), 0, s, tasks)); break;
    case XK_COPY64:
      KL(launch_k(convert_batch_kernel<double, double>, gc, dim3(kBT), 0, s, tasks));
      break;
    case XK_D2F:
      KL(launch_k(convert_batch_kernel<double, float>, gc, dim3(kBT), 0, s, tasks));
      break;
    case XK_F2D:
      KL(launch_k(convert_batch_kernel<float, double>, gc, dim3(kBT), 0, s, tasks));
      break;
    case XK_COARSE:
      KL(launch_k(coarse_solve_batch_kernel<T>, dim3(ntasks), dim3(1024), 2 * (size_t)max_m * sizeof(double), s, tasks));
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
template cudaError_t launch_xfer_batch<float>(int, const XferTask*, int, int64_t, int, cudaStream_t);
template cudaError_t launch_xfer_batch<double>(int, const XferTask*, int, int64_t, int, cudaStream_t);

cudaError_t launch_krylov_batch(int op, const KTask* tasks, int ntasks, int64_t max_n, double* partials,
                                cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  switch (op) {
    case KB_DOT:
      KL(launch_k(reduce_batch_kernel<KB_DOT>, dim3(kDotBlocks, ntasks), dim3(kBT), 0, s, tasks, partials));
      KL(launch_k(reduce_batch_final_kernel, dim3(ntasks), dim3(kDotBlocks), 0, s, tasks, partials));
      break;
    case KB_SUM:
      KL(launch_k(reduce_batch_kernel<KB_SUM>, dim3(kDotBlocks, ntasks), dim3(kBT), 0, s, tasks, partials));
      KL(launch_k(reduce_batch_final_kernel, dim3(ntasks), dim3(kDotBlocks), 0, s, tasks, partials));
      break;
    case KB_SCALARS: KL(launch_k(scalars_batch_kernel, dim3(chunks(ntasks, 32)), dim3(32), 0, s,
                        tasks, ntasks)); break;
    default: {
      dim3 g(std::min<unsigned>(chunks(max_n, kBT), 1216u), (unsigned)ntasks);
      KL(launch_k(vec_batch_kernel, dim3(g), dim3(kBT), 0, s, tasks, op));
    }
  }
  return cudaGetLastError();
}

}  // namespace agca
