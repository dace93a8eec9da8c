// Setup kernels: viscosity hierarchy and flagging (Eq. 2.8, element-wise),
// compaction of the flagged set, batched element-wise Galerkin assembly
// (Eqs. 2.6-2.7, Eq. B.2), level diagonals, the coarsest-grid dense
// Cholesky factor, the lumped pressure mass and the power-iteration start
// vector.  All arithmetic here is FP64.
#include <math.h>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

__global__ void check_eta_kernel(const double* eta, int64_t n, int* status) {
  grid_dep_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = eta[i];
    if (!(isfinite(v) && v > 0.0)) atomicOr(status, 1);
  }
}

// fine element id of child k of coarse element (cube (I,J,K), type t)
__device__ __forceinline__ int64_t child_id(const RefineTables& rt, int nf, int I, int J, int K, int t, int k) {
  const int8_t* c = rt.child[t][k];
  return 6 * ((2 * I + c[0]) + (int64_t)nf * ((2 * J + c[1]) + (int64_t)nf * (2 * K + c[2]))) + c[3];
}

__global__ void coarsen_kernel(const RefineTables rt, int nc, int projection, const double* __restrict__ mean_f,
                               const double* __restrict__ mx_f,
                               const double* __restrict__ mn_f, double nu, double* __restrict__ mean_c,
                               double* __restrict__ mx_c, double* __restrict__ mn_c, uint8_t* __restrict__ flags) {
  grid_dep_entry();
  const int64_t E = nelems(nc);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int t = (int)(e % 6);
  const int64_t cube = e / 6;
  const int I = (int)(cube % nc), J = (int)((cube / nc) % nc), K = (int)(cube / ((int64_t)nc * nc));
  const int nf = 2 * nc;
  double m[8], hi = 0.0, lo = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int64_t f = child_id(rt, nf, I, J, K, t, k);
    m[k] = mean_f[f];
    const double a = mx_f[f], b = mn_f[f];
    hi = k == 0 ? a : fmax(hi, a);
    lo = k == 0 ? b : fmin(lo, b);
  }
  // P0 projection of the children (Sec. 3.2): the arithmetic, harmonic or
  // geometric mean, summed in a fixed pairwise order with explicit roundings
  // (no contraction), /8 exact
  if (projection == 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = __ddiv_rn(1.0, m[k]);
  } else if (projection == 2) {
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = log(m[k]);
  }
  const double s = __dadd_rn(__dadd_rn(__dadd_rn(m[0], m[1]), __dadd_rn(m[2], m[3])),
                             __dadd_rn(__dadd_rn(m[4], m[5]), __dadd_rn(m[6], m[7])));
  mean_c[e] = projection == 1 ? __ddiv_rn(8.0, s) : (projection == 2 ? exp(s * 0.125) : s * 0.125);
  mx_c[e] = hi;
  mn_c[e] = lo;
  flags[e] = hi > __dmul_rn(nu, lo) ? 1 : 0;
}

// Eq. 2.8 on finest element (cube (i, j, k), type t) of a grid of n cubes:
// the norm of the gradient of the P1 interpolant of the nodal viscosity
// eta_v.  The element's path edges are axis-parallel, so gradient component
// perm(t, m) is the difference of the nodal values along the m-th path edge
// times n.  Explicit roundings, IEEE square root.
__device__ __forceinline__ double gradient_norm(const double* __restrict__ eta_v, int n, int i, int j, int k, int t) {
  const int64_t nv = n + 1;
  double prev = eta_v[i + nv * (j + nv * (int64_t)k)], s = 0.0;
  int q = 0;  // cube-corner bits of the current path vertex
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    q |= 1 << perm(t, m);
    const double cur = eta_v[(i + (q & 1)) + nv * ((j + ((q >> 1) & 1)) + nv * (int64_t)(k + ((q >> 2) & 1)))];
    const double d = __dmul_rn(__dsub_rn(cur, prev), (double)n);
    s = __dadd_rn(s, __dmul_rn(d, d));
    prev = cur;
  }
  return __dsqrt_rn(s);
}

// flags of the level above the finest grid: an element is flagged iff the
// gradient norm exceeds nu on one of its 8 finest children
__global__ void gradient_flag_kernel(const RefineTables rt, int nc, const double* __restrict__ eta_v, double nu,
                                     uint8_t* __restrict__ flags) {
  grid_dep_entry();
  const int64_t E = nelems(nc);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int t = (int)(e % 6);
  const int64_t cube = e / 6;
  const int I = (int)(cube % nc), J = (int)((cube / nc) % nc), K = (int)(cube / ((int64_t)nc * nc));
  const int nf = 2 * nc;
  bool f = false;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    const int64_t c = child_id(rt, nf, I, J, K, t, k);
    const int64_t cc = c / 6;
    const int ci = (int)(cc % nf), cj = (int)((cc / nf) % nf), ck = (int)(cc / ((int64_t)nf * nf));
    f = f || gradient_norm(eta_v, nf, ci, cj, ck, (int)(c % 6)) > nu;
  }
  flags[e] = f ? 1 : 0;
}

// coarser levels: flagged iff one of the 8 children is (the maximum over the
// finest descendants exceeds nu)
__global__ void flag_children_kernel(const RefineTables rt, int nc, const uint8_t* __restrict__ flags_f,
                                     uint8_t* __restrict__ flags_c) {
  grid_dep_entry();
  const int64_t E = nelems(nc);
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int t = (int)(e % 6);
  const int64_t cube = e / 6;
  const int I = (int)(cube % nc), J = (int)((cube / nc) % nc), K = (int)(cube / ((int64_t)nc * nc));
  uint8_t f = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) f |= flags_f[child_id(rt, 2 * nc, I, J, K, t, k)];
  flags_c[e] = f ? 1 : 0;
}

constexpr int kCompactChunk = 1024;  // elements per block (256 threads x 4)

__global__ void compact_count_kernel(const uint8_t* flags, int64_t n, int32_t* counts) {
  grid_dep_entry();
  const int64_t base = blockIdx.x * (int64_t)kCompactChunk;
  int c = 0;
  for (int i = threadIdx.x; i < kCompactChunk; i += blockDim.x) {
    const int64_t e = base + i;
    if (e < n && flags[e]) ++c;
  }
  __shared__ int red[256];
  red[threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[blockIdx.x] = red[0];
}

// single block: exclusive scan of counts[0..nb) in place, total in *total
__global__ void compact_scan_kernel(int32_t* counts, int64_t nb, int64_t* total) {
  grid_dep_entry();
  __shared__ int64_t buf[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? counts[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int64_t add = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nb) counts[i] = (int32_t)(carry + buf[threadIdx.x] - v);
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void compact_scatter_kernel(const uint8_t* flags, int64_t n, const int32_t* offsets, int32_t* fidx,
                                       int32_t* list) {
  grid_dep_entry();
  const int64_t base = blockIdx.x * (int64_t)kCompactChunk + 4 * threadIdx.x;
  int f[4], c = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    f[j] = (base + j < n) ? flags[base + j] : 0;
    c += f[j];
  }
  __shared__ int sc[256];
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const int add = threadIdx.x >= off ? sc[threadIdx.x - off] : 0;
    __syncthreads();
    sc[threadIdx.x] += add;
    __syncthreads();
  }
  int pos = offsets[blockIdx.x] + sc[threadIdx.x] - c;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t e = base + j;
    if (e < n) {
      if (f[j]) {
        fidx[e] = pos;
        list[pos] = (int32_t)e;
        ++pos;
      } else {
        fidx[e] = -1;
      }
    }
  }
}

// One block per flagged parent; thread r*12+s computes entry (r, s) of
// A_parent = sum_k (I3 x p_k)^T C_k (I3 x p_k).
__global__ void galerkin_kernel(const RefineTables rt, int nc, const int32_t* __restrict__ list, int nf, int child_finest,
                                const double* __restrict__ coef_f, const int32_t* __restrict__ fidx_f,
                                const double* __restrict__ gca_f, double* __restrict__ gca_c) {
  grid_dep_entry();
  __shared__ int8_t kp[6][144];
  __shared__ double w[8];
  __shared__ int32_t kf[8];
  const int fpar = blockIdx.x;
  const int64_t e = list[fpar];
  const int t = (int)(e % 6);
  const int64_t cube = e / 6;
  const int I = (int)(cube % nc), J = (int)((cube / nc) % nc), K = (int)(cube / ((int64_t)nc * nc));
  const double h6f = 1.0 / (6.0 * nf);
  for (int i = threadIdx.x; i < 6 * 144; i += blockDim.x) kp[i / 144][i % 144] = 0;
  __syncthreads();
  if (threadIdx.x < 144) {
    const int r = threadIdx.x / 12, s = threadIdx.x % 12;
#pragma unroll
    for (int tt = 0; tt < 6; ++tt) kp[tt][threadIdx.x] = (int8_t)kuhn_kprime(tt, r, s);
  }
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    const int64_t f = child_id(rt, nf, I, J, K, t, k);
    w[k] = coef_f[f] * h6f;
    kf[k] = (child_finest || fidx_f == nullptr) ? -1 : fidx_f[f];
  }
  __syncthreads();
  if (threadIdx.x >= 144) return;
  const int r = threadIdx.x / 12, s = threadIdx.x % 12;
  const int c = r >> 2, a = r & 3, d = s >> 2, b = s & 3;
  double acc = 0.0;
  for (int k = 0; k < 8; ++k) {
    const int tc = rt.child[t][k][3];
    const int8_t* p = &rt.pk2[t][k][0][0];  // p[i*4 + j] = 2 lambda_j at child vertex i
    const double* M = kf[k] >= 0 ? gca_f + (int64_t)kf[k] * 144 : nullptr;
    for (int i = 0; i < 4; ++i) {
      const int pia = p[i * 4 + a];
      if (pia == 0) continue;
      for (int j = 0; j < 4; ++j) {
        const int pjb = p[j * 4 + b];
        if (pjb == 0) continue;
        const int rr = c * 4 + i, ss = d * 4 + j;
        const double cv = M ? M[rr * 12 + ss] : w[k] * (double)kp[tc][rr * 12 + ss];
        acc = fma(0.25 * (double)(pia * pjb), cv, acc);
      }
    }
  }
  gca_c[(int64_t)fpar * 144 + threadIdx.x] = acc;
}

__global__ void diag_kernel(const LevelOp<double> op, double* diag, double* invD64, float* invD32) {
  grid_dep_entry();
  const int n = op.n, nv = n + 1;
  const int64_t V = nverts(n);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
  double dg[3] = {0.0, 0.0, 0.0};
  if (inner) {
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int ci = i - (o & 1), cj = j - ((o >> 1) & 1), ck = k - ((o >> 2) & 1);
      const int64_t cube = ci + (int64_t)n * (cj + (int64_t)n * ck);
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int a = corner_local(t, o);
        if (a < 0) continue;
        const int64_t e = 6 * cube + t;
        const int32_t f = op.fidx ? op.fidx[e] : -1;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int r = c * 4 + a;
          if (f >= 0)
            dg[c] += op.gca[(int64_t)f * 144 + r * 13];
          else
            dg[c] += op.coef[e] * op.h6 * (double)kuhn_kprime(t, r, r);
        }
      }
    }
  }
  for (int c = 0; c < 3; ++c) {
    diag[c * V + v] = dg[c];
    const double inv = inner ? 1.0 / dg[c] : 0.0;
    invD64[c * V + v] = inv;
    if (invD32) invD32[c * V + v] = (float)inv;
  }
}

__global__ void gca_to_f32_kernel(int64_t n_flag, const int32_t* list, const double* mx, const double* gca64,
                                  float* gca32, float* scale32) {
  grid_dep_entry();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= n_flag * 144) return;
  const int64_t f = id / 144;
  const double s = mx[list[f]];
  gca32[id] = (float)(gca64[id] / s);
  if (id % 144 == 0) scale32[f] = (float)s;
}

__global__ void d2f_kernel(const double* in, float* out, int64_t n) {
  grid_dep_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void f2d_kernel(const float* in, double* out, int64_t n) {
  grid_dep_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// dense level-1 operator on interior DoFs: row (c, iv), col (d, jv)
__global__ void coarse_assemble_kernel(const LevelOp<double> op, double* dense) {
  grid_dep_entry();
  const int n = op.n, ni = n - 1;
  const int64_t nI = (int64_t)ni * ni * ni, m = 3 * nI;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= m * m) return;
  const int64_t row = id / m, col = id % m;
  const int c = (int)(row / nI), d = (int)(col / nI);
  const int64_t iv = row % nI, jv = col % nI;
  const int i = 1 + (int)(iv % ni), j = 1 + (int)((iv / ni) % ni), k = 1 + (int)(iv / ((int64_t)ni * ni));
  const int wi = 1 + (int)(jv % ni), wj = 1 + (int)((jv / ni) % ni), wk = 1 + (int)(jv / ((int64_t)ni * ni));
  double acc = 0.0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const int ci = i - (o & 1), cj = j - ((o >> 1) & 1), ck = k - ((o >> 2) & 1);
    const int qi = wi - ci, qj = wj - cj, qk = wk - ck;
    if (qi < 0 || qi > 1 || qj < 0 || qj > 1 || qk < 0 || qk > 1) continue;
    const int qw = qi | (qj << 1) | (qk << 2);
    const int64_t cube = ci + (int64_t)n * (cj + (int64_t)n * ck);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int a = corner_local(t, o);
      if (a < 0) continue;
      int b = -1;
#pragma unroll
      for (int bb = 0; bb < 4; ++bb)
        if (tet_corner(t, bb) == qw) b = bb;
      if (b < 0) continue;
      const int64_t e = 6 * cube + t;
      const int32_t f = op.fidx ? op.fidx[e] : -1;
      const int r = c * 4 + a, s = d * 4 + b;
      acc += f >= 0 ? op.gca[(int64_t)f * 144 + r * 12 + s] : op.coef[e] * op.h6 * (double)kuhn_kprime(t, r, s);
    }
  }
  dense[id] = acc;
}

// in-place lower Cholesky of a row-major m x m SPD matrix, one block
__global__ void cholesky_kernel(double* a, int m, int* status) {
  grid_dep_entry();
  __shared__ double piv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      double dk = a[(int64_t)k * m + k];
      if (!(dk > 0.0) || !isfinite(dk)) {
        atomicOr(status, 2);
        dk = 1.0;
      }
      piv = sqrt(dk);
      a[(int64_t)k * m + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < m; i += nt) a[(int64_t)i * m + k] /= piv;
    __syncthreads();
    for (int i = k + 1 + warp; i < m; i += nw) {
      const double lik = a[(int64_t)i * m + k];
      for (int j = k + 1 + lane; j <= i; j += 32) a[(int64_t)i * m + j] -= lik * a[(int64_t)j * m + k];
    }
    __syncthreads();
  }
}

// X = L^-1 (lower), one thread per column; writes column- and row-major copies
__global__ void trinv_kernel(const double* l, int m, double* xcm, double* xrm) {
  grid_dep_entry();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  for (int i = 0; i < j; ++i) {
    xcm[(int64_t)j * m + i] = 0.0;
    xrm[(int64_t)i * m + j] = 0.0;
  }
  for (int i = j; i < m; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < i; ++k) s -= l[(int64_t)i * m + k] * xcm[(int64_t)j * m + k];
    const double x = s / l[(int64_t)i * m + i];
    xcm[(int64_t)j * m + i] = x;
    xrm[(int64_t)i * m + j] = x;
  }
}

// z = L^-T L^-1 r on the interior DoFs of level 1, one block; r, z full-grid.
template <typename T>
__global__ void coarse_solve_kernel(int n, const double* __restrict__ xcm, const double* __restrict__ xrm,
                                    const T* __restrict__ r, T* __restrict__ z) {
  grid_dep_entry();
  extern __shared__ double sm[];
  coarse_solve_block<T>(n, xcm, xrm, r, z, sm);
}

__global__ void pressure_mass_kernel(const RefineTables rt, int np, const double* __restrict__ eta_f, double* pmass, double* pmass_inv) {
  grid_dep_entry();
  const int nv = np + 1;
  const int64_t V = nverts(np);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  const double vol4 = 1.0 / (24.0 * (double)np * np * np);  // |T| / 4
  const int nf = 2 * np;
  double acc = 0.0;
  for (int o = 0; o < 8; ++o) {
    const int ci = i - (o & 1), cj = j - ((o >> 1) & 1), ck = k - ((o >> 2) & 1);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= np || cj >= np || ck >= np) continue;
    for (int t = 0; t < 6; ++t) {
      if (corner_local(t, o) < 0) continue;
      double q[8];
      for (int kk = 0; kk < 8; ++kk) q[kk] = 1.0 / eta_f[child_id(rt, nf, ci, cj, ck, t, kk)];
      const double w = (((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]))) * 0.125;
      acc += w * vol4;
    }
  }
  pmass[v] = acc;
  pmass_inv[v] = 1.0 / acc;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t idx) {
  uint64_t z = (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void start_vector_kernel(int n, double* v) {
  grid_dep_entry();
  const int nv = n + 1;
  const int64_t V = nverts(n);
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < 3 * V; id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = id % V;
    const int i = (int)(p % nv), j = (int)((p / nv) % nv), k = (int)(p / ((int64_t)nv * nv));
    const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
    const double u = (double)(splitmix64((uint64_t)id) >> 11) * 0x1.0p-53;
    v[id] = inner ? 2.0 * u - 1.0 : 0.0;
  }
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t launch_check_eta(const double* eta, int64_t n, int* status, cudaStream_t s) {
  KL(launch_k(check_eta_kernel, dim3(1216), dim3(256), 0, s, eta, n, status));
  return cudaGetLastError();
}

cudaError_t launch_gradient_flags(int nc, const double* eta_v, double nu, const uint8_t* flags_f, uint8_t* flags_c,
                                  cudaStream_t s) {
  const int64_t E = nelems(nc);
  if (eta_v)
    KL(launch_k(gradient_flag_kernel, dim3(blocks_for(E, 256)), dim3(256), 0, s, refine_tables(), nc, eta_v, nu,
                flags_c));
  else
    KL(launch_k(flag_children_kernel, dim3(blocks_for(E, 256)), dim3(256), 0, s, refine_tables(), nc, flags_f,
                flags_c));
  return cudaGetLastError();
}

cudaError_t launch_coarsen(int nc, int projection, const double* mean_f, const double* mx_f, const double* mn_f,
                           double nu, double* mean_c, double* mx_c, double* mn_c, uint8_t* flags, cudaStream_t s) {
  const int64_t E = nelems(nc);
  KL(launch_k(coarsen_kernel, dim3(blocks_for(E, 256)), dim3(256), 0, s,
     refine_tables(), nc, projection, mean_f, mx_f, mn_f, nu, mean_c, mx_c, mn_c, flags));
  return cudaGetLastError();
}

int64_t compact_scratch_blocks(int64_t n) { return (n + kCompactChunk - 1) / kCompactChunk; }

cudaError_t launch_compact(const uint8_t* flags, int64_t n, int32_t* fidx, int32_t* list, int32_t* block_counts,
                           int64_t* total, cudaStream_t s) {
  const int64_t nb = compact_scratch_blocks(n);
  KL(launch_k(compact_count_kernel, dim3((unsigned)nb), dim3(256), 0, s, flags, n, block_counts));
  KL(launch_k(compact_scan_kernel, dim3(1), dim3(1024), 0, s, block_counts, nb, total));
  KL(launch_k(compact_scatter_kernel, dim3((unsigned)nb), dim3(256), 0, s, flags, n, block_counts, fidx, list));
  return cudaGetLastError();
}

cudaError_t launch_galerkin(int nc, int64_t n_flag, const int32_t* list, int nf, bool child_finest,
                            const double* coef_f, const int32_t* fidx_f, const double* gca_f, double* gca_c,
                            cudaStream_t s) {
  if (n_flag == 0) return cudaSuccess;
  KL(launch_k(galerkin_kernel, dim3((unsigned)n_flag), dim3(160), 0, s,
     refine_tables(), nc, list, nf, child_finest ? 1 : 0, coef_f, fidx_f, gca_f, gca_c));
  return cudaGetLastError();
}

cudaError_t launch_diag(const LevelOp<double>& op, double* diag, double* invD64, float* invD32, cudaStream_t s) {
  const int64_t V = nverts(op.n);
  KL(launch_k(diag_kernel, dim3(blocks_for(V, 128)), dim3(128), 0, s, op, diag, invD64, invD32));
  return cudaGetLastError();
}

cudaError_t launch_gca_to_f32(int64_t n_flag, const int32_t* list, const double* mx, const double* gca64,
                              float* gca32, float* scale32, cudaStream_t s) {
  if (n_flag == 0) return cudaSuccess;
  KL(launch_k(gca_to_f32_kernel, dim3(blocks_for(n_flag * 144, 256)), dim3(256), 0, s,
     n_flag, list, mx, gca64, gca32, scale32));
  return cudaGetLastError();
}

cudaError_t launch_d2f(const double* in, float* out, int64_t n, cudaStream_t s) {
  KL(launch_k(d2f_kernel, dim3(1216), dim3(256), 0, s, in, out, n));
  return cudaGetLastError();
}
cudaError_t launch_f2d(const float* in, double* out, int64_t n, cudaStream_t s) {
  KL(launch_k(f2d_kernel, dim3(1216), dim3(256), 0, s, in, out, n));
  return cudaGetLastError();
}

cudaError_t launch_coarse_assemble(const LevelOp<double>& op, double* dense, cudaStream_t s) {
  const int64_t ni = op.n - 1, m = 3 * ni * ni * ni;
  KL(launch_k(coarse_assemble_kernel, dim3(blocks_for(m * m, 128)), dim3(128), 0, s, op, dense));
  return cudaGetLastError();
}

cudaError_t launch_cholesky(double* a, int m, int* status, cudaStream_t s) {
  KL(launch_k(cholesky_kernel, dim3(1), dim3(1024), 0, s, a, m, status));
  return cudaGetLastError();
}

cudaError_t launch_trinv(const double* l, int m, double* linv_cm, double* linv_rm, cudaStream_t s) {
  KL(launch_k(trinv_kernel, dim3(blocks_for(m, 64)), dim3(64), 0, s, l, m, linv_cm, linv_rm));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(int n, const double* linv_cm, const double* linv_rm, const T* r, T* z,
                                cudaStream_t s) {
  const int ni = n - 1, m = 3 * ni * ni * ni;
  const size_t smem = 2 * (size_t)m * sizeof(double);
  KL(launch_k(coarse_solve_kernel<T>, dim3(1), dim3(1024), smem, s, n, linv_cm, linv_rm, r, z));
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(int, const double*, const double*, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(int, const double*, const double*, const double*, double*,
                                                 cudaStream_t);

cudaError_t launch_pressure_mass(int np, const double* eta_f, double* pmass, double* pmass_inv, cudaStream_t s) {
  const int64_t V = nverts(np);
  KL(launch_k(pressure_mass_kernel, dim3(blocks_for(V, 128)), dim3(128), 0, s,
     refine_tables(), np, eta_f, pmass, pmass_inv));
  return cudaGetLastError();
}

cudaError_t launch_start_vector(int n, double* v, cudaStream_t s) {
  KL(launch_k(start_vector_kernel, dim3(1216), dim3(256), 0, s, n, v));
  return cudaGetLastError();
}

}  // namespace agca
