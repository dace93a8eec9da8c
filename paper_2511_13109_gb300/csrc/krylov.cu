// Krylov-side kernels (FP64): deterministic dot products, the preconditioned
// MINRES recurrence of Remark 6 with its scalars kept on the device, the
// pressure block of the block-diagonal preconditioner, the load vector, the
// element sensitivities of the adjoint gradient, and FGMRES's pieces (block
// Gram-Schmidt, the assembled Z of the BFBT Schur block and its
// conjugate-gradient solve).
#include <math.h>

#include <algorithm>
#include <cooperative_groups.h>

#include "agca_internal.cuh"

namespace agca {

namespace {

constexpr int kRedBlocks = 1216;  // 8 per SM; fixed so reductions are deterministic
constexpr int kRedThreads = 256;

struct DotPairs {
  const double* x[3];
  const double* y[3];
};

template <int NP>
__global__ void __launch_bounds__(kRedThreads) dot_partial_kernel(DotPairs p, int64_t n, double* partials) {
  grid_dep_entry();
  double acc[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) acc[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < NP; ++j) acc[j] = fma(p.x[j][i], p.y[j][i], acc[j]);
  }
  __shared__ double red[NP][kRedThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    double v = acc[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[j][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < NP) {
    double v = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) v += red[threadIdx.x][w];
    partials[threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
}

// one block: out[j] = scale * sum_b partials[j*nb + b], fixed tree order
__global__ void reduce_final_kernel(const double* partials, int nb, int np, double* out, double scale) {
  grid_dep_entry();
  __shared__ double red[256];
  for (int j = 0; j < np; ++j) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[j * nb + b];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = scale * red[0];
    __syncthreads();
  }
}

__global__ void sum_partial_kernel(const double* x, int64_t n, double* partials) {
  grid_dep_entry();
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i];
  __shared__ double red[kRedThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) v += red[w];
    partials[blockIdx.x] = v;
  }
}

// ------------------------------------------------------------------ MINRES
// Scalars live in device memory (MinresSlot) so an iteration needs no host
// round trip; the Lanczos vector z is kept unnormalized (z = gamma zhat).
__global__ void lanczos_kernel(int64_t n, const double* __restrict__ kz, const double* __restrict__ v,
                               double* vold_to_vnew, const double* __restrict__ sc) {
  grid_dep_entry();
  if (sc[MS_DONE] != 0.0) return;
  const double g = sc[MS_GAMMA], go = sc[MS_GAMMA_OLD];
  const double ig = 1.0 / g;
  const double delta = sc[MS_DOT_KZZ] * ig * ig;  // z is kept unnormalized: z = gamma * zhat
  const double a = delta * ig, b = g / go;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vold_to_vnew[i] = kz[i] * ig - a * v[i] - b * vold_to_vnew[i];
}

__global__ void minres_scalar_kernel(double* sc) {
  grid_dep_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (sc[MS_DONE] != 0.0) return;
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
  if (!(a1 > 0.0) || !isfinite(a1)) {  // exact convergence or breakdown
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

// w_new = (z/gamma_prev - a3 w_old - a2 w) / a1 into w_old; x += c_new*eta_prev * w_new
__global__ void minres_update_kernel(int64_t n, const double* __restrict__ z, const double* __restrict__ w,
                                     double* wold_to_wnew, double* x, const double* __restrict__ sc) {
  grid_dep_entry();
  if (sc[MS_UPD_SKIP] != 0.0) return;
  const double ig = sc[MS_INV_GAMMA_PREV], a1 = sc[MS_A1], a2 = sc[MS_A2], a3 = sc[MS_A3], xc = sc[MS_XCOEF];
  const double ia1 = 1.0 / a1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double wn = (z[i] * ig - a3 * wold_to_wnew[i] - a2 * w[i]) * ia1;
    wold_to_wnew[i] = wn;
    x[i] = fma(xc, wn, x[i]);
  }
}

__global__ void minres_init_kernel(double* sc, double tol_rel) {
  grid_dep_entry();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double g2 = sc[MS_DOT_ZV];
  const double g = g2 > 0.0 ? sqrt(g2) : 0.0;
  sc[MS_GAMMA] = g;
  sc[MS_GAMMA_OLD] = 1.0;
  sc[MS_ETA] = g;
  sc[MS_ETA0] = g;
  sc[MS_C] = sc[MS_C_OLD] = 1.0;
  sc[MS_S] = sc[MS_S_OLD] = 0.0;
  sc[MS_ITERS] = 0.0;
  sc[MS_UPD_SKIP] = 1.0;
  sc[MS_TOL_ABS] = tol_rel * g;
  sc[MS_DONE] = (g > 0.0) ? 0.0 : 1.0;
}

// ------------------------------------------------------------------ vectors
__global__ void vec_op_kernel(int op, int64_t n, double* y, const double* a, const double* b, const double* c,
                              const double* scal) {
  grid_dep_entry();
  const double s0 = scal ? scal[0] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    switch (op) {
      case VOP_SUB: y[i] = a[i] - b[i]; break;            // y = a - b
      case VOP_ADD: y[i] = a[i] + b[i]; break;            // y = a + b
      case VOP_COPY: y[i] = a[i]; break;                  // y = a
      case VOP_ZERO: y[i] = 0.0; break;                   // y = 0
      case VOP_PDIV: y[i] = (a[i] - s0) * b[i]; break;    // y = (a - mean) * minv
      case VOP_SUBS: y[i] = a[i] - s0; break;             // y = a - s
      case VOP_MUL: y[i] = a[i] * b[i]; break;            // y = a * b
      case VOP_SCALE_RSQRT: y[i] = a[i] * (1.0 / sqrt(s0)); break;  // y = a / sqrt(s)
      case VOP_RECIP: y[i] = a[i] > 0.0 ? 1.0 / a[i] : 0.0; break;  // y = 1 / a (0 where a <= 0)
      default: break;
    }
  }
}

// --------------------------------------------------------------- FE kernels
__global__ void load_vector_kernel(int n, const double* __restrict__ fbar, double* __restrict__ b) {
  grid_dep_entry();
  const int nv = n + 1;
  const int64_t V = nverts(n), E = nelems(n);
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
  const double w = 1.0 / (24.0 * (double)n * n * n);  // |T| / 4
  double acc[3] = {0.0, 0.0, 0.0};
  if (inner) {
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int64_t cube = (i - (o & 1)) + (int64_t)n * ((j - ((o >> 1) & 1)) + (int64_t)n * (k - ((o >> 2) & 1)));
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        if (corner_local(t, o) < 0) continue;
        const int64_t e = 6 * cube + t;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += w * fbar[c * E + e];
      }
    }
  }
  for (int c = 0; c < 3; ++c) b[c * V + v] = acc[c];
}

// g_e = -eta_e (h/12) S(u) : S(lambda), S(w) = Gw + Gw^T the doubled symmetric
// gradient scaled by h (this is -lambda_e^T (eta_e dA_e/deta_e) u_e).
__global__ void sensitivity_kernel(int n, const double* __restrict__ eta, const double* __restrict__ lam,
                                   const double* __restrict__ u, double* __restrict__ g) {
  grid_dep_entry();
  const int nv = n + 1;
  const int64_t V = nverts(n);
  const int64_t cube = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cube >= (int64_t)n * n * n) return;
  const int ci = (int)(cube % n), cj = (int)((cube / n) % n), ck = (int)(cube / ((int64_t)n * n));
  double U[8][3], Lm[8][3];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = ci + (q & 1), j = cj + ((q >> 1) & 1), k = ck + ((q >> 2) & 1);
    const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
    const int64_t v = i + (int64_t)nv * (j + (int64_t)nv * k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      U[q][c] = inner ? u[c * V + v] : 0.0;
      Lm[q][c] = inner ? lam[c * V + v] : 0.0;
    }
  }
  const double h12 = 1.0 / (12.0 * n);
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    double Gu[3][3], Gl[3][3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const int qa = tet_corner(t, kk), qb = tet_corner(t, kk + 1), m = perm(t, kk);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Gu[c][m] = U[qb][c] - U[qa][c];
        Gl[c][m] = Lm[qb][c] - Lm[qa][c];
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) acc += (Gu[a][b] + Gu[b][a]) * (Gl[a][b] + Gl[b][a]);
    const int64_t e = 6 * cube + t;
    g[e] = -eta[e] * h12 * acc;
  }
}

__global__ void mask_boundary_kernel(int n, double* x) {
  grid_dep_entry();
  const int nv = n + 1;
  const int64_t V = nverts(n);
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < 3 * V; id += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = id % V;
    const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
    if (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n) x[id] = 0.0;
  }
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ----------------------------------------------------------- FGMRES pieces
// Gram-Schmidt against a block of vectors V_i = V + i * ld (i < nvec): per
// block and vector the partial sums of w . V_i over the block's grid-stride
// range, in a fixed order (deterministic); the final sums by reduce_final_kernel
__global__ void __launch_bounds__(kRedThreads) block_dot_kernel(int nvec, const double* __restrict__ V, int64_t ld,
                                                                const double* __restrict__ w, int64_t n,
                                                                double* __restrict__ partials) {
  grid_dep_entry();
  __shared__ double red[kRedThreads / 32];
  for (int i = 0; i < nvec; ++i) {
    const double* vi = V + i * ld;
    double acc = 0.0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
      acc = fma(w[q], vi[q], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int k = 0; k < kRedThreads / 32; ++k) v += red[k];
      partials[(int64_t)i * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// w += sign * sum_i coef[i] V_i (coefficients on the device), summed in i order
__global__ void __launch_bounds__(kRedThreads) block_axpy_kernel(int nvec, const double* __restrict__ V, int64_t ld,
                                                                 const double* __restrict__ coef, double sign,
                                                                 double* __restrict__ w, int64_t n) {
  grid_dep_entry();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc = fma(coef[i], V[i * ld + q], acc);
    w[q] = fma(sign, acc, w[q]);
  }
}

// y = a * s (s on the device)
__global__ void scale_kernel(int64_t n, double* __restrict__ y, const double* __restrict__ a,
                             const double* __restrict__ s, int recip) {
  grid_dep_entry();
  const double f = recip ? 1.0 / s[0] : s[0];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = a[q] * f;
}

// conjugate-gradient vector updates on the device scalars sc: x += alpha p,
// r -= alpha q with alpha = sc[0] / sc[1]; p = z + beta p with beta = sc[2] / sc[0]
// Assembled Z = B W^-1 B^T on the pressure grid (np cubes per axis).  A
// pressure hat and a velocity hat overlap only where their Kuhn
// neighbourhoods meet, so Z couples pressure vertices whose offset is a sum
// of two Kuhn offsets: 65 offsets in [-2, 2]^3.  Z is kept as per-vertex
// stencils over those offsets, SoA zs[s * V + v] (slot s in the order
// below).  Applying Z to the indicator of colour (a, b, c) (vertices with
// coordinates = (a, b, c) mod 5) yields, at every vertex l, the one entry
// Z[l][k] of the colour vertex k within distance 2 of l, so 125 colours
// recover every stencil.
struct ZPattern {
  signed char d[65][3];   // offsets (dx, dy, dz), ascending in (dz, dy, dx)
  signed char slot[125];  // (dx + 2) + 5 (dy + 2) + 25 (dz + 2) -> slot, or -1
  int n, centre;
};
constexpr ZPattern make_zpattern() {
  ZPattern p{};
  for (int q = 0; q < 125; ++q) p.slot[q] = -1;
  for (int dz = -2; dz <= 2; ++dz)
    for (int dy = -2; dy <= 2; ++dy)
      for (int dx = -2; dx <= 2; ++dx) {
        bool in = false;
        for (int a = 0; a < 15; ++a)
          for (int b = 0; b < 15; ++b)
            in = in || (kuhn_offset_comp(a, 0) + kuhn_offset_comp(b, 0) == dx &&
                        kuhn_offset_comp(a, 1) + kuhn_offset_comp(b, 1) == dy &&
                        kuhn_offset_comp(a, 2) + kuhn_offset_comp(b, 2) == dz);
        if (!in) continue;
        if (dx == 0 && dy == 0 && dz == 0) p.centre = p.n;
        p.d[p.n][0] = (signed char)dx;
        p.d[p.n][1] = (signed char)dy;
        p.d[p.n][2] = (signed char)dz;
        p.slot[(dx + 2) + 5 * (dy + 2) + 25 * (dz + 2)] = (signed char)p.n;
        ++p.n;
      }
  return p;
}
constexpr ZPattern kZPattern = make_zpattern();
static_assert(kZPattern.n == ZSTENCIL, "sums of two Kuhn offsets: 65 distinct offsets");
__constant__ ZPattern c_zpat = make_zpattern();

__global__ void colour5_kernel(int np, int colour, double* __restrict__ e) {
  grid_dep_entry();
  const int nv = np + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  e[v] = (i % 5) + 5 * (j % 5) + 25 * (k % 5) == colour ? 1.0 : 0.0;
}
__device__ __forceinline__ int offset5(int l, int c) {  // d in [-2, 2] with (l + d) mod 5 == c
  return ((c - l % 5) + 7) % 5 - 2;
}
__global__ void scatter_zrow_kernel(int np, int colour, const double* __restrict__ y, double* __restrict__ zs) {
  grid_dep_entry();
  const int nv = np + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  const int di = offset5(i, colour % 5), dj = offset5(j, (colour / 5) % 5), dk = offset5(k, colour / 25);
  const int s = c_zpat.slot[(di + 2) + 5 * (dj + 2) + 25 * (dk + 2)];
  if (s >= 0) zs[s * V + v] = y[v];  // Z vanishes at the other offsets
}
// inverse diagonal of the assembled Z (0 where it is not positive)
__global__ void zdiag_inv_kernel(int64_t V, const double* __restrict__ zs, double* __restrict__ dinv) {
  grid_dep_entry();
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double d = zs[kZPattern.centre * V + v];
  dinv[v] = d > 0.0 ? 1.0 / d : 0.0;
}

// (Z p)_v from the stencils (neighbours outside the grid contribute nothing)
__device__ __forceinline__ double zrow(const double* __restrict__ zs, const double* __restrict__ p, int64_t V, int nv,
                                       int64_t v) {
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  double acc = 0.0;
#pragma unroll 5
  for (int s = 0; s < ZSTENCIL; ++s) {
    const int ii = i + c_zpat.d[s][0], jj = j + c_zpat.d[s][1], kk = k + c_zpat.d[s][2];
    if (ii < 0 || jj < 0 || kk < 0 || ii >= nv || jj >= nv || kk >= nv) continue;
    acc = fma(zs[s * V + v], p[ii + (int64_t)nv * (jj + (int64_t)nv * kk)], acc);
  }
  return acc;
}

// Sum of one value per thread over the whole grid: block sums into
// partials[blockIdx], a grid barrier, then every block adds the partials in
// index order (the same bits in every block and every run)
__device__ double zcg_grid_sum(cooperative_groups::grid_group& grid, double v, double* partials, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
    partials[blockIdx.x] = b;
  }
  grid.sync();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += partials[b];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  const double total = red[32];
  __syncthreads();  // red is reused by the next sum
  return total;
}

// x = Z^-1 r by `iters` steps of Jacobi-preconditioned conjugate gradients
// from x = 0, in one cooperative launch (grid barriers between the phases
// of a step).  r (mean-free) is overwritten by the residual.  The iterates
// are not projected: r stays mean-free because Z annihilates constants, so
// the constant parts p and x pick up change no inner product, and the
// caller projects x once at the end.  partials: 2 gridDim.x doubles.
__global__ void __launch_bounds__(256) zcg_kernel(int np, const double* __restrict__ zs, const double* __restrict__ dinv,
                                                  double* __restrict__ x, double* __restrict__ r,
                                                  double* __restrict__ p, double* __restrict__ q,
                                                  double* __restrict__ partials, int iters) {
  grid_dep_entry();
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ double red[33];
  const int nv = np + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  double* part[2] = {partials, partials + gridDim.x};  // alternate: consecutive uses are a barrier apart
  double loc = 0.0;
  for (int64_t v = t0; v < V; v += st) {
    const double z = dinv[v] * r[v];
    x[v] = 0.0;
    p[v] = z;
    loc = fma(r[v], z, loc);
  }
  double rho = zcg_grid_sum(grid, loc, part[0], red);
  for (int it = 0; it < iters; ++it) {
    grid.sync();  // p complete
    loc = 0.0;
    for (int64_t v = t0; v < V; v += st) {
      const double qv = zrow(zs, p, V, nv, v);
      q[v] = qv;
      loc = fma(p[v], qv, loc);
    }
    const double pq = zcg_grid_sum(grid, loc, part[1], red);
    const double alpha = pq != 0.0 ? rho / pq : 0.0;
    loc = 0.0;
    for (int64_t v = t0; v < V; v += st) {
      x[v] = fma(alpha, p[v], x[v]);
      const double rv = fma(-alpha, q[v], r[v]);
      r[v] = rv;
      loc = fma(rv, dinv[v] * rv, loc);
    }
    const double rho_new = zcg_grid_sum(grid, loc, part[0], red);
    const double beta = rho != 0.0 ? rho_new / rho : 0.0;
    rho = rho_new;
    for (int64_t v = t0; v < V; v += st) p[v] = fma(beta, p[v], dinv[v] * r[v]);
  }
}

}  // namespace

cudaError_t launch_mask_boundary(int n, double* x, cudaStream_t s) {
  KL(launch_k(mask_boundary_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, x));
  return cudaGetLastError();
}

int dot_blocks() { return kRedBlocks; }

cudaError_t launch_dots(int npairs, const double* const* xs, const double* const* ys, int64_t n, double* partials,
                        double* out, double scale, cudaStream_t s) {
  DotPairs p{};
  for (int j = 0; j < npairs; ++j) {
    p.x[j] = xs[j];
    p.y[j] = ys[j];
  }
  switch (npairs) {
    case 1: KL(launch_k(dot_partial_kernel<1>, dim3(kRedBlocks), dim3(kRedThreads), 0, s, p, n, partials)); break;
    case 2: KL(launch_k(dot_partial_kernel<2>, dim3(kRedBlocks), dim3(kRedThreads), 0, s, p, n, partials)); break;
    case 3: KL(launch_k(dot_partial_kernel<3>, dim3(kRedBlocks), dim3(kRedThreads), 0, s, p, n, partials)); break;
    default: return cudaErrorInvalidValue;
  }
  KL(launch_k(reduce_final_kernel, dim3(1), dim3(256), 0, s, partials, kRedBlocks, npairs, out, scale));
  return cudaGetLastError();
}

cudaError_t launch_sum(const double* x, int64_t n, double* partials, double* out, double scale, cudaStream_t s) {
  KL(launch_k(sum_partial_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, x, n, partials));
  KL(launch_k(reduce_final_kernel, dim3(1), dim3(256), 0, s, partials, kRedBlocks, 1, out, scale));
  return cudaGetLastError();
}

cudaError_t launch_vec_op(int op, int64_t n, double* y, const double* a, const double* b, const double* c,
                          const double* scal, cudaStream_t s) {
  KL(launch_k(vec_op_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, op, n, y, a, b, c, scal));
  return cudaGetLastError();
}

cudaError_t launch_minres_init(double* sc, double tol_rel, cudaStream_t s) {
  KL(launch_k(minres_init_kernel, dim3(1), dim3(32), 0, s, sc, tol_rel));
  return cudaGetLastError();
}

cudaError_t launch_block_dot(int nvec, const double* V, int64_t ld, const double* w, int64_t n, double* partials,
                             double* out, cudaStream_t s) {
  KL(launch_k(block_dot_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, nvec, V, ld, w, n, partials));
  KL(launch_k(reduce_final_kernel, dim3(1), dim3(256), 0, s, (const double*)partials, kRedBlocks, nvec, out, 1.0));
  return cudaGetLastError();
}

cudaError_t launch_block_axpy(int nvec, const double* V, int64_t ld, const double* coef, double sign, double* w,
                              int64_t n, cudaStream_t s) {
  KL(launch_k(block_axpy_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, nvec, V, ld, coef, sign, w, n));
  return cudaGetLastError();
}

cudaError_t launch_scale(int64_t n, double* y, const double* a, const double* s_dev, bool recip, cudaStream_t s) {
  KL(launch_k(scale_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, y, a, s_dev, recip ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t launch_colour5(int np, int colour, double* e, cudaStream_t s) {
  KL(launch_k(colour5_kernel, dim3(blocks_for(nverts(np), 256)), dim3(256), 0, s, np, colour, e));
  return cudaGetLastError();
}

cudaError_t launch_scatter_zrow(int np, int colour, const double* y, double* zs, cudaStream_t s) {
  KL(launch_k(scatter_zrow_kernel, dim3(blocks_for(nverts(np), 256)), dim3(256), 0, s, np, colour, y, zs));
  return cudaGetLastError();
}

cudaError_t launch_zcg(int np, const double* zs, const double* dinv, double* x, double* r, double* p, double* q,
                       double* partials, int64_t partials_cap, int iters, cudaStream_t s) {
  int dev = 0, sms = 152, per = 0, coop = 0;
  KL(cudaGetDevice(&dev));
  KL(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  KL(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return cudaErrorNotSupported;
  KL(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, zcg_kernel, 256, 0));
  // every block resident (a cooperative launch fails rather than waits
  // otherwise); two per SM keep the per-step partial sums short
  int64_t blocks = std::min<int64_t>((int64_t)std::min(per, 2) * sms, blocks_for(nverts(np), 256));
  blocks = std::max<int64_t>(blocks, 1);
  if (2 * blocks > partials_cap) return cudaErrorInvalidValue;
  int np_ = np, iters_ = iters;
  const double* zs_ = zs;
  const double* dinv_ = dinv;
  double *x_ = x, *r_ = r, *p_ = p, *q_ = q, *part_ = partials;
  void* args[] = {&np_, &zs_, &dinv_, &x_, &r_, &p_, &q_, &part_, &iters_};
  KL(cudaLaunchCooperativeKernel((const void*)zcg_kernel, dim3((unsigned)blocks), dim3(256), args, 0, s));
  return cudaGetLastError();
}

cudaError_t launch_zdiag_inv(int np, const double* zs, double* dinv, cudaStream_t s) {
  KL(launch_k(zdiag_inv_kernel, dim3(blocks_for(nverts(np), 256)), dim3(256), 0, s, nverts(np), zs, dinv));
  return cudaGetLastError();
}

cudaError_t launch_lanczos(int64_t n, const double* kz, const double* v, double* vold_to_vnew, const double* sc,
                           cudaStream_t s) {
  KL(launch_k(lanczos_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, kz, v, vold_to_vnew, sc));
  return cudaGetLastError();
}

cudaError_t launch_minres_scalars(double* sc, cudaStream_t s) {
  KL(launch_k(minres_scalar_kernel, dim3(1), dim3(32), 0, s, sc));
  return cudaGetLastError();
}

cudaError_t launch_minres_update(int64_t n, const double* z, const double* w, double* wold_to_wnew, double* x,
                                 const double* sc, cudaStream_t s) {
  KL(launch_k(minres_update_kernel, dim3(kRedBlocks), dim3(kRedThreads), 0, s, n, z, w, wold_to_wnew, x, sc));
  return cudaGetLastError();
}

cudaError_t launch_load_vector(int n, const double* fbar, double* b, cudaStream_t s) {
  KL(launch_k(load_vector_kernel, dim3(blocks_for(nverts(n), 128)), dim3(128), 0, s, n, fbar, b));
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(int n, const double* eta, const double* lam, const double* u, double* g,
                               cudaStream_t s) {
  KL(launch_k(sensitivity_kernel, dim3(blocks_for((int64_t)n * n * n, 128)), dim3(128), 0, s, n, eta, lam, u, g));
  return cudaGetLastError();
}

}  // namespace agca
