// Per-point device arithmetic shared by the single-problem kernels and the
// batched kernels, so that both compute each value with the same operations
// in the same order (a batched cycle is bit-for-bit equal to the cycle of one
// problem).
#pragma once

#include "agca_internal.cuh"

namespace agca {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// ------------------------------------------------------------ element action
// For a tetrahedron with nodal values x_a (a = 0..3) the scaled displacement
// gradient is Gx = sum_a x_a (x) G_a; along the Kuhn path its column p_k is the
// edge difference x_{k+1} - x_k.  With S = Gx + Gx^T, the element
// contribution to local vertex a is y_a = eta (h/6) S G_a, i.e. with the edge
// "fluxes" F_k = eta (h/6) S[:, p_k]:
//   y_0 = -F_0, y_1 = F_0 - F_1, y_2 = F_1 - F_2, y_3 = F_2.
// This equals A_e x_e for the element matrix of Eq. 3.5 and needs only
// differences of nodal values.  Xl / Xh: the cube's corner values on its
// lower / upper z-plane (index qx + 2 qy), c[t]: eta_t h / 6 per type; the
// contributions are added to Y[corner qx + 2 qy + 4 qz][component].
template <typename T, int NC>
__device__ __forceinline__ void cube_dca(const T (&Xl)[4][NC], const T (&Xh)[4][NC], const T (&c)[6], T (&Y)[8][NC]) {
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    T G[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int qa = tet_corner(t, k), qb = tet_corner(t, k + 1), m = perm(t, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T xb = (qb & 4) ? Xh[qb & 3][i] : Xl[qb & 3][i];
        const T xa = (qa & 4) ? Xh[qa & 3][i] : Xl[qa & 3][i];
        G[i][m] = xb - xa;
      }
    }
    const T ct = c[t], nct = -c[t], c2 = c[t] + c[t], nc2 = -c2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int qa = tet_corner(t, k), qb = tet_corner(t, k + 1), m = perm(t, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i == m) {
          Y[qb][i] = fma(c2, G[m][m], Y[qb][i]);
          Y[qa][i] = fma(nc2, G[m][m], Y[qa][i]);
        } else {
          const T sv = G[i][m] + G[m][i];
          Y[qb][i] = fma(ct, sv, Y[qb][i]);
          Y[qa][i] = fma(nct, sv, Y[qa][i]);
        }
      }
    }
  }
}

// Velocity block plus the divergence pieces on the finest grid: with the
// fine-grid pressure q = P p (component 3 of the tile) the element adds
// -(h^2/6) qbar_T G_a to the velocity row of vertex a (that is -B_f^T q with
// B_f the P1-P1 divergence, |T| g = (h^2/6) G) and (h^2/24) tr(Gx) to the
// scalar row of each vertex ((|T|/4) div u).  c[t] = eta_t h/6, hq = h^2/6.
template <typename T>
__device__ __forceinline__ void cube_stokes(const T (&Xl)[4][4], const T (&Xh)[4][4], const T (&c)[6], const T hq,
                                            T (&Y)[8][4]) {
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    T G[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int qa = tet_corner(t, k), qb = tet_corner(t, k + 1), m = perm(t, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T xb = (qb & 4) ? Xh[qb & 3][i] : Xl[qb & 3][i];
        const T xa = (qa & 4) ? Xh[qa & 3][i] : Xl[qa & 3][i];
        G[i][m] = xb - xa;
      }
    }
    T qsum = T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int q = tet_corner(t, a);
      qsum += (q & 4) ? Xh[q & 3][3] : Xl[q & 3][3];
    }
    const T pq = T(0.25) * hq * qsum;  // (h^2/6) qbar
    const T ct = c[t], nct = -c[t], c2 = c[t] + c[t];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int qa = tet_corner(t, k), qb = tet_corner(t, k + 1), m = perm(t, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i == m) {
          const T dm = fma(c2, G[m][m], -pq);
          Y[qb][i] += dm;
          Y[qa][i] -= dm;
        } else {
          const T sv = G[i][m] + G[m][i];
          Y[qb][i] = fma(ct, sv, Y[qb][i]);
          Y[qa][i] = fma(nct, sv, Y[qa][i]);
        }
      }
    }
    const T dv = T(0.25) * hq * (G[0][0] + G[1][1] + G[2][2]);  // (|T|/4) div u
#pragma unroll
    for (int a = 0; a < 4; ++a) Y[tet_corner(t, a)][3] += dv;
  }
}

// The pressure coupling of cube_stokes alone (the viscous part comes from
// the edge form): per tetrahedron -(h^2/6) qbar along the m-component of its
// path edges and (|T|/4) div u at its corners, in component 3
template <typename T>
__device__ __forceinline__ void cube_stokes_b(const T (&Xl)[4][4], const T (&Xh)[4][4], const T hq, T (&Y)[8][4]) {
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    T qsum = T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int q = tet_corner(t, a);
      qsum += (q & 4) ? Xh[q & 3][3] : Xl[q & 3][3];
    }
    const T pq = T(0.25) * hq * qsum;  // (h^2/6) qbar
    T tr = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int qa = tet_corner(t, k), qb = tet_corner(t, k + 1), m = perm(t, k);
      const T xb = (qb & 4) ? Xh[qb & 3][m] : Xl[qb & 3][m];
      const T xa = (qa & 4) ? Xh[qa & 3][m] : Xl[qa & 3][m];
      tr += xb - xa;  // G[m][m]
      Y[qb][m] -= pq;
      Y[qa][m] += pq;
    }
    const T dv = T(0.25) * hq * tr;  // (|T|/4) div u
#pragma unroll
    for (int a = 0; a < 4; ++a) Y[tet_corner(t, a)][3] += dv;
  }
}

// Flagged elements of a coarse level: y_e = s_e A_e x_e (Eq. 2.9, stored
// Galerkin part), one thread per (element, row), written to op.ye for the
// stencil kernel to scatter.  x follows the stencil's input convention
// (boundary entries are zero; CHEB_PRE stages x = s2 D^-1 b).  A separate
// launch spreads the clustered flagged elements over the whole GPU; inside
// the stencil they would serialise in the few warps whose cubes hold them.
// xval(d, v): the operator input (component d, vertex v) on an interior vertex
template <typename T, typename XF>
__device__ __forceinline__ void gca_row_of(const LevelOp<T>& op, const int64_t id, XF xval) {
  const int64_t f = id / 12;
  const int r = (int)(id - f * 12);
  const int e = op.list[f];
  const int cube = e / 6, t = e - cube * 6;
  const int n = op.n, nv = n + 1;
  const int q0 = cube / n, ci = cube - q0 * n, ck = q0 / n, cj = q0 - ck * n;
  const T* M = op.gca + f * 144 + r * 12;
  T acc = T(0);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int q = tet_corner(t, b);
    const int i = ci + (q & 1), j = cj + ((q >> 1) & 1), k = ck + ((q >> 2) & 1);
    const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
    const int v = i + nv * (j + nv * k);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xv = inner ? (T)xval(d, v) : T(0);
      acc = fma(M[d * 4 + b], xv, acc);
    }
  }
  op.ye[f * 12 + r] = op.gscale ? op.gscale[f] * acc : acc;
}

template <typename TS, typename T, bool PRE>
__device__ __forceinline__ void gca_row(const LevelOp<T>& op, const StencilArgs<TS>& a, const int64_t id) {
  const int V = (op.n + 1) * (op.n + 1) * (op.n + 1);
  gca_row_of<T>(op, id, [&](int d, int v) -> TS {
    if (PRE) return a.s2 * __ldg(a.invD + d * V + v) * __ldg(a.b + d * V + v);
    return __ldg(a.x + d * V + v);
  });
}

// Stored-Galerkin part of a coarse operator at interior vertex (i, j, k) of a
// grid with n cubes per axis (Remark 5): g += sum_o S[o] x(v + o) over the 15
// Kuhn offsets, S = op.sten + 135 s for the vertex's stencil index s; Dirichlet
// neighbours contribute nothing.  xval(d, v'): operator input (component d,
// vertex v').  Fixed order: offset, then component.
template <typename T, typename XF>
__device__ __forceinline__ void stencil_gather(const LevelOp<T>& op, const int s, const int i, const int j, const int k,
                                               XF xval, T (&g)[3]) {
  const int n = op.n, nv = n + 1;
  const T* S = op.sten + (int64_t)s * 135;
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int o = 0; o < 15; ++o) {
    const int a = i + kuhn_offset_comp(o, 0), b = j + kuhn_offset_comp(o, 1), c = k + kuhn_offset_comp(o, 2);
    if (a <= 0 || b <= 0 || c <= 0 || a >= n || b >= n || c >= n) continue;
    const int w = a + nv * (b + nv * c);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T xv = (T)xval(d, w);
#pragma unroll
      for (int r = 0; r < 3; ++r) acc[r] = fma(S[o * 9 + r * 3 + d], xv, acc[r]);
    }
  }
  const T sc = op.sscale ? op.sscale[s] : T(1);
#pragma unroll
  for (int r = 0; r < 3; ++r) g[r] = op.sscale ? sc * acc[r] : acc[r];
}

// Result of a fused stencil mode at one vertex from the operator value y =
// (A x)_v, the vertex's own iterate xo, rhs eb, inverse diagonal ed and
// previous iterate ep (Chebyshev steps of Sec. 4; CHEB_PRE starts from x0 = 0
// with xo = x1 = s2 D^-1 b).
template <int MODE, typename TS>
__device__ __forceinline__ TS stencil_epilogue(const TS xo, const TS y, const TS eb, const TS ed, const TS ep,
                                               const TS s0, const TS s1) {
  if (MODE == ST_APPLY || MODE == ST_STOKES) return y;
  if (MODE == ST_STOKES_B) return eb + y;
  if (MODE == ST_RESID) return eb - y;
  if (MODE == ST_CHEB_FIRST) return xo + s0 * ed * (eb - y);
  if (MODE == ST_CHEB_STEP) return xo + s0 * (xo - ep) + s1 * ed * (eb - y);
  return xo + s0 * xo + s1 * ed * (eb - y);  // ST_CHEB_PRE
}

// ------------------------------------------------------------------ transfers
// Linear interpolation between Kuhn grids and its transpose (Sec. 2.1).  Every
// fine vertex is either 2i (a coarse vertex) or the midpoint 2i + d of the
// coarse Kuhn edge (i, i + d), d in {0,1}^3 \ {0} (Kuhn edges join corners
// whose difference has entries of one sign), hence
//   (P e)(2i) = e(i),  (P e)(2i + d) = (e(i) + e(i + d)) / 2,
//   (P^T r)(i) = r(2i) + 1/2 sum_d [ r(2i + d) + r(2i - d) ].
// The weights are known a priori and never stored.

// scale * (P^T r)(I, J, K) for one component r of the fine grid (nf cubes);
// 0 on the coarse boundary when mask is set
template <typename T>
__device__ __forceinline__ T restrict_point(const int nf, const bool mask, const T scale, const T* r, const int I,
                                            const int J, const int K) {
  const int nc = nf / 2, nvf = nf + 1;
  if (mask && (I == 0 || J == 0 || K == 0 || I == nc || J == nc || K == nc)) return T(0);
  const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
  T acc = T(0);
#pragma unroll
  for (int d = 1; d < 8; ++d) {
    const int dx = d & 1, dy = (d >> 1) & 1, dz = (d >> 2) & 1;
    if (fi + dx <= nf && fj + dy <= nf && fk + dz <= nf)
      acc += __ldg(r + (fi + dx) + nvf * ((fj + dy) + nvf * (fk + dz)));
    if (fi - dx >= 0 && fj - dy >= 0 && fk - dz >= 0)
      acc += __ldg(r + (fi - dx) + nvf * ((fj - dy) + nvf * (fk - dz)));
  }
  return scale * (__ldg(r + fi + nvf * (fj + nvf * fk)) + T(0.5) * acc);
}

// (P e)(i, j, k) for one component e of the coarse grid of a fine grid with
// nf cubes; 0 on the fine boundary when mask is set
template <typename T>
__device__ __forceinline__ T prolong_point(const int nf, const bool mask, const T* e, const int i, const int j,
                                           const int k) {
  if (mask && (i == 0 || j == 0 || k == 0 || i == nf || j == nf || k == nf)) return T(0);
  const int nvc = nf / 2 + 1;
  const int I = i >> 1, J = j >> 1, K = k >> 1, dx = i & 1, dy = j & 1, dz = k & 1;
  const T e0 = __ldg(e + I + nvc * (J + nvc * K));
  if (!(dx | dy | dz)) return e0;
  // explicit roundings: x + (P e) then rounds the same in every kernel that adds it
  return mul_rn(T(0.5), add_rn(e0, __ldg(e + (I + dx) + nvc * ((J + dy) + nvc * (K + dz)))));
}

// ------------------------------------------------------------- coarsest solve
// z = L^-T L^-1 r on the interior DoFs of the coarsest grid (n cubes), by one
// thread block: one warp per row of each triangular product with coalesced
// row reads (X row-major for t = X r, X column-major for z = X^T t); r, z are
// full-grid vectors, sm holds 2 * 3 (n-1)^3 doubles.  Every row's sum is
// formed by one warp in a fixed order, whatever the block size.
template <typename T>
__device__ __forceinline__ void coarse_solve_block(const int n, const double* __restrict__ xcm,
                                                   const double* __restrict__ xrm, const T* r, T* z, double* sm) {
  const int nv = n + 1, ni = n - 1;
  const int64_t V = nverts(n);
  const int nI = ni * ni * ni, m = 3 * nI;
  double* rs = sm;
  double* ts = sm + m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < m; q += blockDim.x) {
    const int c = q / nI, iv = q % nI;
    const int i = 1 + iv % ni, j = 1 + (iv / ni) % ni, k = 1 + iv / (ni * ni);
    rs[q] = (double)__ldg(r + c * V + i + (int64_t)nv * (j + (int64_t)nv * k));
  }
  __syncthreads();
  for (int q = warp; q < m; q += nw) {
    double s = 0.0;
    for (int p = lane; p <= q; p += 32) s = fma(xrm[(int64_t)q * m + p], rs[p], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) ts[q] = s;
  }
  __syncthreads();
  for (int q = warp; q < m; q += nw) {
    double s = 0.0;
    for (int p = q + lane; p < m; p += 32) s = fma(xcm[(int64_t)q * m + p], ts[p], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) rs[q] = s;
  }
  __syncthreads();
  for (int id = threadIdx.x; id < 3 * (int)V; id += blockDim.x) {
    const int c = id / (int)V, v = id - c * (int)V;
    const int t = v / nv, i = v - t * nv, k = t / nv, j = t - k * nv;
    const bool inner = i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
    T out = T(0);
    if (inner) out = (T)rs[c * nI + (i - 1) + ni * ((j - 1) + ni * (k - 1))];
    z[id] = out;
  }
}

}  // namespace agca
