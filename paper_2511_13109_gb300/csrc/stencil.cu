// Matrix-free operator application on a Kuhn cube grid, fused with the
// smoother and residual epilogues (Eq. 2.3 on the finest level, the
// heterogeneous AGCA operator of Eq. 2.9 on coarse levels).
//
// Element action.  For a tetrahedron with nodal values x_a (a = 0..3) the
// scaled displacement gradient is Gx = sum_a x_a (x) G_a; along the Kuhn path
// its column p_k is the edge difference x_{k+1} - x_k.  With S = Gx + Gx^T,
// the element contribution to local vertex a is y_a = eta (h/6) S G_a, i.e.
// with the edge "fluxes" F_k = eta (h/6) S[:, p_k]:
//   y_0 = -F_0, y_1 = F_0 - F_1, y_2 = F_1 - F_2, y_3 = F_2.
// This equals A_e x_e for the element matrix of Eq. 3.5 and needs only
// differences of nodal values.
//
// Tiling (GB300): a CTA of BX x BY threads owns a (BX-1) x (BY-1) column of
// vertices and marches through a chunk of z-planes.  Thread (tx, ty) computes
// the cube whose (1,1) xy-corner is its own vertex.  Per cube layer the CTA
// stages the next vertex plane of x in shared memory (coalesced rows), each
// thread computes its cube's 6 tetrahedra once, corner contributions are
// combined along x with warp shuffles and along y through shared memory, and
// each owner finishes its vertex in registers (owner-computes: no atomics,
// deterministic summation order).  HBM traffic per vertex is one read of x,
// the 6 element coefficients and the epilogue vectors, and one write.
#include "agca_internal.cuh"

namespace agca {

namespace {

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

template <typename T>
__device__ __forceinline__ void load6(const T* p, T (&c)[6]);
template <>
__device__ __forceinline__ void load6<float>(const float* p, float (&c)[6]) {
  const float2* q = reinterpret_cast<const float2*>(p);
  float2 a = __ldg(q), b = __ldg(q + 1), d = __ldg(q + 2);
  c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y; c[4] = d.x; c[5] = d.y;
}
template <>
__device__ __forceinline__ void load6<double>(const double* p, double (&c)[6]) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1), d = __ldg(q + 2);
  c[0] = a.x; c[1] = a.y; c[2] = b.x; c[3] = b.y; c[4] = d.x; c[5] = d.y;
}

template <typename TS, typename T, int BX, int BY, int MODE, bool COARSE>
__global__ void __launch_bounds__(BX* BY) stencil_kernel(const LevelOp<T> op, const StencilArgs<TS> a, const int zch) {
  constexpr int NC = (MODE == ST_STOKES) ? 4 : 3;  // tile fields: velocity (+ fine-grid pressure)
  const int n = op.n;
  const int nv = n + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const int x0 = blockIdx.x * (BX - 1), y0 = blockIdx.y * (BY - 1);
  const int z0 = blockIdx.z * zch;
  const int z1 = min(z0 + zch, nv);
  const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;
  const bool cube_xy = (cx >= 0) && (cx < n) && (cy >= 0) && (cy < n);
  const int vx = x0 + tx, vy = y0 + ty;
  const bool owner = (tx < BX - 1) && (ty < BY - 1) && (vx < nv) && (vy < nv);
  const bool inner_xy = (vx > 0) && (vx < n) && (vy > 0) && (vy < n);

  __shared__ T xs[NC][BY + 1][BX + 1];
  __shared__ T cs[2][NC][BY][BX];

  auto load_plane = [&](int z) {
    const bool zin = (z > 0) && (z < n);
    for (int idx = tid; idx < (BX + 1) * (BY + 1); idx += BX * BY) {
      const int lx = idx % (BX + 1), ly = idx / (BX + 1);
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
      const bool in = zin && gx > 0 && gx < n && gy > 0 && gy < n;
      const int64_t v = gx + (int64_t)nv * (gy + (int64_t)nv * z);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T val = T(0);
        if (in) {
          if (MODE == ST_CHEB_PRE)
            val = (T)(a.s2 * __ldg(a.invD + c * V + v) * __ldg(a.b + c * V + v));
          else
            val = (T)__ldg(a.x + c * V + v);
        }
        xs[c][ly][lx] = val;
      }
      if (MODE == ST_STOKES) {  // fine-grid pressure q = P p lives on every vertex
        const bool qin = z >= 0 && z <= n && gx >= 0 && gx <= n && gy >= 0 && gy <= n;
        xs[NC - 1][ly][lx] = qin ? (T)__ldg(a.q + v) : T(0);
      }
    }
  };

  T Xl[4][NC], Xh[4][NC];
  const int zs = z0 - 1;
  load_plane(zs);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < NC; ++c) Xl[q][c] = xs[c][ty + (q >> 1)][tx + (q & 1)];
  __syncthreads();

  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  for (int k = zs; k < z1; ++k) {
    if (k + 1 <= n) load_plane(k + 1);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) Xh[q][c] = (k + 1 <= n) ? xs[c][ty + (q >> 1)][tx + (q & 1)] : T(0);

    T Y[8][NC];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) Y[q][c] = T(0);

    if (cube_xy && k >= 0 && k < n) {
      const int64_t cube = cx + (int64_t)n * (cy + (int64_t)n * k);
      T cf[6];
      load6<T>(op.coef + 6 * cube, cf);
#pragma unroll
      for (int t = 0; t < 6; ++t) cf[t] *= op.h6;
      if constexpr (COARSE) {
        int32_t f[6];
        const int2* fp = reinterpret_cast<const int2*>(op.fidx + 6 * cube);
        int2 f01 = __ldg(fp), f23 = __ldg(fp + 1), f45 = __ldg(fp + 2);
        f[0] = f01.x; f[1] = f01.y; f[2] = f23.x; f[3] = f23.y; f[4] = f45.x; f[5] = f45.y;
#pragma unroll
        for (int t = 0; t < 6; ++t)
          if (f[t] >= 0) cf[t] = T(0);
        cube_dca<T, NC>(Xl, Xh, cf, Y);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          if (f[t] >= 0) {
            const T* M = op.gca + (int64_t)f[t] * 144;
            const T sc = op.gscale ? op.gscale[f[t]] : T(1);
            T xl[12];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const int q = tet_corner(t, b);
                xl[d * 4 + b] = (q & 4) ? Xh[q & 3][d] : Xl[q & 3][d];
              }
#pragma unroll
            for (int r = 0; r < 12; ++r) {
              T yr = T(0);
#pragma unroll
              for (int s2 = 0; s2 < 12; ++s2) yr = fma(M[r * 12 + s2], xl[s2], yr);
              const int q = tet_corner(t, r & 3);
              Y[q][r >> 2] = fma(sc, yr, Y[q][r >> 2]);
            }
          }
        }
      } else if constexpr (MODE == ST_STOKES) {
        cube_stokes<T>(Xl, Xh, cf, op.hq, Y);
      } else {
        cube_dca<T, NC>(Xl, Xh, cf, Y);
      }
    }

    // combine along x (lane tx+1 holds the neighbouring cube), then along y
    T s1[2][NC];
#pragma unroll
    for (int qz = 0; qz < 2; ++qz)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        // corners (qx, qy, qz): index qx + 2 qy + 4 qz
        const T from_right_y1 = __shfl_down_sync(0xffffffffu, Y[4 * qz + 2][c], 1);
        const T from_right_y0 = __shfl_down_sync(0xffffffffu, Y[4 * qz + 0][c], 1);
        s1[qz][c] = Y[4 * qz + 3][c] + from_right_y1;           // row qy = 1 (own vertex row)
        cs[qz][c][ty][tx] = Y[4 * qz + 1][c] + from_right_y0;   // row qy = 0, for thread ty-1
      }
    __syncthreads();

    if (owner) {
      T yk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        yk[c] = acc[c] + (s1[0][c] + cs[0][c][ty + 1][tx]);
        acc[c] = s1[1][c] + cs[1][c][ty + 1][tx];
      }
      if (k >= z0) {
        const int64_t v = vx + (int64_t)nv * (vy + (int64_t)nv * k);
        const bool inner = inner_xy && k > 0 && k < n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int64_t i = c * V + v;
          TS o = TS(0);
          if (inner) {
            const TS xo = (TS)Xl[3][c];  // own vertex value on plane k
            const TS y = (TS)yk[c];
            if (MODE == ST_APPLY || MODE == ST_STOKES) {
              o = y;
            } else if (MODE == ST_RESID) {
              o = __ldg(a.b + i) - y;
            } else if (MODE == ST_CHEB_FIRST) {
              o = xo + a.s0 * __ldg(a.invD + i) * (__ldg(a.b + i) - y);
            } else if (MODE == ST_CHEB_STEP) {
              const TS xp = a.xprev[i];
              o = xo + a.s0 * (xo - xp) + a.s1 * __ldg(a.invD + i) * (__ldg(a.b + i) - y);
            } else {  // ST_CHEB_PRE: x1 = s2 D^-1 b staged in the tile, x0 = 0
              o = xo + a.s0 * xo + a.s1 * __ldg(a.invD + i) * (__ldg(a.b + i) - y);
            }
          }
          a.out[i] = o;
        }
        if (MODE == ST_STOKES) a.out2[v] = (TS)yk[NC - 1];  // (B_f u) on every fine vertex
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) Xl[q][c] = Xh[q][c];
  }
}

template <typename TS, typename T, int BX, int BY, bool COARSE>
cudaError_t launch_mode(int mode, const LevelOp<T>& op, const StencilArgs<TS>& a, cudaStream_t s) {
  const int nv = op.n + 1;
  const int gx = (nv + BX - 2) / (BX - 1), gy = (nv + BY - 2) / (BY - 1);
  int gz = (608 + gx * gy - 1) / (gx * gy);
  int zch = (nv + gz - 1) / gz;
  if (zch < 4) zch = 4;
  if (zch > nv) zch = nv;
  gz = (nv + zch - 1) / zch;
  dim3 grid(gx, gy, gz), block(BX, BY);
  switch (mode) {
    case ST_APPLY: stencil_kernel<TS, T, BX, BY, ST_APPLY, COARSE><<<grid, block, 0, s>>>(op, a, zch); break;
    case ST_RESID: stencil_kernel<TS, T, BX, BY, ST_RESID, COARSE><<<grid, block, 0, s>>>(op, a, zch); break;
    case ST_CHEB_FIRST: stencil_kernel<TS, T, BX, BY, ST_CHEB_FIRST, COARSE><<<grid, block, 0, s>>>(op, a, zch); break;
    case ST_CHEB_STEP: stencil_kernel<TS, T, BX, BY, ST_CHEB_STEP, COARSE><<<grid, block, 0, s>>>(op, a, zch); break;
    case ST_CHEB_PRE: stencil_kernel<TS, T, BX, BY, ST_CHEB_PRE, COARSE><<<grid, block, 0, s>>>(op, a, zch); break;
    case ST_STOKES:
      if (COARSE) return cudaErrorInvalidValue;
      stencil_kernel<TS, T, BX, BY, ST_STOKES, false><<<grid, block, 0, s>>>(op, a, zch);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

template <typename TS, typename T>
cudaError_t launch_stencil(int mode, const LevelOp<T>& op, const StencilArgs<TS>& a, cudaStream_t s) {
  if (op.fidx) return launch_mode<TS, T, 32, 8, true>(mode, op, a, s);
  return launch_mode<TS, T, 32, 8, false>(mode, op, a, s);
}

template cudaError_t launch_stencil<float, float>(int, const LevelOp<float>&, const StencilArgs<float>&,
                                                  cudaStream_t);
template cudaError_t launch_stencil<double, double>(int, const LevelOp<double>&, const StencilArgs<double>&,
                                                    cudaStream_t);
template cudaError_t launch_stencil<double, float>(int, const LevelOp<float>&, const StencilArgs<double>&,
                                                   cudaStream_t);

}  // namespace agca
