// FP64 finest-level operator in edge form (Eq. 2.3 with the element matrices
// of Eq. 3.5), fused with the smoother and residual epilogues.
//
// On a Kuhn grid every edge of a tetrahedron's path is an axis edge of the
// grid, and the element action reduces to fluxes along those edges (see
// cube_dca in device_ops.cuh): with S = Gx + Gx^T, the tetrahedron t adds
// F = eta_t S[:, m] to the end vertex of its m-edge and subtracts it from the
// start vertex.  Summing over the 6 tetrahedra around a grid edge E = (v, m)
// (v to v + e_m), with d_E = x(v + e_m) - x(v):
//   F_E[m] = 2 H_E d_E[m],
//   F_E[c] = H_E d_E[c] + sum_{t around E} eta_t d_{e_t(c)}[m]   (c != m),
// where H_E is the sum of eta_t around E and e_t(c) the c-edge of t's path,
// and the operator is y_v = (h/6) sum_m (F_(v - e_m, m) - F_(v, m)).
// Per vertex this is 9 edge differences, 3 x 16 flux products and 15
// divergence terms: about 75 FP64 instructions against about 190 for the
// per-tetrahedron form.  FP64 arithmetic is the bound of this operator on
// GB300 (one FP64 fused multiply-add per 64 FP32 ones), so the per-vertex
// edge sums H (3 per vertex) are formed once per set-up (edge_sum_kernel)
// and the neighbours' edge differences are shared through shared memory
// instead of being recomputed.
//
// Tiling: a CTA of 32 x 8 threads, thread (tx, ty) <-> vertex column
// (x0 - 1 + tx, y0 - 1 + ty), marches a chunk of z-planes.  Per plane k it
// stages the x plane k + 2 (cp.async, one plane ahead), forms the edge
// differences of plane k + 1 for its (34 x 10)-vertex tile, computes the three
// fluxes of its vertex's forward edges from the differences of planes
// k - 1..k + 1 and the coefficients of cube layers k - 1, k, exchanges the x
// and y fluxes through shared memory (the z flux stays in registers for the
// next plane), and the threads with tx, ty >= 1 finish their vertex
// (owner-computes: no atomics; every vertex sums its fluxes in one fixed
// order, whatever the tile shape or z-chunk).
#include <algorithm>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

constexpr int EBX = 32, EBY = 8, ENT = EBX * EBY;
constexpr int XW = EBX + 3, XH = EBY + 3, XT = XW * XH;  // x tile: vertices (x0-2 .., y0-2 ..)
constexpr int DW = EBX + 2, DH = EBY + 2, DT = DW * DH;  // edge-difference tile
constexpr int CW = EBX + 1, CH = EBY + 1, CT = CW * CH;  // cube tile: origins (x0-2 .., y0-2 ..)
constexpr int DRING = 84;                                // halo entries of the difference tile
// off-diagonal edge-difference components kept in shared memory:
// (edge axis, component) = xy, xz, yx, yz, zx, zy
enum { XY = 0, XZ, YX, YZ, ZX, ZY };

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int MODE>
__host__ __device__ constexpr size_t edge_smem_elems() {
  // x ring [3][3][XT] (+ D^-1 ring for the step from zero), difference ring
  // [3][6][DT], coefficient ring [2][6][CT], y-flux exchange [3][ENT]: in
  // FP64 111 KB (two CTAs per SM) or, with the D^-1 ring, 139 KB; in FP32
  // half of that (three CTAs per SM)
  return (size_t)(MODE == ST_CHEB_PRE ? 2 : 1) * 3 * 3 * XT + (size_t)3 * 6 * DT + (size_t)2 * 6 * CT +
         (size_t)3 * ENT;
}
// resident CTAs per SM the shared memory (and, in FP32, the register file) allows
// (the FP32 form is not used: its per-copy staging arithmetic saturated the
// integer pipe, 1600 instructions per vertex against 530 for the per-cube kernel)
template <typename T, int MODE>
__host__ __device__ constexpr int edge_min_blocks() {
  return sizeof(T) == 4 ? 3 : (MODE == ST_CHEB_PRE ? 1 : 2);
}
template <typename T>
__device__ __forceinline__ void cpT(T* smem, const T* gmem, bool ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int src = ok ? (int)sizeof(T) : 0;
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src) : "memory");
}

// difference-tile coordinates of halo entry r (0..83): rows 0 and DH-1, then
// columns 0 and DW-1 of the rows between
__device__ __forceinline__ void ring_entry(int r, int& i, int& j) {
  if (r < 2 * DW) {
    i = r % DW;
    j = r < DW ? 0 : DH - 1;
  } else {
    const int q = r - 2 * DW;
    i = (q & 1) ? DW - 1 : 0;
    j = 1 + (q >> 1);
  }
}

template <typename T, int MODE>
__device__ __forceinline__ void stencil_edge_block(const LevelOp<T>& op, const StencilArgs<T>& a, const int zch,
                                                   const int x0, const int y0, const int bz, const int tid,
                                                   T* __restrict__ sm) {
  const int n = op.n, nv = n + 1, V = nv * nv * nv;
  const int tx = tid & (EBX - 1), ty = tid >> 5;
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const int za = bz * zch, zb = min(za + zch, nv);
  const bool owner = tx >= 1 && ty >= 1 && gx <= n && gy <= n;
  const bool inner_xy = gx > 0 && gx < n && gy > 0 && gy < n;
  constexpr bool PRE = MODE == ST_CHEB_PRE;

  T* xs = sm;                                    // [3][3][XT]
  T* xa = xs + 3 * 3 * XT;                       // PRE: D^-1 ring [3][3][XT]
  T* ds = xa + (PRE ? 3 * 3 * XT : 0);           // [3][6][DT]
  T* cs = ds + 3 * 6 * DT;                       // [2][6][CT]
  T* fy = cs + 2 * 6 * CT;                       // [3][ENT]

  const int zs = za - 2;  // planes zs + i use ring slot i mod 3, cube layers zs + i slot i mod 2
  auto slot = [&](int p) { return (p - zs) % 3; };
  auto cslot = [&](int q) { return (q - zs) & 1; };

  // stage x plane p (PRE: b and D^-1) for the x tile; Dirichlet and outside
  // vertices read as zero
  auto issue_x = [&](int p) {
    T* dst = xs + slot(p) * 3 * XT;
    T* dsa = xa + slot(p) * 3 * XT;
    const bool zin = p > 0 && p < n;
    for (int e = tid; e < 3 * XT; e += ENT) {
      const int c = e / XT, r = e - c * XT;
      const int j = r / XW, i = r - j * XW;
      const int vx = x0 - 2 + i, vy = y0 - 2 + j;
      const bool in = zin && vx > 0 && vx < n && vy > 0 && vy < n;
      const int g = in ? c * V + vx + nv * (vy + nv * p) : 0;
      if (PRE) {
        cpT(dst + e, a.b + g, in);
        cpT(dsa + e, a.invD + g, in);
      } else {
        cpT(dst + e, a.x + g, in);
      }
    }
  };
  // PRE: the first Chebyshev iterate x1 = (s2 D^-1) b of the entries this
  // thread staged (the same operations as the per-tetrahedron kernel)
  auto convert_x = [&](int p) {
    if (!PRE) return;
    T* dst = xs + slot(p) * 3 * XT;
    const T* dsa = xa + slot(p) * 3 * XT;
    for (int e = tid; e < 3 * XT; e += ENT) dst[e] = a.s2 * dsa[e] * dst[e];
  };
  // stage the 6 coefficients of every cube of the cube tile on layer q
  auto issue_coef = [&](int q) {
    T* dst = cs + cslot(q) * 6 * CT;
    const bool qin = q >= 0 && q < n;
    for (int e = tid; e < 6 * CT; e += ENT) {
      const int j = e / (6 * CW), r = e - j * 6 * CW;
      const int i = r / 6, t = r - i * 6;
      const int cx = x0 - 2 + i, cy = y0 - 2 + j;
      const bool in = qin && cx >= 0 && cx < n && cy >= 0 && cy < n;
      const int g = in ? 6 * (cx + n * (cy + n * q)) + t : 0;
      cpT(dst + t * CT + j * CW + i, (op.coefm ? op.coefm : op.coef) + g, in);
    }
  };
  // edge differences of plane p from x planes p, p + 1: difference-tile
  // entry (i, j) <-> x-tile entry (i, j); the 6 off-diagonal components go to
  // the ring, the thread's own vertex (entry (tx+1, ty+1)) keeps all 9
  auto diffs_at = [&](const T* xl, const T* xh, int i, int j, T (&d)[3][3]) {
    const int e = j * XW + i;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T x0v = xl[c * XT + e];
      d[0][c] = xl[c * XT + e + 1] - x0v;
      d[1][c] = xl[c * XT + e + XW] - x0v;
      d[2][c] = xh[c * XT + e] - x0v;
    }
  };
  auto store_d = [&](T* dp, int i, int j, const T (&d)[3][3]) {
    const int e = j * DW + i;
    dp[XY * DT + e] = d[0][1];
    dp[XZ * DT + e] = d[0][2];
    dp[YX * DT + e] = d[1][0];
    dp[YZ * DT + e] = d[1][2];
    dp[ZX * DT + e] = d[2][0];
    dp[ZY * DT + e] = d[2][1];
  };
  auto compute_d = [&](int p, T (&own)[3][3]) {
    const T* xl = xs + slot(p) * 3 * XT;
    const T* xh = xs + slot(p + 1) * 3 * XT;
    T* dp = ds + slot(p) * 6 * DT;
    diffs_at(xl, xh, tx + 1, ty + 1, own);
    store_d(dp, tx + 1, ty + 1, own);
    if (tid < DRING) {
      int i, j;
      ring_entry(tid, i, j);
      T d[3][3];
      diffs_at(xl, xh, i, j, d);
      store_d(dp, i, j, d);
    }
  };

  // prologue: x planes za-2 .. za, coefficient layers za-2, za-1; edge
  // differences of planes za-2 and za-1
  issue_x(zs);
  issue_x(zs + 1);
  issue_x(zs + 2);
  issue_coef(zs);
  issue_coef(zs + 1);
  cp_commit();
  cp_wait_all();
  convert_x(zs);
  convert_x(zs + 1);
  convert_x(zs + 2);
  __syncthreads();
  T dcur[3][3], dnext[3][3];
  compute_d(zs, dnext);
  compute_d(zs + 1, dcur);
  __syncthreads();
  issue_x(za + 1);
  cp_commit();

  const int I = tx + 1, J = ty + 1;  // own entry of the difference and cube tiles
  T fzp[3] = {T(0), T(0), T(0)};    // flux of the z edge below the vertex

  for (int k = za - 1; k < zb; ++k) {
    cp_wait_all();
    convert_x(k + 2);
    __syncthreads();  // x plane k+2 and coefficient layer k staged; ring slots of k-2 free
    compute_d(k + 1, dnext);
    __syncthreads();  // differences of plane k+1 visible; x slot of plane k free
    if (k + 1 < zb) issue_x(k + 3);
    cp_commit();

    // own edge sums and epilogue inputs of plane k, read early
    const bool kin = k >= 0 && k <= n && gx >= 0 && gx <= n && gy >= 0 && gy <= n;
    const int vo = kin ? gx + nv * (gy + nv * k) : 0;
    T H[3] = {T(0), T(0), T(0)};
    if (kin) {
#pragma unroll
      for (int m = 0; m < 3; ++m) H[m] = __ldg(op.hedge + m * V + vo);
    }
    const bool out_k = owner && k >= za;
    const bool inner = out_k && inner_xy && k > 0 && k < n;
    T eb[3] = {T(0), T(0), T(0)}, ed[3] = {T(0), T(0), T(0)}, ep[3] = {T(0), T(0), T(0)}, xo[3] = {T(0), T(0), T(0)};
    if (inner) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (MODE != ST_APPLY) eb[c] = __ldg(a.b + c * V + vo);
        if (MODE == ST_CHEB_FIRST || MODE == ST_CHEB_STEP || MODE == ST_CHEB_PRE) ed[c] = __ldg(a.invD + c * V + vo);
        if (MODE == ST_CHEB_STEP) ep[c] = a.xprev[c * V + vo];
        if (MODE == ST_CHEB_FIRST || MODE == ST_CHEB_STEP) xo[c] = __ldg(a.x + c * V + vo);
      }
    }

    const T* dm = ds + slot(k - 1) * 6 * DT;  // plane k-1
    const T* d0 = ds + slot(k) * 6 * DT;      // plane k
    const T* dp = ds + slot(k + 1) * 6 * DT;  // plane k+1
    const T* cm = cs + cslot(k - 1) * 6 * CT;  // cube layer k-1
    const T* c0 = cs + cslot(k) * 6 * CT;      // cube layer k
    auto D = [&](const T* p, int comp, int di, int dj) { return p[comp * DT + (J + dj) * DW + I + di]; };
    auto C = [&](const T* p, int t, int di, int dj) { return p[t * CT + (J + dj) * CW + I + di]; };
    // coefficients of the 7 cubes around the vertex that touch its forward edges
    const T v0 = C(c0, 0, 0, 0), v1 = C(c0, 1, 0, 0), v2 = C(c0, 2, 0, 0), v3 = C(c0, 3, 0, 0),
                 v4 = C(c0, 4, 0, 0), v5 = C(c0, 5, 0, 0);
    const T mx0 = C(c0, 0, -1, 0), mx1 = C(c0, 1, -1, 0);      // cube v - ex
    const T my2 = C(c0, 2, 0, -1), my3 = C(c0, 3, 0, -1);      // v - ey
    const T mxy0 = C(c0, 0, -1, -1), mxy2 = C(c0, 2, -1, -1);  // v - ex - ey
    const T mz4 = C(cm, 4, 0, 0), mz5 = C(cm, 5, 0, 0);        // v - ez
    const T myz3 = C(cm, 3, 0, -1), myz5 = C(cm, 5, 0, -1);    // v - ey - ez
    const T mxz1 = C(cm, 1, -1, 0), mxz4 = C(cm, 4, -1, 0);    // v - ex - ez

    T Fx[3], Fy[3], Fz[3];
    // x edge (v, v + ex)
    {
      const T h = H[0];
      Fx[0] = T(2) * (h * dcur[0][0]);
      T s = h * dcur[0][1];
      s = fma(D(d0, YX, 1, 0), v0, s);
      s = fma(D(d0, YX, 1, 0), mz4, s);
      s = fma(D(d0, YX, 0, -1), my2, s);
      s = fma(D(d0, YX, 0, -1), myz5, s);
      s = fma(D(dp, YX, 1, 0), v1, s);
      Fx[1] = fma(D(dm, YX, 0, -1), myz3, s);
      s = h * dcur[0][2];
      s = fma(D(d0, ZX, 1, 0), v1, s);
      s = fma(D(d0, ZX, 1, 0), my2, s);
      s = fma(D(dm, ZX, 0, 0), mz4, s);
      s = fma(D(dm, ZX, 0, 0), myz3, s);
      s = fma(D(d0, ZX, 1, 1), v0, s);
      Fx[2] = fma(D(dm, ZX, 0, -1), myz5, s);
    }
    // y edge (v, v + ey)
    {
      const T h = H[1];
      Fy[1] = T(2) * (h * dcur[1][1]);
      T s = h * dcur[1][0];
      s = fma(D(d0, XY, 0, 1), v2, s);
      s = fma(D(d0, XY, 0, 1), mz5, s);
      s = fma(D(d0, XY, -1, 0), mx0, s);
      s = fma(D(d0, XY, -1, 0), mxz4, s);
      s = fma(D(dp, XY, 0, 1), v3, s);
      Fy[0] = fma(D(dm, XY, -1, 0), mxz1, s);
      s = h * dcur[1][2];
      s = fma(D(d0, ZY, 0, 1), v3, s);
      s = fma(D(d0, ZY, 0, 1), mx0, s);
      s = fma(D(dm, ZY, 0, 0), mz5, s);
      s = fma(D(dm, ZY, 0, 0), mxz1, s);
      s = fma(D(d0, ZY, 1, 1), v2, s);
      Fy[2] = fma(D(dm, ZY, -1, 0), mxz4, s);
    }
    // z edge (v, v + ez)
    {
      const T h = H[2];
      Fz[2] = T(2) * (h * dcur[2][2]);
      T s = h * dcur[2][0];
      s = fma(D(dp, XZ, 0, 0), v4, s);
      s = fma(D(dp, XZ, 0, 0), my3, s);
      s = fma(D(d0, XZ, -1, 0), mx1, s);
      s = fma(D(d0, XZ, -1, 0), mxy2, s);
      s = fma(D(dp, XZ, 0, 1), v5, s);
      Fz[0] = fma(D(d0, XZ, -1, -1), mxy0, s);
      s = h * dcur[2][1];
      s = fma(D(dp, YZ, 0, 0), v5, s);
      s = fma(D(dp, YZ, 0, 0), mx1, s);
      s = fma(D(d0, YZ, 0, -1), my3, s);
      s = fma(D(d0, YZ, 0, -1), mxy0, s);
      s = fma(D(dp, YZ, 1, 0), v4, s);
      Fz[1] = fma(D(d0, YZ, -1, -1), mxy2, s);
    }
    // the x edge ending at v belongs to lane tx - 1 of the same row (a warp)
    T fl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fl[c] = __shfl_up_sync(0xffffffffu, Fx[c], 1);
      fy[c * ENT + tid] = Fy[c];
    }
    __syncthreads();  // y fluxes of the tile visible; coefficient layer k-1 free
    if (k + 1 < zb) issue_coef(k + 1);
    cp_commit();
    T gs[3] = {T(0), T(0), T(0)};  // stored-Galerkin part (coarse levels)
    if (op.sten && inner) {
      const int sv = op.sidx[vo];
      if (sv >= 0)
        stencil_gather<T>(op, sv, gx, gy, k, [&](int d, int w) -> T {
          if (PRE) return a.s2 * __ldg(a.invD + d * V + w) * __ldg(a.b + d * V + w);
          return __ldg(a.x + d * V + w);
        }, gs);
    }
    if (out_k) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T fd = fy[c * ENT + tid - EBX];  // flux of the y edge ending at v
        // the DCA fluxes carry the unscaled coefficient (y = (h/6) sum), the
        // stencils the scaled operator
        const T sum = ((fl[c] - Fx[c]) + (fd - Fy[c])) + (fzp[c] - Fz[c]);
        T o = T(0);
        if (inner) {
          if (MODE == ST_APPLY) {
            o = op.sten ? fma(op.h6, sum, gs[c]) : op.h6 * sum;
          } else {
            const T r = op.sten ? eb[c] - fma(op.h6, sum, gs[c]) : fma(-op.h6, sum, eb[c]);  // b - A x
            if (MODE == ST_RESID) o = r;
            if (MODE == ST_CHEB_FIRST) o = fma(a.s0, ed[c] * r, xo[c]);
            if (MODE == ST_CHEB_STEP) o = fma(a.s1, ed[c] * r, fma(a.s0, xo[c] - ep[c], xo[c]));
            if (MODE == ST_CHEB_PRE) {
              const T x1 = a.s2 * ed[c] * eb[c];
              o = fma(a.s1, ed[c] * r, fma(a.s0, x1, x1));
            }
          }
        }
        if (a.out64)
          a.out64[c * V + vo] = (double)o;  // the mixed cycle's result, widened
        else
          a.out[c * V + vo] = o;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fzp[c] = Fz[c];
#pragma unroll
      for (int q = 0; q < 3; ++q) dcur[c][q] = dnext[c][q];
    }
  }
  cp_wait_all();  // no copy may be in flight when the block (or tile) ends
}

template <typename T, int MODE>
__global__ void __launch_bounds__(ENT, edge_min_blocks<T, MODE>())
    stencil_edge_kernel(const LevelOp<T> op, const StencilArgs<T> a, const int zch, const int gxw) {
  grid_dep_entry();
  extern __shared__ __align__(16) unsigned char sm_edge_raw[];
  const int t = blockIdx.x;
  stencil_edge_block<T, MODE>(op, a, zch, (t % gxw) * (EBX - 1), (t / gxw) * (EBY - 1), blockIdx.y, threadIdx.x,
                              reinterpret_cast<T*>(sm_edge_raw));
}

template <typename T, int MODE>
__global__ void __launch_bounds__(ENT, edge_min_blocks<T, MODE>())
    stencil_edge_batch_kernel(const StencilTask<T, T>* __restrict__ tasks, const int ntasks, const int64_t ntiles) {
  grid_dep_entry();
  extern __shared__ __align__(16) unsigned char sm_edge_raw[];
  for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int lo = 0, hi = ntasks - 1;  // last task with tile0 <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const StencilTask<T, T>& tk = tasks[lo];
    if (tk.sc && tk.sc[MS_DONE] != 0.0) continue;  // converged problem
    const int local = (int)(it - tk.tile0), per = tk.tg.per_z();
    const int bz = local / per, t = local % per;
    stencil_edge_block<T, MODE>(tk.op, tk.a, tk.tg.zch, (t % tk.tg.gxw) * (EBX - 1), (t / tk.tg.gxw) * (EBY - 1),
                                bz, threadIdx.x, reinterpret_cast<T*>(sm_edge_raw));
    __syncthreads();  // the shared-memory rings are reused by the next tile
  }
}

// H[m][v] = sum of eta over the 6 tetrahedra around the edge (v, v + e_m)
// (0 where the edge leaves the grid), in a fixed order; cube offsets and
// types as in stencil_edge_block
template <typename T>
__global__ void edge_sum_kernel(const int n, const T* __restrict__ eta, T* __restrict__ hedge) {
  const int nv = n + 1;
  const int64_t V = (int64_t)nv * nv * nv;
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int i = (int)(v % nv), j = (int)((v / nv) % nv), k = (int)(v / ((int64_t)nv * nv));
  auto c = [&](int di, int dj, int dk, int t) -> T {
    const int ci = i + di, cj = j + dj, ck = k + dk;
    if (ci < 0 || cj < 0 || ck < 0 || ci >= n || cj >= n || ck >= n) return T(0);
    return __ldg(eta + 6 * (ci + (int64_t)n * (cj + (int64_t)n * ck)) + t);
  };
  hedge[v] = ((c(0, 0, 0, 0) + c(0, 0, 0, 1)) + (c(0, -1, 0, 2) + c(0, 0, -1, 4))) + (c(0, -1, -1, 3) + c(0, -1, -1, 5));
  hedge[V + v] =
      ((c(0, 0, 0, 2) + c(0, 0, 0, 3)) + (c(-1, 0, 0, 0) + c(0, 0, -1, 5))) + (c(-1, 0, -1, 1) + c(-1, 0, -1, 4));
  hedge[2 * V + v] =
      ((c(0, 0, 0, 4) + c(0, 0, 0, 5)) + (c(-1, 0, 0, 1) + c(0, -1, 0, 3))) + (c(-1, -1, 0, 0) + c(-1, -1, 0, 2));
}

}  // namespace

TileGrid edge_tiles(int n, int zch_req) {
  const int nv = n + 1;
  TileGrid g;
  g.gxw = (nv + EBX - 2) / (EBX - 1);
  g.gyw = (nv + EBY - 2) / (EBY - 1);
  g.gxn = g.gyn = 0;
  g.x0n = 31 * g.gxw;
  const int per = g.per_z();
  // default: about four waves of one resident block per SM; long chunks
  // amortise the two prologue planes of each chunk
  int gz = (4 * 152 + per - 1) / per;
  int zch = zch_req > 0 ? zch_req : (nv + gz - 1) / gz;
  zch = std::max(zch, 1);
  zch = std::min(zch, nv);
  g.gz = (nv + zch - 1) / zch;
  g.zch = zch;
  return g;
}

template <typename T>
cudaError_t launch_edge_sums(int n, const T* eta, T* hedge, cudaStream_t s) {
  const int64_t V = nverts(n);
  return launch_k(edge_sum_kernel<T>, dim3((unsigned)((V + 255) / 256)), dim3(256), 0, s, n, eta, hedge);
}
template cudaError_t launch_edge_sums<double>(int, const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_stencil_edge(int mode, const LevelOp<T>& op, const StencilArgs<T>& a, cudaStream_t s, int zch_req) {
  const TileGrid tg = edge_tiles(op.n, zch_req);
  int dev = 0;
  KL(cudaGetDevice(&dev));
  const dim3 grid((unsigned)tg.per_z(), (unsigned)tg.gz), block(ENT);
#define AGCA_ELAUNCH(M)                                                                                     \
  do {                                                                                                      \
    static bool attr_set[64] = {};                                                                         \
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;                                                \
    if (!attr_set[dev]) {                                                                                   \
      KL(cudaFuncSetAttribute(stencil_edge_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                              (int)(edge_smem_elems<M>() * sizeof(T))));                                    \
      attr_set[dev] = true;                                                                                 \
    }                                                                                                       \
    KL(launch_k(stencil_edge_kernel<T, M>, grid, block, edge_smem_elems<M>() * sizeof(T), s, op, a, tg.zch,     \
                tg.gxw));                                                                                   \
  } while (0)
  switch (mode) {
    case ST_APPLY: AGCA_ELAUNCH(ST_APPLY); break;
    case ST_RESID: AGCA_ELAUNCH(ST_RESID); break;
    case ST_CHEB_FIRST: AGCA_ELAUNCH(ST_CHEB_FIRST); break;
    case ST_CHEB_STEP: AGCA_ELAUNCH(ST_CHEB_STEP); break;
    case ST_CHEB_PRE: AGCA_ELAUNCH(ST_CHEB_PRE); break;
    default: return cudaErrorInvalidValue;
  }
#undef AGCA_ELAUNCH
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stencil_edge_batch(int mode, const StencilTask<T, T>* tasks, int ntasks, int64_t ntiles,
                                      cudaStream_t s) {
  if (ntasks <= 0 || ntiles <= 0) return cudaSuccess;
  int dev = 0, sms = 152;
  KL(cudaGetDevice(&dev));
  KL(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const dim3 grid((unsigned)std::min<int64_t>(ntiles, (int64_t)edge_min_blocks<T, ST_RESID>() * sms)), block(ENT);
#define AGCA_EBLAUNCH(M)                                                                                      \
  do {                                                                                                        \
    static bool attr_set[64] = {};                                                                           \
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;                                                  \
    if (!attr_set[dev]) {                                                                                     \
      KL(cudaFuncSetAttribute(stencil_edge_batch_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                              (int)(edge_smem_elems<M>() * sizeof(T))));                                      \
      attr_set[dev] = true;                                                                                   \
    }                                                                                                         \
    KL(launch_k(stencil_edge_batch_kernel<T, M>, grid, block, edge_smem_elems<M>() * sizeof(T), s, tasks,     \
                ntasks, ntiles));                                                                             \
  } while (0)
  switch (mode) {
    case ST_RESID: AGCA_EBLAUNCH(ST_RESID); break;
    case ST_CHEB_FIRST: AGCA_EBLAUNCH(ST_CHEB_FIRST); break;
    case ST_CHEB_STEP: AGCA_EBLAUNCH(ST_CHEB_STEP); break;
    case ST_CHEB_PRE: AGCA_EBLAUNCH(ST_CHEB_PRE); break;
    default: return cudaErrorInvalidValue;
  }
#undef AGCA_EBLAUNCH
  return cudaGetLastError();
}

template cudaError_t launch_stencil_edge<double>(int, const LevelOp<double>&, const StencilArgs<double>&,
                                                  cudaStream_t, int);
template cudaError_t launch_stencil_edge_batch<double>(int, const StencilTask<double, double>*, int, int64_t,
                                                       cudaStream_t);

}  // namespace agca
