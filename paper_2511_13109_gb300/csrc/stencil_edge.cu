// FP64 operator in edge form (Eq. 2.3 with the element matrices of Eq. 3.5;
// on coarse levels the DCA part of Eq. 2.9), fused with the smoother and
// residual epilogues: every level of an FP64 context.
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
// Per vertex the coefficients enter through a record of 27 combinations
// (EREC, edge_record): the three edge sums H_m and, for each forward edge m
// and component c != m, the weights of the four distinct c-edge differences
// around the edge (two of them the sum of the two tetrahedra sharing that
// difference).  The kernel then does 9 edge differences, 3 x 20 flux flops
// and 15 divergence terms per vertex, against about 190 for the
// per-tetrahedron form; the neighbours' edge differences are shared through
// shared memory instead of being recomputed.
//
// GB300 runs one FP64 fused multiply-add per 64 FP32 ones, so FP64
// arithmetic bounds the operator; the records are formed once per viscosity
// (edge_record_kernel) and read by each vertex's own thread.  (The FP32
// cycle keeps the per-cube kernel: an FP32 instance of this kernel, records
// formed in-kernel from staged cube rows, issued about 1,600 instructions per
// vertex, mostly integer, and ran 2.3x slower.)
//
// Tiling: a CTA of 32 x 8 threads, thread (tx, ty) <-> vertex column
// (x0 - 1 + tx, y0 - 1 + ty), marches a chunk of z-planes.  Per plane k it
// stages the x plane k + 2 (cp.async, one plane ahead), forms the edge
// differences of plane k + 1 for its
// (34 x 10)-vertex tile, computes the three fluxes of its vertex's forward
// edges from the differences of planes k - 1..k + 1 and its vertex's
// coefficient record, exchanges the x and y fluxes (warp shuffle, shared
// memory; the z flux stays in registers for the next plane), and the threads
// with tx, ty >= 1 finish their vertex (owner-computes: no atomics; every
// vertex sums its fluxes in one fixed order, whatever the tile shape or
// z-chunk).  Staging copies whole tile rows per warp: a row's geometry is
// warp-uniform and each lane's column bounds are fixed for the block, so a
// copy costs an address add and a predicate.
#include <algorithm>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

constexpr int EBX = 32, EBY = 8, ENT = EBX * EBY, NWARP = ENT / 32;
constexpr int XW = EBX + 3, XH = EBY + 3, XT = XW * XH;  // x tile: vertices (x0-2 .., y0-2 ..)
constexpr int DW = EBX + 2, DH = EBY + 2, DT = DW * DH;  // edge-difference tile
constexpr int DRING = 84;                                // halo entries of the difference tile
static_assert(EBX == 32, "a tile row is one warp");
static_assert(XW - 32 <= 32, "row staging covers an x-tile row in at most 2 warp copies");
// off-diagonal edge-difference components kept in shared memory:
// (edge axis, component) = xy, xz, yx, yz, zx, zy
enum { XY = 0, XZ, YX, YZ, ZX, ZY };

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T, int MODE>
__host__ __device__ constexpr size_t edge_smem_elems() {
  // x ring [3][3][XT] (+ D^-1 ring for the step from zero), difference ring
  // [3][6][DT], y-flux exchange [3][ENT]: in FP64 82 KB, or 110 KB with the
  // D^-1 ring
  return (size_t)(MODE == ST_CHEB_PRE ? 2 : 1) * 3 * 3 * XT + (size_t)3 * 6 * DT + (size_t)3 * ENT;
}
// resident CTAs per SM (shared memory and the 128-register budget)
template <typename T, int MODE>
__host__ __device__ constexpr int edge_min_blocks() {
  return 2;
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

// The coefficient record of vertex v = (i, j, k) from the coefficients of
// the cubes around it, named by the cube's offset from v and the tetrahedron
// type: v0..v5 cube (i, j, k); mx cube (i-1, j, k), my (i, j-1, k),
// mxy (i-1, j-1, k), mz (i, j, k-1), myz (i, j-1, k-1), mxz (i-1, j, k-1)
// (0 for a cube outside the grid).
//   q = 0..2   H_x, H_y, H_z (sums over the 6 tetrahedra around each edge)
//   q = 3..10  x edge: component y, then z
//   q = 11..18 y edge: component x, then z
//   q = 19..26 z edge: component x, then y
// each (edge, component) block holding the weights of its four difference
// terms in the order stencil_edge_block reads them; the four add up to H_m.
template <typename T>
__device__ __forceinline__ void edge_record(T v0, T v1, T v2, T v3, T v4, T v5, T mx0, T mx1, T my2, T my3, T mxy0,
                                            T mxy2, T mz4, T mz5, T myz3, T myz5, T mxz1, T mxz4, T (&r)[EREC]) {
  r[0] = ((v0 + v1) + (my2 + mz4)) + (myz3 + myz5);
  r[1] = ((v2 + v3) + (mx0 + mz5)) + (mxz1 + mxz4);
  r[2] = ((v4 + v5) + (mx1 + my3)) + (mxy0 + mxy2);
  r[3] = v0 + mz4, r[4] = my2 + myz5, r[5] = v1, r[6] = myz3;
  r[7] = v1 + my2, r[8] = mz4 + myz3, r[9] = v0, r[10] = myz5;
  r[11] = v2 + mz5, r[12] = mx0 + mxz4, r[13] = v3, r[14] = mxz1;
  r[15] = v3 + mx0, r[16] = mz5 + mxz1, r[17] = v2, r[18] = mxz4;
  r[19] = v4 + my3, r[20] = mx1 + mxy2, r[21] = v5, r[22] = mxy0;
  r[23] = v5 + mx1, r[24] = my3 + mxy0, r[25] = v4, r[26] = mxy2;
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
  const int tx = tid & (EBX - 1), ty = tid >> 5;  // lane, warp
  const int gx = x0 - 1 + tx, gy = y0 - 1 + ty;
  const int za = bz * zch, zb = min(za + zch, nv);
  const bool owner = tx >= 1 && ty >= 1 && gx <= n && gy <= n;
  const bool inner_xy = gx > 0 && gx < n && gy > 0 && gy < n;
  constexpr bool PRE = MODE == ST_CHEB_PRE;

  T* xs = sm;                                    // [3][3][XT]
  T* xa = xs + 3 * 3 * XT;                       // PRE: D^-1 ring [3][3][XT]
  T* ds = xa + (PRE ? 3 * 3 * XT : 0);           // [3][6][DT]
  T* fy = ds + 3 * 6 * DT;                       // [3][ENT]

  const int zs = za - 2;  // planes zs + i use ring slot i mod 3
  auto slot = [&](int p) { return (p - zs) % 3; };

  // this lane's columns of the x tile (x0 - 2 + tx, and x0 + 30 + tx for the
  // last XW - 32 lanes): interior in x?  Dirichlet and outside vertices read 0
  const bool inx0 = x0 - 2 + tx > 0 && x0 - 2 + tx < n;
  const bool inx1 = tx < XW - 32 && x0 + 30 + tx > 0 && x0 + 30 + tx < n;
  // stage x plane p (PRE: b and D^-1): warp ty copies the rows r = ty, ty + 8, ..
  // of the [3][XH] rows of the tile
  auto issue_x = [&](int p) {
    T* dst = xs + slot(p) * 3 * XT;
    T* dsa = xa + slot(p) * 3 * XT;
    const bool zin = p > 0 && p < n;
    for (int r = ty; r < 3 * XH; r += NWARP) {
      const int c = r / XH, j = r - c * XH;
      const int vy = y0 - 2 + j;
      const bool rin = zin && vy > 0 && vy < n;
      const int g = c * V + (x0 - 2) + nv * (vy + nv * p);  // valid when rin (then vy >= 1, so g >= 0)
      const int e = c * XT + j * XW + tx;
      const bool ok0 = rin && inx0, ok1 = rin && inx1;
      const int g0 = ok0 ? g + tx : 0, g1 = ok1 ? g + 32 + tx : 0;
      if (PRE) {
        cpT(dst + e, a.b + g0, ok0);
        cpT(dsa + e, a.invD + g0, ok0);
        if (tx < XW - 32) {
          cpT(dst + e + 32, a.b + g1, ok1);
          cpT(dsa + e + 32, a.invD + g1, ok1);
        }
      } else {
        cpT(dst + e, a.x + g0, ok0);
        if (tx < XW - 32) cpT(dst + e + 32, a.x + g1, ok1);
      }
    }
  };
  // PRE: the first Chebyshev iterate x1 = (s2 D^-1) b of the entries this
  // thread staged (the same operations as the per-tetrahedron kernel)
  auto convert_x = [&](int p) {
    if (!PRE) return;
    T* dst = xs + slot(p) * 3 * XT;
    const T* dsa = xa + slot(p) * 3 * XT;
    for (int r = ty; r < 3 * XH; r += NWARP) {
      const int c = r / XH, j = r - c * XH;
      const int e = c * XT + j * XW + tx;
      dst[e] = a.s2 * dsa[e] * dst[e];
      if (tx < XW - 32) dst[e + 32] = a.s2 * dsa[e + 32] * dst[e + 32];
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

  // prologue: x planes za-2 .. za; edge differences of planes za-2 and za-1
  issue_x(zs);
  issue_x(zs + 1);
  issue_x(zs + 2);
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
    __syncthreads();  // x plane k+2 staged; ring slots of k-2 free
    compute_d(k + 1, dnext);
    __syncthreads();  // differences of plane k+1 visible; x slot of plane k free
    if (k + 1 < zb) issue_x(k + 3);
    cp_commit();

    // own coefficient record and epilogue inputs of plane k, read early
    const bool kin = k >= 0 && k <= n && gx >= 0 && gx <= n && gy >= 0 && gy <= n;
    const int vo = kin ? gx + nv * (gy + nv * k) : 0;
    const T* rec = op.hedge + vo;
    auto R = [&](int q) { return kin ? __ldg(rec + (int64_t)q * V) : T(0); };
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
    auto D = [&](const T* p, int comp, int di, int dj) { return p[comp * DT + (J + dj) * DW + I + di]; };

    // the halo row (warp 0) supplies only the y fluxes of row 1, and the
    // halo plane za-1 only the z fluxes of plane za (warp-uniform branches)
    const bool need_x = ty != 0 && k >= za, need_y = k >= za, need_z = ty != 0;
    T Fx[3] = {T(0), T(0), T(0)}, Fy[3] = {T(0), T(0), T(0)}, Fz[3] = {T(0), T(0), T(0)};
    // flux component c != m of edge m: the H_m term and the four distinct
    // c-edge differences around the edge, weighted by the record (EREC order)
    auto flux = [&](int q0, T hd, T da, T db, T dc, T dd) {
      T f = fma(da, R(q0), hd);
      f = fma(db, R(q0 + 1), f);
      f = fma(dc, R(q0 + 2), f);
      return fma(dd, R(q0 + 3), f);
    };
    if (need_x) {  // x edge (v, v + ex)
      const T h = R(0);
      Fx[0] = T(2) * (h * dcur[0][0]);
      Fx[1] = flux(3, h * dcur[0][1], D(d0, YX, 1, 0), D(d0, YX, 0, -1), D(dp, YX, 1, 0), D(dm, YX, 0, -1));
      Fx[2] = flux(7, h * dcur[0][2], D(d0, ZX, 1, 0), D(dm, ZX, 0, 0), D(d0, ZX, 1, 1), D(dm, ZX, 0, -1));
    }
    if (need_y) {  // y edge (v, v + ey)
      const T h = R(1);
      Fy[1] = T(2) * (h * dcur[1][1]);
      Fy[0] = flux(11, h * dcur[1][0], D(d0, XY, 0, 1), D(d0, XY, -1, 0), D(dp, XY, 0, 1), D(dm, XY, -1, 0));
      Fy[2] = flux(15, h * dcur[1][2], D(d0, ZY, 0, 1), D(dm, ZY, 0, 0), D(d0, ZY, 1, 1), D(dm, ZY, -1, 0));
    }
    if (need_z) {  // z edge (v, v + ez)
      const T h = R(2);
      Fz[2] = T(2) * (h * dcur[2][2]);
      Fz[0] = flux(19, h * dcur[2][0], D(dp, XZ, 0, 0), D(d0, XZ, -1, 0), D(dp, XZ, 0, 1), D(d0, XZ, -1, -1));
      Fz[1] = flux(23, h * dcur[2][1], D(dp, YZ, 0, 0), D(d0, YZ, 0, -1), D(dp, YZ, 1, 0), D(d0, YZ, -1, -1));
    }
    // the x edge ending at v belongs to lane tx - 1 of the same row (a warp)
    T fl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fl[c] = __shfl_up_sync(0xffffffffu, Fx[c], 1);
      fy[c * ENT + tid] = Fy[c];
    }
    __syncthreads();  // y fluxes of the tile visible
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

// the coefficient record of every vertex, rec[q][v], q < EREC (edge_record)
template <typename T>
__global__ void edge_record_kernel(const int n, const T* __restrict__ eta, T* __restrict__ rec) {
  grid_dep_entry();  // the coefficients may come from the kernel before (masked_coef_kernel)
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
  T r[EREC];
  edge_record<T>(c(0, 0, 0, 0), c(0, 0, 0, 1), c(0, 0, 0, 2), c(0, 0, 0, 3), c(0, 0, 0, 4), c(0, 0, 0, 5),
                 c(-1, 0, 0, 0), c(-1, 0, 0, 1), c(0, -1, 0, 2), c(0, -1, 0, 3), c(-1, -1, 0, 0), c(-1, -1, 0, 2),
                 c(0, 0, -1, 4), c(0, 0, -1, 5), c(0, -1, -1, 3), c(0, -1, -1, 5), c(-1, 0, -1, 1), c(-1, 0, -1, 4),
                 r);
#pragma unroll
  for (int q = 0; q < EREC; ++q) rec[q * V + v] = r[q];
}

}  // namespace

TileGrid edge_tiles(int n, int zch_req, int slots) {
  const int nv = n + 1;
  TileGrid g;
  g.gxw = (nv + EBX - 2) / (EBX - 1);
  g.gyw = (nv + EBY - 2) / (EBY - 1);
  g.gxn = g.gyn = 0;
  g.x0n = 31 * g.gxw;
  const int per = g.per_z();
  int zch = zch_req;
  if (zch <= 0) {
    // default: the z-chunk with the least modelled time: whole waves of
    // `slots` resident blocks times the planes a block marches (its chunk
    // plus about one plane's worth of prologue); longer chunks win ties
    const int sl = slots > 0 ? slots : 2 * 152;
    double best = 1e300;
    for (int gz = 1; gz <= nv; ++gz) {
      const int z = (nv + gz - 1) / gz;
      if ((nv + z - 1) / z != gz) continue;  // the same chunk as a smaller gz
      const double waves = (double)(((int64_t)per * gz + sl - 1) / sl);
      const double cost = waves * (z + 1.0);
      if (cost < best - 1e-9) {
        best = cost;
        zch = z;
      }
    }
  }
  zch = std::max(zch, 1);
  zch = std::min(zch, nv);
  g.gz = (nv + zch - 1) / zch;
  g.zch = zch;
  return g;
}

template <typename T>
cudaError_t launch_edge_records(int n, const T* eta, T* rec, cudaStream_t s) {
  const int64_t V = nverts(n);
  return launch_k(edge_record_kernel<T>, dim3((unsigned)((V + 255) / 256)), dim3(256), 0, s, n, eta, rec);
}
template cudaError_t launch_edge_records<double>(int, const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_stencil_edge(int mode, const LevelOp<T>& op, const StencilArgs<T>& a, cudaStream_t s, int zch_req) {
  int dev = 0, sms = 152;
  KL(cudaGetDevice(&dev));
  KL(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const TileGrid tg = edge_tiles(op.n, zch_req, edge_min_blocks<T, ST_RESID>() * sms);
  const dim3 grid((unsigned)tg.per_z(), (unsigned)tg.gz), block(ENT);
#define AGCA_ELAUNCH(M)                                                                                     \
  do {                                                                                                      \
    static bool attr_set[64] = {};                                                                         \
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;                                                \
    if (!attr_set[dev]) {                                                                                   \
      KL(cudaFuncSetAttribute(stencil_edge_kernel<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                              (int)(edge_smem_elems<T, M>() * sizeof(T))));                                    \
      attr_set[dev] = true;                                                                                 \
    }                                                                                                       \
    KL(launch_k(stencil_edge_kernel<T, M>, grid, block, edge_smem_elems<T, M>() * sizeof(T), s, op, a, tg.zch,     \
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
                              (int)(edge_smem_elems<T, M>() * sizeof(T))));                                      \
      attr_set[dev] = true;                                                                                   \
    }                                                                                                         \
    KL(launch_k(stencil_edge_batch_kernel<T, M>, grid, block, edge_smem_elems<T, M>() * sizeof(T), s, tasks,     \
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
