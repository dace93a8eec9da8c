// Matrix-free operator application on a Kuhn cube grid, fused with the
// smoother and residual epilogues (Eq. 2.3 on the finest level, the
// heterogeneous AGCA operator of Eq. 2.9 on coarse levels); the per-cube
// element action (cube_dca) is in device_ops.cuh.
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
//
// Summation order at vertex (i, j, k), Y(cube)[corner] the cube's corner sums
// (zero for cubes outside the grid):
//   [(Y(i-1,j-1,k-1)[7] + Y(i,j-1,k-1)[6]) + (Y(i-1,j,k-1)[5] + Y(i,j,k-1)[4])]
//   + [(Y(i-1,j-1,k)[3] + Y(i,j-1,k)[2]) + (Y(i-1,j,k)[1] + Y(i,j,k)[0])]
// whatever the tile shape (results do not depend on it).
#include <algorithm>
#include <type_traits>

#include "agca_internal.cuh"
#include "device_ops.cuh"

namespace agca {

namespace {

// cp.async (LDGSTS) helpers: asynchronous global -> shared copies, zero fill
// when src_bytes == 0 (the source address is then not read).
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes, bool ok) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int src = ok ? bytes : 0;
  if (bytes == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int MODE, typename TS>
__host__ __device__ constexpr int stencil_tile_fields() {
  return MODE == ST_CHEB_PRE ? 9 : ((MODE == ST_STOKES || MODE == ST_STOKES_B) ? 4 : 3);
}

// FP32 tiles keep the operator input of a vertex as one float4 (its 3 or 4
// components), so a corner is one 16-byte shared load and the y-exchange one
// 16-byte store and load per cube layer; FP64 tiles keep one array per field
template <typename TS>
__host__ __device__ constexpr bool stencil_aos() {
  return sizeof(TS) == 4;
}
// TS elements of one ring slot: AoS [4 * TSZ] (+ CHEB_PRE: b and D^-1 as
// [6][TSZ], padded to whole float4s), or SoA [NF][TSZ]
template <typename TS, int BX, int BY, int MODE>
__host__ __device__ constexpr int stencil_slot_elems() {
  constexpr int TSZ = (BX + 1) * (BY + 1);
  return stencil_aos<TS>() ? 4 * TSZ + (MODE == ST_CHEB_PRE ? (6 * TSZ + 3) / 4 * 4 : 0)
                           : stencil_tile_fields<MODE, TS>() * TSZ;
}

// dynamic shared memory of one block: tile ring [3][slot] of TS, then
// (128-byte aligned, as the 8/16-byte async copies need) the coefficient ring
// [2][BX*BY][6] of T and the y-exchange ([2][BX*BY][4] AoS or [2][NC][BX*BY]) of T
template <typename TS, int BX, int BY, int MODE>
__host__ __device__ constexpr size_t stencil_tile_bytes() {
  return ((size_t)3 * stencil_slot_elems<TS, BX, BY, MODE>() * sizeof(TS) + 127) / 128 * 128;
}
// Stokes operator with FP64 vectors and FP32 arithmetic: every staged value
// is converted once, by the thread that copied it, into an FP32 copy of the
// ring (FP64 -> FP32 conversions issue at the FP64 rate on this GPU, so
// converting at each of the up to 4 corner reads of a value costs more than
// the element arithmetic)
template <typename TS, typename T, int MODE>
__host__ __device__ constexpr bool stencil_converts() {
  return MODE == ST_STOKES && sizeof(TS) != sizeof(T);
}
template <typename TS, typename T, int BX, int BY, int MODE>
__host__ __device__ constexpr size_t stencil_smem_bytes() {
  constexpr int NC = (MODE == ST_STOKES || MODE == ST_STOKES_B) ? 4 : 3;
  return stencil_tile_bytes<TS, BX, BY, MODE>() + (size_t)2 * BX * BY * 6 * sizeof(T) +
         (size_t)2 * (stencil_aos<TS>() ? 4 : NC) * BX * BY * sizeof(T) +
         (stencil_converts<TS, T, MODE>() ? (size_t)3 * NC * (BX + 1) * (BY + 1) * sizeof(T) : 0);
}

// One CTA tile of the stencil: vertex columns x0.. and rows y0.. (origin of
// the owned (BX-1) x (BY-1) block), z-chunk bz; thread (tx, ty) with
// tid = ty * BX + tx, so a warp spans 32 / BX rows of the tile (BX = 32 or 8;
// the shuffle along x then crosses rows only into the non-owning last
// column).  Called by the single-operator kernel and by the persistent
// batched kernel.
template <typename TS, typename T, int BX, int BY, int MODE, bool COARSE>
__device__ __forceinline__ void stencil_block(const LevelOp<T>& op, const StencilArgs<TS>& a, const int zch,
                                              const int x0, const int y0, const int bz, const int tx, const int ty,
                                              unsigned char* __restrict__ smem_raw) {
  static_assert(BX == 32 || BX == 8, "a tile row is a whole warp or a quarter of one");
  constexpr int NC = (MODE == ST_STOKES || MODE == ST_STOKES_B) ? 4 : 3;  // combined fields: velocity (+ divergence)
  constexpr int NF = stencil_tile_fields<MODE, TS>();
  constexpr int TW = BX + 1, TSZ = (BX + 1) * (BY + 1), NT = BX * BY;
  constexpr int NSLOT = (TSZ + NT - 1) / NT;
  constexpr bool AOS = stencil_aos<TS>();
  constexpr int SS = stencil_slot_elems<TS, BX, BY, MODE>();
  TS* xs = reinterpret_cast<TS*>(smem_raw);
  T* cfs = reinterpret_cast<T*>(smem_raw + stencil_tile_bytes<TS, BX, BY, MODE>());
  T* cs = cfs + 2 * NT * 6;
  constexpr bool CONV = stencil_converts<TS, T, MODE>();
  static_assert(!(AOS && CONV), "an FP32 tile needs no conversion");
  T* xcv = cs + 2 * NC * NT;  // CONV: FP32 ring [3][NC][TSZ]

  // 32-bit indices: the host limits grids to 3 (n+1)^3 < 2^31 and 6 n^3 < 2^31
  const int n = op.n;
  const int nv = n + 1;
  const int V = nv * nv * nv;
  const int plane = nv * nv;
  const int tid = ty * BX + tx;
  const int z0 = bz * zch;
  const int z1 = min(z0 + zch, nv);
  const int cx = x0 - 1 + tx, cy = y0 - 1 + ty;
  const bool cube_xy = (cx >= 0) && (cx < n) && (cy >= 0) && (cy < n);
  const int cube_col = cx + n * cy;
  const int vx = x0 + tx, vy = y0 + ty;
  const bool owner = (tx < BX - 1) && (ty < BY - 1) && (vx < nv) && (vy < nv);
  const bool inner_xy = (vx > 0) && (vx < n) && (vy > 0) && (vy < n);
  const int vcol = vx + nv * vy;

  // tile slots of this thread (fixed for the whole z-march)
  int s_col[NSLOT];
  unsigned s_flags = 0;  // bit 2j: slot valid, 2j+1: interior in xy; bit 16+j: pressure-valid in xy
#pragma unroll
  for (int j = 0; j < NSLOT; ++j) {
    const int idx = tid + j * NT;
    const int lx = idx % TW, ly = idx / TW;
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    s_col[j] = gx + nv * gy;
    if (idx < TSZ) {
      s_flags |= 1u << (2 * j);
      if (gx > 0 && gx < n && gy > 0 && gy < n) s_flags |= 2u << (2 * j);
      if (gx >= 0 && gx <= n && gy >= 0 && gy <= n) s_flags |= 1u << (16 + j);
    }
  }

  const int zs = z0 - 1;
  // plane z goes to ring slot `slot` (plane zs + i uses slot i mod 3)
  auto issue_tile = [&](int z, int slot) {
    TS* dst = xs + slot * SS;
    TS* soa = AOS ? dst + 4 * TSZ : dst;  // CHEB_PRE: b, D^-1
    const bool zin = (z > 0) && (z < n);
    const bool zq = (z >= 0) && (z <= n);
    const int pb = z * plane;
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
      if (!(s_flags & (1u << (2 * j)))) continue;
      const int idx = tid + j * NT;
      const bool in = zin && (s_flags & (2u << (2 * j)));
      const int v = in ? pb + s_col[j] : 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (MODE == ST_CHEB_PRE) {
          cp_async(soa + c * TSZ + idx, a.b + (c * V + v), sizeof(TS), in);
          cp_async(soa + (3 + c) * TSZ + idx, a.invD + (c * V + v), sizeof(TS), in);
        } else {
          cp_async(AOS ? dst + 4 * idx + c : dst + c * TSZ + idx, a.x + (c * V + v), sizeof(TS), in);
        }
      }
      if (MODE == ST_STOKES || MODE == ST_STOKES_B) {  // fine-grid pressure q = P p lives on every vertex
        const bool qin = zq && (s_flags & (1u << (16 + j)));
        cp_async(AOS ? dst + 4 * idx + 3 : dst + 3 * TSZ + idx, a.q + (qin ? pb + s_col[j] : 0), sizeof(TS),
                 qin);
      }
    }
  };
  auto issue_coef = [&](int kc) {
    if (MODE == ST_STOKES_B) return;  // no viscous part: the coefficients are not read
    T* dst = cfs + (((kc - zs) & 1) * NT + tid) * 6;
    const bool ok = cube_xy && kc >= 0 && kc < n;
    const T* src = op.coef + (ok ? 6 * (cube_col + kc * n * n) : 0);
    if (sizeof(T) == 4) {
#pragma unroll
      for (int i = 0; i < 3; ++i) cp_async(dst + 2 * i, src + 2 * i, 8, ok);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) cp_async(dst + 2 * i, src + 2 * i, 16, ok);
    }
  };
  // CHEB_PRE: the first Chebyshev iterate x1 = s2 D^-1 b of the slots this
  // thread copied, formed once in shared memory (fields 6..8)
  auto convert_plane = [&](int slot) {
    TS* t = xs + slot * SS;
    const TS* soa = AOS ? t + 4 * TSZ : t;
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
      if (!(s_flags & (1u << (2 * j)))) continue;
      const int idx = tid + j * NT;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const TS x1 = a.s2 * soa[(3 + c) * TSZ + idx] * soa[c * TSZ + idx];
        if constexpr (AOS)
          t[4 * idx + c] = x1;
        else
          t[(6 + c) * TSZ + idx] = x1;
      }
    }
  };
  // CONV: the FP32 copy of the slots this thread copied
  auto convert_slots = [&](int slot) {
    const TS* t = xs + slot * SS;
    T* o = xcv + slot * NC * TSZ;
#pragma unroll
    for (int j = 0; j < NSLOT; ++j) {
      if (!(s_flags & (1u << (2 * j)))) continue;
      const int idx = tid + j * NT;
#pragma unroll
      for (int c = 0; c < NC; ++c) o[c * TSZ + idx] = (T)t[c * TSZ + idx];
    }
  };
  auto tile_val = [&](const TS* t, int c, int li) -> T {
    if (MODE == ST_CHEB_PRE && c < 3) return (T)t[(6 + c) * TSZ + li];
    return (T)t[c * TSZ + li];
  };
  // the NC operator-input components of tile vertex li of a ring slot
  auto load_vertex = [&](const TS* t, int li, T (&v)[NC]) {
    if constexpr (AOS) {
      const float4 q = *reinterpret_cast<const float4*>(t + 4 * li);
      v[0] = q.x;
      v[1] = q.y;
      v[2] = q.z;
      if constexpr (NC == 4) v[3] = q.w;
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = tile_val(t, c, li);
    }
  };

  // prologue: planes zs, zs+1 and the coefficients of cube layer zs
  issue_tile(zs, 0);
  if (zs + 1 <= n) issue_tile(zs + 1, 1);
  issue_coef(zs);
  cp_commit();

  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);

  // one cube layer k: Xl holds plane k (loaded here when k == zs), Xh
  // receives plane k+1; rk = ring slot of plane k
  auto layer = [&](const int k, const int rk, T(&Xl)[4][NC], T(&Xh)[4][NC]) {
    const int rk1 = rk == 2 ? 0 : rk + 1, rk2 = rk1 == 2 ? 0 : rk1 + 1;
    // prefetch plane k+2 and the coefficients of layer k+1 while layer k computes
    if (k + 1 < z1) {
      if (k + 2 <= n) issue_tile(k + 2, rk2);
      issue_coef(k + 1);
    }
    cp_commit();
    // epilogue inputs of plane k, read early so their latency overlaps the compute
    const bool out_k = owner && k >= z0;
    const bool inner = out_k && inner_xy && k > 0 && k < n;
    const int vo = vcol + k * plane;
    TS eb[3], ed[3], ep[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      eb[c] = ed[c] = ep[c] = TS(0);
      if (inner) {
        if (MODE == ST_RESID || MODE == ST_CHEB_FIRST || MODE == ST_CHEB_STEP || MODE == ST_STOKES_B)
          eb[c] = __ldg(a.b + (c * V + vo));  // STOKES_B: A u
        if (MODE == ST_CHEB_FIRST || MODE == ST_CHEB_STEP) ed[c] = __ldg(a.invD + (c * V + vo));
        if (MODE == ST_CHEB_STEP) ep[c] = a.xprev[c * V + vo];
      }
    }
    int32_t f[6];
    if constexpr (COARSE) {
      if (cube_xy && k >= 0 && k < n) {
        const int2* fp = reinterpret_cast<const int2*>(op.fidx + 6 * (cube_col + k * n * n));
        int2 f01 = __ldg(fp), f23 = __ldg(fp + 1), f45 = __ldg(fp + 2);
        f[0] = f01.x; f[1] = f01.y; f[2] = f23.x; f[3] = f23.y; f[4] = f45.x; f[5] = f45.y;
      } else {
#pragma unroll
        for (int t = 0; t < 6; ++t) f[t] = -1;
      }
    }
    cp_wait1();
    if (MODE == ST_CHEB_PRE) {
      if (k == zs) convert_plane(rk);
      if (k + 1 <= n) convert_plane(rk1);
    }
    if constexpr (CONV) {
      if (k == zs) convert_slots(rk);
      if (k + 1 <= n) convert_slots(rk1);
    }
    __syncthreads();
    {
      const TS* tl = xs + rk * SS;
      const TS* th = xs + rk1 * SS;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int li = (ty + (q >> 1)) * TW + tx + (q & 1);
        if constexpr (CONV) {
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (k == zs) Xl[q][c] = xcv[(rk * NC + c) * TSZ + li];
            Xh[q][c] = (k + 1 <= n) ? xcv[(rk1 * NC + c) * TSZ + li] : T(0);
          }
        } else {
          if (k == zs) load_vertex(tl, li, Xl[q]);
          if (k + 1 <= n) {
            load_vertex(th, li, Xh[q]);
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) Xh[q][c] = T(0);
          }
        }
      }
      if (MODE == ST_CHEB_PRE && inner) {  // own b and D^-1 on plane k, before the ring slot is reused
        const int li = (ty + 1) * TW + tx + 1;
        const TS* soa = AOS ? tl + 4 * TSZ : tl;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          eb[c] = soa[c * TSZ + li];
          ed[c] = soa[(3 + c) * TSZ + li];
        }
      }
    }

    T Y[8][NC];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int c = 0; c < NC; ++c) Y[q][c] = T(0);

    if (cube_xy && k >= 0 && k < n) {
      // this cube's 6 coefficients: three 8-byte (FP32) or 16-byte (FP64) shared loads
      const T* cp = cfs + (((k - zs) & 1) * NT + tid) * 6;
      T cf[6];
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 v = reinterpret_cast<const float2*>(cp)[i];
          cf[2 * i] = v.x * op.h6;
          cf[2 * i + 1] = v.y * op.h6;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double2 v = reinterpret_cast<const double2*>(cp)[i];
          cf[2 * i] = v.x * op.h6;
          cf[2 * i + 1] = v.y * op.h6;
        }
      }
      if constexpr (COARSE) {
#pragma unroll
        for (int t = 0; t < 6; ++t)
          if (f[t] >= 0) cf[t] = T(0);
        cube_dca<T, NC>(Xl, Xh, cf, Y);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          if (f[t] >= 0 && !op.sten) {  // stored Galerkin element: s_e A_e x_e precomputed by gca_apply_kernel
            const T* yv = op.ye + f[t] * 12;
#pragma unroll
            for (int r = 0; r < 12; ++r) {
              const int q = tet_corner(t, r & 3);
              Y[q][r >> 2] += yv[r];
            }
          }
        }
      } else if constexpr (MODE == ST_STOKES) {
        cube_stokes<T>(Xl, Xh, cf, op.hq, Y);
      } else if constexpr (MODE == ST_STOKES_B) {
        cube_stokes_b<T>(Xl, Xh, op.hq, Y);
      } else {
        cube_dca<T, NC>(Xl, Xh, cf, Y);
      }
    }

    // combine along x (lane tx+1 holds the neighbouring cube), then along y
    T s1[2][NC];
#pragma unroll
    for (int qz = 0; qz < 2; ++qz) {
      T s0[4];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        // corners (qx, qy, qz): index qx + 2 qy + 4 qz
        const T from_right_y1 = __shfl_down_sync(0xffffffffu, Y[4 * qz + 2][c], 1);
        const T from_right_y0 = __shfl_down_sync(0xffffffffu, Y[4 * qz + 0][c], 1);
        s1[qz][c] = Y[4 * qz + 3][c] + from_right_y1;  // row qy = 1 (own vertex row)
        s0[c] = Y[4 * qz + 1][c] + from_right_y0;      // row qy = 0, for thread ty-1
      }
      if constexpr (AOS) {
        reinterpret_cast<float4*>(cs)[qz * NT + tid] = make_float4(s0[0], s0[1], s0[2], NC == 4 ? s0[3] : 0.f);
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) cs[(qz * NC + c) * NT + tid] = s0[c];
      }
    }
    __syncthreads();

    if (owner) {
      T up[2][4];  // row qy = 0 sums of the cube above, per qz
      if constexpr (AOS) {
#pragma unroll
        for (int qz = 0; qz < 2; ++qz) {
          const float4 u = reinterpret_cast<const float4*>(cs)[qz * NT + tid + BX];
          up[qz][0] = u.x;
          up[qz][1] = u.y;
          up[qz][2] = u.z;
          up[qz][3] = u.w;
        }
      } else {
#pragma unroll
        for (int qz = 0; qz < 2; ++qz)
#pragma unroll
          for (int c = 0; c < NC; ++c) up[qz][c] = cs[(qz * NC + c) * NT + tid + BX];
      }
      T yk[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        yk[c] = acc[c] + (s1[0][c] + up[0][c]);
        acc[c] = s1[1][c] + up[1][c];
      }
      if constexpr (COARSE) {
        // stored-Galerkin part of the touched vertices (stencil storage)
        if (op.sten && inner) {
          const int sv = op.sidx[vo];
          if (sv >= 0) {
            T g[3];
            stencil_gather<T>(op, sv, vx, vy, k, [&](int d, int w) -> TS {
              if (MODE == ST_CHEB_PRE) return a.s2 * __ldg(a.invD + d * V + w) * __ldg(a.b + d * V + w);
              return __ldg(a.x + d * V + w);
            }, g);
#pragma unroll
            for (int c = 0; c < 3; ++c) yk[c] += g[c];
          }
        }
      }
      if (out_k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int i = c * V + vo;
          // own vertex value on plane k (CHEB_PRE: x1 = s2 D^-1 b staged in the tile)
          const TS o = inner ? stencil_epilogue<MODE, TS>((TS)Xl[3][c], (TS)yk[c], eb[c], ed[c], ep[c], a.s0, a.s1)
                             : TS(0);
          if (MODE != ST_STOKES && MODE != ST_STOKES_B && a.out64)
            a.out64[i] = (double)o;
          else
            a.out[i] = o;
        }
        if (MODE == ST_STOKES || MODE == ST_STOKES_B) a.out2[vo] = (TS)yk[NC - 1];  // (B_f u) on every fine vertex
      }
    }
  };

  T Xa[4][NC], Xb[4][NC];
  int rk = 0;
  if constexpr (sizeof(T) == 4 && MODE != ST_STOKES && MODE != ST_STOKES_B) {
    // the z-march unrolled by two so that the plane registers alternate roles
    // (no copy of the upper plane into the lower one per layer)
    for (int k = zs; k < z1; k += 2) {
      layer(k, rk, Xa, Xb);
      if (k + 1 >= z1) break;
      const int rk1 = rk == 2 ? 0 : rk + 1;
      layer(k + 1, rk1, Xb, Xa);
      rk = rk1 == 2 ? 0 : rk1 + 1;
    }
  } else {  // larger per-layer state: one copy of the layer body keeps it in registers
    for (int k = zs; k < z1; ++k) {
      layer(k, rk, Xa, Xb);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) Xa[q][c] = Xb[q][c];
      rk = rk == 2 ? 0 : rk + 1;
    }
  }
}

template <typename T, int BY>
__host__ __device__ constexpr int stencil_min_blocks() {
  return sizeof(T) == 4 ? (BY <= 8 ? 3 : (BY <= 12 ? 2 : 1)) : 2;
}
// the persistent batched form keeps its task's fields in registers: two
// FP32 CTAs per SM (128 registers) instead of three, without spills
template <typename T, int BY>
__host__ __device__ constexpr int stencil_batch_min_blocks() {
  return sizeof(T) == 4 && BY <= 8 ? 2 : stencil_min_blocks<T, BY>();
}

// Single-operator launch over two tile classes: wide tiles (32 x BY threads,
// 31 x (BY-1) owned vertices) cover the first gxw * 31 vertex columns, narrow
// tiles (8 x 4BY threads, 7 x (4BY-1) owned) the columns x0n.. left over.
// A vertex row of n+1 = 129 columns is then 4 wide + 1 narrow strip instead
// of 5 wide strips whose last one would keep 26 of 32 lanes idle.  Both
// classes have 32 * BY threads and the same shared-memory layout size class.
template <typename TS, typename T, int BY, int MODE, bool COARSE>
__global__ void __launch_bounds__(32 * BY, stencil_min_blocks<T, BY>())
    stencil_kernel(const LevelOp<T> op, const StencilArgs<TS> a, const int zch, const int gxw, const int gyw,
                   const int gxn, const int x0n) {
  grid_dep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int t = blockIdx.x, nw = gxw * gyw;
  if (t < nw) {
    stencil_block<TS, T, 32, BY, MODE, COARSE>(op, a, zch, (t % gxw) * 31, (t / gxw) * (BY - 1), blockIdx.y,
                                               tid & 31, tid >> 5, smem_raw);
  } else {
    constexpr int BYN = 4 * BY;
    const int u = t - nw;
    stencil_block<TS, T, 8, BYN, MODE, COARSE>(op, a, zch, x0n + (u % gxn) * 7, (u / gxn) * (BYN - 1), blockIdx.y,
                                               tid & 7, tid >> 3, smem_raw);
  }
}

// Persistent batched form: one launch applies the same stencil mode to many
// independent problems; every CTA walks the flattened (problem, tile) work
// list (both tile classes, as stencil_kernel), skipping problems whose MINRES
// has converged.
template <typename TS, typename T, int BY, int MODE, bool COARSE>
__global__ void __launch_bounds__(32 * BY, stencil_batch_min_blocks<T, BY>())
    stencil_batch_kernel(const StencilTask<TS, T>* __restrict__ tasks, const int ntasks, const int64_t ntiles) {
  grid_dep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  for (int64_t it = blockIdx.x; it < ntiles; it += gridDim.x) {
    int lo = 0, hi = ntasks - 1;  // last task with tile0 <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const StencilTask<TS, T>& tk = tasks[lo];
    if (tk.sc && tk.sc[MS_DONE] != 0.0) continue;  // converged problem
    const TileGrid tg = tk.tg;
    const int local = (int)(it - tk.tile0), per = tg.per_z();
    const int bz = local / per, t = local % per, nw = tg.gxw * tg.gyw;
    if (t < nw) {
      stencil_block<TS, T, 32, BY, MODE, COARSE>(tk.op, tk.a, tg.zch, (t % tg.gxw) * 31, (t / tg.gxw) * (BY - 1), bz,
                                                 tid & 31, tid >> 5, smem_raw);
    } else {
      constexpr int BYN = 4 * BY;
      const int u = t - nw;
      stencil_block<TS, T, 8, BYN, MODE, COARSE>(tk.op, tk.a, tg.zch, tg.x0n + (u % tg.gxn) * 7,
                                                 (u / tg.gxn) * (BYN - 1), bz, tid & 7, tid >> 3, smem_raw);
    }
    __syncthreads();  // the shared-memory rings are reused by the next tile
  }
}


template <typename TS, typename T, bool PRE>
__global__ void gca_apply_kernel(const LevelOp<T> op, const StencilArgs<TS> a) {
  grid_dep_entry();
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= op.n_flag * 12) return;
  gca_row<TS, T, PRE>(op, a, id);
}

template <typename TS, typename T, bool PRE>
__global__ void gca_apply_batch_kernel(const StencilTask<TS, T>* __restrict__ tasks) {
  grid_dep_entry();
  const StencilTask<TS, T>& tk = tasks[blockIdx.y];
  if (tk.sc && tk.sc[MS_DONE] != 0.0) return;
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= tk.op.n_flag * 12) return;
  gca_row<TS, T, PRE>(tk.op, tk.a, id);
}

template <typename TS, typename T, int BY, bool COARSE>
cudaError_t launch_mode(int mode, const LevelOp<T>& op, const StencilArgs<TS>& a, cudaStream_t s, int zch_req) {
  const TileGrid tg = stencil_tiles(op.n, BY, zch_req);
  if (COARSE && op.n_flag > 0 && !op.sten) {
    const unsigned gb = (unsigned)((op.n_flag * 12 + 127) / 128);
    if (mode == ST_CHEB_PRE)
      KL(launch_k(gca_apply_kernel<TS, T, true>, dim3(gb), dim3(128), 0, s, op, a));
    else
      KL(launch_k(gca_apply_kernel<TS, T, false>, dim3(gb), dim3(128), 0, s, op, a));
  }
  const dim3 grid((unsigned)tg.per_z(), (unsigned)tg.gz), block(32 * BY);
#define AGCA_LAUNCH(M, C)                                                                                  \
  do {                                                                                                     \
    constexpr size_t smem = std::max(stencil_smem_bytes<TS, T, 32, BY, M>(),                              \
                                     stencil_smem_bytes<TS, T, 8, 4 * BY, M>());                          \
    static bool attr_set[64] = {};                                                                        \
    int dev_ = 0;                                                                                         \
    cudaError_t e = cudaGetDevice(&dev_);                                                                 \
    if (e != cudaSuccess) return e;                                                                       \
    if (smem > 48 * 1024 && dev_ >= 0 && dev_ < 64 && !attr_set[dev_]) {                                  \
      e = cudaFuncSetAttribute(stencil_kernel<TS, T, BY, M, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)smem);                                                                \
      if (e != cudaSuccess) return e;                                                                     \
      attr_set[dev_] = true;                                                                              \
    }                                                                                                     \
    KL(launch_k(stencil_kernel<TS, T, BY, M, C>, grid, block, smem, s, op, a, tg.zch, tg.gxw, tg.gyw, tg.gxn, \
                tg.x0n));                                                                                 \
  } while (0)
  switch (mode) {
    case ST_APPLY: AGCA_LAUNCH(ST_APPLY, COARSE); break;
    case ST_RESID: AGCA_LAUNCH(ST_RESID, COARSE); break;
    case ST_CHEB_FIRST: AGCA_LAUNCH(ST_CHEB_FIRST, COARSE); break;
    case ST_CHEB_STEP: AGCA_LAUNCH(ST_CHEB_STEP, COARSE); break;
    case ST_CHEB_PRE: AGCA_LAUNCH(ST_CHEB_PRE, COARSE); break;
    case ST_STOKES:
      if constexpr (COARSE) {
        return cudaErrorInvalidValue;
      } else {
        AGCA_LAUNCH(ST_STOKES, false);
      }
      break;
    case ST_STOKES_B:
      if constexpr (COARSE || sizeof(T) != 8 || sizeof(TS) != 8) {
        return cudaErrorInvalidValue;
      } else {
        AGCA_LAUNCH(ST_STOKES_B, false);
      }
      break;
    default: return cudaErrorInvalidValue;
  }
#undef AGCA_LAUNCH
  return cudaGetLastError();
}

template <typename TS, typename T, int BY, bool COARSE>
cudaError_t launch_batch_mode(int mode, const StencilTask<TS, T>* tasks, int ntasks, int64_t ntiles,
                              int64_t max_gca_rows, cudaStream_t s) {
  if (ntasks <= 0 || ntiles <= 0) return cudaSuccess;
  if (COARSE && max_gca_rows > 0) {
    const dim3 g((unsigned)((max_gca_rows + 127) / 128), (unsigned)ntasks);
    if (mode == ST_CHEB_PRE)
      KL(launch_k(gca_apply_batch_kernel<TS, T, true>, g, dim3(128), 0, s, tasks));
    else
      KL(launch_k(gca_apply_batch_kernel<TS, T, false>, g, dim3(128), 0, s, tasks));
  }
  int dev = 0, sms = 152;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t nb = std::min<int64_t>(ntiles, (int64_t)sms * stencil_batch_min_blocks<T, BY>());
  const dim3 grid((unsigned)nb), block(32 * BY);
#define AGCA_BLAUNCH(M, C)                                                                                 \
  do {                                                                                                     \
    constexpr size_t smem = std::max(stencil_smem_bytes<TS, T, 32, BY, M>(),                              \
                                     stencil_smem_bytes<TS, T, 8, 4 * BY, M>());                          \
    static bool attr_set[64] = {};                                                                        \
    if (smem > 48 * 1024 && dev >= 0 && dev < 64 && !attr_set[dev]) {                                    \
      e = cudaFuncSetAttribute(stencil_batch_kernel<TS, T, BY, M, C>,                                     \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                   \
      if (e != cudaSuccess) return e;                                                                     \
      attr_set[dev] = true;                                                                               \
    }                                                                                                     \
    KL(launch_k(stencil_batch_kernel<TS, T, BY, M, C>, grid, block, smem, s, tasks, ntasks, ntiles));     \
  } while (0)
  switch (mode) {
    case ST_RESID: AGCA_BLAUNCH(ST_RESID, COARSE); break;
    case ST_CHEB_FIRST: AGCA_BLAUNCH(ST_CHEB_FIRST, COARSE); break;
    case ST_CHEB_STEP: AGCA_BLAUNCH(ST_CHEB_STEP, COARSE); break;
    case ST_CHEB_PRE: AGCA_BLAUNCH(ST_CHEB_PRE, COARSE); break;
    case ST_STOKES:
      if constexpr (COARSE) {
        return cudaErrorInvalidValue;
      } else {
        AGCA_BLAUNCH(ST_STOKES, false);
      }
      break;
    default: return cudaErrorInvalidValue;
  }
#undef AGCA_BLAUNCH
  return cudaGetLastError();
}

}  // namespace

TileGrid stencil_tiles(int n, int BY, int zch_req) {
  const int nv = n + 1;
  const int BYN = 4 * BY;
  TileGrid g;
  g.gyw = (nv + BY - 2) / (BY - 1);
  g.gyn = (nv + BYN - 2) / (BYN - 1);
  // strips of 31 columns (wide) while they are full, the rest in strips of
  // 7 (narrow) if that takes fewer blocks than one more wide strip
  const int full = nv / 31, rem = nv - 31 * full;
  const int nar = (rem + 6) / 7;
  if (rem == 0 || nar * g.gyn < g.gyw) {
    g.gxw = full;
    g.gxn = nar;
  } else {
    g.gxw = full + 1;
    g.gxn = 0;
  }
  g.x0n = 31 * g.gxw;
  if (g.gxn == 0) g.gyn = 0;
  const int per = g.per_z();
  // default: enough blocks for two waves of 3 resident 256-thread blocks per
  // SM; small grids get short z-chunks (latency bound), large ones long
  // chunks (less z-halo).  zch_req > 0 (autotuner, batches) overrides
  int gz = (912 * 8 / BY + per - 1) / per;
  int zch = zch_req > 0 ? zch_req : (nv + gz - 1) / gz;
  if (zch < 1) zch = 1;
  if (zch > nv) zch = nv;
  g.gz = (nv + zch - 1) / zch;
  g.zch = zch;
  return g;
}

template <typename TS, typename T>
cudaError_t launch_stencil_batch(int mode, bool coarse, const StencilTask<TS, T>* tasks, int ntasks, int64_t ntiles,
                                 int64_t max_gca_rows, cudaStream_t s) {
  if constexpr (std::is_same<TS, double>::value && std::is_same<T, double>::value) {
    if (edge_form_step<TS, T>(mode, coarse)) return launch_stencil_edge_batch<T>(mode, tasks, ntasks, ntiles, s);
  }
  if (coarse) return launch_batch_mode<TS, T, 8, true>(mode, tasks, ntasks, ntiles, max_gca_rows, s);
  return launch_batch_mode<TS, T, 8, false>(mode, tasks, ntasks, ntiles, 0, s);
}
template cudaError_t launch_stencil_batch<float, float>(int, bool, const StencilTask<float, float>*, int, int64_t,
                                                        int64_t, cudaStream_t);
template cudaError_t launch_stencil_batch<double, double>(int, bool, const StencilTask<double, double>*, int, int64_t,
                                                          int64_t, cudaStream_t);
template cudaError_t launch_stencil_batch<double, float>(int, bool, const StencilTask<double, float>*, int, int64_t,
                                                         int64_t, cudaStream_t);

template <typename TS, typename T>
cudaError_t launch_stencil(int mode, const LevelOp<T>& op, const StencilArgs<TS>& a, cudaStream_t s,
                           const TileCfg* cfg) {
  const int by = cfg ? cfg->by : 8, zch = cfg ? cfg->zch : 0;
  if constexpr (std::is_same<TS, double>::value && std::is_same<T, double>::value) {
    // FP64 levels run the edge form (their coefficient records exist in FP64 contexts)
    if (op.hedge && mode != ST_STOKES && mode != ST_STOKES_B) return launch_stencil_edge<T>(mode, op, a, s, zch);
  }
  if constexpr (sizeof(T) == 4 && sizeof(TS) == 4) {
    if (by == 12) {
      if (op.fidx) return launch_mode<TS, T, 12, true>(mode, op, a, s, zch);
      return launch_mode<TS, T, 12, false>(mode, op, a, s, zch);
    }
    if (by == 16) {
      if (op.fidx) return launch_mode<TS, T, 16, true>(mode, op, a, s, zch);
      return launch_mode<TS, T, 16, false>(mode, op, a, s, zch);
    }
  }
  // 8 block rows otherwise (a tile shape never changes the result)
  if (op.fidx) return launch_mode<TS, T, 8, true>(mode, op, a, s, zch);
  return launch_mode<TS, T, 8, false>(mode, op, a, s, zch);
}

template cudaError_t launch_stencil<float, float>(int, const LevelOp<float>&, const StencilArgs<float>&,
                                                  cudaStream_t, const TileCfg*);
template cudaError_t launch_stencil<double, double>(int, const LevelOp<double>&, const StencilArgs<double>&,
                                                    cudaStream_t, const TileCfg*);
template cudaError_t launch_stencil<double, float>(int, const LevelOp<float>&, const StencilArgs<double>&,
                                                   cudaStream_t, const TileCfg*);

}  // namespace agca
