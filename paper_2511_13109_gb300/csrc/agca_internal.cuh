// Internal declarations shared by the CUDA translation units of libagca.
//
// Kuhn grid conventions (the same as include/agca.h): tetrahedron t of a cube
// follows the t-th lexicographic permutation p of (0,1,2); its local vertices
// lie on the cube corners 0, 1<<p0, (1<<p0)|(1<<p1), 7 (corner bit m = offset
// along axis m).  The barycentric gradients on a cube of size h are g = G/h
// with G_0 = -e_p0, G_1 = e_p0 - e_p1, G_2 = e_p1 - e_p2, G_3 = e_p2 and the
// volume is h^3/6, so the viscous element matrix of Eq. 3.5,
//   [A_e]_{(a,c),(b,d)} = eta_e |T| (delta_cd g_a.g_b + g_{a,d} g_{b,c}),
// equals eta_e * (h/6) * K'_t with K'_t = delta_cd G_a.G_b + G_{a,d} G_{b,c},
// an integer matrix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/agca.h"

namespace agca {

// ---------------------------------------------------------------- Kuhn tables
__host__ __device__ constexpr int perm(int t, int k) {
  return t == 0   ? (k == 0 ? 0 : k == 1 ? 1 : 2)
         : t == 1 ? (k == 0 ? 0 : k == 1 ? 2 : 1)
         : t == 2 ? (k == 0 ? 1 : k == 1 ? 0 : 2)
         : t == 3 ? (k == 0 ? 1 : k == 1 ? 2 : 0)
         : t == 4 ? (k == 0 ? 2 : k == 1 ? 0 : 1)
                  : (k == 0 ? 2 : k == 1 ? 1 : 0);
}
// cube corner (bits x,y,z) of local vertex a of a type-t tetrahedron
__host__ __device__ constexpr int tet_corner(int t, int a) {
  return a == 0 ? 0 : a == 1 ? (1 << perm(t, 0)) : a == 2 ? ((1 << perm(t, 0)) | (1 << perm(t, 1))) : 7;
}
// component m of the scaled gradient G_a of local vertex a (values -1, 0, 1)
__host__ __device__ constexpr int kuhn_grad(int t, int a, int m) {
  return a == 0   ? -(perm(t, 0) == m)
         : a == 1 ? (perm(t, 0) == m) - (perm(t, 1) == m)
         : a == 2 ? (perm(t, 1) == m) - (perm(t, 2) == m)
                  : (perm(t, 2) == m);
}
// K'_t entry for local DoFs r = c*4+a, s = d*4+b
__host__ __device__ constexpr int kuhn_kprime(int t, int r, int s) {
  return ((r >> 2) == (s >> 2) ? (kuhn_grad(t, r & 3, 0) * kuhn_grad(t, s & 3, 0) +
                                  kuhn_grad(t, r & 3, 1) * kuhn_grad(t, s & 3, 1) +
                                  kuhn_grad(t, r & 3, 2) * kuhn_grad(t, s & 3, 2))
                               : 0) +
         kuhn_grad(t, r & 3, s >> 2) * kuhn_grad(t, s & 3, r >> 2);
}
// local index a of cube corner q in tetrahedron t, or -1
__host__ __device__ constexpr int corner_local(int t, int q) {
  return q == 0 ? 0 : q == 7 ? 3 : q == tet_corner(t, 1) ? 1 : q == tet_corner(t, 2) ? 2 : -1;
}

// The 15 Kuhn offsets of a vertex stencil (the vertex and the 14 neighbours it
// shares an element edge with), in the order 0, +-e_x, +-e_y, +-e_z,
// +-(e_x+e_y), +-(e_x+e_z), +-(e_y+e_z), +-(1,1,1): index of offset
// (dx, dy, dz) (entries of one sign) and the offset of index o
__host__ __device__ constexpr int kuhn_offset_index(int dx, int dy, int dz) {
  return (dx | dy | dz) == 0 ? 0
         : 1 + 2 * ((((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 1)   ? 0
                    : (((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 2) ? 1
                    : (((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 4) ? 2
                    : (((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 3) ? 3
                    : (((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 5) ? 4
                    : (((dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)) == 6) ? 5
                                                                          : 6) +
               ((dx < 0 || dy < 0 || dz < 0) ? 1 : 0);
}
__host__ __device__ constexpr int kuhn_offset_comp(int o, int axis) {
  // pattern of offset pair (o - 1) / 2: x, y, z, xy, xz, yz, xyz
  return o == 0 ? 0
                : (((((o - 1) >> 1) == 0 || ((o - 1) >> 1) == 3 || ((o - 1) >> 1) == 4 || ((o - 1) >> 1) == 6) && axis == 0) ||
                   ((((o - 1) >> 1) == 1 || ((o - 1) >> 1) == 3 || ((o - 1) >> 1) == 5 || ((o - 1) >> 1) == 6) && axis == 1) ||
                   ((((o - 1) >> 1) == 2 || ((o - 1) >> 1) == 4 || ((o - 1) >> 1) == 5 || ((o - 1) >> 1) == 6) && axis == 2))
                      ? (((o - 1) & 1) ? -1 : 1)
                      : 0;
}

// Refinement tables, built once on the host from the Kuhn ordering rule and
// passed to kernels by value (kernel-parameter constant bank; see tables.cu):
//  child[t][k] = {ox, oy, oz, t'}: k-th child (ascending fine element id) of a
//                type-t parent: fine cube 2*C + o, fine type t'.
//  pk2[t][k][i][j] = 2 * lambda_j(parent) at local vertex i of child k.
struct RefineTables {
  int8_t child[6][8][4];
  int8_t pk2[6][8][4][4];
};
void build_refine_tables(RefineTables* out);
const RefineTables& refine_tables();

// ---------------------------------------------------------------- level views
template <typename T>
struct LevelOp {
  int n;               // cubes per axis
  T h6;                // h / 6
  T hq;                // h^2 / 6 (divergence terms, finest level)
  const T* coef;       // per-element coefficient: eta (finest) or child mean (coarse)
  const int32_t* fidx; // compact Galerkin index per element or -1; nullptr on finest
  const T* gca;        // stored Galerkin matrices (n_flag * 144)
  const T* gscale;     // per flagged element scale (mixed) or nullptr
  const int32_t* list; // flagged element ids (coarse levels)
  int64_t n_flag;      // number of flagged elements
  T* ye;               // n_flag * 12 scratch: s_e A_e x_e of the flagged elements
  const T* hedge;      // FP64 levels: per-vertex coefficient records [EREC][V] of the edge form, or nullptr
  const T* coefm;      // FP64 coarse levels: DCA coefficient with flagged elements zeroed (edge form), or nullptr
  // stored-Galerkin part as per-vertex stencils (Remark 5): stencil index of a
  // vertex or -1, 15 x 3 x 3 couplings per touched vertex, FP32 scale (mixed)
  const int32_t* sidx;
  const T* sten;
  const T* sscale;
};

__host__ __device__ inline int64_t nverts(int n) { return (int64_t)(n + 1) * (n + 1) * (n + 1); }
__host__ __device__ inline int64_t nelems(int n) { return (int64_t)6 * n * n * n; }

// ---------------------------------------------------------------- dependent launch
// Programmatic dependent launch: a hot-path kernel is launched while its
// predecessor in the stream is still running, so the launch latency of the
// ~50 short kernels of a V-cycle or MINRES iteration overlaps the previous
// kernel.  Every kernel begins with grid_dep_entry(): each thread waits until
// all grids it depends on have completed and their writes are visible (a
// no-op when the kernel was launched normally), then allows the next grid to
// begin launching.  Waiting in every thread before any memory access keeps
// the stream's ordering transitive (a grid completes only after the grids
// before it) and rules out write-after-read races with the predecessor.
__device__ __forceinline__ void grid_dep_entry() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Whether launches carry the programmatic-serialization attribute (on unless
// the environment sets AGCA_PDL=0; never on the legacy default stream).
bool pdl_enabled(cudaStream_t s);

template <typename... KP, typename... A>
cudaError_t launch_k(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled(s) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}
// return the error of a launch from the enclosing cudaError_t function
#define KL(...)                                  \
  do {                                           \
    const cudaError_t e_ = (__VA_ARGS__);        \
    if (e_ != cudaSuccess) return e_;            \
  } while (0)

// ---------------------------------------------------------------- launchers
enum StencilMode { ST_APPLY = 0, ST_RESID = 1, ST_CHEB_FIRST = 2, ST_CHEB_STEP = 3, ST_CHEB_PRE = 4, ST_STOKES = 5 };
// internal (FP64 contexts, not tunable): the pressure coupling of the Stokes
// operator added to a.b = A u from the edge form, out = a.b - B_f^T q,
// out2 = B_f u
constexpr int ST_STOKES_B = 6;

template <typename T>
struct StencilArgs {
  const T* x;      // input field (ST_CHEB_PRE: unused)
  const T* b;      // right-hand side (RESID, CHEB*)
  const T* invD;   // inverse diagonal (CHEB*)
  const T* xprev;  // previous iterate (CHEB_STEP), may alias out
  const T* q;      // fine-grid pressure P p (STOKES)
  T* out;
  T* out2;         // B_f u on the fine grid (STOKES)
  double* out64;   // if set, the result is written here widened to FP64 instead of to out
  T s0, s1, s2;    // mode scalars
};

// Tile shape of a stencil launch: block rows BY (8, 12 or 16 for FP32; 8
// otherwise) and the z-chunk (0 = automatic).  Chosen by the autotuner.
struct TileCfg {
  int by = 8;
  int zch = 0;
};

// TS: storage type of the vectors; T: compute type (and type of the level data)
template <typename TS, typename T>
cudaError_t launch_stencil(int mode, const LevelOp<T>& op, const StencilArgs<TS>& a, cudaStream_t s,
                           const TileCfg* cfg = nullptr);

// Tiles of a stencil launch: wide tiles (32 x BY threads) over vertex
// columns 0 .. 31*gxw-1, narrow tiles (8 x 4BY threads) over x0n .. n; grid =
// (per_z(), gz) blocks of 32*BY threads.
struct TileGrid {
  int gxw = 0, gyw = 0, gxn = 0, gyn = 0, x0n = 0, gz = 0, zch = 0;
  __host__ __device__ int per_z() const { return gxw * gyw + gxn * gyn; }
};
TileGrid stencil_tiles(int n, int by, int zch_req);

// FP64 operator in edge form (stencil_edge.cu): modes APPLY, RESID and the
// Chebyshev steps, with op.hedge = the per-vertex coefficient records
// (EREC values per vertex, launch_edge_records): the sums of eta over the 6
// tetrahedra around each forward axis edge and the weights of the edge
// differences in the off-axis flux components
constexpr int EREC = 27;
// tile grid of the edge form; zch_req 0 picks the z-chunk for `slots`
// resident blocks (0: 304)
TileGrid edge_tiles(int n, int zch_req, int slots = 0);
template <typename T>
cudaError_t launch_edge_records(int n, const T* eta, T* rec, cudaStream_t s);
template <typename T>
cudaError_t launch_stencil_edge(int mode, const LevelOp<T>& op, const StencilArgs<T>& a, cudaStream_t s, int zch_req);

// ------------------------------------------------------------ batched forms
// One (problem, level) operator application inside a batched launch.
template <typename TS, typename T>
struct StencilTask {
  LevelOp<T> op;
  StencilArgs<TS> a;
  TileGrid tg;          // tiles of this problem (8 block rows), tg.per_z() * tg.gz of them
  int64_t tile0;        // first tile of this task in the flattened work list
  const double* sc;     // MINRES scalars of the problem (skip when sc[MS_DONE] != 0) or nullptr
};
// tasks: device array, ntiles = total tiles of all tasks; coarse launches
// first run the stored-Galerkin products of every task (max_gca_rows = the
// largest n_flag * 12)
template <typename TS, typename T>
cudaError_t launch_stencil_batch(int mode, bool coarse, const StencilTask<TS, T>* tasks, int ntasks, int64_t ntiles,
                                 int64_t max_gca_rows, cudaStream_t s);
// the edge form for a batch of tasks (tiles from edge_tiles)
template <typename T>
cudaError_t launch_stencil_edge_batch(int mode, const StencilTask<T, T>* tasks, int ntasks, int64_t ntiles,
                                      cudaStream_t s);
// whether a step of this kind runs the edge form: every level of an FP64
// context (its coefficient records exist on every level); the FP32 cycle and
// the Stokes operator run the per-cube kernel
template <typename TS, typename T>
constexpr bool edge_form_step(int mode, bool coarse) {
  (void)coarse;
  return sizeof(TS) == 8 && sizeof(T) == 8 && mode != ST_STOKES;
}

// Element-wise batched tasks (transfers, conversions, coarsest solves).
struct XferTask {
  int nf;               // fine cubes per axis (transfers) or cubes per axis (coarse solve)
  int ncomp;            // components (transfers)
  int mask;             // zero Dirichlet rows (transfers)
  double scale;         // restriction scale
  int64_t count;        // work items of the task
  const void* src;
  void* dst;
  const double* m1;     // coarsest solve: L^-1 column-major
  const double* m2;     // coarsest solve: L^-1 row-major
  const double* sc;     // skip when sc[MS_DONE] != 0, or nullptr
};
enum XferKind { XK_RESTRICT = 0, XK_PROLONG_ADD, XK_D2F, XK_F2D, XK_COARSE, XK_PROLONG, XK_COPY64 };
template <typename T>
cudaError_t launch_xfer_batch(int kind, const XferTask* tasks, int ntasks, int64_t max_count, int max_m,
                              cudaStream_t s);

// grid transfers (transfer.cu)
template <typename T>
cudaError_t launch_restrict(int nf, int ncomp, bool mask, T scale, const T* rf, T* rc, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong(int nf, int ncomp, bool mask, bool add, const T* ec, T* xf, cudaStream_t s);

// setup kernels (setup.cu)
cudaError_t launch_check_eta(const double* eta, int64_t n, int* status, cudaStream_t s);
// Eq. 2.8 flags of a coarse level (nc cubes): from the finest nodal viscosity
// eta_v when given (the level above the finest), else from the flags of the
// next finer level flags_f
cudaError_t launch_gradient_flags(int nc, const double* eta_v, double nu, const uint8_t* flags_f, uint8_t* flags_c,
                                  cudaStream_t s);
// projection: coarse coefficient as the children's arithmetic (0), harmonic (1) or geometric (2) mean
cudaError_t launch_coarsen(int nc, int projection, const double* mean_f, const double* mx_f, const double* mn_f,
                           double nu, double* mean_c, double* mx_c, double* mn_c, uint8_t* flags, cudaStream_t s);
cudaError_t launch_compact(const uint8_t* flags, int64_t n, int32_t* fidx, int32_t* list, int32_t* block_counts,
                           int64_t* total, cudaStream_t s);
int64_t compact_scratch_blocks(int64_t n);
cudaError_t launch_galerkin(int nc, int64_t n_flag, const int32_t* list, int nf, bool child_finest,
                            const double* coef_f, const int32_t* fidx_f, const double* gca_f, double* gca_c,
                            cudaStream_t s);
cudaError_t launch_diag(const LevelOp<double>& op, double* diag, double* invD64, float* invD32, cudaStream_t s);
cudaError_t launch_gca_to_f32(int64_t n_flag, const int32_t* list, const double* mx, const double* gca64,
                              float* gca32, float* scale32, cudaStream_t s);
cudaError_t launch_d2f(const double* in, float* out, int64_t n, cudaStream_t s);
cudaError_t launch_f2d(const float* in, double* out, int64_t n, cudaStream_t s);
cudaError_t launch_coarse_assemble(const LevelOp<double>& op, double* dense, cudaStream_t s);
cudaError_t launch_cholesky(double* a, int m, int* status, cudaStream_t s);
cudaError_t launch_trinv(const double* l, int m, double* linv_cm, double* linv_rm, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(int n, const double* linv_cm, const double* linv_rm, const T* r, T* z,
                                cudaStream_t s);
cudaError_t launch_pressure_mass(int np, const double* eta_f, double* pmass, double* pmass_inv, cudaStream_t s);
// stencil storage of the flagged elements' Galerkin matrices (stencil_store.cu)
cudaError_t launch_mark_vertices(int n, const uint8_t* flags, uint8_t* mark, cudaStream_t s);
cudaError_t launch_stencil_assemble(int n, int64_t n_sv, const int32_t* slist, const int32_t* fidx, const double* gca,
                                    double* sten, cudaStream_t s);
cudaError_t launch_stencil_to_f32(int64_t n_sv, const double* s64, float* s32, float* scale, cudaStream_t s);
cudaError_t launch_masked_coef(int64_t E, const double* mean, const int32_t* fidx, double* coefm, cudaStream_t s);
cudaError_t launch_start_vector(int n, double* v, cudaStream_t s);

// Stokes / Krylov kernels (krylov.cu)
// device-resident MINRES scalar slots
enum MinresSlot {
  MS_GAMMA = 0, MS_GAMMA_OLD, MS_ETA, MS_ETA0, MS_C, MS_C_OLD, MS_S, MS_S_OLD, MS_A1, MS_A2, MS_A3, MS_XCOEF,
  MS_INV_GAMMA_PREV, MS_UPD_SKIP, MS_DONE, MS_ITERS, MS_TOL_ABS, MS_DOT_KZZ, MS_DOT_ZV, MS_TMP0, MS_TMP1, MS_TMP2,
  MS_COUNT
};
enum VecOp { VOP_SUB = 0, VOP_ADD, VOP_COPY, VOP_ZERO, VOP_PDIV, VOP_SUBS, VOP_MUL, VOP_SCALE_RSQRT, VOP_RECIP };
int dot_blocks();
// out[j] = scale * sum_i xs[j][i] * ys[j][i] for npairs <= 3, deterministic
cudaError_t launch_dots(int npairs, const double* const* xs, const double* const* ys, int64_t n, double* partials,
                        double* out, double scale, cudaStream_t s);
cudaError_t launch_sum(const double* x, int64_t n, double* partials, double* out, double scale, cudaStream_t s);
cudaError_t launch_vec_op(int op, int64_t n, double* y, const double* a, const double* b, const double* c,
                          const double* scal, cudaStream_t s);
cudaError_t launch_minres_init(double* sc, double tol_rel, cudaStream_t s);
cudaError_t launch_lanczos(int64_t n, const double* kz, const double* v, double* vold_to_vnew, const double* sc,
                           cudaStream_t s);
cudaError_t launch_minres_scalars(double* sc, cudaStream_t s);
cudaError_t launch_minres_update(int64_t n, const double* z, const double* w, double* wold_to_wnew, double* x,
                                 const double* sc, cudaStream_t s);
cudaError_t launch_load_vector(int n, const double* fbar, double* b, cudaStream_t s);
// batched MINRES pieces: one task per problem (pointers per problem)
struct KTask {
  int64_t n;            // vector length
  double* sc;           // MINRES scalars of the problem
  const double* a;
  const double* b;
  double* c;
  double* d;
  int slot;             // scalar slot written by reductions
  double scale;         // reduction scale
};
enum KBatchOp { KB_DOT = 0, KB_SUM, KB_LANCZOS, KB_UPDATE, KB_SCALARS, KB_PDIV, KB_SUBS };
cudaError_t launch_krylov_batch(int op, const KTask* tasks, int ntasks, int64_t max_n, double* partials,
                                cudaStream_t s);
cudaError_t launch_mask_boundary(int n, double* x, cudaStream_t s);
// FGMRES pieces: out[i] = w . V_i (i < nvec, V_i = V + i ld); w += sign sum_i coef[i] V_i;
// y = a * s or a / s (s on the device)
cudaError_t launch_block_dot(int nvec, const double* V, int64_t ld, const double* w, int64_t n, double* partials,
                             double* out, cudaStream_t s);
cudaError_t launch_block_axpy(int nvec, const double* V, int64_t ld, const double* coef, double sign, double* w,
                              int64_t n, cudaStream_t s);
cudaError_t launch_scale(int64_t n, double* y, const double* a, const double* s_dev, bool recip, cudaStream_t s);
// assembled Z = B W^-1 B^T on the pressure grid as per-vertex stencils over
// the ZSTENCIL offsets that are sums of two Kuhn offsets, SoA [ZSTENCIL][V]
constexpr int ZSTENCIL = 65;
cudaError_t launch_colour5(int np, int colour, double* e, cudaStream_t s);
cudaError_t launch_scatter_zrow(int np, int colour, const double* y, double* zs, cudaStream_t s);
// x = Z^-1 r by `iters` Jacobi-PCG steps from 0 in one cooperative launch (r
// mean-free on entry, overwritten; x not projected); partials: partials_cap
// doubles of scratch
cudaError_t launch_zcg(int np, const double* zs, const double* dinv, double* x, double* r, double* p, double* q,
                       double* partials, int64_t partials_cap, int iters, cudaStream_t s);
cudaError_t launch_zdiag_inv(int np, const double* zs, double* dinv, cudaStream_t s);
cudaError_t launch_sensitivity(int n, const double* eta, const double* lam, const double* u, double* g,
                               cudaStream_t s);

}  // namespace agca
