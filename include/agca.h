/*
 * agca.h — C ABI of the GB300 (sm_103a) AGCA multigrid library.
 *
 * Adaptive Galerkin coarse-grid approximation (AGCA) multigrid for the
 * generalized variable-viscosity Stokes problem of arXiv 2511.13109:
 *   -div(2 eta eps(u)) + grad p = f,  -div u = 0 in the unit cube, u = 0 on
 *   the boundary (Eq. 3.1), discretized with the P1-iso-P2 / P1 pair (Eq. 3.3)
 *   on uniformly refined Kuhn tetrahedral grids (Eq. 2.2).
 *
 * Grid and vector conventions (every pointer argument below follows them):
 *  - N pressure cubes per axis; the velocity grid has n_L = 2N cubes per axis.
 *    Level l = 1 (coarsest) .. L (finest) has n_l = n_L / 2^(L-l) cubes per
 *    axis, V_l = (n_l+1)^3 vertices and E_l = 6 n_l^3 tetrahedra.
 *  - Vertex id = i + (n+1)*(j + (n+1)*k).  Cube id = i + n*(j + n*k); cube
 *    (i,j,k) is split along its main diagonal into 6 tetrahedra, type t being
 *    the t-th permutation p of (0,1,2) in lexicographic order, with local
 *    vertices v0 = origin, v1 = v0 + e_p0, v2 = v1 + e_p1, v3 = v0 + (1,1,1).
 *    Element id = 6*cube_id + t.
 *  - Velocity vectors are SoA: value of component c at vertex v is x[c*V + v],
 *    boundary vertices included.  Boundary entries of inputs are ignored;
 *    boundary entries of outputs are written as 0 (homogeneous Dirichlet).
 *  - Stokes vectors x = [u; p] hold 3*V_L velocity values followed by the
 *    (N+1)^3 pressure values of the level-(L-1) grid.
 *  - Local element DoF (vertex a, component c) has index c*4 + a; stored
 *    Galerkin matrices are 12x12 row-major in that index.
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller.  The
 * library allocates no device memory: the caller queries the workspace size,
 * allocates it (e.g. a torch uint8 tensor) and binds it; the size of the
 * Galerkin store is only known after flagging and is bound separately.
 * All calls run on the CUDA stream given at creation and are asynchronous,
 * except agca_flag, agca_setup, agca_solve, agca_adjoint_gradient,
 * agca_level_info, which synchronize that stream before returning.
 *
 * Errors: every call returns an agca_status; the library never aborts or
 * traps.  agca_last_error() gives a message for the last failing call on a
 * context.  A context is not thread safe.
 */
#ifndef AGCA_H_
#define AGCA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct agca_ctx agca_ctx;

typedef enum {
  AGCA_OK = 0,
  AGCA_EINVAL = 1,     /* bad argument (size, level, null pointer, NaN/<=0 viscosity) */
  AGCA_ENOMEM = 2,     /* bound workspace or Galerkin store too small */
  AGCA_ECUDA = 3,      /* a CUDA runtime call failed */
  AGCA_ENOTCONV = 4,   /* solver stopped at maxit above the tolerance */
  AGCA_ETIMEOUT = 5,   /* a bounded device wait gave up */
  AGCA_EINTERNAL = 6,  /* device-detected inconsistency (e.g. non-SPD coarsest matrix) */
  AGCA_ESTATE = 7      /* call out of order (e.g. apply before setup) */
} agca_status;

typedef enum { AGCA_FP64 = 0, AGCA_MIXED = 1 } agca_precision;
typedef enum { AGCA_F64 = 0, AGCA_F32 = 1 } agca_dtype;

/* Level data fields for agca_get_level_data. */
typedef enum {
  AGCA_FIELD_MEAN = 0,   /* double[E_l]: element viscosity (finest) or child mean (coarse) */
  AGCA_FIELD_MAX = 1,    /* double[E_l]: max finest viscosity under the element */
  AGCA_FIELD_MIN = 2,    /* double[E_l]: min finest viscosity under the element */
  AGCA_FIELD_FLAGS = 3,  /* uint8[E_l]: 1 if Galerkin-coarsened */
  AGCA_FIELD_LIST = 4,   /* int32[n_flag]: flagged element ids, ascending */
  AGCA_FIELD_GCA = 5,    /* double[n_flag*144]: stored Galerkin matrices, list order */
  AGCA_FIELD_DIAG = 6,   /* double[3*V_l]: diagonal of the level operator (0 on boundary) */
  AGCA_FIELD_COARSE = 7, /* double[m*m]: dense coarsest operator on interior DoFs (level 1 only) */
  AGCA_FIELD_PMASS = 8,  /* double[(N+1)^3]: viscosity-weighted lumped pressure mass (level L-1) */
  AGCA_FIELD_SIDX = 9,   /* int32[V_l]: stencil index of a vertex touched by a flagged element, else -1
                            (coarse levels, after agca_flag; touched vertices numbered in ascending order) */
  AGCA_FIELD_STENCIL = 10 /* double[n_stencil*135]: per touched vertex, the stored-Galerkin part of the
                            level operator as 15 Kuhn-offset blocks of 3x3 couplings, [offset][row c][column d],
                            offsets 0, +-x, +-y, +-z, +-(x+y), +-(x+z), +-(y+z), +-(x+y+z) (Remark 5) */
} agca_field;

typedef struct {
  int n;            /* cubes per axis */
  int64_t vertices; /* V_l */
  int64_t elements; /* E_l */
  int64_t n_flag;   /* flagged elements (0 on the finest level) */
  double lambda;    /* power-iteration estimate of lambda_max(D^-1 A_l) (0 on level 1) */
  int64_t n_stencil; /* vertices touched by flagged elements: stored stencils (0 on the finest level) */
} agca_level_info_t;

/* Human-readable name of a status code (static string). */
const char* agca_status_string(agca_status s);

/* Create a context for a velocity grid of 2N cubes per axis with n_levels
 * levels (1 <= N <= 256; 2N must be divisible by 2^(n_levels-1) with at
 * least 2 cubes per axis on level 1).  prec selects the V-cycle precision: AGCA_FP64, or
 * AGCA_MIXED (FP32 smoothing, transfers and coarse applies; FP64 Galerkin
 * assembly, coarsest solve and Krylov recurrence).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  Host-only; *out is owned by
 * the caller and released with agca_destroy. */
agca_status agca_create(int N, int n_levels, int prec, void* cuda_stream, agca_ctx** out);
void agca_destroy(agca_ctx* ctx);
const char* agca_last_error(const agca_ctx* ctx);

/* Smoother parameters (Section 4: Chebyshev smoother on D^-1 A): polynomial
 * degree, interval [lo, hi] * lambda_hat and the number of power iterations
 * for lambda_hat.  Defaults 2, 0.1, 1.1, 20.  Call before agca_setup. */
agca_status agca_set_smoother(agca_ctx* ctx, int degree, double lo, double hi, int power_iters);

/* Solver options: in mixed contexts each residual-refinement step runs
 * MINRES until the preconditioned residual norm has dropped by at least
 * mixed_inner_rtol (default 1e-4; the FP32 cycle and operator limit how far
 * one inner solve can usefully go); check_every MINRES iterations pass
 * between host-side convergence checks (default 4). */
agca_status agca_set_solver_options(agca_ctx* ctx, double mixed_inner_rtol, int check_every);

/* Coarse DCA coefficient of a coarse element from its 8 children's values
 * (Sec. 3.2, Fig. 6: the piecewise-constant projections): 0 = arithmetic
 * mean (default), 1 = harmonic mean 8 / sum(1/c_k), 2 = geometric mean
 * exp(sum(log c_k) / 8), sums in the fixed pairwise order
 * ((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)).  Takes effect at the next agca_flag.
 * Host only; AGCA_EINVAL for another kind. */
agca_status agca_set_coarse_projection(agca_ctx* ctx, int kind);

/* Bytes of device workspace the context needs (excluding the Galerkin store). */
agca_status agca_workspace_size(const agca_ctx* ctx, size_t* bytes);
/* Bind caller-owned device memory of at least agca_workspace_size bytes,
 * 256-byte aligned.  The memory must outlive the context's use. */
agca_status agca_bind_workspace(agca_ctx* ctx, void* dev_ptr, size_t bytes);

/* Copy the finest element viscosities eta (double[E_L], device) into the
 * workspace.  Every value must be finite and > 0 (checked on the device at
 * agca_flag: AGCA_EINVAL otherwise).  Eq. 3.5: only the element mean of eta
 * enters a P1 element matrix (Remark 3). */
agca_status agca_set_viscosity(agca_ctx* ctx, const double* eta_dev);

/* Build the viscosity hierarchy (per coarse element: mean, max and min over
 * its 8 children) and flag elements with max > nu * min for Galerkin
 * coarsening (element-wise form of Eq. 2.8); compact the flagged elements of
 * every coarse level in ascending id order.  Returns in *gca_bytes the size
 * of the Galerkin store to bind next.  Synchronizes. */
agca_status agca_flag(agca_ctx* ctx, double nu, size_t* gca_bytes);
/* As agca_flag, with the paper's own flag rule (Eq. 2.8) at element
 * granularity: a coarse element is flagged iff the norm of the gradient of
 * the P1 interpolant of the viscosity exceeds nu on at least one finest
 * element it covers.  eta_vertex_dev: the viscosity at the finest-grid
 * vertices (double[V_L], device, vertex order as for vectors, every value
 * finite and > 0; read during the call only).  The hierarchy of means,
 * maxima and minima is built as by agca_flag.  Synchronizes. */
agca_status agca_flag_gradient(agca_ctx* ctx, const double* eta_vertex_dev, double nu, size_t* gca_bytes);
/* Bind caller-owned device memory for the stored Galerkin matrices. */
agca_status agca_bind_gca_store(agca_ctx* ctx, void* dev_ptr, size_t bytes);

/* Direct coarse-grid approximation with a coefficient evaluated on the coarse
 * grid itself (Eq. 2.5; the coefficient approximations of Sec. 3.2): replace
 * the DCA coefficient of coarse level 1 <= level < L by coef_dev
 * (double[E_level], device, element order as on the finest level, every
 * value finite and > 0), e.g. the analytic viscosity's mean over the coarse
 * element's quadrature points or the mean of its P1 interpolant on the
 * coarse grid.  Call after agca_flag (which projects the children's means)
 * and before agca_setup; the flags and the per-element maxima and minima
 * stay those of the finest descendants, and coarser levels keep the
 * coefficients agca_flag projected.  Copies asynchronously on the context
 * stream.  AGCA_ESTATE before agca_flag; AGCA_EINVAL for a bad level. */
agca_status agca_set_level_coefficient(agca_ctx* ctx, int level, const double* coef_dev);

/* Assemble the local Galerkin matrices of all flagged elements, finest to
 * coarsest (Eqs. 2.6-2.7, Eq. B.2), the level diagonals, lambda_hat per level,
 * the dense Cholesky factor of the coarsest operator and the pressure mass.
 * Synchronizes. */
agca_status agca_setup(agca_ctx* ctx);

/* y = A_l x for level l (Eq. 2.3 at l = L; the heterogeneous AGCA operator of
 * Eq. 2.9 for l < L).  dtype AGCA_F64 uses the FP64 data; AGCA_F32 (mixed
 * contexts only) the FP32 data.  x, y: dtype[3*V_l]. */
agca_status agca_apply(agca_ctx* ctx, int level, int dtype, const void* x_dev, void* y_dev);
/* r_c = P^T r_f from level l to l-1 (linear interpolation transpose, Sec. 2.1);
 * boundary rows of r_c are 0.  r_f: dtype[3*V_l], r_c: dtype[3*V_{l-1}]. */
agca_status agca_restrict(agca_ctx* ctx, int level, int dtype, const void* rf_dev, void* rc_dev);
/* x_f += P e_c from level l-1 to l. */
agca_status agca_prolong_add(agca_ctx* ctx, int level, int dtype, const void* ec_dev, void* xf_dev);
/* One V-cycle z = V(r) on the velocity block from z = 0 (Section 4: Chebyshev
 * pre/post smoothing, AGCA coarse operators, exact coarsest solve).
 * r, z: double[3*V_L]; in mixed contexts the cycle runs in FP32. */
agca_status agca_vcycle(agca_ctx* ctx, const double* r_dev, double* z_dev);

/* Stokes operator y = K x, K = [[A, B^T], [B, 0]] with B = -D,
 * D_kj = int psi_k div Phi_j (Eqs. 3.4-3.5).  x, y: double[3*V_L + (N+1)^3]. */
agca_status agca_stokes_apply(agca_ctx* ctx, const double* x_dev, double* y_dev);
/* Block-diagonal preconditioner z = diag(V-cycle, Pi M^-1 Pi) r with M the
 * lumped 1/eta-weighted pressure mass and Pi the mean-zero projection. */
agca_status agca_precondition(agca_ctx* ctx, const double* r_dev, double* z_dev);
/* Right-hand side b = [f; 0] with f_(a,c) = sum_T |T| fbar_c(T) / 4 for the
 * element-mean forcing fbar: double[3*E_L] (SoA by component). */
agca_status agca_load_vector(agca_ctx* ctx, const double* fbar_dev, double* b_dev);

/* Solve K x = b to ||b - K x||_2 <= rtol ||b||_2 on the true FP64 residual:
 * residual refinement around preconditioned MINRES (Remark 6), at most maxit
 * MINRES iterations in total.  x is overwritten (initial guess 0); the
 * pressure is returned with zero mean.  *iters, *relres (host) receive the
 * iteration count and final relative residual.  Synchronizes.  Returns
 * AGCA_ENOTCONV if the tolerance was not met. */
agca_status agca_solve(agca_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit,
                       int* iters, double* relres);

/* The paper's outer solver (Sec. 4): flexible GMRES, restarted every
 * `restart` iterations, right-preconditioned by the block-triangular
 * preconditioner of Eq. 4.1 (z_p = -S~^-1 r_p, z_u = V-cycle(r_u - B^T z_p),
 * the signs of K = [[A, B^T], [B, 0]] with B = -D), stopping when the
 * residual norm of the Arnoldi process, then of the true FP64 residual, is
 * at most rtol ||b|| (Eq. 4.3).  schur: 0 = S~^-1 the mean-free lumped 1/eta
 * pressure mass; 1 = the diag(A)-BFBT of Eq. 4.2, S~^-1 = Z^-1 (B W^-1 A
 * W^-1 B^T) Z^-1 with W = diag(A), Z = B W^-1 B^T assembled at each call
 * on the pressure grid (App. B; Z couples pressure vertices whose offset is
 * a sum of two Kuhn offsets, 65 in all, and 125 matrix-free applies to
 * colour indicators give those stencils) and Z^-1 by z_iters steps of
 * Jacobi-preconditioned conjugate gradients on the mean-free pressures (one
 * cooperative launch per solve; the device must support cooperative
 * launches, else the call fails with AGCA_ECUDA).
 * work_dev: caller-owned device memory of agca_fgmres_workspace_size bytes
 * (256-byte aligned; holds the 2 restart + 1 Krylov vectors and Z).  x is
 * overwritten (initial guess 0; pressure returned mean-free).  *iters,
 * *relres (host): iterations and the final true relative residual.
 * Synchronizes (once per iteration).  AGCA_ENOTCONV above the tolerance
 * after maxit iterations. */
agca_status agca_fgmres_workspace_size(const agca_ctx* ctx, int restart, size_t* bytes);
agca_status agca_solve_fgmres(agca_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit, int restart,
                              int schur, int z_iters, void* work_dev, size_t work_bytes, int* iters, double* relres);

/* Element sensitivities g_e = -lambda_e^T (dA_e/dtheta_e) u_e for theta =
 * log(eta) (the viscous element matrix is linear in eta_e).  lam_u, u:
 * double[3*V_L]; g: double[E_L]. */
agca_status agca_element_sensitivity(agca_ctx* ctx, const double* lam_u_dev, const double* u_dev,
                                     double* g_dev);
/* Adjoint gradient of J(u) w.r.t. theta = log(eta): solves K lambda =
 * (dJ/du, 0) with the same preconditioned solver (K is symmetric) to rtol,
 * then g = agca_element_sensitivity(lambda_u, u).  x: the forward solution
 * [u; p]; dJdu: double[3*V_L]; g: double[E_L].  Synchronizes. */
agca_status agca_adjoint_gradient(agca_ctx* ctx, const double* x_dev, const double* dJdu_dev,
                                  double* g_dev, double rtol, int maxit, int* iters);

/* Allocation-free Stokes apply y = K x on the finest grid of N pressure cubes
 * per axis, for callers that cannot allocate device memory themselves (code
 * whose device memory belongs to another allocator or pool it must not
 * bypass, or loops that cannot afford an allocation).  No context, workspace
 * or allocation: the operator's two fine-grid scratch fields live in a fixed
 * device array inside the library, held by every GPU that loads it until the
 * process exits.  The paper has no counterpart of this entry point.
 *   N: 1..32 (AGCA_EINVAL beyond: the scratch holds 2 (2N+1)^3 doubles);
 *   eta: double[6 (2N)^3] element viscosities (as agca_set_viscosity);
 *   x, y: double[3 (2N+1)^3 + (N+1)^3] Stokes vectors as agca_stokes_apply;
 *   cuda_stream: cudaStream_t (NULL = legacy default stream).
 * eta, x and y must be device memory of the current device (AGCA_EINVAL
 * otherwise); the stream must belong to the current device.
 * The scratch array's device address belongs to a CUDA context: the first
 * call under each context (normally once per device, in its primary
 * context) looks it up and caches it by the context's unique ID, so a call
 * under another context never uses a stale address.  Make that first call
 * before any stream capture.  Every call uses the same scratch and
 * overwrites all of it that it reads, so nothing needs clearing; calls that
 * overlap on the GPU (other streams, other host threads) race on it.
 * Asynchronous; returns AGCA_ECUDA if a launch fails. */
agca_status agca_stokes_apply_static(int N, const double* eta_dev, const double* x_dev, double* y_dev,
                                     void* cuda_stream);

/* Autotuner: for every level >= 2 and V-cycle stencil mode (0 apply,
 * 1 residual, 2 first and 3 later Chebyshev steps, 4 pre-smoothing step from
 * zero), time the candidate tile shapes (block rows 8/12/16 in FP32, 8 in
 * FP64; z-chunks 1..64) with CUDA events on the context stream, reps
 * launches each, and keep the fastest for the context's later launches.
 * cache_path (nullable): text file of earlier results, read first and
 * rewritten.  Uses the cycle vectors as scratch.  Synchronizes. */
agca_status agca_autotune(agca_ctx* ctx, int reps, const char* cache_path);
/* The tile shape in use for (level, mode): block rows and z-chunk (0 = automatic). */
agca_status agca_tile_config(const agca_ctx* ctx, int level, int mode, int* by, int* zch);
/* Set the tile shape of (level, mode) by hand (mode 5: the Stokes operator
 * on the finest level): by = 8, 12 or 16 block rows (12 and 16 in FP32 only),
 * zch = z-chunk in vertex planes (0 = automatic, at most 4096).  Results do
 * not depend on the tile shape: every vertex sums its element contributions
 * in the same order.  Host only; AGCA_EINVAL for other values. */
agca_status agca_set_tile_config(agca_ctx* ctx, int level, int mode, int by, int zch);
/* The tile grid the stencil kernels use on a grid of n cubes per axis with
 * by block rows and z-chunk request zch (0 = automatic): out[0..6] = wide
 * strips in x, wide tile rows in y, narrow strips in x, narrow tile rows in
 * y, first vertex column of the narrow strips, z-chunks, vertex planes per
 * z-chunk.  Wide tiles own 31 x (by - 1) vertex columns x rows, narrow tiles
 * 7 x (4 by - 1); every vertex of the (n+1)^2 plane is owned by exactly one
 * tile and every vertex plane by exactly one z-chunk.  out is a host array
 * of 7 ints.  Host only, no context; AGCA_EINVAL for n < 1, n > 1024, by not
 * 8, 12 or 16, or zch < 0. */
agca_status agca_stencil_tiles(int n, int by, int zch, int* out);

/* Number of CUDA kernels this context has launched so far (host counter). */
agca_status agca_launch_count(const agca_ctx* ctx, int64_t* launches);
/* Per-launch timing of the finest-level stencil kernels (the dominant
 * kernels of the V-cycle), with CUDA events on the context stream.
 * enable = 1 starts recording (up to 65536 launches); enable = 0 stops,
 * synchronizes and returns the summed kernel time in *ms, their compulsory
 * HBM bytes (element coefficients and vectors read/written once) in *bytes,
 * their algorithmic arithmetic in *flops (the edge form of the element
 * action of Eq. 3.5 with per-vertex coefficient records: 84 flops per
 * vertex for the operator plus the epilogue's, a fused multiply-add
 * counting 2) and the number of timed launches.  Output pointers are host
 * pointers and may be NULL. */
agca_status agca_profile_fine(agca_ctx* ctx, int enable, double* ms, double* bytes, double* flops,
                              int64_t* launches);

/* ------------------------------------------------------------------------
 * Batched solves of many independent problems (uneven sizes allowed).
 * Every problem keeps its own hierarchy; the MINRES iterations of all
 * problems run in lockstep, each launch covering every problem: the stencil
 * launches are persistent (every CTA walks the flattened (problem, tile)
 * work list) and one lockstep iteration pair is captured once as a CUDA graph
 * (when the stream is not the legacy default stream) and replayed.
 * Converged problems are skipped on the device.  The batch owns its
 * sub-contexts; device memory is bound by the caller as for one context.
 * ---------------------------------------------------------------------- */
typedef struct agca_batch agca_batch;
/* n problems with Ns[i] pressure cubes per axis, default level counts
 * (coarsen while the velocity grid stays even with >= 4 cubes), one
 * precision for all; degree-2 Chebyshev smoothing. */
agca_status agca_batch_create(int n, const int* Ns, int prec, void* cuda_stream, agca_batch** out);
void agca_batch_destroy(agca_batch* b);
const char* agca_batch_last_error(const agca_batch* b);
agca_status agca_batch_workspace_size(const agca_batch* b, size_t* bytes);
agca_status agca_batch_bind_workspace(agca_batch* b, void* dev_ptr, size_t bytes);
/* as agca_set_viscosity for problem i */
agca_status agca_batch_set_viscosity(agca_batch* b, int i, const double* eta_dev);
/* as agca_flag for every problem; *gca_bytes: the total Galerkin store */
agca_status agca_batch_flag(agca_batch* b, double nu, size_t* gca_bytes);
agca_status agca_batch_bind_gca_store(agca_batch* b, void* dev_ptr, size_t bytes);
/* as agca_setup for every problem, then builds the batched task tables and
 * captures the lockstep iteration graph.  Synchronizes. */
agca_status agca_batch_setup(agca_batch* b);
/* as agca_load_vector for problem i */
agca_status agca_batch_load_vector(agca_batch* b, int i, const double* fbar_dev, double* b_dev);
/* One V-cycle for every problem: z_devs[i] = V_i(r_devs[i]) (host arrays of
 * n device pointers).  Synchronizes. */
agca_status agca_batch_vcycle(agca_batch* b, const double* const* r_devs, double* const* z_devs);
/* Solve every problem to ||b_i - K_i x_i|| <= rtol ||b_i|| (as agca_solve);
 * iters, relres: host arrays of n (may be NULL).  Synchronizes. */
agca_status agca_batch_solve(agca_batch* b, const double* const* b_devs, double* const* x_devs, double rtol, int maxit,
                             int* iters, double* relres);
/* The context of problem i (owned by the batch): parity hooks such as
 * agca_get_level_data, agca_apply, agca_level_info. */
agca_ctx* agca_batch_context(agca_batch* b, int i);

/* Level metadata (host struct).  Synchronizes. */
agca_status agca_level_info(agca_ctx* ctx, int level, agca_level_info_t* out);
/* Copy a level field (agca_field) into caller device memory. */
agca_status agca_get_level_data(agca_ctx* ctx, int level, int field, void* dst_dev);

#ifdef __cplusplus
}
#endif
#endif /* AGCA_H_ */
