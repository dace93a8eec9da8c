// C ABI of libagca (include/agca.h): context, workspace layout, setup
// sequence, V-cycle and Krylov drivers.  Host code only; every numerical
// step runs in the kernels of stencil.cu, transfer.cu, setup.cu, krylov.cu.
#include <math.h>

#include <algorithm>
#include <array>
#include <fstream>
#include <map>
#include <sstream>
#include <type_traits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "agca_internal.cuh"

using namespace agca;

namespace {

constexpr size_t kAlign = 256;

struct Level {
  int n = 0;
  int64_t V = 0, E = 0;
  // FP64 data
  double* mean = nullptr;  // eta on the finest level
  double* mx = nullptr;    // == mean on the finest level
  double* mn = nullptr;
  uint8_t* flags = nullptr;
  int32_t* fidx = nullptr;
  int32_t* list = nullptr;
  int64_t n_flag = 0;
  double* gca64 = nullptr;
  double* hedge = nullptr;  // FP64 contexts: per-vertex coefficient records [EREC][V] of the edge form
  double* coefm = nullptr;  // FP64 coarse levels: DCA coefficient with flagged elements zeroed (edge form)
  // stencil storage of the flagged elements' Galerkin matrices (Remark 5)
  uint8_t* vmark = nullptr;   // vertex touched by a flagged element
  int32_t* sidx = nullptr;    // stencil index of a vertex or -1
  int32_t* slist = nullptr;   // touched vertices, ascending
  int64_t n_sv = 0;
  double* sten64 = nullptr;   // n_sv * 135
  float* sten32 = nullptr;    // mixed: S / s_v
  float* sscale32 = nullptr;  // mixed: s_v
  double* diag = nullptr;
  double* invD64 = nullptr;
  // FP32 copies (mixed)
  float* mean32 = nullptr;
  float* invD32 = nullptr;
  float* gca32 = nullptr;
  float* gscale32 = nullptr;
  // s_e A_e x_e of the flagged elements (coarse-apply scratch)
  double* ye64 = nullptr;
  float* ye32 = nullptr;
  // V-cycle vectors in the cycle precision: rhs, two iterate buffers, residual
  void* vb = nullptr;
  void* vx = nullptr;
  void* vt = nullptr;
  void* vr = nullptr;
  double lambda = 0.0;
};

enum KVec { KV_VOLD = 0, KV_V, KV_Z, KV_ZNEW, KV_WOLD, KV_W, KV_KZ, KV_R, KV_D, KV_B, KV_ARHS, KV_ALAM, KV_COUNT };

}  // namespace

struct agca_ctx {
  int N = 0, L = 0, prec = 0;
  cudaStream_t stream = nullptr;
  int cheb_degree = 2;
  double cheb_lo = 0.1, cheb_hi = 1.1;
  int power_iters = 20;
  double mixed_inner = 1e-4;  // floor of the inner MINRES tolerance in mixed refinement
  int projection = 0;         // coarse DCA coefficient: 0 arithmetic, 1 harmonic, 2 geometric mean
  int check_every = 4;        // MINRES iterations between host convergence checks
  std::vector<Level> lev;  // 1..L
  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0, ws_need = 0;
  char* gs = nullptr;
  size_t gs_bytes = 0, gs_need = 0;
  // coarsest
  int mc = 0;
  double *cdense = nullptr, *cfac = nullptr, *linv_cm = nullptr, *linv_rm = nullptr;
  // pressure
  int64_t Vp = 0;
  double *pmass = nullptr, *pmass_inv = nullptr, *qfine = nullptr, *sfine = nullptr;
  // krylov
  int64_t nt = 0;
  double* kv[KV_COUNT] = {};
  double* sc = nullptr;
  double* partials = nullptr;
  int* status = nullptr;
  int64_t* totals = nullptr;
  int32_t* block_counts = nullptr;
  double nu = 10.0;
  bool have_eta = false, flagged = false, setup_done = false;
  std::string err;
  // kernel launches issued by this context, and optional per-launch timing
  // of the finest-level stencil kernels (agca_profile_fine)
  int64_t launches = 0;
  // tile shape per level and stencil mode (autotuner; default by = 8, automatic z-chunk)
  std::vector<std::array<TileCfg, 6>> tune;
  // V-cycles replayed from CUDA graphs, keyed by their (input, output) pointers
  struct GraphEntry {
    const void* r;
    void* z;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<GraphEntry> graphs;
  // two MINRES iterations (the buffer rotation returns after two) replayed
  // from a CUDA graph; [0]: FP64 operator, [1]: FP32-compute operator
  cudaGraphExec_t minres_graph[2] = {nullptr, nullptr};
  const double* minres_key[2] = {nullptr, nullptr};  // the correction vector d the graph updates
  int64_t minres_launches[2] = {0, 0};
  bool use_graphs = true;
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  double prof_bytes = 0.0;
  double prof_flops = 0.0;
  int64_t prof_launches = 0;

  ~agca_ctx() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    clear_graphs();
  }
  void clear_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    for (int i = 0; i < 2; ++i) {
      if (minres_graph[i]) cudaGraphExecDestroy(minres_graph[i]);
      minres_graph[i] = nullptr;
      minres_key[i] = nullptr;
    }
  }

  agca_status fail(agca_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  size_t cyc() const { return prec == AGCA_MIXED ? sizeof(float) : sizeof(double); }
};

#define CK(...)                                                                                      \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      return ctx->fail(AGCA_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));       \
  } while (0)
#define LK(count, ...)          \
  do {                          \
    CK(__VA_ARGS__);            \
    ctx->launches += (count);   \
  } while (0)
#define CKS(expr)                  \
  do {                             \
    agca_status s_ = (expr);       \
    if (s_ != AGCA_OK) return s_;  \
  } while (0)

namespace {

// Assigns 256-byte aligned offsets; with base == nullptr it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <typename T>
  T* take(int64_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (size_t)count * sizeof(T);
    return p;
  }
};

void carve_workspace(agca_ctx* ctx, char* base) {
  Carver cv(base);
  const bool mixed = ctx->prec == AGCA_MIXED;
  int64_t max_coarse_e = 1;
  for (int l = 1; l <= ctx->L; ++l) {
    Level& lv = ctx->lev[l];
    lv.mean = cv.take<double>(lv.E);
    if (l < ctx->L) {
      lv.mx = cv.take<double>(lv.E);
      lv.mn = cv.take<double>(lv.E);
      lv.flags = cv.take<uint8_t>(lv.E);
      lv.fidx = cv.take<int32_t>(lv.E);
      lv.list = cv.take<int32_t>(lv.E);
      max_coarse_e = std::max(max_coarse_e, lv.E);
    } else {
      lv.mx = lv.mean;
      lv.mn = lv.mean;
    }
    if (mixed) lv.mean32 = cv.take<float>(lv.E);
    if (!mixed) lv.hedge = cv.take<double>(EREC * lv.V);
    if (!mixed && l < ctx->L) lv.coefm = cv.take<double>(lv.E);
    if (l < ctx->L) {
      lv.vmark = cv.take<uint8_t>(lv.V);
      lv.sidx = cv.take<int32_t>(lv.V);
      lv.slist = cv.take<int32_t>(lv.V);
    }
    lv.diag = cv.take<double>(3 * lv.V);
    lv.invD64 = cv.take<double>(3 * lv.V);
    if (mixed) lv.invD32 = cv.take<float>(3 * lv.V);
    const size_t es = ctx->cyc();
    lv.vb = cv.take<char>(3 * lv.V * (int64_t)es);
    lv.vx = cv.take<char>(3 * lv.V * (int64_t)es);
    lv.vt = cv.take<char>(3 * lv.V * (int64_t)es);
    lv.vr = cv.take<char>(3 * lv.V * (int64_t)es);
  }
  ctx->block_counts = cv.take<int32_t>(compact_scratch_blocks(max_coarse_e) + 1);
  ctx->totals = cv.take<int64_t>(2 * (ctx->L + 1));  // flagged elements, then touched vertices, per level
  ctx->status = cv.take<int>(4);
  ctx->sc = cv.take<double>(64);
  ctx->partials = cv.take<double>(3 * (int64_t)dot_blocks());
  const int64_t m2 = (int64_t)ctx->mc * ctx->mc;
  ctx->cdense = cv.take<double>(m2);
  ctx->cfac = cv.take<double>(m2);
  ctx->linv_cm = cv.take<double>(m2);
  ctx->linv_rm = cv.take<double>(m2);
  ctx->pmass = cv.take<double>(ctx->Vp);
  ctx->pmass_inv = cv.take<double>(ctx->Vp);
  ctx->qfine = cv.take<double>(ctx->lev[ctx->L].V);
  ctx->sfine = cv.take<double>(ctx->lev[ctx->L].V);
  for (int i = 0; i < KV_COUNT; ++i) ctx->kv[i] = cv.take<double>(ctx->nt);
  ctx->ws_need = (cv.off + kAlign - 1) / kAlign * kAlign;
}

void carve_gca(agca_ctx* ctx, char* base) {
  Carver cv(base);
  const bool mixed = ctx->prec == AGCA_MIXED;
  for (int l = 1; l < ctx->L; ++l) {
    Level& lv = ctx->lev[l];
    lv.gca64 = cv.take<double>(std::max<int64_t>(1, lv.n_flag * 144));
    lv.ye64 = cv.take<double>(std::max<int64_t>(1, lv.n_flag * 12));
    lv.sten64 = cv.take<double>(std::max<int64_t>(1, lv.n_sv * 135));
    if (mixed) {
      lv.ye32 = cv.take<float>(std::max<int64_t>(1, lv.n_flag * 12));
      lv.gca32 = cv.take<float>(std::max<int64_t>(1, lv.n_flag * 144));
      lv.gscale32 = cv.take<float>(std::max<int64_t>(1, lv.n_flag));
      lv.sten32 = cv.take<float>(std::max<int64_t>(1, lv.n_sv * 135));
      lv.sscale32 = cv.take<float>(std::max<int64_t>(1, lv.n_sv));
    }
  }
  ctx->gs_need = (cv.off + kAlign - 1) / kAlign * kAlign;
}

LevelOp<double> op64(const agca_ctx* ctx, int l) {
  const Level& lv = ctx->lev[l];
  LevelOp<double> op{};
  op.n = lv.n;
  op.h6 = 1.0 / (6.0 * lv.n);
  op.hq = 1.0 / (6.0 * (double)lv.n * lv.n);
  op.coef = lv.mean;
  op.hedge = lv.hedge;
  if (l < ctx->L) {
    op.coefm = lv.coefm;
    op.sidx = lv.sidx;
    op.sten = lv.n_sv > 0 ? lv.sten64 : nullptr;
    op.fidx = lv.fidx;
    op.gca = lv.gca64;
    op.list = lv.list;
    op.n_flag = lv.n_flag;
    op.ye = lv.ye64;
  }
  return op;
}

LevelOp<float> op32(const agca_ctx* ctx, int l) {
  const Level& lv = ctx->lev[l];
  LevelOp<float> op{};
  op.n = lv.n;
  op.h6 = (float)(1.0 / (6.0 * lv.n));
  op.hq = (float)(1.0 / (6.0 * (double)lv.n * lv.n));
  op.coef = lv.mean32;
  if (l < ctx->L) {
    op.sidx = lv.sidx;
    op.sten = lv.n_sv > 0 ? lv.sten32 : nullptr;
    op.sscale = lv.n_sv > 0 ? lv.sscale32 : nullptr;
    op.fidx = lv.fidx;
    op.gca = lv.gca32;
    op.gscale = lv.gscale32;
    op.list = lv.list;
    op.n_flag = lv.n_flag;
    op.ye = lv.ye32;
  }
  return op;
}

template <typename T>
LevelOp<T> level_op(const agca_ctx* ctx, int l);
template <>
LevelOp<double> level_op<double>(const agca_ctx* ctx, int l) {
  return op64(ctx, l);
}
template <>
LevelOp<float> level_op<float>(const agca_ctx* ctx, int l) {
  return op32(ctx, l);
}

template <typename T>
const T* invD_of(const Level& lv);
template <>
const double* invD_of<double>(const Level& lv) {
  return lv.invD64;
}
template <>
const float* invD_of<float>(const Level& lv) {
  return lv.invD32;
}

struct Cheb {
  double theta, delta, sigma;
};
Cheb cheb_params(const agca_ctx* ctx, int l) {
  const double lam = ctx->lev[l].lambda;
  const double a = ctx->cheb_lo * lam, b = ctx->cheb_hi * lam;
  Cheb c;
  c.theta = 0.5 * (b + a);
  c.delta = 0.5 * (b - a);
  c.sigma = c.theta / c.delta;
  return c;
}

// Compulsory HBM bytes per vertex of one finest-level stencil launch: the
// element coefficients (6 per vertex) plus every vector read and written
// once (3 components each).
double stencil_bytes(int mode, size_t s) {
  const double coef = 6.0 * s, vec = 3.0 * s;
  switch (mode) {
    case ST_APPLY: return coef + 2 * vec;        // x in, y out
    case ST_RESID: return coef + 3 * vec;        // x, b in, r out
    case ST_CHEB_FIRST: return coef + 4 * vec;   // x, b, D^-1 in, x' out
    case ST_CHEB_STEP: return coef + 5 * vec;    // x, x_prev, b, D^-1 in, x' out
    case ST_CHEB_PRE: return coef + 3 * vec;     // b, D^-1 in, x' out
    default: return 0.0;
  }
}

// Algorithmic arithmetic per vertex of one finest-level stencil launch (flops;
// a fused multiply-add counts 2), from the edge form of Eq. 3.5 on a Kuhn
// grid with the per-vertex coefficient records: 9 edge differences (3 axis
// edges x 3 components); per axis edge the on-axis flux 2 H d (2) and two
// off-axis components H d + four weighted differences (2 x 9); the
// divergence of the 6 fluxes at the vertex (15): 84 in all (the
// per-tetrahedron form of the same operator takes 129).  The scaling by h/6
// folds into the epilogue (3 products, or a fused b - (h/6) y).  The
// Chebyshev epilogues add per component: residual 2, first step 5, later
// step 8, step from zero 7 plus 2 for its staged first iterate.
double stencil_flops(int mode) {
  const double op = 9.0 + 3.0 * (2.0 + 2.0 * 9.0) + 15.0;
  switch (mode) {
    case ST_APPLY: return op + 3.0;
    case ST_RESID: return op + 3.0 * 2.0;
    case ST_CHEB_FIRST: return op + 3.0 * 5.0;
    case ST_CHEB_STEP: return op + 3.0 * 8.0;
    case ST_CHEB_PRE: return op + 3.0 * (7.0 + 2.0);
    default: return 0.0;
  }
}

template <typename T>
agca_status stencil(agca_ctx* ctx, int mode, int l, const T* x, const T* b, const T* xprev, T* out, double s0,
                    double s1, double s2, double* out64 = nullptr) {
  const Level& lv = ctx->lev[l];
  StencilArgs<T> a{};
  a.x = x;
  a.b = b;
  a.invD = invD_of<T>(lv);
  a.xprev = xprev;
  a.out = out;
  a.out64 = out64;
  a.s0 = (T)s0;
  a.s1 = (T)s1;
  a.s2 = (T)s2;
  const bool timed = ctx->prof && l == ctx->L && ctx->ev_used + 2 <= ctx->ev.size();
  if (timed) CK(cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream));
  const TileCfg* cfg = (mode >= 0 && mode < 6) ? &ctx->tune[l][mode] : nullptr;
  LK((l < ctx->L && lv.n_flag > 0) ? 2 : 1, launch_stencil<T, T>(mode, level_op<T>(ctx, l), a, ctx->stream, cfg));
  if (timed) {
    CK(cudaEventRecord(ctx->ev[ctx->ev_used + 1], ctx->stream));
    ctx->ev_used += 2;
    // an FP64-widened result writes 3 * (8 - sizeof(T)) more bytes per vertex
    const double wide = out64 ? 3.0 * (sizeof(double) - sizeof(T)) : 0.0;
    ctx->prof_bytes += (stencil_bytes(mode, sizeof(T)) + wide) * (double)lv.V;
    ctx->prof_flops += stencil_flops(mode) * (double)lv.V;
    ctx->prof_launches += 1;
  }
  return AGCA_OK;
}

// Chebyshev smoothing of A_l x = b (Section 4).  from_zero: start at x = 0
// (the result of the first step is staged on the fly); otherwise start at
// *cur.  cur/other are the two iterate buffers; returns the result buffer.
// final64: if set, the last step writes its result there, widened to FP64,
// instead of to the iterate buffers (the end of a mixed-precision cycle).
template <typename T>
agca_status chebyshev(agca_ctx* ctx, int l, const T* b, bool from_zero, T** cur, T** other,
                      double* final64 = nullptr) {
  const Cheb c = cheb_params(ctx, l);
  const int k = ctx->cheb_degree;
  double rho = 1.0 / c.sigma;
  int step = 1;
  if (from_zero && k == 2) {
    const double rn = 1.0 / (2.0 * c.sigma - rho);
    CKS(stencil<T>(ctx, ST_CHEB_PRE, l, nullptr, b, nullptr, *cur, rn * rho, 2.0 * rn / c.delta, 1.0 / c.theta));
    return AGCA_OK;
  }
  if (from_zero) CK(cudaMemsetAsync(*cur, 0, 3 * ctx->lev[l].V * sizeof(T), ctx->stream));
  // first step: other = cur + D^-1 (b - A cur) / theta
  CKS(stencil<T>(ctx, ST_CHEB_FIRST, l, *cur, b, nullptr, *other, 1.0 / c.theta, 0.0, 0.0,
                 k == 1 ? final64 : nullptr));
  std::swap(*cur, *other);  // cur = x1, other = x0
  for (step = 1; step < k; ++step) {
    const double rn = 1.0 / (2.0 * c.sigma - rho);
    // x_{i+1} = x_i + rn*rho (x_i - x_{i-1}) + (2 rn / delta) D^-1 (b - A x_i), written over x_{i-1}
    CKS(stencil<T>(ctx, ST_CHEB_STEP, l, *cur, b, *other, *other, rn * rho, 2.0 * rn / c.delta, 0.0,
                   step + 1 == k ? final64 : nullptr));
    std::swap(*cur, *other);
    rho = rn;
  }
  return AGCA_OK;
}

// V-cycle on level l for rhs b; X, Tb are the iterate buffers.  Returns the
// buffer holding the result in *res, or writes it to final64 (FP64) if set.
template <typename T>
agca_status cycle(agca_ctx* ctx, int l, const T* b, T* X, T* Tb, T** res, double* final64 = nullptr) {
  if (l == 1) {
    LK(1, launch_coarse_solve<T>(ctx->lev[1].n, ctx->linv_cm, ctx->linv_rm, b, X, ctx->stream));
    *res = X;
    return AGCA_OK;
  }
  Level& lv = ctx->lev[l];
  Level& lc = ctx->lev[l - 1];
  T* cur = X;
  T* other = Tb;
  CKS(chebyshev<T>(ctx, l, b, true, &cur, &other));
  T* r = static_cast<T*>(lv.vr);
  CKS(stencil<T>(ctx, ST_RESID, l, cur, b, nullptr, r, 0, 0, 0));
  T* bc = static_cast<T*>(lc.vb);
  LK(1, launch_restrict<T>(lv.n, 3, true, T(1), r, bc, ctx->stream));
  T* ec = nullptr;
  CKS(cycle<T>(ctx, l - 1, bc, static_cast<T*>(lc.vx), static_cast<T*>(lc.vt), &ec));
  LK(1, launch_prolong<T>(lv.n, 3, true, true, ec, cur, ctx->stream));
  CKS(chebyshev<T>(ctx, l, b, false, &cur, &other, final64));
  *res = cur;
  return AGCA_OK;
}

agca_status vcycle_direct(agca_ctx* ctx, const double* r, double* z) {
  const int L = ctx->L;
  Level& lf = ctx->lev[L];
  const int64_t n3 = 3 * lf.V;
  if (ctx->prec == AGCA_FP64) {
    double* res = nullptr;
    CKS(cycle<double>(ctx, L, r, z, static_cast<double*>(lf.vt), &res));
    if (res != z) CK(cudaMemcpyAsync(z, res, n3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    float* b32 = static_cast<float*>(lf.vb);
    LK(1, launch_d2f(r, b32, n3, ctx->stream));
    float* res = nullptr;
    CKS(cycle<float>(ctx, L, b32, static_cast<float*>(lf.vx), static_cast<float*>(lf.vt), &res, z));
  }
  return AGCA_OK;
}

// One V-cycle, replayed from a CUDA graph captured on first use for this
// (r, z) pair: the cycle is a fixed sequence of ~40 launches whose
// parameters only change at setup.  Direct launches when the stream is the
// legacy default stream, is already being captured by the caller, or while
// per-launch timing is on.
agca_status vcycle_impl(agca_ctx* ctx, const double* r, double* z) {
  cudaStream_t s = ctx->stream;
  bool graph = ctx->use_graphs && !ctx->prof && s != nullptr;
  if (graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    graph = (cs == cudaStreamCaptureStatusNone);
  }
  if (!graph) return vcycle_direct(ctx, r, z);
  for (auto& g : ctx->graphs) {
    if (g.r == r && g.z == z) {
      CK(cudaGraphLaunch(g.exec, s));
      ctx->launches += g.launches;
      return AGCA_OK;
    }
  }
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->use_graphs = false;
    return vcycle_direct(ctx, r, z);
  }
  const int64_t l0 = ctx->launches;
  const agca_status st = vcycle_direct(ctx, r, z);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(s, &g);
  const int64_t nl = ctx->launches - l0;
  ctx->launches = l0;
  if (st != AGCA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ee != cudaSuccess) return ctx->fail(AGCA_ECUDA, std::string("V-cycle capture: ") + cudaGetErrorString(ee));
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return ctx->fail(AGCA_ECUDA, std::string("V-cycle graph: ") + cudaGetErrorString(ie));
  if (ctx->graphs.size() >= 16) {
    cudaGraphExecDestroy(ctx->graphs.front().exec);
    ctx->graphs.erase(ctx->graphs.begin());
  }
  ctx->graphs.push_back({r, z, exec, nl});
  CK(cudaGraphLaunch(exec, s));
  ctx->launches += nl;
  return AGCA_OK;
}

// K x = [A u + B^T p ; B u], B = -P^T B_f, B^T p = -B_f^T (P p)
template <typename TC>
agca_status stokes_impl(agca_ctx* ctx, const double* x, double* y) {
  const int L = ctx->L;
  const Level& lf = ctx->lev[L];
  const int64_t n3 = 3 * lf.V;
  LK(1, launch_prolong<double>(lf.n, 1, false, false, x + n3, ctx->qfine, ctx->stream));
  StencilArgs<double> a{};
  a.x = x;
  a.q = ctx->qfine;
  a.out = y;
  a.out2 = ctx->sfine;
  if (std::is_same<TC, double>::value && lf.hedge) {
    // FP64 context: the viscous block in edge form (A u into y), then the
    // pressure coupling per cube added to it (y = A u - B_f^T q, B_f u)
    StencilArgs<double> e{};
    e.x = x;
    e.out = y;
    LK(1, launch_stencil<double, double>(ST_APPLY, op64(ctx, L), e, ctx->stream));
    a.b = y;
    LK(1, launch_stencil<double, double>(ST_STOKES_B, op64(ctx, L), a, ctx->stream));
  } else {
    LK(1, launch_stencil<double, TC>(ST_STOKES, level_op<TC>(ctx, L), a, ctx->stream));
  }
  LK(1, launch_restrict<double>(lf.n, 1, false, -1.0, ctx->sfine, y + n3, ctx->stream));
  return AGCA_OK;
}

agca_status stokes_dispatch(agca_ctx* ctx, const double* x, double* y, bool low) {
  if (low && ctx->prec == AGCA_MIXED) return stokes_impl<float>(ctx, x, y);
  return stokes_impl<double>(ctx, x, y);
}

agca_status precond_impl(agca_ctx* ctx, const double* r, double* z) {
  const int64_t n3 = 3 * ctx->lev[ctx->L].V;
  CKS(vcycle_impl(ctx, r, z));
  const double* rp = r + n3;
  double* zp = z + n3;
  const double inv = 1.0 / (double)ctx->Vp;
  LK(2, launch_sum(rp, ctx->Vp, ctx->partials, ctx->sc + MS_TMP0, inv, ctx->stream));
  LK(1, launch_vec_op(VOP_PDIV, ctx->Vp, zp, rp, ctx->pmass_inv, nullptr, ctx->sc + MS_TMP0, ctx->stream));
  LK(2, launch_sum(zp, ctx->Vp, ctx->partials, ctx->sc + MS_TMP1, inv, ctx->stream));
  LK(1, launch_vec_op(VOP_SUBS, ctx->Vp, zp, zp, nullptr, nullptr, ctx->sc + MS_TMP1, ctx->stream));
  return AGCA_OK;
}

agca_status dot1(agca_ctx* ctx, const double* x, const double* y, int64_t n, double* out_dev) {
  const double* xs[1] = {x};
  const double* ys[1] = {y};
  LK(2, launch_dots(1, xs, ys, n, ctx->partials, out_dev, 1.0, ctx->stream));
  return AGCA_OK;
}

agca_status read_scalar(agca_ctx* ctx, const double* dev, double* host) {
  CK(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return AGCA_OK;
}

// Preconditioned MINRES for K d = b from d = 0 until the preconditioned
// residual norm drops by tol_rel (Remark 6).  low: inner operator applied
// with FP32 arithmetic in mixed contexts.
agca_status minres_impl(agca_ctx* ctx, const double* b, double* d, double tol_rel, int maxit, bool low,
                        int* iters) {
  const int64_t nt = ctx->nt;
  cudaStream_t s = ctx->stream;
  double* vold = ctx->kv[KV_VOLD];
  double* v = ctx->kv[KV_V];
  double* z = ctx->kv[KV_Z];
  double* zn = ctx->kv[KV_ZNEW];
  double* wold = ctx->kv[KV_WOLD];
  double* w = ctx->kv[KV_W];
  double* kz = ctx->kv[KV_KZ];
  LK(1, launch_vec_op(VOP_ZERO, nt, d, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_ZERO, nt, vold, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_ZERO, nt, wold, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_ZERO, nt, w, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_COPY, nt, v, b, nullptr, nullptr, nullptr, s));
  CKS(precond_impl(ctx, v, z));
  CKS(dot1(ctx, z, v, nt, ctx->sc + MS_DOT_ZV));
  LK(1, launch_minres_init(ctx->sc, tol_rel, s));
  // one iteration; after it the buffer roles rotate (v, z, w pairs swap)
  auto iteration = [&]() -> agca_status {
    CKS(stokes_dispatch(ctx, z, kz, low));
    CKS(dot1(ctx, kz, z, nt, ctx->sc + MS_DOT_KZZ));
    LK(1, launch_lanczos(nt, kz, v, vold, ctx->sc, s));  // vold <- v_new
    CKS(precond_impl(ctx, vold, zn));
    CKS(dot1(ctx, zn, vold, nt, ctx->sc + MS_DOT_ZV));
    LK(1, launch_minres_scalars(ctx->sc, s));
    LK(1, launch_minres_update(nt, z, w, wold, d, ctx->sc, s));  // wold <- w_new
    std::swap(vold, v);
    std::swap(z, zn);
    std::swap(wold, w);
    return AGCA_OK;
  };
  // iterations past convergence change nothing (the device scalars freeze the
  // update), so the loop may run a few beyond it between host checks
  const int gi = low ? 1 : 0;
  bool graph = ctx->use_graphs && !ctx->prof && s != nullptr;
  if (graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    graph = (cs == cudaStreamCaptureStatusNone);
  }
  if (graph && (ctx->minres_graph[gi] == nullptr || ctx->minres_key[gi] != d)) {
    if (ctx->minres_graph[gi]) cudaGraphExecDestroy(ctx->minres_graph[gi]);
    ctx->minres_graph[gi] = nullptr;
    const int64_t l0 = ctx->launches;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    agca_status st = iteration();
    if (st == AGCA_OK) st = iteration();
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    ctx->minres_launches[gi] = ctx->launches - l0;
    ctx->launches = l0;
    if (st != AGCA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (ee != cudaSuccess) return ctx->fail(AGCA_ECUDA, std::string("MINRES capture: ") + cudaGetErrorString(ee));
    const cudaError_t ie = cudaGraphInstantiate(&ctx->minres_graph[gi], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return ctx->fail(AGCA_ECUDA, std::string("MINRES graph: ") + cudaGetErrorString(ie));
    ctx->minres_key[gi] = d;
  }
  const int check_every = ctx->check_every;
  int it = 0;
  while (it < maxit) {
    if (graph && maxit - it >= 2) {  // two iterations per replay: the buffer roles return
      CK(cudaGraphLaunch(ctx->minres_graph[gi], s));
      ctx->launches += ctx->minres_launches[gi];
      it += 2;
    } else {
      CKS(iteration());
      it += 1;
    }
    if (it % check_every < (graph ? 2 : 1) || it >= maxit) {
      double done = 0.0;
      CKS(read_scalar(ctx, ctx->sc + MS_DONE, &done));
      if (done != 0.0) break;
    }
  }
  double its = 0.0;
  CKS(read_scalar(ctx, ctx->sc + MS_ITERS, &its));
  *iters = (int)its;
  return AGCA_OK;
}

agca_status project_pressure(agca_ctx* ctx, double* x) {
  const int64_t n3 = 3 * ctx->lev[ctx->L].V;
  LK(2, launch_sum(x + n3, ctx->Vp, ctx->partials, ctx->sc + MS_TMP2, 1.0 / (double)ctx->Vp, ctx->stream));
  LK(1, launch_vec_op(VOP_SUBS, ctx->Vp, x + n3, x + n3, nullptr, nullptr, ctx->sc + MS_TMP2, ctx->stream));
  return AGCA_OK;
}

agca_status solve_impl(agca_ctx* ctx, const double* b_in, double* x, double rtol, int maxit, int* iters,
                       double* relres) {
  const int64_t nt = ctx->nt;
  cudaStream_t s = ctx->stream;
  double* r = ctx->kv[KV_R];
  double* d = ctx->kv[KV_D];
  double* kx = ctx->kv[KV_KZ];
  // Dirichlet rows carry no equation: work on a copy of b with them zeroed
  double* bm = ctx->kv[KV_B];
  LK(1, launch_vec_op(VOP_COPY, nt, bm, b_in, nullptr, nullptr, nullptr, s));
  LK(1, launch_mask_boundary(ctx->lev[ctx->L].n, bm, s));
  const double* b = bm;
  LK(1, launch_vec_op(VOP_ZERO, nt, x, nullptr, nullptr, nullptr, nullptr, s));
  double nb2 = 0.0;
  CKS(dot1(ctx, b, b, nt, ctx->sc + MS_TMP0));
  CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &nb2));
  const double nb = sqrt(nb2);
  int total = 0;
  double rel = nb > 0.0 ? 1.0 : 0.0;
  const bool mixed = ctx->prec == AGCA_MIXED;
  for (int outer = 0; outer < 60 && nb > 0.0; ++outer) {
    CKS(stokes_dispatch(ctx, x, kx, false));
    LK(1, launch_vec_op(VOP_SUB, nt, r, b, kx, nullptr, nullptr, s));
    double nr2 = 0.0;
    CKS(dot1(ctx, r, r, nt, ctx->sc + MS_TMP0));
    CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &nr2));
    rel = sqrt(nr2) / nb;
    if (!(rel > rtol) || total >= maxit) break;
    double inner = 0.1 * rtol / rel;
    if (mixed) inner = std::max(inner, ctx->mixed_inner);
    inner = std::max(inner, 1e-14);
    int its = 0;
    CKS(minres_impl(ctx, r, d, inner, maxit - total, mixed, &its));
    total += its;
    LK(1, launch_vec_op(VOP_ADD, nt, x, x, d, nullptr, nullptr, s));
    CKS(project_pressure(ctx, x));
    if (its == 0) break;
  }
  if (iters) *iters = total;
  if (relres) *relres = rel;
  if (!(rel <= rtol)) return ctx->fail(AGCA_ENOTCONV, "solver stopped above the tolerance");
  return AGCA_OK;
}

// ------------------------------------------------------------------ FGMRES
// The paper's outer solver (Sec. 4): flexible GMRES (restarted, right
// preconditioning by a map that may vary between iterations), with the
// block-triangular preconditioner of Eq. 4.1,
//   z_p = -S~^-1 r_p,  z_u = A~^-1 (r_u - B^T z_p)
// (the signs of K = [[A, B^T], [B, 0]] with B = -D, so that exact blocks give
// K Q^-1 = [[I, 0], [B A^-1, I]]), A~^-1 one AGCA V-cycle and S~^-1 either
// the mean-free lumped 1/eta pressure mass (the MINRES preconditioner's
// pressure block) or the diag(A)-BFBT of Eq. 4.2,
//   S~^-1 = Z^-1 (B W^-1 A W^-1 B^T) Z^-1,  W = diag(A),  Z = B W^-1 B^T,
// with the middle factor applied matrix-free (one Stokes apply of
// [W^-1 B^T t; 0] gives A W^-1 B^T t) and Z assembled on the pressure grid as
// it is in the paper (App. B): Z couples pressure vertices at most 2 cells
// apart, so 125 applies of the matrix-free Z to colour indicators (vertices
// equal mod 5 per axis) give every row as a 5x5x5 stencil; Z^-1 by
// Jacobi-preconditioned conjugate gradients on the mean-free pressures.  In
// mixed contexts the preconditioner's Stokes applies use FP32 arithmetic;
// the outer K z stays FP64.  Arnoldi by classical
// Gram-Schmidt with one reorthogonalisation (two block dot products and two
// block updates per iteration); the small Hessenberg least-squares problem
// by Givens rotations on the host.
struct FgmresWork {
  double *V, *Z, *w, *t1, *t2, *partials, *hbuf, *ycoef, *zdinv, *cx, *cr, *cz, *cp, *cq, *m, *sc, *zsten;
  int64_t npartials;
  size_t need;
};

FgmresWork fgmres_layout(const agca_ctx* ctx, int restart, char* base) {
  Carver cv(base);
  const int64_t nt = ctx->nt, np = ctx->Vp;
  FgmresWork w{};
  w.V = cv.take<double>((int64_t)(restart + 1) * nt);
  w.Z = cv.take<double>((int64_t)restart * nt);
  w.w = cv.take<double>(nt);
  w.t1 = cv.take<double>(nt);
  w.t2 = cv.take<double>(nt);
  w.npartials = (int64_t)(restart + 1) * dot_blocks();
  w.partials = cv.take<double>(w.npartials);
  w.hbuf = cv.take<double>(2 * (restart + 1) + 8);
  w.ycoef = cv.take<double>(restart + 1);
  w.zdinv = cv.take<double>(np);
  w.cx = cv.take<double>(np);
  w.cr = cv.take<double>(np);
  w.cz = cv.take<double>(np);
  w.cp = cv.take<double>(np);
  w.cq = cv.take<double>(np);
  w.m = cv.take<double>(np);
  w.sc = cv.take<double>(8);
  w.zsten = cv.take<double>(np * ZSTENCIL);
  w.need = (cv.off + kAlign - 1) / kAlign * kAlign;
  return w;
}

// t2 = K [W^-1 B^T p; 0]: pressure part Z p, velocity part A W^-1 B^T p (t1 scratch)
agca_status z_apply(agca_ctx* ctx, const FgmresWork& W, const double* p) {
  const int64_t n3 = 3 * ctx->lev[ctx->L].V, np = ctx->Vp;
  cudaStream_t s = ctx->stream;
  LK(1, launch_vec_op(VOP_ZERO, n3, W.t1, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_COPY, np, W.t1 + n3, p, nullptr, nullptr, nullptr, s));
  CKS(stokes_dispatch(ctx, W.t1, W.t2, true));  // t2_u = B^T p
  LK(1, launch_vec_op(VOP_MUL, n3, W.t1, W.t2, ctx->lev[ctx->L].invD64, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_ZERO, np, W.t1 + n3, nullptr, nullptr, nullptr, nullptr, s));
  CKS(stokes_dispatch(ctx, W.t1, W.t2, true));  // [A W^-1 B^T p; Z p]
  return AGCA_OK;
}

// y = y - mean(y) over the pressure DoFs
agca_status mean_free(agca_ctx* ctx, double* y) {
  const int64_t np = ctx->Vp;
  LK(2, launch_sum(y, np, ctx->partials, ctx->sc + MS_TMP2, 1.0 / (double)np, ctx->stream));
  LK(1, launch_vec_op(VOP_SUBS, np, y, y, nullptr, nullptr, ctx->sc + MS_TMP2, ctx->stream));
  return AGCA_OK;
}

// x = Z^-1 rhs on the mean-free pressures: iters steps of Jacobi-preconditioned CG from 0
agca_status z_solve(agca_ctx* ctx, const FgmresWork& W, const double* rhs, double* x, int iters) {
  const int64_t np = ctx->Vp;
  cudaStream_t s = ctx->stream;
  LK(1, launch_vec_op(VOP_COPY, np, W.cr, rhs, nullptr, nullptr, nullptr, s));
  CKS(mean_free(ctx, W.cr));
  LK(1, launch_zcg(ctx->N, W.zsten, W.zdinv, x, W.cr, W.cp, W.cq, W.partials, W.npartials, iters, s));
  CKS(mean_free(ctx, x));
  return AGCA_OK;
}

// Z assembled by probing with the 125 colours (i, j, k) mod 5, and its inverse diagonal
agca_status z_assemble(agca_ctx* ctx, const FgmresWork& W) {
  const int64_t n3 = 3 * ctx->lev[ctx->L].V;
  cudaStream_t s = ctx->stream;
  for (int c = 0; c < 125; ++c) {
    LK(1, launch_colour5(ctx->N, c, W.cp, s));
    CKS(z_apply(ctx, W, W.cp));
    LK(1, launch_scatter_zrow(ctx->N, c, W.t2 + n3, W.zsten, s));
  }
  LK(1, launch_zdiag_inv(ctx->N, W.zsten, W.zdinv, s));
  return AGCA_OK;
}

// z = Q^-1 r (Eq. 4.1); schur 0: lumped mass, 1: BFBT with z_iters CG steps per Z solve
agca_status blocktri_precond(agca_ctx* ctx, const FgmresWork& W, const double* r, double* z, int schur, int z_iters) {
  const int64_t n3 = 3 * ctx->lev[ctx->L].V, np = ctx->Vp;
  cudaStream_t s = ctx->stream;
  const double* rp = r + n3;
  double* zp = z + n3;
  if (schur == 0) {
    const double inv = 1.0 / (double)np;
    LK(2, launch_sum(rp, np, ctx->partials, ctx->sc + MS_TMP0, inv, s));
    LK(1, launch_vec_op(VOP_PDIV, np, zp, rp, ctx->pmass_inv, nullptr, ctx->sc + MS_TMP0, s));
    CKS(mean_free(ctx, zp));
  } else {
    CKS(z_solve(ctx, W, rp, W.m, z_iters));                 // t = Z^-1 r_p
    CKS(z_apply(ctx, W, W.m));                              // t2_u = A W^-1 B^T t
    LK(1, launch_vec_op(VOP_MUL, n3, W.t1, W.t2, ctx->lev[ctx->L].invD64, nullptr, nullptr, s));
    LK(1, launch_vec_op(VOP_ZERO, np, W.t1 + n3, nullptr, nullptr, nullptr, nullptr, s));
    CKS(stokes_dispatch(ctx, W.t1, W.t2, true));          // t2_p = B W^-1 A W^-1 B^T t
    LK(1, launch_vec_op(VOP_COPY, np, W.m, W.t2 + n3, nullptr, nullptr, nullptr, s));
    CKS(z_solve(ctx, W, W.m, zp, z_iters));                 // S~^-1 r_p
  }
  // z_p = -S~^-1 r_p
  LK(1, launch_vec_op(VOP_ZERO, np, W.cq, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_SUB, np, zp, W.cq, zp, nullptr, nullptr, s));
  // z_u = A~^-1 (r_u - B^T z_p)
  LK(1, launch_vec_op(VOP_ZERO, n3, W.t1, nullptr, nullptr, nullptr, nullptr, s));
  LK(1, launch_vec_op(VOP_COPY, np, W.t1 + n3, zp, nullptr, nullptr, nullptr, s));
  CKS(stokes_dispatch(ctx, W.t1, W.t2, true));  // t2_u = B^T z_p
  LK(1, launch_vec_op(VOP_SUB, n3, W.t1, r, W.t2, nullptr, nullptr, s));
  CKS(vcycle_impl(ctx, W.t1, z));
  return AGCA_OK;
}

agca_status fgmres_impl(agca_ctx* ctx, const FgmresWork& W, int restart, const double* b_in, double* x, double rtol,
                        int maxit, int schur, int z_iters, int* iters, double* relres) {
  const int64_t nt = ctx->nt;
  cudaStream_t s = ctx->stream;
  double* r = ctx->kv[KV_R];
  double* kx = ctx->kv[KV_KZ];
  double* bm = ctx->kv[KV_B];
  LK(1, launch_vec_op(VOP_COPY, nt, bm, b_in, nullptr, nullptr, nullptr, s));
  LK(1, launch_mask_boundary(ctx->lev[ctx->L].n, bm, s));
  LK(1, launch_vec_op(VOP_ZERO, nt, x, nullptr, nullptr, nullptr, nullptr, s));
  if (schur == 1) CKS(z_assemble(ctx, W));
  double nb2 = 0.0;
  CKS(dot1(ctx, bm, bm, nt, ctx->sc + MS_TMP0));
  CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &nb2));
  const double nb = sqrt(nb2);
  int its = 0;
  double rel = nb > 0.0 ? 1.0 : 0.0;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart),
      hv(2 * (restart + 1) + 1);
  auto Hh = [&](int i, int j) -> double& { return H[(size_t)i * restart + j]; };
  double* const hdev = W.hbuf;                     // [0, restart+1): first pass, then second pass, then |w|^2
  double* const h2dev = W.hbuf + (restart + 1);
  double* const wn2 = W.hbuf + 2 * (restart + 1);
  while (nb > 0.0) {
    CKS(stokes_dispatch(ctx, x, kx, false));
    LK(1, launch_vec_op(VOP_SUB, nt, r, bm, kx, nullptr, nullptr, s));
    double beta2 = 0.0;
    CKS(dot1(ctx, r, r, nt, ctx->sc + MS_TMP0));
    CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &beta2));
    const double beta = sqrt(beta2);
    rel = beta / nb;
    if (!(rel > rtol) || its >= maxit) break;
    LK(1, launch_vec_op(VOP_SCALE_RSQRT, nt, W.V, r, nullptr, nullptr, ctx->sc + MS_TMP0, s));  // v0 = r / beta
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int m = 0;
    for (int j = 0; j < restart; ++j) {
      double* vj = W.V + (int64_t)j * nt;
      double* zj = W.Z + (int64_t)j * nt;
      CKS(blocktri_precond(ctx, W, vj, zj, schur, z_iters));
      CKS(stokes_dispatch(ctx, zj, W.w, false));
      // classical Gram-Schmidt, twice
      LK(2, launch_block_dot(j + 1, W.V, nt, W.w, nt, W.partials, hdev, s));
      LK(1, launch_block_axpy(j + 1, W.V, nt, hdev, -1.0, W.w, nt, s));
      LK(2, launch_block_dot(j + 1, W.V, nt, W.w, nt, W.partials, h2dev, s));
      LK(1, launch_block_axpy(j + 1, W.V, nt, h2dev, -1.0, W.w, nt, s));
      CKS(dot1(ctx, W.w, W.w, nt, wn2));
      LK(1, launch_vec_op(VOP_SCALE_RSQRT, nt, W.V + (int64_t)(j + 1) * nt, W.w, nullptr, nullptr, wn2, s));
      CK(cudaMemcpyAsync(hv.data(), W.hbuf, (2 * (restart + 1) + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) Hh(i, j) = hv[i] + hv[restart + 1 + i];
      const double hn = sqrt(std::max(hv[2 * (restart + 1)], 0.0));
      // previous rotations, then the one that annihilates H(j+1, j)
      for (int i = 0; i < j; ++i) {
        const double a = Hh(i, j), b = Hh(i + 1, j);
        Hh(i, j) = cs[i] * a + sn[i] * b;
        Hh(i + 1, j) = -sn[i] * a + cs[i] * b;
      }
      const double a = Hh(j, j);
      const double den = sqrt(a * a + hn * hn);
      cs[j] = den > 0.0 ? a / den : 1.0;
      sn[j] = den > 0.0 ? hn / den : 0.0;
      Hh(j, j) = den;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      m = j + 1;
      if (std::fabs(g[j + 1]) <= rtol * nb || its >= maxit || hn == 0.0) break;
    }
    // x += Z y with R y = g (back substitution)
    for (int i = m - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < m; ++k) acc -= Hh(i, k) * y[k];
      y[i] = Hh(i, i) != 0.0 ? acc / Hh(i, i) : 0.0;
    }
    CK(cudaMemcpyAsync(W.ycoef, y.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    LK(1, launch_block_axpy(m, W.Z, nt, W.ycoef, 1.0, x, nt, s));
    CKS(project_pressure(ctx, x));
  }
  if (iters) *iters = its;
  if (relres) *relres = rel;
  if (!(rel <= rtol)) return ctx->fail(AGCA_ENOTCONV, "FGMRES stopped above the tolerance");
  return AGCA_OK;
}

agca_status check_status(agca_ctx* ctx, const char* where) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st & 1) return ctx->fail(AGCA_EINVAL, std::string(where) + ": viscosity must be finite and > 0");
  if (st & 2) return ctx->fail(AGCA_EINTERNAL, std::string(where) + ": coarsest operator is not SPD");
  return AGCA_OK;
}

agca_status power_lambda(agca_ctx* ctx, int l, double* lam) {
  const Level& lv = ctx->lev[l];
  const int64_t n3 = 3 * lv.V;
  cudaStream_t s = ctx->stream;
  double* v = ctx->kv[KV_VOLD];
  double* w = ctx->kv[KV_V];
  LK(1, launch_start_vector(lv.n, v, s));
  for (int it = 0; it < ctx->power_iters; ++it) {
    CKS(stencil<double>(ctx, ST_APPLY, l, v, nullptr, nullptr, w, 0, 0, 0));
    LK(1, launch_vec_op(VOP_MUL, n3, w, w, lv.invD64, nullptr, nullptr, s));
    CKS(dot1(ctx, w, w, n3, ctx->sc + MS_TMP0));
    LK(1, launch_vec_op(VOP_SCALE_RSQRT, n3, v, w, nullptr, nullptr, ctx->sc + MS_TMP0, s));
  }
  CKS(stencil<double>(ctx, ST_APPLY, l, v, nullptr, nullptr, w, 0, 0, 0));
  CKS(dot1(ctx, v, w, n3, ctx->sc + MS_TMP0));
  LK(1, launch_vec_op(VOP_MUL, n3, w, v, lv.diag, nullptr, nullptr, s));
  CKS(dot1(ctx, v, w, n3, ctx->sc + MS_TMP1));
  double num = 0.0, den = 0.0;
  CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &num));
  CKS(read_scalar(ctx, ctx->sc + MS_TMP1, &den));
  *lam = num / den;
  return AGCA_OK;
}

bool valid_level(const agca_ctx* ctx, int l) { return l >= 1 && l <= ctx->L; }

// Autotuner: times every candidate tile shape (block rows, z-chunk) of the
// V-cycle stencil launches on each level with CUDA events on the context
// stream and keeps the fastest; results can be cached in a text file keyed
// by (precision, cubes per axis, mode, coarse).
template <typename T>
agca_status tune_level(agca_ctx* ctx, int l, int reps, std::map<std::string, TileCfg>& cache) {
  Level& lv = ctx->lev[l];
  const int64_t n3 = 3 * lv.V;
  cudaStream_t s = ctx->stream;
  for (void* p : {lv.vb, lv.vx, lv.vt, lv.vr}) CK(cudaMemsetAsync(p, 0, n3 * sizeof(T), s));
  const bool f32 = sizeof(T) == 4;
  // the edge form (every FP64 level) has one tile shape
  const bool edge = !f32;
  std::vector<int> bys = edge ? std::vector<int>{8} : std::vector<int>{8, 12, 16};
  const int nv = lv.n + 1;
  int dev = 0, sms = 152;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // z-chunk candidates: a fixed ladder plus, per block-row count, the chunks
  // whose block count fills k = 1..16 whole waves of resident blocks (no
  // partly filled last wave)
  auto candidates = [&](int by) {
    std::vector<int> zs = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64};
    const int per_sm = edge ? 2 : (by <= 8 ? 3 : (by <= 12 ? 2 : 1));
    const int per_z = edge ? edge_tiles(lv.n, 1).per_z() : stencil_tiles(lv.n, by, 1).per_z();
    for (int k = 1; k <= 16; ++k) {
      const int gz = std::max(1, k * sms * per_sm / per_z);
      zs.push_back((nv + gz - 1) / gz);
    }
    std::sort(zs.begin() + 1, zs.end());
    zs.erase(std::unique(zs.begin() + 1, zs.end()), zs.end());
    return zs;
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int modes[4] = {ST_CHEB_PRE, ST_RESID, ST_CHEB_FIRST, ST_CHEB_STEP};
  agca_status st = AGCA_OK;
  for (int mode : modes) {
    std::ostringstream key;
    key << (f32 ? "f32" : "f64") << ' ' << lv.n << ' ' << mode << ' ' << (l < ctx->L ? 1 : 0);
    auto it = cache.find(key.str());
    if (it != cache.end()) {
      ctx->tune[l][mode] = it->second;
      continue;
    }
    TileCfg best;
    float best_ms = 1e30f;
    for (int by : bys) {
      int last_zch = -1;
      for (int zr : candidates(by)) {
        if (zr > nv) continue;
        const int zch = edge ? edge_tiles(lv.n, zr, 2 * sms).zch : stencil_tiles(lv.n, by, zr).zch;
        if (zch == last_zch) continue;
        last_zch = zch;
        TileCfg c;
        c.by = by;
        c.zch = zch;
        ctx->tune[l][mode] = c;
        T* X = static_cast<T*>(lv.vx);
        T* Bv = static_cast<T*>(lv.vb);
        T* Tb = static_cast<T*>(lv.vt);
        T* R = static_cast<T*>(lv.vr);
        auto once = [&]() -> agca_status {
          switch (mode) {
            case ST_CHEB_PRE: return stencil<T>(ctx, mode, l, nullptr, Bv, nullptr, X, 0.5, 0.5, 0.5);
            case ST_RESID: return stencil<T>(ctx, mode, l, X, Bv, nullptr, R, 0, 0, 0);
            case ST_CHEB_FIRST: return stencil<T>(ctx, mode, l, X, Bv, nullptr, Tb, 0.5, 0, 0);
            default: return stencil<T>(ctx, mode, l, Tb, Bv, X, X, 0.5, 0.5, 0);
          }
        };
        if ((st = once()) != AGCA_OK) break;
        if ((st = once()) != AGCA_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) break;
        for (int r = 0; r < reps && st == AGCA_OK; ++r) st = once();
        if (st != AGCA_OK) break;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
      if (st != AGCA_OK) break;
    }
    if (st != AGCA_OK) break;
    ctx->tune[l][mode] = best;
    cache[key.str()] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// ===================================================================== batch
// Many independent problems solved together: every problem has its own
// context (hierarchy, workspace slice, MINRES state); the MINRES iteration of
// all problems runs in lockstep as one CUDA graph whose launches each cover
// every problem (persistent stencil launches over the (problem, tile) work
// list, 2-D element-wise grids over (chunk, problem)), skipping converged
// problems on the device.
struct BatchStep {
  int kind;        // 0 stencil, 1 xfer, 2 krylov
  int mode;        // stencil mode / xfer kind / krylov op
  int prec;        // 0: <double,double>, 1: <float,float>, 2: <double,float>
  bool coarse;
  size_t off;      // byte offset of the task array in the task table
  int ntasks;
  int64_t work;    // tiles (stencil), max count (xfer), max n (krylov)
  int64_t gca;     // max gca rows (coarse stencil)
  int max_m;       // coarsest solve size
};

}  // namespace

struct agca_batch {
  int n = 0, prec = 0;
  int sms = 152;             // multiprocessors of the device (read at setup)
  cudaStream_t stream = nullptr;
  std::vector<agca_ctx*> ctx;
  std::vector<size_t> ws_off, gs_off;
  size_t ws_need = 0, gs_need = 0, tab_bytes = 0;
  char* ws = nullptr;
  char* gs = nullptr;
  char* tab = nullptr;       // device task tables
  std::vector<int> members;       // problems the table builders cover
  std::vector<int> iter_members;  // problems the captured iteration graph covers
  double* partials = nullptr;
  std::vector<char> host_tab;
  std::vector<BatchStep> iter_steps[2];  // MINRES iteration, by buffer parity
  cudaGraphExec_t iter_graph = nullptr;
  int64_t iter_launches = 0;
  bool setup_done = false;
  std::string err;
  agca_status fail(agca_status s, const std::string& m) {
    err = m;
    return s;
  }
  ~agca_batch() {
    if (iter_graph) cudaGraphExecDestroy(iter_graph);
    for (agca_ctx* c : ctx) delete c;
  }
};

#define BCK(...)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (__VA_ARGS__);                                                                  \
    if (e_ != cudaSuccess)                                                                           \
      return b->fail(AGCA_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));         \
  } while (0)
#define BCKS(expr)                                                                                   \
  do {                                                                                               \
    agca_status s_ = (expr);                                                                         \
    if (s_ != AGCA_OK) return s_;                                                                    \
  } while (0)

namespace {

template <typename TaskT>
size_t push_tasks(agca_batch* b, const std::vector<TaskT>& t) {
  size_t off = (b->host_tab.size() + 255) / 256 * 256;
  b->host_tab.resize(off + t.size() * sizeof(TaskT));
  if (!t.empty()) std::memcpy(b->host_tab.data() + off, t.data(), t.size() * sizeof(TaskT));
  return off;
}

template <typename TS, typename T>
StencilTask<TS, T> make_task(agca_ctx* c, int l, int mode, const TS* x, const TS* bb, const TS* xprev, TS* out,
                             double s0, double s1, double s2, const double* sc) {
  StencilTask<TS, T> tk{};
  tk.op = level_op<T>(c, l);
  tk.a.x = x;
  tk.a.b = bb;
  tk.a.invD = (const TS*)invD_of<T>(c->lev[l]);
  tk.a.xprev = xprev;
  tk.a.out = out;
  tk.a.s0 = (TS)s0;
  tk.a.s1 = (TS)s1;
  tk.a.s2 = (TS)s2;
  tk.sc = sc;  // tiles: push_stencil
  (void)mode;
  return tk;
}

template <typename TS, typename T>
void push_stencil(agca_batch* b, std::vector<BatchStep>& steps, int mode, bool coarse, std::vector<StencilTask<TS, T>> t,
                  int prec) {
  if (t.empty()) return;
  // one z-chunk for the whole step: about six waves of resident blocks over
  // all problems (the batch supplies the parallelism, so chunks stay long and
  // the z-halo small), between 4 and 32 planes
  int64_t cols = 0;
  for (const auto& tk : t) cols += (int64_t)stencil_tiles(tk.op.n, 8, 0).per_z() * (tk.op.n + 1);
  const int64_t slots = 6 * (int64_t)b->sms * 3;
  const int zch = (int)std::min<int64_t>(32, std::max<int64_t>(4, (cols + slots - 1) / slots));
  int64_t tiles = 0, gca = 0;
  for (auto& tk : t) {
    tk.tg = edge_form_step<TS, T>(mode, coarse) ? edge_tiles(tk.op.n, zch) : stencil_tiles(tk.op.n, 8, zch);
    tk.tile0 = tiles;
    tiles += (int64_t)tk.tg.per_z() * tk.tg.gz;
    gca = std::max<int64_t>(gca, tk.op.sten ? 0 : tk.op.n_flag * 12);  // stencils need no product launch
  }
  BatchStep st{0, mode, prec, coarse, push_tasks(b, t), (int)t.size(), tiles, coarse ? gca : 0, 0};
  steps.push_back(st);
}

void push_xfer(agca_batch* b, std::vector<BatchStep>& steps, int kind, const std::vector<XferTask>& t, int prec) {
  if (t.empty()) return;
  int64_t mx = 0;
  int mm = 0;
  for (auto& tk : t) {
    mx = std::max(mx, tk.count);
    if (kind == XK_COARSE) mm = std::max(mm, 3 * (tk.nf - 1) * (tk.nf - 1) * (tk.nf - 1));
  }
  BatchStep st{1, kind, prec, false, push_tasks(b, t), (int)t.size(), mx, 0, mm};
  steps.push_back(st);
}

void push_krylov(agca_batch* b, std::vector<BatchStep>& steps, int op, const std::vector<KTask>& t) {
  if (t.empty()) return;
  int64_t mx = 0;
  for (auto& tk : t) mx = std::max(mx, tk.n);
  BatchStep st{2, op, 0, false, push_tasks(b, t), (int)t.size(), mx, 0, 0};
  steps.push_back(st);
}

// Batched V(2,2) cycle z_p = V_p(r_p) (degree-2 Chebyshev), result copied to z_p.
template <typename T>
void build_cycle(agca_batch* b, std::vector<BatchStep>& steps, const std::vector<const double*>& r,
                 const std::vector<double*>& z, bool skip_done) {
  const int P = b->n;
  const int pr = std::is_same<T, float>::value ? 1 : 0;
  const bool mixed = std::is_same<T, float>::value;
  int maxL = 0;
  for (int p : b->members) maxL = std::max(maxL, b->ctx[p]->L);
  auto sc_of = [&](int p) -> const double* { return skip_done ? b->ctx[p]->sc : nullptr; };
  auto bfine = [&](int p) -> const T* {
    agca_ctx* c = b->ctx[p];
    return mixed ? static_cast<const T*>(c->lev[c->L].vb) : reinterpret_cast<const T*>(r[p]);
  };
  if (mixed) {
    std::vector<XferTask> t;
    for (int p : b->members) {
      agca_ctx* c = b->ctx[p];
      XferTask x{};
      x.count = 3 * c->lev[c->L].V;
      x.src = r[p];
      x.dst = c->lev[c->L].vb;
      x.sc = sc_of(p);
      t.push_back(x);
    }
    push_xfer(b, steps, XK_D2F, t, 1);
  }
  // down-sweep by depth below each problem's finest level
  for (int d = 0; d <= maxL - 2; ++d) {
    std::vector<StencilTask<T, T>> pre, res;
    std::vector<XferTask> rst;
    for (int p : b->members) {
      agca_ctx* c = b->ctx[p];
      const int l = c->L - d;
      if (l < 2) continue;
      Level& lv = c->lev[l];
      const T* bl = (d == 0) ? bfine(p) : static_cast<const T*>(lv.vb);
      T* X = static_cast<T*>(lv.vx);
      const Cheb ch = cheb_params(c, l);
      const double rho = 1.0 / ch.sigma, rn = 1.0 / (2.0 * ch.sigma - rho);
      pre.push_back(make_task<T, T>(c, l, ST_CHEB_PRE, nullptr, bl, nullptr, X, rn * rho, 2.0 * rn / ch.delta,
                                    1.0 / ch.theta, sc_of(p)));
      res.push_back(make_task<T, T>(c, l, ST_RESID, X, bl, nullptr, static_cast<T*>(lv.vr), 0, 0, 0, sc_of(p)));
      XferTask x{};
      x.nf = lv.n;
      x.ncomp = 3;
      x.mask = 1;
      x.scale = 1.0;
      x.count = c->lev[l - 1].V;
      x.src = lv.vr;
      x.dst = c->lev[l - 1].vb;
      x.sc = sc_of(p);
      rst.push_back(x);
    }
    push_stencil<T, T>(b, steps, ST_CHEB_PRE, d > 0, pre, pr);
    push_stencil<T, T>(b, steps, ST_RESID, d > 0, res, pr);
    push_xfer(b, steps, XK_RESTRICT, rst, pr);
  }
  {
    std::vector<XferTask> t;
    for (int p : b->members) {
      agca_ctx* c = b->ctx[p];
      XferTask x{};
      x.nf = c->lev[1].n;
      x.count = 1;
      x.src = c->lev[1].vb;
      x.dst = c->lev[1].vx;
      x.m1 = c->linv_cm;
      x.m2 = c->linv_rm;
      x.sc = sc_of(p);
      t.push_back(x);
    }
    push_xfer(b, steps, XK_COARSE, t, pr);
  }
  for (int d = maxL - 2; d >= 0; --d) {
    std::vector<StencilTask<T, T>> first, step;
    std::vector<XferTask> pro;
    for (int p : b->members) {
      agca_ctx* c = b->ctx[p];
      const int l = c->L - d;
      if (l < 2) continue;
      Level& lv = c->lev[l];
      const T* bl = (d == 0) ? bfine(p) : static_cast<const T*>(lv.vb);
      T* X = static_cast<T*>(lv.vx);
      T* Tb = static_cast<T*>(lv.vt);
      XferTask x{};
      x.nf = lv.n;
      x.ncomp = 3;
      x.mask = 1;
      x.count = lv.V;
      x.src = c->lev[l - 1].vx;
      x.dst = X;
      x.sc = sc_of(p);
      pro.push_back(x);
      const Cheb ch = cheb_params(c, l);
      const double rho = 1.0 / ch.sigma, rn = 1.0 / (2.0 * ch.sigma - rho);
      first.push_back(make_task<T, T>(c, l, ST_CHEB_FIRST, X, bl, nullptr, Tb, 1.0 / ch.theta, 0, 0, sc_of(p)));
      step.push_back(make_task<T, T>(c, l, ST_CHEB_STEP, Tb, bl, X, X, rn * rho, 2.0 * rn / ch.delta, 0, sc_of(p)));
    }
    push_xfer(b, steps, XK_PROLONG_ADD, pro, pr);
    push_stencil<T, T>(b, steps, ST_CHEB_FIRST, d > 0, first, pr);
    push_stencil<T, T>(b, steps, ST_CHEB_STEP, d > 0, step, pr);
  }
  {
    std::vector<XferTask> t;
    for (int p : b->members) {
      agca_ctx* c = b->ctx[p];
      XferTask x{};
      x.count = 3 * c->lev[c->L].V;
      x.src = c->lev[c->L].vx;
      x.dst = z[p];
      x.sc = sc_of(p);
      t.push_back(x);
    }
    push_xfer(b, steps, mixed ? XK_F2D : XK_COPY64, t, pr);
  }
}

// K x for every problem (x_p, y_p: Stokes vectors), FP32 compute when low
void build_stokes(agca_batch* b, std::vector<BatchStep>& steps, const std::vector<const double*>& x,
                  const std::vector<double*>& y, bool low, bool skip_done) {
  const int P = b->n;
  std::vector<XferTask> pro, rst;
  std::vector<StencilTask<double, double>> t64;
  std::vector<StencilTask<double, float>> t32;
  for (int p : b->members) {
    agca_ctx* c = b->ctx[p];
    const Level& lf = c->lev[c->L];
    const int64_t n3 = 3 * lf.V;
    const double* sc = skip_done ? c->sc : nullptr;
    XferTask a{};
    a.nf = lf.n;
    a.ncomp = 1;
    a.mask = 0;
    a.count = lf.V;
    a.src = x[p] + n3;
    a.dst = c->qfine;
    a.sc = sc;
    pro.push_back(a);
    if (low) {
      StencilTask<double, float> tk{};
      tk.op = op32(c, c->L);
      tk.a.x = x[p];
      tk.a.q = c->qfine;
      tk.a.out = y[p];
      tk.a.out2 = c->sfine;
      tk.sc = sc;
      t32.push_back(tk);
    } else {
      StencilTask<double, double> tk{};
      tk.op = op64(c, c->L);
      tk.a.x = x[p];
      tk.a.q = c->qfine;
      tk.a.out = y[p];
      tk.a.out2 = c->sfine;
      tk.sc = sc;
      t64.push_back(tk);
    }
    XferTask r{};
    r.nf = lf.n;
    r.ncomp = 1;
    r.mask = 0;
    r.scale = -1.0;
    r.count = c->Vp;
    r.src = c->sfine;
    r.dst = y[p] + n3;
    r.sc = sc;
    rst.push_back(r);
  }
  push_xfer(b, steps, XK_PROLONG, pro, 0);
  if (low)
    push_stencil<double, float>(b, steps, ST_STOKES, false, t32, 2);
  else
    push_stencil<double, double>(b, steps, ST_STOKES, false, t64, 0);
  push_xfer(b, steps, XK_RESTRICT, rst, 0);
}

// One MINRES iteration for every problem at buffer parity par (see minres_impl).
void build_iteration(agca_batch* b, int par) {
  std::vector<BatchStep>& steps = b->iter_steps[par];
  steps.clear();
  const int P = b->n;
  const bool mixed = b->prec == AGCA_MIXED;
  std::vector<const double*> z(P), vnew_c(P);
  std::vector<double*> kz(P), vnew(P), zn(P);
  for (int p : b->members) {
    agca_ctx* c = b->ctx[p];
    z[p] = c->kv[par ? KV_ZNEW : KV_Z];
    zn[p] = c->kv[par ? KV_Z : KV_ZNEW];
    kz[p] = c->kv[KV_KZ];
    vnew[p] = c->kv[par ? KV_V : KV_VOLD];
    vnew_c[p] = vnew[p];
  }
  build_stokes(b, steps, z, kz, mixed, true);
  std::vector<KTask> dk, lz, pz, ps, pd, pm, dz, up, sc;
  for (int p : b->members) {
    agca_ctx* c = b->ctx[p];
    const int64_t nt = c->nt, n3 = nt - c->Vp;
    const double* v = c->kv[par ? KV_VOLD : KV_V];
    const double* w = c->kv[par ? KV_WOLD : KV_W];
    double* wold = c->kv[par ? KV_W : KV_WOLD];
    dk.push_back({nt, c->sc, kz[p], z[p], nullptr, nullptr, MS_DOT_KZZ, 1.0});
    lz.push_back({nt, c->sc, kz[p], v, vnew[p], nullptr, 0, 0.0});
    ps.push_back({c->Vp, c->sc, vnew[p] + n3, nullptr, nullptr, nullptr, MS_TMP0, 1.0 / (double)c->Vp});
    pd.push_back({c->Vp, c->sc, vnew[p] + n3, c->pmass_inv, zn[p] + n3, nullptr, MS_TMP0, 0.0});
    pm.push_back({c->Vp, c->sc, zn[p] + n3, nullptr, nullptr, nullptr, MS_TMP1, 1.0 / (double)c->Vp});
    pz.push_back({c->Vp, c->sc, zn[p] + n3, nullptr, zn[p] + n3, nullptr, MS_TMP1, 0.0});
    dz.push_back({nt, c->sc, zn[p], vnew[p], nullptr, nullptr, MS_DOT_ZV, 1.0});
    sc.push_back({0, c->sc, nullptr, nullptr, nullptr, nullptr, 0, 0.0});
    up.push_back({nt, c->sc, z[p], w, wold, c->kv[KV_D], 0, 0.0});
  }
  push_krylov(b, steps, KB_DOT, dk);
  push_krylov(b, steps, KB_LANCZOS, lz);
  if (mixed)
    build_cycle<float>(b, steps, vnew_c, zn, true);
  else
    build_cycle<double>(b, steps, vnew_c, zn, true);
  push_krylov(b, steps, KB_SUM, ps);
  push_krylov(b, steps, KB_PDIV, pd);
  push_krylov(b, steps, KB_SUM, pm);
  push_krylov(b, steps, KB_SUBS, pz);
  push_krylov(b, steps, KB_DOT, dz);
  push_krylov(b, steps, KB_SCALARS, sc);
  push_krylov(b, steps, KB_UPDATE, up);
}

agca_status run_steps(agca_batch* b, const std::vector<BatchStep>& steps, int64_t* launches) {
  cudaStream_t s = b->stream;
  for (const BatchStep& st : steps) {
    const void* t = b->tab + st.off;
    if (st.kind == 0) {
      if (st.prec == 0)
        BCK(launch_stencil_batch<double, double>(st.mode, st.coarse, (const StencilTask<double, double>*)t, st.ntasks,
                                                 st.work, st.gca, s));
      else if (st.prec == 1)
        BCK(launch_stencil_batch<float, float>(st.mode, st.coarse, (const StencilTask<float, float>*)t, st.ntasks,
                                               st.work, st.gca, s));
      else
        BCK(launch_stencil_batch<double, float>(st.mode, st.coarse, (const StencilTask<double, float>*)t, st.ntasks,
                                                st.work, st.gca, s));
      *launches += (st.coarse && st.gca > 0) ? 2 : 1;
    } else if (st.kind == 1) {
      if (st.prec == 1)
        BCK(launch_xfer_batch<float>(st.mode, (const XferTask*)t, st.ntasks, st.work, st.max_m, s));
      else
        BCK(launch_xfer_batch<double>(st.mode, (const XferTask*)t, st.ntasks, st.work, st.max_m, s));
      *launches += 1;
    } else {
      BCK(launch_krylov_batch(st.mode, (const KTask*)t, st.ntasks, st.work, b->partials, s));
      *launches += (st.mode == KB_DOT || st.mode == KB_SUM) ? 2 : 1;
    }
  }
  return AGCA_OK;
}

bool batch_valid(const agca_batch* b, int i) { return b && i >= 0 && i < b->n; }

}  // namespace


extern "C" {

const char* agca_status_string(agca_status s) {
  switch (s) {
    case AGCA_OK: return "AGCA_OK";
    case AGCA_EINVAL: return "AGCA_EINVAL";
    case AGCA_ENOMEM: return "AGCA_ENOMEM";
    case AGCA_ECUDA: return "AGCA_ECUDA";
    case AGCA_ENOTCONV: return "AGCA_ENOTCONV";
    case AGCA_ETIMEOUT: return "AGCA_ETIMEOUT";
    case AGCA_EINTERNAL: return "AGCA_EINTERNAL";
    case AGCA_ESTATE: return "AGCA_ESTATE";
  }
  return "unknown";
}

agca_status agca_create(int N, int n_levels, int prec, void* cuda_stream, agca_ctx** out) {
  if (!out) return AGCA_EINVAL;
  *out = nullptr;
  // N <= 256 keeps every per-level index below 2^31 (3 (2N+1)^3 vertex entries,
  // 6 (2N)^3 elements): the kernels index with 32-bit integers
  if (N < 1 || N > 256 || n_levels < 2 || n_levels > 12 || (prec != AGCA_FP64 && prec != AGCA_MIXED))
    return AGCA_EINVAL;
  const int nL = 2 * N;
  if (nL % (1 << (n_levels - 1)) != 0 || (nL >> (n_levels - 1)) < 2) return AGCA_EINVAL;
  if (nL > 1024) return AGCA_EINVAL;
  agca_ctx* ctx = new agca_ctx();
  ctx->N = N;
  ctx->L = n_levels;
  ctx->prec = prec;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->lev.resize(n_levels + 1);
  for (int l = 1; l <= n_levels; ++l) {
    Level& lv = ctx->lev[l];
    lv.n = nL >> (n_levels - l);
    lv.V = nverts(lv.n);
    lv.E = nelems(lv.n);
  }
  const int n1 = ctx->lev[1].n;
  ctx->mc = 3 * (n1 - 1) * (n1 - 1) * (n1 - 1);
  if (ctx->mc > 3000) {  // the coarsest dense factor must stay small (solve staged in 48 KB of shared memory)
    delete ctx;
    return AGCA_EINVAL;
  }
  ctx->Vp = nverts(nL / 2);
  ctx->nt = 3 * ctx->lev[n_levels].V + ctx->Vp;
  ctx->tune.assign(n_levels + 1, std::array<TileCfg, 6>{});
  carve_workspace(ctx, nullptr);
  *out = ctx;
  return AGCA_OK;
}

void agca_destroy(agca_ctx* ctx) { delete ctx; }

const char* agca_last_error(const agca_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

agca_status agca_set_smoother(agca_ctx* ctx, int degree, double lo, double hi, int power_iters) {
  if (!ctx) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (degree < 2 || degree > 8 || !(lo > 0.0) || !(hi > lo) || power_iters < 1 || power_iters > 1000)
    return ctx->fail(AGCA_EINVAL, "smoother parameters out of range");
  ctx->cheb_degree = degree;
  ctx->cheb_lo = lo;
  ctx->cheb_hi = hi;
  ctx->power_iters = power_iters;
  ctx->setup_done = false;
  return AGCA_OK;
}

agca_status agca_set_solver_options(agca_ctx* ctx, double mixed_inner_rtol, int check_every) {
  if (!ctx) return AGCA_EINVAL;
  if (!(mixed_inner_rtol > 0.0 && mixed_inner_rtol < 1.0) || check_every < 1 || check_every > 1000)
    return ctx->fail(AGCA_EINVAL, "solver options out of range");
  ctx->mixed_inner = mixed_inner_rtol;
  ctx->check_every = check_every;
  return AGCA_OK;
}

agca_status agca_set_coarse_projection(agca_ctx* ctx, int kind) {
  if (!ctx) return AGCA_EINVAL;
  if (kind < 0 || kind > 2) return ctx->fail(AGCA_EINVAL, "projection must be 0, 1 or 2");
  ctx->projection = kind;
  return AGCA_OK;
}

agca_status agca_workspace_size(const agca_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return AGCA_EINVAL;
  *bytes = ctx->ws_need;
  return AGCA_OK;
}

agca_status agca_bind_workspace(agca_ctx* ctx, void* dev_ptr, size_t bytes) {
  if (!ctx) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign) != 0) return ctx->fail(AGCA_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < ctx->ws_need) return ctx->fail(AGCA_ENOMEM, "workspace too small");
  ctx->ws = static_cast<char*>(dev_ptr);
  ctx->ws_bytes = bytes;
  carve_workspace(ctx, ctx->ws);
  ctx->have_eta = ctx->flagged = ctx->setup_done = false;
  ctx->gs = nullptr;
  return AGCA_OK;
}

agca_status agca_set_viscosity(agca_ctx* ctx, const double* eta_dev) {
  if (!ctx || !eta_dev) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (!ctx->ws) return ctx->fail(AGCA_ESTATE, "bind the workspace first");
  Level& lf = ctx->lev[ctx->L];
  CK(cudaMemcpyAsync(lf.mean, eta_dev, lf.E * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (lf.hedge) LK(1, launch_edge_records(lf.n, lf.mean, lf.hedge, ctx->stream));
  ctx->have_eta = true;
  ctx->flagged = ctx->setup_done = false;
  return AGCA_OK;
}

}  // extern "C"

namespace {
// viscosity hierarchy and flags: by the element-wise ratio rule, or (eta_v
// set) by the gradient rule of Eq. 2.8 on the finest nodal viscosity
agca_status flag_impl(agca_ctx* ctx, double nu, const double* eta_v, size_t* gca_bytes) {
  if (!ctx || !gca_bytes) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (!ctx->have_eta) return ctx->fail(AGCA_ESTATE, "set the viscosity first");
  if (!(nu >= 0.0) || !isfinite(nu)) return ctx->fail(AGCA_EINVAL, "nu must be finite and >= 0");
  cudaStream_t s = ctx->stream;
  const int L = ctx->L;
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), s));
  LK(1, launch_check_eta(ctx->lev[L].mean, ctx->lev[L].E, ctx->status, s));
  if (eta_v) LK(1, launch_check_eta(eta_v, ctx->lev[L].V, ctx->status, s));
  CKS(check_status(ctx, "agca_flag"));
  ctx->nu = nu;
  for (int l = L - 1; l >= 1; --l) {
    Level& lc = ctx->lev[l];
    const Level& lf = ctx->lev[l + 1];
    LK(1, launch_coarsen(lc.n, ctx->projection, lf.mean, lf.mx, lf.mn, nu, lc.mean, lc.mx, lc.mn, lc.flags, s));
    if (eta_v)
      LK(1, launch_gradient_flags(lc.n, l == L - 1 ? eta_v : nullptr, nu, l == L - 1 ? nullptr : lf.flags, lc.flags,
                                  s));
  }
  for (int l = 1; l < L; ++l) {
    Level& lc = ctx->lev[l];
    LK(3, launch_compact(lc.flags, lc.E, lc.fidx, lc.list, ctx->block_counts, ctx->totals + l, s));
    // vertices of flagged elements: the stencil store (Remark 5)
    LK(1, launch_mark_vertices(lc.n, lc.flags, lc.vmark, s));
    LK(3, launch_compact(lc.vmark, lc.V, lc.sidx, lc.slist, ctx->block_counts, ctx->totals + (L + 1) + l, s));
  }
  std::vector<int64_t> tot(2 * (L + 1), 0);
  CK(cudaMemcpyAsync(tot.data(), ctx->totals, 2 * (L + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int l = 1; l < L; ++l) {
    ctx->lev[l].n_flag = tot[l];
    ctx->lev[l].n_sv = tot[L + 1 + l];
  }
  carve_gca(ctx, nullptr);
  *gca_bytes = ctx->gs_need;
  ctx->flagged = true;
  ctx->setup_done = false;
  ctx->gs = nullptr;
  return AGCA_OK;
}
}  // namespace

extern "C" {

agca_status agca_flag(agca_ctx* ctx, double nu, size_t* gca_bytes) { return flag_impl(ctx, nu, nullptr, gca_bytes); }

agca_status agca_flag_gradient(agca_ctx* ctx, const double* eta_vertex_dev, double nu, size_t* gca_bytes) {
  if (!eta_vertex_dev) return ctx ? ctx->fail(AGCA_EINVAL, "nodal viscosity missing") : AGCA_EINVAL;
  return flag_impl(ctx, nu, eta_vertex_dev, gca_bytes);
}

agca_status agca_bind_gca_store(agca_ctx* ctx, void* dev_ptr, size_t bytes) {
  if (!ctx) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (!ctx->flagged) return ctx->fail(AGCA_ESTATE, "flag first");
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign) != 0) return ctx->fail(AGCA_EINVAL, "store must be 256-byte aligned");
  if (bytes < ctx->gs_need) return ctx->fail(AGCA_ENOMEM, "Galerkin store too small");
  ctx->gs = static_cast<char*>(dev_ptr);
  ctx->gs_bytes = bytes;
  carve_gca(ctx, ctx->gs);
  return AGCA_OK;
}

agca_status agca_set_level_coefficient(agca_ctx* ctx, int level, const double* coef_dev) {
  if (!ctx || !coef_dev) return AGCA_EINVAL;
  if (level < 1 || level >= ctx->L) return ctx->fail(AGCA_EINVAL, "level must be a coarse level");
  if (!ctx->flagged) return ctx->fail(AGCA_ESTATE, "flag first");
  ctx->clear_graphs();
  Level& lv = ctx->lev[level];
  CK(cudaMemcpyAsync(lv.mean, coef_dev, lv.E * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  LK(1, launch_check_eta(lv.mean, lv.E, ctx->status, ctx->stream));
  CKS(check_status(ctx, "agca_set_level_coefficient"));
  ctx->setup_done = false;
  return AGCA_OK;
}

agca_status agca_setup(agca_ctx* ctx) {
  if (!ctx) return AGCA_EINVAL;
  ctx->clear_graphs();
  if (!ctx->flagged || !ctx->gs) return ctx->fail(AGCA_ESTATE, "flag and bind the Galerkin store first");
  cudaStream_t s = ctx->stream;
  const int L = ctx->L;
  const bool mixed = ctx->prec == AGCA_MIXED;
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), s));
  // Galerkin matrices, finest to coarsest (Eq. 2.7)
  for (int l = L - 1; l >= 1; --l) {
    Level& lc = ctx->lev[l];
    const Level& lf = ctx->lev[l + 1];
    const bool child_finest = (l + 1 == L);
    LK(1, launch_galerkin(lc.n, lc.n_flag, lc.list, lf.n, child_finest, lf.mean, child_finest ? nullptr : lf.fidx,
                       child_finest ? nullptr : lf.gca64, lc.gca64, s));
  }
  // stencil storage of the stored-Galerkin part (Remark 5) and, in FP64, the
  // edge-form data of the coarse DCA part (flagged elements masked)
  for (int l = 1; l < L; ++l) {
    Level& lc = ctx->lev[l];
    LK(1, launch_stencil_assemble(lc.n, lc.n_sv, lc.slist, lc.fidx, lc.gca64, lc.sten64, s));
    if (mixed) {
      LK(1, launch_stencil_to_f32(lc.n_sv, lc.sten64, lc.sten32, lc.sscale32, s));
    } else {
      LK(1, launch_masked_coef(lc.E, lc.mean, lc.fidx, lc.coefm, s));
      LK(1, launch_edge_records(lc.n, lc.coefm, lc.hedge, s));
    }
  }
  for (int l = 1; l <= L; ++l) {
    Level& lv = ctx->lev[l];
    if (mixed) {
      LK(1, launch_d2f(lv.mean, lv.mean32, lv.E, s));
      if (l < L) LK(1, launch_gca_to_f32(lv.n_flag, lv.list, lv.mx, lv.gca64, lv.gca32, lv.gscale32, s));
    }
    LK(1, launch_diag(op64(ctx, l), lv.diag, lv.invD64, mixed ? lv.invD32 : nullptr, s));
  }
  // coarsest operator: dense assembly, Cholesky, explicit inverse factor
  LK(1, launch_coarse_assemble(op64(ctx, 1), ctx->cdense, s));
  CK(cudaMemcpyAsync(ctx->cfac, ctx->cdense, (size_t)ctx->mc * ctx->mc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  LK(1, launch_cholesky(ctx->cfac, ctx->mc, ctx->status, s));
  LK(1, launch_trinv(ctx->cfac, ctx->mc, ctx->linv_cm, ctx->linv_rm, s));
  CKS(check_status(ctx, "agca_setup"));
  for (int l = 2; l <= L; ++l) CKS(power_lambda(ctx, l, &ctx->lev[l].lambda));
  LK(1, launch_pressure_mass(ctx->lev[L].n / 2, ctx->lev[L].mean, ctx->pmass, ctx->pmass_inv, s));
  CK(cudaStreamSynchronize(s));
  ctx->setup_done = true;
  return AGCA_OK;
}

agca_status agca_apply(agca_ctx* ctx, int level, int dtype, const void* x_dev, void* y_dev) {
  if (!ctx || !x_dev || !y_dev) return AGCA_EINVAL;
  if (!valid_level(ctx, level)) return ctx->fail(AGCA_EINVAL, "level out of range");
  if (!ctx->setup_done && !(level == ctx->L && ctx->have_eta && dtype == AGCA_F64))
    return ctx->fail(AGCA_ESTATE, "setup first");
  if (dtype == AGCA_F64)
    return stencil<double>(ctx, ST_APPLY, level, static_cast<const double*>(x_dev), nullptr, nullptr,
                           static_cast<double*>(y_dev), 0, 0, 0);
  if (dtype == AGCA_F32 && ctx->prec == AGCA_MIXED)
    return stencil<float>(ctx, ST_APPLY, level, static_cast<const float*>(x_dev), nullptr, nullptr,
                          static_cast<float*>(y_dev), 0, 0, 0);
  return ctx->fail(AGCA_EINVAL, "dtype not available in this context");
}

agca_status agca_restrict(agca_ctx* ctx, int level, int dtype, const void* rf_dev, void* rc_dev) {
  if (!ctx || !rf_dev || !rc_dev) return AGCA_EINVAL;
  if (level < 2 || level > ctx->L) return ctx->fail(AGCA_EINVAL, "level out of range");
  const int nf = ctx->lev[level].n;
  if (dtype == AGCA_F64)
    LK(1, launch_restrict<double>(nf, 3, true, 1.0, static_cast<const double*>(rf_dev), static_cast<double*>(rc_dev),
                               ctx->stream));
  else if (dtype == AGCA_F32)
    LK(1, launch_restrict<float>(nf, 3, true, 1.0f, static_cast<const float*>(rf_dev), static_cast<float*>(rc_dev),
                              ctx->stream));
  else
    return ctx->fail(AGCA_EINVAL, "bad dtype");
  return AGCA_OK;
}

agca_status agca_prolong_add(agca_ctx* ctx, int level, int dtype, const void* ec_dev, void* xf_dev) {
  if (!ctx || !ec_dev || !xf_dev) return AGCA_EINVAL;
  if (level < 2 || level > ctx->L) return ctx->fail(AGCA_EINVAL, "level out of range");
  const int nf = ctx->lev[level].n;
  if (dtype == AGCA_F64)
    LK(1, launch_prolong<double>(nf, 3, true, true, static_cast<const double*>(ec_dev), static_cast<double*>(xf_dev),
                              ctx->stream));
  else if (dtype == AGCA_F32)
    LK(1, launch_prolong<float>(nf, 3, true, true, static_cast<const float*>(ec_dev), static_cast<float*>(xf_dev),
                             ctx->stream));
  else
    return ctx->fail(AGCA_EINVAL, "bad dtype");
  return AGCA_OK;
}

agca_status agca_vcycle(agca_ctx* ctx, const double* r_dev, double* z_dev) {
  if (!ctx || !r_dev || !z_dev) return AGCA_EINVAL;
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  return vcycle_impl(ctx, r_dev, z_dev);
}

agca_status agca_stokes_apply(agca_ctx* ctx, const double* x_dev, double* y_dev) {
  if (!ctx || !x_dev || !y_dev) return AGCA_EINVAL;
  if (!ctx->have_eta) return ctx->fail(AGCA_ESTATE, "set the viscosity first");
  return stokes_impl<double>(ctx, x_dev, y_dev);
}

agca_status agca_precondition(agca_ctx* ctx, const double* r_dev, double* z_dev) {
  if (!ctx || !r_dev || !z_dev) return AGCA_EINVAL;
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  return precond_impl(ctx, r_dev, z_dev);
}

agca_status agca_load_vector(agca_ctx* ctx, const double* fbar_dev, double* b_dev) {
  if (!ctx || !fbar_dev || !b_dev) return AGCA_EINVAL;
  const Level& lf = ctx->lev[ctx->L];
  LK(1, launch_load_vector(lf.n, fbar_dev, b_dev, ctx->stream));
  CK(cudaMemsetAsync(b_dev + 3 * lf.V, 0, ctx->Vp * sizeof(double), ctx->stream));
  return AGCA_OK;
}

agca_status agca_solve(agca_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit, int* iters,
                       double* relres) {
  if (!ctx || !b_dev || !x_dev) return AGCA_EINVAL;
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  if (!(rtol > 0.0) || maxit < 1) return ctx->fail(AGCA_EINVAL, "rtol must be > 0 and maxit >= 1");
  return solve_impl(ctx, b_dev, x_dev, rtol, maxit, iters, relres);
}

agca_status agca_fgmres_workspace_size(const agca_ctx* ctx, int restart, size_t* bytes) {
  if (!ctx || !bytes || restart < 1 || restart > 500) return AGCA_EINVAL;
  *bytes = fgmres_layout(ctx, restart, nullptr).need;
  return AGCA_OK;
}

agca_status agca_solve_fgmres(agca_ctx* ctx, const double* b_dev, double* x_dev, double rtol, int maxit, int restart,
                              int schur, int z_iters, void* work_dev, size_t work_bytes, int* iters, double* relres) {
  if (!ctx || !b_dev || !x_dev || !work_dev) return AGCA_EINVAL;
  if (restart < 1 || restart > 500 || maxit < 1 || !(rtol > 0.0) || (schur != 0 && schur != 1) || z_iters < 0)
    return ctx->fail(AGCA_EINVAL, "bad FGMRES parameters");
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  if (((uintptr_t)work_dev % kAlign) != 0) return ctx->fail(AGCA_EINVAL, "workspace must be 256-byte aligned");
  const FgmresWork W = fgmres_layout(ctx, restart, static_cast<char*>(work_dev));
  if (work_bytes < W.need) return ctx->fail(AGCA_ENOMEM, "FGMRES workspace too small");
  return fgmres_impl(ctx, W, restart, b_dev, x_dev, rtol, maxit, schur, z_iters, iters, relres);
}

agca_status agca_element_sensitivity(agca_ctx* ctx, const double* lam_u_dev, const double* u_dev, double* g_dev) {
  if (!ctx || !lam_u_dev || !u_dev || !g_dev) return AGCA_EINVAL;
  if (!ctx->have_eta) return ctx->fail(AGCA_ESTATE, "set the viscosity first");
  const Level& lf = ctx->lev[ctx->L];
  LK(1, launch_sensitivity(lf.n, lf.mean, lam_u_dev, u_dev, g_dev, ctx->stream));
  return AGCA_OK;
}

agca_status agca_adjoint_gradient(agca_ctx* ctx, const double* x_dev, const double* dJdu_dev, double* g_dev,
                                  double rtol, int maxit, int* iters) {
  if (!ctx || !x_dev || !dJdu_dev || !g_dev) return AGCA_EINVAL;
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  if (!(rtol > 0.0) || maxit < 1) return ctx->fail(AGCA_EINVAL, "rtol must be > 0 and maxit >= 1");
  const Level& lf = ctx->lev[ctx->L];
  const int64_t n3 = 3 * lf.V;
  double* rhs = ctx->kv[KV_ARHS];
  double* lam = ctx->kv[KV_ALAM];
  CK(cudaMemcpyAsync(rhs, dJdu_dev, n3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemsetAsync(rhs + n3, 0, ctx->Vp * sizeof(double), ctx->stream));
  double rel = 0.0;
  int its = 0;
  const agca_status st = solve_impl(ctx, rhs, lam, rtol, maxit, &its, &rel);
  if (iters) *iters = its;
  if (st != AGCA_OK) return st;
  LK(1, launch_sensitivity(lf.n, lf.mean, lam, x_dev, g_dev, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return AGCA_OK;
}

agca_status agca_autotune(agca_ctx* ctx, int reps, const char* cache_path) {
  if (!ctx) return AGCA_EINVAL;
  if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
  if (reps < 1 || reps > 10000) return ctx->fail(AGCA_EINVAL, "reps out of range");
  ctx->clear_graphs();
  std::map<std::string, TileCfg> cache;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string pr;
    int n, mode, coarse, by, zch;
    while (in >> pr >> n >> mode >> coarse >> by >> zch) {
      std::ostringstream key;
      key << pr << ' ' << n << ' ' << mode << ' ' << coarse;
      TileCfg c;
      c.by = by;
      c.zch = zch;
      cache[key.str()] = c;
    }
  }
  for (int l = 2; l <= ctx->L; ++l) {
    const agca_status st = ctx->prec == AGCA_MIXED ? tune_level<float>(ctx, l, reps, cache)
                                                   : tune_level<double>(ctx, l, reps, cache);
    if (st != AGCA_OK) return st;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (cache_path) {
    std::ofstream out(cache_path);
    for (auto& kv : cache) out << kv.first << ' ' << kv.second.by << ' ' << kv.second.zch << '\n';
  }
  return AGCA_OK;
}

agca_status agca_tile_config(const agca_ctx* ctx, int level, int mode, int* by, int* zch) {
  if (!ctx || !by || !zch || level < 1 || level > ctx->L || mode < 0 || mode > 5) return AGCA_EINVAL;
  *by = ctx->tune[level][mode].by;
  *zch = ctx->tune[level][mode].zch;
  return AGCA_OK;
}

agca_status agca_set_tile_config(agca_ctx* ctx, int level, int mode, int by, int zch) {
  if (!ctx) return AGCA_EINVAL;
  if (level < 1 || level > ctx->L || mode < 0 || mode > 5 || zch < 0 || zch > 4096)
    return ctx->fail(AGCA_EINVAL, "tile config out of range");
  if (!(by == 8 || ((by == 12 || by == 16) && ctx->prec == AGCA_MIXED && mode != ST_STOKES)))
    return ctx->fail(AGCA_EINVAL, "block rows must be 8 (or 12, 16 for FP32 cycle launches)");
  ctx->clear_graphs();
  ctx->tune[level][mode].by = by;
  ctx->tune[level][mode].zch = zch;
  return AGCA_OK;
}

agca_status agca_stencil_tiles(int n, int by, int zch, int* out) {
  if (!out || n < 1 || n > 1024 || !(by == 8 || by == 12 || by == 16) || zch < 0) return AGCA_EINVAL;
  const TileGrid g = stencil_tiles(n, by, zch);
  const int v[7] = {g.gxw, g.gyw, g.gxn, g.gyn, g.x0n, g.gz, g.zch};
  for (int i = 0; i < 7; ++i) out[i] = v[i];
  return AGCA_OK;
}

agca_status agca_launch_count(const agca_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return AGCA_EINVAL;
  *launches = ctx->launches;
  return AGCA_OK;
}

agca_status agca_profile_fine(agca_ctx* ctx, int enable, double* ms, double* bytes, double* flops,
                              int64_t* launches) {
  if (!ctx) return AGCA_EINVAL;
  if (enable) {
    const size_t want = 2 * 65536;
    while (ctx->ev.size() < want) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ctx->ev.push_back(e);
    }
    ctx->ev_used = 0;
    ctx->prof_bytes = 0.0;
    ctx->prof_flops = 0.0;
    ctx->prof_launches = 0;
    ctx->prof = true;
    return AGCA_OK;
  }
  ctx->prof = false;
  CK(cudaStreamSynchronize(ctx->stream));
  double total = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
    total += t;
  }
  if (ms) *ms = total;
  if (bytes) *bytes = ctx->prof_bytes;
  if (flops) *flops = ctx->prof_flops;
  if (launches) *launches = ctx->prof_launches;
  ctx->ev_used = 0;
  return AGCA_OK;
}

agca_status agca_level_info(agca_ctx* ctx, int level, agca_level_info_t* out) {
  if (!ctx || !out) return AGCA_EINVAL;
  if (!valid_level(ctx, level)) return ctx->fail(AGCA_EINVAL, "level out of range");
  const Level& lv = ctx->lev[level];
  out->n = lv.n;
  out->vertices = lv.V;
  out->elements = lv.E;
  out->n_flag = level < ctx->L ? lv.n_flag : 0;
  out->n_stencil = level < ctx->L ? lv.n_sv : 0;
  out->lambda = lv.lambda;
  return AGCA_OK;
}

agca_status agca_get_level_data(agca_ctx* ctx, int level, int field, void* dst_dev) {
  if (!ctx || !dst_dev) return AGCA_EINVAL;
  if (!valid_level(ctx, level)) return ctx->fail(AGCA_EINVAL, "level out of range");
  const Level& lv = ctx->lev[level];
  const void* src = nullptr;
  size_t bytes = 0;
  const bool coarse = level < ctx->L;
  switch (field) {
    case AGCA_FIELD_MEAN: src = lv.mean; bytes = lv.E * sizeof(double); break;
    case AGCA_FIELD_MAX: src = lv.mx; bytes = lv.E * sizeof(double); break;
    case AGCA_FIELD_MIN: src = lv.mn; bytes = lv.E * sizeof(double); break;
    case AGCA_FIELD_FLAGS:
      if (!coarse) return ctx->fail(AGCA_EINVAL, "no flags on the finest level");
      src = lv.flags; bytes = lv.E; break;
    case AGCA_FIELD_LIST:
      if (!coarse) return ctx->fail(AGCA_EINVAL, "no flags on the finest level");
      src = lv.list; bytes = lv.n_flag * sizeof(int32_t); break;
    case AGCA_FIELD_GCA:
      if (!coarse || !ctx->setup_done) return ctx->fail(AGCA_ESTATE, "no Galerkin matrices here");
      src = lv.gca64; bytes = lv.n_flag * 144 * sizeof(double); break;
    case AGCA_FIELD_DIAG:
      if (!ctx->setup_done) return ctx->fail(AGCA_ESTATE, "setup first");
      src = lv.diag; bytes = 3 * lv.V * sizeof(double); break;
    case AGCA_FIELD_COARSE:
      if (level != 1 || !ctx->setup_done) return ctx->fail(AGCA_ESTATE, "coarse matrix: level 1 after setup");
      src = ctx->cdense; bytes = (size_t)ctx->mc * ctx->mc * sizeof(double); break;
    case AGCA_FIELD_PMASS:
      if (level != ctx->L - 1 || !ctx->setup_done) return ctx->fail(AGCA_ESTATE, "pressure mass: level L-1 after setup");
      src = ctx->pmass; bytes = ctx->Vp * sizeof(double); break;
    case AGCA_FIELD_SIDX:
      if (!coarse || !ctx->flagged) return ctx->fail(AGCA_ESTATE, "stencil indices: coarse level after agca_flag");
      src = lv.sidx; bytes = lv.V * sizeof(int32_t); break;
    case AGCA_FIELD_STENCIL:
      if (!coarse || !ctx->setup_done) return ctx->fail(AGCA_ESTATE, "stencils: coarse level after setup");
      src = lv.sten64; bytes = lv.n_sv * 135 * sizeof(double); break;
    default: return ctx->fail(AGCA_EINVAL, "unknown field");
  }
  if (bytes) CK(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return AGCA_OK;
}

// ============================================================== batch C ABI
static int default_levels_for(int N) {
  int n = 2 * N, L = 1;
  while (n % 2 == 0 && n / 2 >= 4) {
    n /= 2;
    ++L;
  }
  return L;
}

agca_status agca_batch_create(int n, const int* Ns, int prec, void* cuda_stream, agca_batch** out) {
  if (!out || !Ns || n < 1 || n > 4096) return AGCA_EINVAL;
  *out = nullptr;
  agca_batch* b = new agca_batch();
  b->n = n;
  b->prec = prec;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  size_t off = 0;
  size_t max_task = std::max(sizeof(StencilTask<double, double>), std::max(sizeof(XferTask), sizeof(KTask)));
  for (int i = 0; i < n; ++i) {
    agca_ctx* c = nullptr;
    const agca_status st = agca_create(Ns[i], default_levels_for(Ns[i]), prec, cuda_stream, &c);
    if (st != AGCA_OK) {
      delete b;
      return st;
    }
    b->ctx.push_back(c);
    b->ws_off.push_back(off);
    off += (c->ws_need + kAlign - 1) / kAlign * kAlign;
  }
  // task tables: two MINRES iteration parities plus one per-call V-cycle set,
  // at most ~8 steps per level and 24 fixed steps, one task per problem each
  int maxL = 0;
  for (auto* c : b->ctx) maxL = std::max(maxL, c->L);
  const size_t steps = (size_t)8 * maxL + 32;
  b->tab_bytes = 3 * steps * ((size_t)n * max_task + 256) + (1 << 16);
  b->ws_off.push_back(off);  // table
  off += (b->tab_bytes + kAlign - 1) / kAlign * kAlign;
  b->ws_off.push_back(off);  // reduction partials and done flags
  off += ((size_t)n * 64 + n) * sizeof(double);
  b->ws_need = (off + kAlign - 1) / kAlign * kAlign;
  *out = b;
  return AGCA_OK;
}

void agca_batch_destroy(agca_batch* b) { delete b; }

const char* agca_batch_last_error(const agca_batch* b) { return b ? b->err.c_str() : "null batch"; }

agca_status agca_batch_workspace_size(const agca_batch* b, size_t* bytes) {
  if (!b || !bytes) return AGCA_EINVAL;
  *bytes = b->ws_need;
  return AGCA_OK;
}

agca_status agca_batch_bind_workspace(agca_batch* b, void* dev_ptr, size_t bytes) {
  if (!b) return AGCA_EINVAL;
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign) != 0) return b->fail(AGCA_EINVAL, "workspace must be 256-byte aligned");
  if (bytes < b->ws_need) return b->fail(AGCA_ENOMEM, "workspace too small");
  b->ws = static_cast<char*>(dev_ptr);
  for (int i = 0; i < b->n; ++i) {
    const agca_status st = agca_bind_workspace(b->ctx[i], b->ws + b->ws_off[i], b->ctx[i]->ws_need);
    if (st != AGCA_OK) return b->fail(st, b->ctx[i]->err);
  }
  b->tab = b->ws + b->ws_off[b->n];
  b->partials = reinterpret_cast<double*>(b->ws + b->ws_off[b->n + 1]);
  b->setup_done = false;
  return AGCA_OK;
}

agca_status agca_batch_set_viscosity(agca_batch* b, int i, const double* eta_dev) {
  if (!batch_valid(b, i) || !eta_dev) return AGCA_EINVAL;
  b->setup_done = false;
  const agca_status st = agca_set_viscosity(b->ctx[i], eta_dev);
  return st == AGCA_OK ? st : b->fail(st, b->ctx[i]->err);
}

agca_status agca_batch_flag(agca_batch* b, double nu, size_t* gca_bytes) {
  if (!b || !gca_bytes) return AGCA_EINVAL;
  b->gs_off.assign(b->n + 1, 0);
  size_t off = 0;
  for (int i = 0; i < b->n; ++i) {
    size_t g = 0;
    const agca_status st = agca_flag(b->ctx[i], nu, &g);
    if (st != AGCA_OK) return b->fail(st, b->ctx[i]->err);
    b->gs_off[i] = off;
    off += (g + kAlign - 1) / kAlign * kAlign;
  }
  b->gs_off[b->n] = off;
  b->gs_need = off;
  *gca_bytes = off;
  b->setup_done = false;
  return AGCA_OK;
}

agca_status agca_batch_bind_gca_store(agca_batch* b, void* dev_ptr, size_t bytes) {
  if (!b) return AGCA_EINVAL;
  if (b->gs_off.empty()) return b->fail(AGCA_ESTATE, "flag first");
  if (!dev_ptr || ((uintptr_t)dev_ptr % kAlign) != 0) return b->fail(AGCA_EINVAL, "store must be 256-byte aligned");
  if (bytes < b->gs_need) return b->fail(AGCA_ENOMEM, "Galerkin store too small");
  b->gs = static_cast<char*>(dev_ptr);
  for (int i = 0; i < b->n; ++i) {
    const agca_status st = agca_bind_gca_store(b->ctx[i], b->gs + b->gs_off[i], b->ctx[i]->gs_need);
    if (st != AGCA_OK) return b->fail(st, b->ctx[i]->err);
  }
  return AGCA_OK;
}

// Task tables and captured graph of the lockstep MINRES iteration (both
// buffer parities) for the problems in b->members.
agca_status build_iteration_graph(agca_batch* b) {
  b->iter_members.clear();
  b->host_tab.clear();
  build_iteration(b, 0);
  build_iteration(b, 1);
  // publish every member's done flag into one contiguous array (by problem) as well
  double* done = b->partials + (size_t)b->n * 64;
  for (int par = 0; par < 2; ++par)
    for (BatchStep& st : b->iter_steps[par])
      if (st.kind == 2 && st.mode == KB_SCALARS)
        for (int i = 0; i < st.ntasks; ++i) {
          KTask* t = reinterpret_cast<KTask*>(b->host_tab.data() + st.off) + i;
          t->c = done + b->members[i];
        }
  if (b->host_tab.size() > b->tab_bytes / 3 * 2) return b->fail(AGCA_EINTERNAL, "batch task table overflow");
  BCK(cudaMemcpyAsync(b->tab, b->host_tab.data(), b->host_tab.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (b->iter_graph) {
    cudaGraphExecDestroy(b->iter_graph);
    b->iter_graph = nullptr;
  }
  b->iter_launches = 0;
  if (b->stream != nullptr) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int64_t nl = 0;
    agca_status st = run_steps(b, b->iter_steps[0], &nl);
    if (st == AGCA_OK) st = run_steps(b, b->iter_steps[1], &nl);
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (st != AGCA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    BCK(ee);
    const cudaError_t ie = cudaGraphInstantiate(&b->iter_graph, g, 0);
    cudaGraphDestroy(g);
    BCK(ie);
    b->iter_launches = nl;
  }
  b->iter_members = b->members;
  return AGCA_OK;
}

agca_status agca_batch_setup(agca_batch* b) {
  if (!b) return AGCA_EINVAL;
  if (!b->ws || !b->gs) return b->fail(AGCA_ESTATE, "bind the workspace and the Galerkin store first");
  for (int i = 0; i < b->n; ++i) {
    const agca_status st = agca_setup(b->ctx[i]);
    if (st != AGCA_OK) return b->fail(st, b->ctx[i]->err);
  }
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
  b->members.resize(b->n);
  for (int i = 0; i < b->n; ++i) b->members[i] = i;
  BCKS(build_iteration_graph(b));
  b->setup_done = true;
  return AGCA_OK;
}

agca_status agca_batch_load_vector(agca_batch* b, int i, const double* fbar_dev, double* b_dev) {
  if (!batch_valid(b, i)) return AGCA_EINVAL;
  const agca_status st = agca_load_vector(b->ctx[i], fbar_dev, b_dev);
  return st == AGCA_OK ? st : b->fail(st, b->ctx[i]->err);
}

agca_status agca_batch_vcycle(agca_batch* b, const double* const* r_devs, double* const* z_devs) {
  if (!b || !r_devs || !z_devs) return AGCA_EINVAL;
  if (!b->setup_done) return b->fail(AGCA_ESTATE, "setup first");
  std::vector<const double*> r(r_devs, r_devs + b->n);
  std::vector<double*> z(z_devs, z_devs + b->n);
  b->members.resize(b->n);  // a batched V-cycle covers every problem
  for (int p = 0; p < b->n; ++p) b->members[p] = p;
  std::vector<BatchStep> steps;
  const size_t base = b->host_tab.size();
  if (b->prec == AGCA_MIXED)
    build_cycle<float>(b, steps, r, z, false);
  else
    build_cycle<double>(b, steps, r, z, false);
  const size_t used = b->host_tab.size() - base;
  if (b->host_tab.size() > b->tab_bytes) {
    b->host_tab.resize(base);
    return b->fail(AGCA_EINTERNAL, "batch task table overflow");
  }
  BCK(cudaMemcpyAsync(b->tab + base, b->host_tab.data() + base, used, cudaMemcpyHostToDevice, b->stream));
  int64_t nl = 0;
  const agca_status st = run_steps(b, steps, &nl);
  BCK(cudaStreamSynchronize(b->stream));  // the table region is reused by the next call
  b->host_tab.resize(base);
  return st;
}

agca_status agca_batch_solve(agca_batch* b, const double* const* b_devs, double* const* x_devs, double rtol, int maxit,
                             int* iters, double* relres) {
  if (!b || !b_devs || !x_devs) return AGCA_EINVAL;
  if (!b->setup_done) return b->fail(AGCA_ESTATE, "setup first");
  if (!(rtol > 0.0) || maxit < 1) return b->fail(AGCA_EINVAL, "rtol must be > 0 and maxit >= 1");
  const int P = b->n;
  const bool mixed = b->prec == AGCA_MIXED;
  std::vector<double> nb(P, 0.0), rel(P, 0.0);
  std::vector<int> total(P, 0);
  std::vector<char> active(P, 0);
  static const double one = 1.0;
  for (int p = 0; p < P; ++p) {
    agca_ctx* ctx = b->ctx[p];
    const int64_t nt = ctx->nt;
    double* bm = ctx->kv[KV_B];
    LK(1, launch_vec_op(VOP_COPY, nt, bm, b_devs[p], nullptr, nullptr, nullptr, b->stream));
    LK(1, launch_mask_boundary(ctx->lev[ctx->L].n, bm, b->stream));
    LK(1, launch_vec_op(VOP_ZERO, nt, x_devs[p], nullptr, nullptr, nullptr, nullptr, b->stream));
    double nb2 = 0.0;
    CKS(dot1(ctx, bm, bm, nt, ctx->sc + MS_TMP0));
    CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &nb2));
    nb[p] = sqrt(nb2);
    rel[p] = nb[p] > 0.0 ? 1.0 : 0.0;
  }
  double* done_dev = b->partials + (size_t)P * 64;
  std::vector<double> done(P, 0.0);
  for (int outer = 0; outer < 60; ++outer) {
    bool any = false;
    for (int p = 0; p < P; ++p) {
      agca_ctx* ctx = b->ctx[p];
      const int64_t nt = ctx->nt;
      active[p] = 0;
      if (!(nb[p] > 0.0)) continue;
      CKS(stokes_dispatch(ctx, x_devs[p], ctx->kv[KV_KZ], false));
      LK(1, launch_vec_op(VOP_SUB, nt, ctx->kv[KV_R], ctx->kv[KV_B], ctx->kv[KV_KZ], nullptr, nullptr, b->stream));
      double nr2 = 0.0;
      CKS(dot1(ctx, ctx->kv[KV_R], ctx->kv[KV_R], nt, ctx->sc + MS_TMP0));
      CKS(read_scalar(ctx, ctx->sc + MS_TMP0, &nr2));
      rel[p] = sqrt(nr2) / nb[p];
      active[p] = (rel[p] > rtol && total[p] < maxit) ? 1 : 0;
      any = any || active[p];
    }
    if (!any) break;
    // the lockstep tables cover the problems still above the tolerance
    std::vector<int> act;
    for (int p = 0; p < P; ++p)
      if (active[p]) act.push_back(p);
    if (act != b->iter_members) {
      b->members = act;
      BCKS(build_iteration_graph(b));
    }
    int budget = 0;
    for (int p = 0; p < P; ++p) {
      agca_ctx* ctx = b->ctx[p];
      const int64_t nt = ctx->nt;
      cudaStream_t s = b->stream;
      if (!active[p]) {
        CK(cudaMemcpyAsync(ctx->sc + MS_DONE, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->sc + MS_UPD_SKIP, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        continue;
      }
      budget = std::max(budget, maxit - total[p]);
      double inner = 0.1 * rtol / rel[p];
      if (mixed) inner = std::max(inner, ctx->mixed_inner);
      inner = std::max(inner, 1e-14);
      LK(1, launch_vec_op(VOP_ZERO, nt, ctx->kv[KV_D], nullptr, nullptr, nullptr, nullptr, s));
      LK(1, launch_vec_op(VOP_ZERO, nt, ctx->kv[KV_VOLD], nullptr, nullptr, nullptr, nullptr, s));
      LK(1, launch_vec_op(VOP_ZERO, nt, ctx->kv[KV_WOLD], nullptr, nullptr, nullptr, nullptr, s));
      LK(1, launch_vec_op(VOP_ZERO, nt, ctx->kv[KV_W], nullptr, nullptr, nullptr, nullptr, s));
      LK(1, launch_vec_op(VOP_COPY, nt, ctx->kv[KV_V], ctx->kv[KV_R], nullptr, nullptr, nullptr, s));
      CKS(precond_impl(ctx, ctx->kv[KV_V], ctx->kv[KV_Z]));
      CKS(dot1(ctx, ctx->kv[KV_Z], ctx->kv[KV_V], nt, ctx->sc + MS_DOT_ZV));
      LK(1, launch_minres_init(ctx->sc, inner, s));
    }
    // lockstep iterations, two per graph replay (buffer parity returns)
    int64_t launches = 0;
    for (int it = 0; it < budget; it += 2) {
      if (b->iter_graph) {
        BCK(cudaGraphLaunch(b->iter_graph, b->stream));
        launches += b->iter_launches;
      } else {
        BCKS(run_steps(b, b->iter_steps[0], &launches));
        BCKS(run_steps(b, b->iter_steps[1], &launches));
      }
      if ((it / 2 + 1) % 4 == 0 || it + 2 >= budget) {
        BCK(cudaMemcpyAsync(done.data(), done_dev, P * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        std::vector<int> running;
        for (int p : b->iter_members)
          if (done[p] == 0.0) running.push_back(p);
        if (running.empty()) break;
        // once a quarter of the lockstep problems have converged, drop them
        // from the tables: their launches no longer walk converged work
        if (4 * running.size() <= 3 * b->iter_members.size()) {
          b->members = running;
          BCKS(build_iteration_graph(b));
        }
      }
    }
    for (int p = 0; p < P; ++p) {
      if (!active[p]) continue;
      agca_ctx* ctx = b->ctx[p];
      double its = 0.0;
      CKS(read_scalar(ctx, ctx->sc + MS_ITERS, &its));
      total[p] += (int)its;
      LK(1, launch_vec_op(VOP_ADD, ctx->nt, x_devs[p], x_devs[p], ctx->kv[KV_D], nullptr, nullptr, b->stream));
      CKS(project_pressure(ctx, x_devs[p]));
    }
    b->ctx[0]->launches += launches;
  }
  bool ok = true;
  for (int p = 0; p < P; ++p) {
    if (iters) iters[p] = total[p];
    if (relres) relres[p] = rel[p];
    if (!(rel[p] <= rtol)) ok = false;
  }
  if (!ok) return b->fail(AGCA_ENOTCONV, "some problems stopped above the tolerance");
  return AGCA_OK;
}

agca_ctx* agca_batch_context(agca_batch* b, int i) { return batch_valid(b, i) ? b->ctx[i] : nullptr; }

}  // extern "C"
