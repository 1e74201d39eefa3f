// C ABI of the SEIRD Newton-Krylov-Schwarz step (include/seird.h) and the
// host-side drivers: context set-up, Newton with backtracking (Section 2.2),
// right-preconditioned restarted FGMRES with CGS2 (Section 3.2), and the
// RAS + coarse preconditioner (Eq. RAS, Section 3.1).  Every arithmetic step
// of the path runs in the library's CUDA kernels; the host only sequences
// launches and reads back scalars (norms, the GMRES residual estimate).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"
#include <nvtx3/nvToolsExt.h>
#include "kernels.cuh"

namespace seird {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }
void coarse_init();

}  // namespace seird

using namespace seird;

namespace {

thread_local std::string g_create_error;

}  // namespace

void seird::set_global_error(const std::string& msg) { g_create_error = msg; }

namespace {

int fail(seird_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  else g_create_error = msg;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, SEIRD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(expr)          \
  do {                     \
    int rc_ = (expr);      \
    if (rc_ != SEIRD_OK) { \
      return rc_;          \
    }                      \
  } while (0)

// Host exceptions end as error codes and never cross the C ABI: chiefly a failed
// host allocation (the set-up of a paper-scale mesh holds several GB of host
// arrays), reported as SEIRD_ENOMEM.
void note_error(seird_ctx* ctx, const char* msg) noexcept {
  try {
    if (ctx) ctx->last_error = msg;
    else g_create_error = msg;
  } catch (...) {
  }
}

template <class F>
int host_guard(seird_ctx* ctx, F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    note_error(ctx, "host allocation failed");
    return SEIRD_ENOMEM;
  } catch (const std::length_error&) {
    note_error(ctx, "host allocation failed (size beyond the container limit)");
    return SEIRD_ENOMEM;
  } catch (const std::exception& e) {
    note_error(ctx, e.what());
    return SEIRD_EINVAL;
  } catch (...) {
    note_error(ctx, "unknown host exception");
    return SEIRD_EINVAL;
  }
}

template <class T>
int dalloc(seird_ctx* ctx, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, SEIRD_ENOMEM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes: " +
                                       cudaGetErrorString(e));
  }
  try {
    ctx->allocations.push_back((void*)*p);
  } catch (...) {
    cudaFree(*p);
    *p = nullptr;
    throw;
  }
  ctx->device_bytes += (int64_t)(sizeof(T) * count);
  return SEIRD_OK;
}

template <class T>
int upload(seird_ctx* ctx, T** p, const std::vector<T>& v) {
  TRY(dalloc(ctx, p, v.size()));
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return SEIRD_OK;
}

// beta(t) of the sigmoid schedule (Eq. beta_ie)
double beta_time(const seird_beta_schedule& s, double t) { return s.b0 - s.b1 / (1.0 + std::exp(s.t_mid - t)); }

// Rates of the step that ends at ctx->t + dt.
Rates make_rates(const seird_ctx* ctx) {
  Rates r{};
  const seird_params& p = ctx->params;
  r.A = p.A;
  r.bi = p.beta_i;
  r.be = p.beta_e;
  if (ctx->sched_on) r.bi = r.be = beta_time(ctx->sched, ctx->t + ctx->opt.dt);
  if (ctx->rtab) {
    r.tab = ctx->rtab;
    r.nper = ctx->n_per_sample;
  }
  r.sigma = p.sigma;
  r.ge = p.gamma_e;
  r.gr = p.gamma_r;
  r.gd = p.gamma_d;
  r.alpha = p.alpha;
  r.mu = p.mu;
  for (int c = 0; c < 4; ++c) r.nu[c] = p.nu[c];
  r.dt = ctx->opt.dt;
  return r;
}

// transmission multiplier field in use (NULL: none)
const double* bfield_of(const seird_ctx* ctx) { return ctx->sched_on ? ctx->bsched : ctx->bfield; }

int64_t vlen(const seird_ctx* ctx) { return 5 * ctx->hs.n; }

bool mixed(const seird_ctx* ctx) { return ctx->opt.precision == 1; }

int check_flags(seird_ctx* ctx, const char* where) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int32_t f = *ctx->h_err;
  if (!f) return SEIRD_OK;
  CK(cudaMemsetAsync(ctx->err, 0, sizeof(int32_t), ctx->stream));
  *ctx->h_err = 0;
  if (f & ERR_NONPOS_N) return fail(ctx, SEIRD_ENONFINITE, std::string(where) + ": N <= 0 at a quadrature point");
  if (f & ERR_SINGULAR) return fail(ctx, SEIRD_ESINGULAR, std::string(where) + ": singular 5x5 pivot block");
  if (f & ERR_TIMEOUT) return fail(ctx, SEIRD_ETIMEOUT, std::string(where) + ": bounded wait expired");
  return fail(ctx, SEIRD_ENONFINITE, std::string(where) + ": non-finite value");
}

// ---- tracing ------------------------------------------------------------------

// NVTX range around a phase of the step (no-op unless a profiler is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// ---- kernel-class timing ----------------------------------------------------

// Records a start event on construction and an end event on destruction, on the
// context's stream, when options.timing is set.
struct KTimer {
  seird_ctx* c;
  size_t slot = (size_t)-1;
  KTimer(seird_ctx* ctx, int cls) : c(ctx) {
    if (!c->opt.timing) return;
    if (c->ev_used + 2 > c->evpool.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->evpool.push_back(e);
      }
    }
    slot = c->ev_used;
    c->ev_used += 2;
    c->ev_class.push_back(cls);
    cudaEventRecord(c->evpool[slot], c->stream);
  }
  ~KTimer() {
    if (slot != (size_t)-1) cudaEventRecord(c->evpool[slot + 1], c->stream);
  }
};

void timing_reset(seird_ctx* ctx) {
  ctx->ev_used = 0;
  ctx->ev_class.clear();
  for (int k = 0; k < SEIRD_K_COUNT; ++k) ctx->abytes[k] = 0.0;
}

void timing_collect(seird_ctx* ctx, seird_stats* S) {
  for (int k = 0; k < SEIRD_K_COUNT; ++k) {
    S->kernel_ms[k] = 0.0;
    S->kernel_calls[k] = 0;
    S->alg_bytes[k] = ctx->abytes[k];
  }
  if (!ctx->opt.timing) return;
  cudaStreamSynchronize(ctx->stream);
  for (size_t q = 0; q < ctx->ev_class.size(); ++q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->evpool[2 * q], ctx->evpool[2 * q + 1]) == cudaSuccess) {
      S->kernel_ms[ctx->ev_class[q]] += ms;
      S->kernel_calls[ctx->ev_class[q]] += 1;
    }
  }
  timing_reset(ctx);
}

// ---- algorithmic bytes per kernel class (seird_stats.alg_bytes) ---------------
// What each launch group must move at least: every array it needs, read or
// written once, at the precision it runs in (w = 4 for the mixed path's FP32
// matrix, factors and preconditioned basis); scratch that a class keeps between
// its own kernels (element vectors, work vectors of the sweeps) is not counted.
// Vectors of the state are 5n doubles = 40n bytes.

double wv(const seird_ctx* c) { return c->opt.precision == 1 ? 4.0 : 8.0; }
void add_bytes(seird_ctx* c, int cls, double b) { c->abytes[cls] += b; }
double nnzb_of(const seird_ctx* c) { return (double)c->hs.col.size(); }
// U and u^n read (80n), xy (16n), triangles (12m), F written (40n)
double bytes_residual(const seird_ctx* c) { return 136.0 * c->hs.n + 12.0 * c->hs.m; }
// U (40n) and xy (16n) read, triangles (12m) and block incidence lists (36m), blocks written
double bytes_jacobian(const seird_ctx* c) { return 56.0 * c->hs.n + 48.0 * c->hs.m + 25.0 * wv(c) * nnzb_of(c); }
// J blocks gathered with their global ids and local columns, factor blocks and inverted pivots written
double bytes_ilu_factor(const seird_ctx* c) {
  return (double)c->hs.l_col.size() * (50.0 * wv(c) + 8.0) + (double)c->hs.sd_node.size() * 25.0 * wv(c);
}
// J blocks read once with their segment order, plus the J Z blocks written for the two-grid
double bytes_coarse_setup(const seird_ctx* c) {
  return nnzb_of(c) * (25.0 * wv(c) + 4.0) + (c->opt.coarse >= 2 ? 25.0 * wv(c) * c->hs.az_unit.size() : 0.0);
}
// values with column indices, row pointers, x once (wx), y written, b read when fused (y = b - J x)
double bytes_spmv(const seird_ctx* c, double wx, bool fused) {
  const double n = (double)c->hs.n;
  return nnzb_of(c) * (25.0 * wv(c) + 4.0) + 4.0 * (n + 1) + 5.0 * n * wx + 40.0 * n + (fused ? 40.0 * n : 0.0);
}
// every local block once (strictly lower, inverted pivots, strictly upper) with its column,
// two 16-byte row records, r read per local row, z written per owned row (wz)
double bytes_ilu_solve(const seird_ctx* c, double wz) {
  return (double)c->hs.l_col.size() * (25.0 * wv(c) + 4.0) + 72.0 * c->hs.sd_node.size() + 5.0 * c->hs.n * wz;
}
// Z^T r (r read), A_c^{-1} (explicit inverse or band factors read once), z += Z y (read and
// written at wz, unit map), and with J Z: its blocks and segment maps read, t read and written
double bytes_coarse_solve(const seird_ctx* c) {
  const double nc = 5.0 * c->hs.Pc;
  const double inv = c->ainvT ? nc * nc * 8.0 : (double)c->hs.Pc * (2.0 * c->hs.cband + 2.0) * 200.0;
  return 40.0 * c->hs.n + inv;
}
double bytes_coarse_prolong(const seird_ctx* c, double wz) { return 10.0 * c->hs.n * wz + 4.0 * c->hs.n; }
double bytes_az_sub(const seird_ctx* c, double wa) {
  return (double)c->hs.az_unit.size() * (25.0 * wa + 4.0) + 8.0 * c->hs.n + 80.0 * c->hs.n;
}
// Arnoldi iteration with nv basis vectors: one classical Gram-Schmidt pass reads V and w
// (dots), then V and w again and writes w (update and norm), then w -> v_{nv}; CGS2 adds a
// fused update-and-dots pass
double bytes_arnoldi(const seird_ctx* c, int nv) {
  const double vec = 40.0 * c->hs.n;
  return (c->opt.gmres_one_pass == 1 ? 2.0 * nv + 5.0 : 3.0 * nv + 7.0) * vec;
}

// ---- building blocks --------------------------------------------------------

// F = F(U; Un), returns ||F||_2 in *fn (synchronises)
int residual(seird_ctx* ctx, const double* U, const double* Un, double* F, double* fn) {
  Range rg_("seird residual");
  const HostSetup& hs = ctx->hs;
  {
    KTimer kt_(ctx, SEIRD_K_RESIDUAL);
    add_bytes(ctx, SEIRD_K_RESIDUAL, bytes_residual(ctx));
    launch_residual(hs.n, hs.m, ctx->tri, ctx->xy, ctx->geo, U, Un, bfield_of(ctx), make_rates(ctx),
                    ctx->opt.quadrature, ctx->nodebuf, ctx->elem, ctx->node_inc_ptr, ctx->node_inc, F, ctx->partial,
                    ctx->scal, ctx->err, ctx->stream);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TRY(check_flags(ctx, "residual"));
  const double v = ctx->h_scal[0];
  if (!std::isfinite(v)) return fail(ctx, SEIRD_ENONFINITE, "residual: non-finite norm");
  *fn = std::sqrt(v);
  return SEIRD_OK;
}

// Assembles dF/dU at U (picard = false) or the Picard matrix of Eq.
// weak_vec_implicit with its coefficients frozen at U (picard = true).
int jacobian(seird_ctx* ctx, const double* U, bool picard = false) {
  Range rg_("seird jacobian");
  const HostSetup& hs = ctx->hs;
  KTimer kt_(ctx, SEIRD_K_JACOBIAN);
  add_bytes(ctx, SEIRD_K_JACOBIAN, bytes_jacobian(ctx));
  // the mixed path assembles the Jacobian straight into its FP32 copy (FP32
  // arithmetic); it only feeds the FP32 operator and the FP32 factors
  launch_jacobian((int64_t)hs.col.size(), hs.m, ctx->tri, ctx->xy, ctx->geo, U, bfield_of(ctx), make_rates(ctx),
                  ctx->opt.quadrature, ctx->rec, ctx->blk_inc_ptr, ctx->blk_inc,
                  mixed(ctx) ? (void*)ctx->val32 : (void*)ctx->val, mixed(ctx), picard, ctx->err, ctx->stream);
  CK(cudaGetLastError());
  ctx->jac_ready = true;  // an existing preconditioner stays usable (lagged set-up, options.pc_lag)
  return SEIRD_OK;
}

RasDev ras_dev(seird_ctx* ctx) {
  RasDev d;
  d.P = ctx->hs.P;
  d.sd_sched = ctx->sd_sched;
  d.sd_row0 = ctx->sd_row0;
  d.sd_node = ctx->sd_node;
  d.l_row_ptr = ctx->l_row_ptr;
  d.l_col = ctx->l_col;
  d.l_gblk = ctx->l_gblk;
  d.l_diag = ctx->l_diag;
  d.upd_ptr = ctx->upd_ptr;
  d.upd = ctx->upd;
  d.fwd_order = ctx->fwd_order;
  d.fwd_lev = ctx->fwd_lev;
  d.sd_fwd_lev0 = ctx->sd_fwd_lev0;
  d.bwd_order = ctx->bwd_order;
  d.bwd_lev = ctx->bwd_lev;
  d.sd_bwd_lev0 = ctx->sd_bwd_lev0;
  d.own_ptr = ctx->own_ptr;
  d.fval = ctx->fval;
  d.dinv = ctx->dinv;
  d.ywork = ctx->ywork;
  d.zwork = ctx->zwork;
  d.fval32 = ctx->fval32;
  d.dinv32 = ctx->dinv32;
  d.ywork32 = ctx->ywork32;
  d.zwork32 = ctx->zwork32;
  auto plan = [](const seird_ctx::PlanPtrs& q) {
    SolvePlanDev s;
    s.row = q.row;
    s.start = q.start;
    s.cnt = q.cnt;
    s.levpos = q.levpos;
    s.levblk = q.levblk;
    s.sd_lev0 = q.sd_lev0;
    s.info = reinterpret_cast<const int4*>(q.info);
    return s;
  };
  d.fwd = plan(ctx->pf);
  d.bwd = plan(ctx->pb);
  d.fL = ctx->fL;
  d.bU = ctx->bU;
  d.fL32 = ctx->fL32;
  d.bU32 = ctx->bU32;
  d.wait_polls = ctx->wait_polls;
  d.solve_ch = ctx->ilu_ch;
  d.solve_warps = ctx->ilu_warps;
  d.solve_ring = ctx->ilu_ring;
  return d;
}

CoarseDev coarse_dev(seird_ctx* ctx) {
  CoarseDev c;
  c.P = ctx->hs.Pc;  // coarse units (groups of cG subdomains)
  c.band = ctx->hs.cband;
  c.cpos = ctx->cpos;
  c.owner = ctx->cunit;
  c.own_ptr = ctx->cunit_ptr;
  c.cseg_blk = ctx->cseg_blk;
  c.cchunk_ptr = ctx->cchunk_ptr;
  c.nchunk = (int32_t)ctx->hs.cchunk_ptr.size() - 1;
  c.cdst_ptr = ctx->cdst_ptr;
  c.cdst_idx = ctx->cdst_idx;
  c.ndst = (int32_t)ctx->hs.cdst_idx.size();
  c.cpart = ctx->cpart;
  c.cband = ctx->cband;
  c.cdinv = ctx->cdinv;
  c.crhs = ctx->crhs;
  c.ainvT = ctx->ainvT;
  c.y32 = ctx->cy32;
  return c;
}

int pc_setup(seird_ctx* ctx) {
  Range rg_("seird preconditioner setup");
  if (!ctx->jac_ready) return fail(ctx, SEIRD_EINVAL, "preconditioner setup needs an assembled Jacobian");
  {
    KTimer kt_(ctx, SEIRD_K_ILU_FACTOR);
    add_bytes(ctx, SEIRD_K_ILU_FACTOR, bytes_ilu_factor(ctx));
    const RasDev d = ras_dev(ctx);
    launch_ilu_factor(d, ctx->val, ctx->val32, ctx->err, mixed(ctx), ctx->stream);
    launch_ilu_reorg(d, (int64_t)ctx->hs.sp_fwd.src.size(), (int64_t)ctx->hs.sp_bwd.src.size(), ctx->pf.src,
                     ctx->pf.col, ctx->pb.src, ctx->pb.col, mixed(ctx), ctx->stream);
  }
  CK(cudaGetLastError());
  if (ctx->opt.coarse) {
    KTimer kt_(ctx, SEIRD_K_COARSE_SETUP);
    add_bytes(ctx, SEIRD_K_COARSE_SETUP, bytes_coarse_setup(ctx));
    const CoarseDev c = coarse_dev(ctx);
    launch_coarse_assemble(c, ctx->val, ctx->val32, ctx->stream);
    if (!ctx->coarse_graph) {
      // capture on a private stream (the caller's stream may be the legacy default stream,
      // which cannot be captured); the replays run on the context's stream
      cudaStream_t cs;
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      const int64_t k0 = launch_total();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        launch_coarse_factor(c, ctx->err, cs);
        e = cudaStreamEndCapture(cs, &g);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->coarse_graph, g, 0);
      if (g) cudaGraphDestroy(g);
      cudaStreamDestroy(cs);
      ctx->coarse_graph_kernels = launch_total() - k0;
      count_launches(-ctx->coarse_graph_kernels);  // captured, not run
      if (e != cudaSuccess) {
        ctx->coarse_graph = nullptr;
        return fail(ctx, SEIRD_ECUDA, std::string("coarse factorisation graph: ") + cudaGetErrorString(e));
      }
    }
    CK(cudaGraphLaunch(ctx->coarse_graph, ctx->stream));
    count_launches(ctx->coarse_graph_kernels);
    if (ctx->opt.coarse >= 2)  // (J Z) of this set-up: the residual update after the coarse correction
      launch_az_build((int64_t)ctx->hs.az_unit.size(), ctx->az_blk, ctx->val, ctx->val32, ctx->azval, ctx->azval32,
                      mixed(ctx), ctx->stream);
    CK(cudaGetLastError());
  }
  TRY(check_flags(ctx, "preconditioner setup"));
  ctx->pc_ready = true;
  ctx->pc_age_steps = 0;
  return SEIRD_OK;
}

int spmv32(seird_ctx* ctx, const float* x, double* y, const double* b = nullptr);
int spmv(seird_ctx* ctx, const double* x, double* y, const double* b = nullptr);

// z = M^{-1} r with FP32 subdomain factors and an FP32 result (mixed path)
int pc_apply32(seird_ctx* ctx, const double* r, float* z) {
  const int64_t len = vlen(ctx);
  if (ctx->opt.coarse == 3) {  // coarse correction, then RAS on the residual it leaves
    const CoarseDev cd = coarse_dev(ctx);
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_solve(ctx) + 80.0 * ctx->hs.n + bytes_az_sub(ctx, 4.0));
      launch_coarse_solve(cd, r, ctx->stream);
      launch_coarse_y32(cd, ctx->stream);
      CK(cudaMemcpyAsync(ctx->pct, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, ctx->stream));
      launch_az_sub(cd, ctx->hs.n, ctx->az_ptr, ctx->az_unit, ctx->azval, ctx->azval32, true, ctx->pct, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
      add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 4.0));
      launch_ilu_solve32(ras_dev(ctx), ctx->pct, z, ctx->err, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_prolong(ctx, 4.0));
      launch_coarse_prolong32(cd, ctx->hs.n, z, ctx->stream);
    }
    CK(cudaGetLastError());
    return SEIRD_OK;
  }
  {
    KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
    add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 4.0));
    launch_ilu_solve32(ras_dev(ctx), r, z, ctx->err, ctx->stream);
  }
  if (ctx->opt.coarse == 1) {
    KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
    add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_solve(ctx) + bytes_coarse_prolong(ctx, 4.0));
    const CoarseDev cd = coarse_dev(ctx);
    launch_coarse_solve(cd, r, ctx->stream);
    launch_coarse_y32(cd, ctx->stream);
    launch_coarse_prolong32(cd, ctx->hs.n, z, ctx->stream);
  } else if (ctx->opt.coarse == 2) {  // Eq. RAS_2L: coarse on r - J z, then RAS on the new residual
    TRY(spmv32(ctx, z, ctx->pct, r));  // r - J z
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY,
                bytes_coarse_solve(ctx) + bytes_coarse_prolong(ctx, 4.0) + bytes_az_sub(ctx, 4.0));
      const CoarseDev cd = coarse_dev(ctx);
      launch_coarse_solve(cd, ctx->pct, ctx->stream);
      launch_coarse_y32(cd, ctx->stream);
      launch_coarse_prolong32(cd, ctx->hs.n, z, ctx->stream);
      // r - J (z + Z y) = (r - J z) - (J Z) y, with J Z summed at set-up
      launch_az_sub(cd, ctx->hs.n, ctx->az_ptr, ctx->az_unit, ctx->azval, ctx->azval32, true, ctx->pct, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
      add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 4.0));
      launch_ilu_solve32(ras_dev(ctx), ctx->pct, ctx->pcu32, ctx->err, ctx->stream);
    }
    launch_add32(len, ctx->pcu32, z, ctx->stream);
  }
  CK(cudaGetLastError());
  return SEIRD_OK;
}

// z = M^{-1} r  (every node is owned by exactly one subdomain, so the RAS part
// writes every entry of z; the coarse part adds to it).  On the mixed path the
// FP32 result is widened into z.
int pc_apply(seird_ctx* ctx, const double* r, double* z) {
  if (mixed(ctx)) {
    TRY(pc_apply32(ctx, r, ctx->Z32));
    launch_f32_to_f64(vlen(ctx), ctx->Z32, z, ctx->stream);
    CK(cudaGetLastError());
    return SEIRD_OK;
  }
  if (ctx->opt.coarse == 3) {  // coarse correction, then RAS on the residual it leaves
    const int64_t len = vlen(ctx);
    const CoarseDev cd = coarse_dev(ctx);
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_solve(ctx) + 80.0 * ctx->hs.n + bytes_az_sub(ctx, 8.0));
      launch_coarse_solve(cd, r, ctx->stream);
      CK(cudaMemcpyAsync(ctx->pct, r, sizeof(double) * len, cudaMemcpyDeviceToDevice, ctx->stream));
      launch_az_sub(cd, ctx->hs.n, ctx->az_ptr, ctx->az_unit, ctx->azval, ctx->azval32, false, ctx->pct, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
      add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 8.0));
      launch_ilu_solve(ras_dev(ctx), ctx->pct, z, ctx->err, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_prolong(ctx, 8.0));
      launch_coarse_prolong<double>(cd, ctx->hs.n, z, ctx->stream);
    }
    CK(cudaGetLastError());
    return SEIRD_OK;
  }
  {
    KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
    add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 8.0));
    launch_ilu_solve(ras_dev(ctx), r, z, ctx->err, ctx->stream);
  }
  if (ctx->opt.coarse == 1) {
    KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
    add_bytes(ctx, SEIRD_K_COARSE_APPLY, bytes_coarse_solve(ctx) + bytes_coarse_prolong(ctx, 8.0));
    launch_coarse_apply_add<double>(coarse_dev(ctx), ctx->hs.n, r, z, ctx->stream);
  } else if (ctx->opt.coarse == 2) {  // Eq. RAS_2L: coarse on r - J z, then RAS on the new residual
    const int64_t len = vlen(ctx);
    TRY(spmv(ctx, z, ctx->pct, r));  // r - J z
    {
      KTimer kt_(ctx, SEIRD_K_COARSE_APPLY);
      add_bytes(ctx, SEIRD_K_COARSE_APPLY,
                bytes_coarse_solve(ctx) + bytes_coarse_prolong(ctx, 8.0) + bytes_az_sub(ctx, 8.0));
      const CoarseDev cd = coarse_dev(ctx);
      launch_coarse_apply_add<double>(cd, ctx->hs.n, ctx->pct, z, ctx->stream);
      // r - J (z + Z y) = (r - J z) - (J Z) y, with J Z summed at set-up
      launch_az_sub(cd, ctx->hs.n, ctx->az_ptr, ctx->az_unit, ctx->azval, ctx->azval32, false, ctx->pct, ctx->stream);
    }
    {
      KTimer kt_(ctx, SEIRD_K_ILU_SOLVE);
      add_bytes(ctx, SEIRD_K_ILU_SOLVE, bytes_ilu_solve(ctx, 8.0));
      launch_ilu_solve(ras_dev(ctx), ctx->pct, ctx->pcu, ctx->err, ctx->stream);
    }
    launch_axpby(len, 1.0, z, 1.0, ctx->pcu, z, ctx->stream);
  }
  CK(cudaGetLastError());
  return SEIRD_OK;
}

// y = J x, or y = b - J x when b != NULL
int spmv(seird_ctx* ctx, const double* x, double* y, const double* b) {
  KTimer kt_(ctx, SEIRD_K_SPMV);
  add_bytes(ctx, SEIRD_K_SPMV, bytes_spmv(ctx, 8.0, b != nullptr));
  if (mixed(ctx))
    launch_spmv<float>(ctx->hs.n, ctx->row_ptr, ctx->col, ctx->val32, x, y, ctx->stream, ctx->spmv_tb, b);
  else launch_spmv<double>(ctx->hs.n, ctx->row_ptr, ctx->col, ctx->val, x, y, ctx->stream, ctx->spmv_tb, b);
  CK(cudaGetLastError());
  return SEIRD_OK;
}

// y = J x (or b - J x) with the FP32 matrix copy and FP32 x (mixed path)
int spmv32(seird_ctx* ctx, const float* x, double* y, const double* b) {
  KTimer kt_(ctx, SEIRD_K_SPMV);
  add_bytes(ctx, SEIRD_K_SPMV, bytes_spmv(ctx, 4.0, b != nullptr));
  launch_spmv32(ctx->hs.n, ctx->row_ptr, ctx->col, ctx->val32, x, y, ctx->stream, ctx->spmv_tb, b);
  CK(cudaGetLastError());
  return SEIRD_OK;
}

int read_scalars(seird_ctx* ctx, int first, int count) {
  CK(cudaMemcpyAsync(ctx->h_scal + first, ctx->scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SEIRD_OK;
}

// read_scalars plus the device error word in the same synchronisation: a set flag
// (a subdomain solve that timed out, a singular pivot) ends the caller's loop at once
int read_scalars_checked(seird_ctx* ctx, int first, int count, const char* where) {
  CK(cudaMemcpyAsync(ctx->h_scal + first, ctx->scal + first, sizeof(double) * count, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_err, ctx->err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (*ctx->h_err) return check_flags(ctx, where);
  return SEIRD_OK;
}

int norm2(seird_ctx* ctx, const double* x, double* out) {
  launch_norm2(vlen(ctx), x, ctx->partial, ctx->red_grid, ctx->scal + 4, ctx->stream);
  CK(cudaGetLastError());
  TRY(read_scalars(ctx, 4, 1));
  *out = std::sqrt(std::max(ctx->h_scal[4], 0.0));
  return SEIRD_OK;
}

// Right-preconditioned restarted FGMRES (Z_j = M^{-1} V_j kept), CGS2, x0 = 0.
// Stops on ||r|| <= max(rtol ||b||, atol); dtol divergence and non-finite
// estimates are errors; hitting the iteration limit returns SEIRD_OK with
// *converged = false (Newton then takes the inexact step).
bool verbose();

// Largest stage of the solve plans in blocks (a stage has to fit the factor ring).
int64_t solve_max_stage_blocks(const seird_ctx* ctx) {
  return std::max<int64_t>(ctx->hs.sp_fwd.max_lev_blocks, ctx->hs.sp_bwd.max_lev_blocks);
}

// Launch-shape autotuner (options.autotune): times the candidates on the context's own
// vectors (V[0] holds the first Krylov vector; the Gram-Schmidt candidates run at depth 8
// with V[1..7] set to copies of it, which GMRES overwrites later) and keeps the fastest.
int autotune(seird_ctx* ctx) {
  ctx->tuned = true;
  const int64_t len = vlen(ctx);
  const cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto best_of = [&](auto&& launch) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      launch();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  float tbest = 1e30f;
  int best_ch = 0;
  for (int tb : {128, 256, 512}) {
    const float t = best_of([&] {
      if (mixed(ctx)) launch_spmv32(ctx->hs.n, ctx->row_ptr, ctx->col, ctx->val32, ctx->Z32, ctx->tune_buf, s, tb);
      else launch_spmv<double>(ctx->hs.n, ctx->row_ptr, ctx->col, ctx->val, ctx->V, ctx->tune_buf, s, tb);
    });
    if (t < tbest) {
      tbest = t;
      ctx->spmv_tb = tb;
    }
  }
  const int nv = 8;
  for (int k = 1; k < nv; ++k)
    CK(cudaMemcpyAsync(ctx->V + (int64_t)k * len, ctx->V, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(ctx->tune_buf, ctx->V, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  tbest = 1e30f;
  for (int per_sm : {2, 3, 4, 6}) {
    const int grid = per_sm * ctx->sms;
    for (int tile : {128, 256}) {
      const float t = best_of([&] {
        launch_mdot(len, nv, ctx->V, len, ctx->tune_buf, ctx->partial, grid, ctx->hcol, s, tile);
        launch_update_norm(len, nv, ctx->V, len, ctx->hcol, ctx->tune_buf, ctx->partial, grid, ctx->scal + 7, s);
      });
      if (t < tbest) {
        tbest = t;
        ctx->red_grid = grid;
        ctx->cgs_tile = tile;
      }
    }
  }
  // subdomain solves: the dependency-load batch and the consumer warps per CTA, on the
  // context's own factors with V[0] as the right-hand side (every choice forms the same
  // sums; only the time differs)
  if (ctx->pc_ready) {
    tbest = 1e30f;
    const int keep_ch = ctx->ilu_ch, keep_w = ctx->ilu_warps, keep_r = ctx->ilu_ring;
    int best_w = 0, best_r = 0;
    const bool half_ok = solve_max_stage_blocks(ctx) <= SOLVE_RING_HALF;
    for (int ring : {SOLVE_RING_FULL, SOLVE_RING_HALF}) {
      if (ring == SOLVE_RING_HALF && !half_ok) continue;
      for (int nw : {7, 3}) {
        for (int ch : {1, 2, 3, 4}) {
          ctx->ilu_ch = ch;
          ctx->ilu_warps = nw;
          ctx->ilu_ring = ring;
          const RasDev d = ras_dev(ctx);
          const float t = best_of([&] {
            if (mixed(ctx)) launch_ilu_solve32(d, ctx->V, reinterpret_cast<float*>(ctx->tune_buf), ctx->err, s);
            else launch_ilu_solve(d, ctx->V, ctx->tune_buf, ctx->err, s);
          });
          if (t < tbest) {
            tbest = t;
            best_ch = ch;
            best_w = nw;
            best_r = ring;
          }
        }
      }
    }
    ctx->ilu_ch = best_ch > 0 ? best_ch : keep_ch;
    ctx->ilu_warps = best_w > 0 ? best_w : keep_w;
    ctx->ilu_ring = best_r > 0 ? best_r : keep_r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  if (verbose())
    std::fprintf(stderr, "[seird] autotune: spmv %d threads, gram-schmidt %d CTAs, tile %d, ilu batch %d warps %d "
                 "ring %d\n", ctx->spmv_tb, ctx->red_grid, ctx->cgs_tile, ctx->ilu_ch, ctx->ilu_warps, ctx->ilu_ring);
  return SEIRD_OK;
}

// Arnoldi iteration j of the FGMRES cycle: z_j = M^{-1} v_j, w = J z_j, Gram-Schmidt of w
// against v_0..v_j, Givens update of H and g, v_{j+1} = w / ||w||.  Device work only, so
// that a restart cycle can be captured into a CUDA graph.
static int arnoldi_iteration(seird_ctx* ctx, int j, const CycleCtl& cc) {
  const int64_t len = vlen(ctx);
  const int ldh = ctx->opt.gmres_restart + 1;
  const cudaStream_t s = ctx->stream;
  double* h1 = ctx->hcol;
  double* h2 = ctx->hcol + NV_STRIDE;
  double* Vj = ctx->V + (int64_t)j * len;
  if (mixed(ctx)) {  // FP32 preconditioner and operator inside the FP64 FGMRES
    float* Zj = ctx->Z32 + (int64_t)j * len;
    TRY(pc_apply32(ctx, Vj, Zj));
    TRY(spmv32(ctx, Zj, ctx->w));
  } else {
    double* Zj = ctx->Z + (int64_t)j * len;
    TRY(pc_apply(ctx, Vj, Zj));
    TRY(spmv(ctx, Zj, ctx->w));
  }
  KTimer kt_(ctx, SEIRD_K_KRYLOV);
  add_bytes(ctx, SEIRD_K_KRYLOV, bytes_arnoldi(ctx, j + 1));
  launch_mdot(len, j + 1, ctx->V, len, ctx->w, ctx->partial, ctx->red_grid, h1, s, ctx->cgs_tile);
  if (ctx->opt.gmres_one_pass == 1) {
    launch_update_norm(len, j + 1, ctx->V, len, h1, ctx->w, ctx->partial, ctx->red_grid, ctx->scal + 5, s);
  } else {
    launch_update_mdot(len, j + 1, ctx->V, len, h1, ctx->w, ctx->partial, ctx->red_grid, nullptr, s,
                       ctx->cgs_tile);
    launch_reduce_cols(ctx->red_grid, j + 1, ctx->partial, h2, 0, s);
    launch_update_norm(len, j + 1, ctx->V, len, h2, ctx->w, ctx->partial, ctx->red_grid, ctx->scal + 5, s);
  }
  launch_givens(j, ctx->gm, h1, h2, ctx->scal + 5, ldh, ctx->scal + 2, s, cc);
  launch_scale(len, ctx->w, ctx->scal + 3, 1, ctx->V + (int64_t)(j + 1) * len, s);
  CK(cudaGetLastError());
  return SEIRD_OK;
}

// Captures one restart cycle (options.graph) as nested conditional IF nodes: the body
// of node j holds Arnoldi iteration j followed by node j + 1, whose condition the Givens
// kernel of iteration j sets (k_givens).  Node 0's condition defaults to 1 at every
// launch.  A replay thus runs iterations until convergence, dtol or the cycle's limit
// (ctl[1]) with no host round trip, and once a condition is 0 the rest of the cycle is
// skipped as a whole.  The graph bakes in the Krylov, preconditioner and matrix buffers
// and the launch shapes, which are fixed once the autotuner has run.
static int build_cycle_graph(seird_ctx* ctx) {
  const int m = ctx->opt.gmres_restart;
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle hnd = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hnd, g, 1u, cudaGraphCondAssignDefault);
  const cudaStream_t saved_stream = ctx->stream;
  ctx->stream = cs;  // the launchers capture on the context's stream
  int rc = SEIRD_OK;
  std::vector<int64_t> launches(1, 0);
  double saved[SEIRD_K_COUNT];
  for (int c = 0; c < SEIRD_K_COUNT; ++c) saved[c] = ctx->abytes[c];
  std::vector<double> cbytes((size_t)(m + 1) * SEIRD_K_COUNT, 0.0);
  cudaGraph_t parent = g;
  cudaGraphNode_t dep = nullptr;  // node j's predecessor inside its parent
  for (int j = 0; j < m && e == cudaSuccess && rc == SEIRD_OK; ++j) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, parent, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &np);
    if (e != cudaSuccess) break;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CycleCtl cc;
    cc.ctl = ctx->cyc_ctl;
    cc.tol = ctx->scal + 10;
    cc.has_next = j + 1 < m;
    if (cc.has_next) {  // the next node's condition, set by this iteration's Givens kernel
      e = cudaGraphConditionalHandleCreate(&cc.next, body, 0u, 0);
      if (e != cudaSuccess) break;
    }
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) break;
    const int64_t k0 = launch_total();
    rc = arnoldi_iteration(ctx, j, cc);
    launches.push_back(launches.back() + launch_total() - k0);
    count_launches(k0 - launch_total());  // captured, not run
    for (int c = 0; c < SEIRD_K_COUNT; ++c) cbytes[(size_t)(j + 1) * SEIRD_K_COUNT + c] = ctx->abytes[c] - saved[c];
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* last = nullptr;
    size_t nlast = 0;
    e = cudaStreamGetCaptureInfo(cs, &st, nullptr, nullptr, &last, nullptr, &nlast);
    dep = (e == cudaSuccess && nlast == 1) ? last[0] : nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &body);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && !dep) e = cudaErrorStreamCaptureUnjoined;  // the capture must end in one node
    parent = body;
    hnd = cc.next;
  }
  ctx->stream = saved_stream;
  for (int c = 0; c < SEIRD_K_COUNT; ++c) ctx->abytes[c] = saved[c];  // counted per replay instead
  if (e == cudaSuccess && rc == SEIRD_OK) e = cudaGraphInstantiate(&ctx->cycle_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (rc) return rc;
  if (e != cudaSuccess) {
    ctx->cycle_exec = nullptr;
    cudaGetLastError();
    return fail(ctx, SEIRD_ECUDA, std::string("gmres: capture of the restart cycle failed: ") +
                                       cudaGetErrorString(e));
  }
  ctx->cycle_m = m;
  ctx->cycle_launches = launches;
  ctx->cycle_bytes = cbytes;
  return SEIRD_OK;
}

int gmres(seird_ctx* ctx, const double* b, double* x, double rtol, int* its_out, bool* converged) {
  Range rg_("seird gmres");
  const int64_t len = vlen(ctx);
  const int m = ctx->opt.gmres_restart;
  const int ldh = m + 1;
  const cudaStream_t s = ctx->stream;
  double* h2 = ctx->hcol + NV_STRIDE;
  *its_out = 0;
  *converged = false;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * len, s));
  double bnorm;
  TRY(norm2(ctx, b, &bnorm));
  if (!std::isfinite(bnorm)) return fail(ctx, SEIRD_ENONFINITE, "gmres: non-finite right-hand side");
  if (bnorm == 0.0) {
    *converged = true;
    return SEIRD_OK;
  }
  const double tol = std::max(rtol * bnorm, ctx->opt.gmres_atol);
  const double* r = b;
  double rnorm = bnorm;
  int its = 0;
  std::vector<double> g0(ldh, 0.0);
  double* gbuf = ctx->gm + (int64_t)ldh * m + 2 * m;  // g inside the GMRES small state
  if (ctx->opt.gmres_one_pass == 1)
    CK(cudaMemsetAsync(h2, 0, sizeof(double) * NV_STRIDE, s));  // no second-pass coefficients
  // captured cycles: not under per-kernel timing (events cannot sit in conditional bodies)
  // nor while the adjoint has J^T swapped in
  const bool graph = ctx->opt.graph == 1 && !ctx->opt.timing && !ctx->eager_cycles;
  if (graph) {  // the cycle's tolerances, read by k_givens
    ctx->h_scal[10] = tol;
    ctx->h_scal[11] = ctx->opt.gmres_dtol * bnorm;
    CK(cudaMemcpyAsync(ctx->scal + 10, ctx->h_scal + 10, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  while (true) {
    launch_axpby(len, 1.0 / rnorm, r, 0.0, r, ctx->V, s);
    if (ctx->opt.autotune && !ctx->tuned) TRY(autotune(ctx));
    g0.assign(ldh, 0.0);
    g0[0] = rnorm;
    CK(cudaMemcpyAsync(gbuf, g0.data(), sizeof(double) * ldh, cudaMemcpyHostToDevice, s));
    int k = 0;
    bool done = false;
    if (graph) {
      if (!ctx->cycle_exec || ctx->cycle_m != m) TRY(build_cycle_graph(ctx));
      int* hin = ctx->h_cyc;
      int* hout = ctx->h_cyc + 4;
      hin[0] = 0;
      hin[1] = std::min(m, ctx->opt.gmres_maxit - its);
      hin[2] = 0;
      hin[3] = 0;
      CK(cudaMemcpyAsync(ctx->cyc_ctl, hin, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
      CK(cudaGraphLaunch(ctx->cycle_exec, s));
      CK(cudaMemcpyAsync(hout, ctx->cyc_ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(read_scalars_checked(ctx, 2, 2, "gmres"));
      k = hout[0];
      its += k;
      if (k < 1 || k > m) return fail(ctx, SEIRD_ECUDA, "gmres: captured cycle reported no iterations");
      count_launches(ctx->cycle_launches[k]);
      for (int c = 0; c < SEIRD_K_COUNT; ++c) ctx->abytes[c] += ctx->cycle_bytes[(size_t)k * SEIRD_K_COUNT + c];
      if (hout[2] == 2) {
        if (!std::isfinite(ctx->h_scal[2])) return fail(ctx, SEIRD_ENONFINITE, "gmres: non-finite residual estimate");
        return fail(ctx, SEIRD_EGMRES, "gmres: diverged (dtol)");
      }
      done = hout[2] == 1;
    } else {
      for (int j = 0; j < m; ++j) {
        TRY(arnoldi_iteration(ctx, j, CycleCtl()));
        TRY(read_scalars_checked(ctx, 2, 2, "gmres"));
        ++its;
        k = j + 1;
        const double res = ctx->h_scal[2], hn = ctx->h_scal[3];
        if (!std::isfinite(res)) return fail(ctx, SEIRD_ENONFINITE, "gmres: non-finite residual estimate");
        if (res > ctx->opt.gmres_dtol * bnorm) return fail(ctx, SEIRD_EGMRES, "gmres: diverged (dtol)");
        if (res <= tol || hn == 0.0) {
          done = true;
          break;
        }
        if (its >= ctx->opt.gmres_maxit) break;
      }
    }
    {
      KTimer kt_(ctx, SEIRD_K_KRYLOV);
      // x += Z y: k preconditioned vectors read, x read and written
      add_bytes(ctx, SEIRD_K_KRYLOV, (5.0 * k * wv(ctx) + 80.0) * ctx->hs.n);
      launch_hsolve(k, ctx->gm, ldh, s);
      if (mixed(ctx)) launch_multi_axpy32(len, k, ctx->Z32, len, gbuf + ldh, x, s);
      else launch_multi_axpy(len, k, ctx->Z, len, gbuf + ldh, x, s);  // y lives right after g
    }
    CK(cudaGetLastError());
    if (done) {
      *converged = true;
      break;
    }
    if (its >= ctx->opt.gmres_maxit) break;
    // restart from the residual r = b - J x of the operator GMRES works with
    TRY(spmv(ctx, x, ctx->w, b));
    TRY(norm2(ctx, ctx->w, &rnorm));
    if (!std::isfinite(rnorm)) return fail(ctx, SEIRD_ENONFINITE, "gmres: non-finite restart residual");
    if (rnorm <= tol) {
      *converged = true;
      break;
    }
    r = ctx->w;
  }
  *its_out = its;
  // a subdomain solve whose bounded wait gave up (or a singular pivot) fails the solve here
  return check_flags(ctx, "gmres");
}

bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("SEIRD_VERBOSE");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v == 1;
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// One step by the coupled Picard iteration of Eq. weak_vec_implicit, written in
// correction form: the Picard matrix P(U^k) satisfies P(U^k) U^k - M U^n =
// F(U^k), so U^{k+1} = U^k + dU with P(U^k) dU = -F(U^k) solves
// P(U^k) U^{k+1} = M U^n.  Full steps, no line search; stops on the update
// measure of Eq. picardtol (picard_tol > 0) or on the residual test.
int picard_step(seird_ctx* ctx, seird_stats* st) {
  using clk = std::chrono::steady_clock;
  const auto t_begin = clk::now();
  const int64_t len = vlen(ctx);
  const cudaStream_t s = ctx->stream;
  seird_stats S;
  std::memset(&S, 0, sizeof(S));
  timing_reset(ctx);
  CK(cudaMemcpyAsync(ctx->Un, ctx->U, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  auto t0 = clk::now();
  double f;
  int rc = residual(ctx, ctx->U, ctx->Un, ctx->F, &f);
  S.ms_assemble += ms_since(t0);
  if (rc) return rc;
  const double f0 = f;
  S.res0 = f0;
  double unorm;
  TRY(norm2(ctx, ctx->Un, &unorm));
  auto restore = [&](int code) {
    cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    return code;
  };
  const double ptol = ctx->opt.picard_tol;
  int its = 0;
  double eps = 0.0;
  for (;;) {
    const bool done = ptol > 0 ? (its > 0 && eps <= ptol) : (f <= ctx->opt.newton_rtol * f0 + ctx->opt.newton_atol);
    if (done) break;
    if (its >= ctx->opt.newton_maxit) return restore(fail(ctx, SEIRD_ENEWTON_MAXIT, "picard: iteration limit"));
    t0 = clk::now();
    rc = jacobian(ctx, ctx->U, true);
    if (rc) return restore(rc);
    CK(cudaStreamSynchronize(s));
    S.ms_assemble += ms_since(t0);
    if (its % std::max(1, ctx->opt.pc_lag) == 0 || !ctx->pc_ready) {
      t0 = clk::now();
      rc = pc_setup(ctx);
      S.ms_setup += ms_since(t0);
      if (rc) return restore(rc);
      S.pc_setups++;
    }
    launch_axpby(len, -1.0, ctx->F, 0.0, ctx->F, ctx->stage, s);
    t0 = clk::now();
    int lits = 0;
    bool conv = false;
    rc = gmres(ctx, ctx->stage, ctx->dU, ctx->opt.gmres_rtol, &lits, &conv);
    S.ms_solve += ms_since(t0);
    S.gmres_its += lits;
    if (rc) return restore(rc);
    t0 = clk::now();
    launch_axpby(len, 1.0, ctx->U, 1.0, ctx->dU, ctx->Ut, s);
    double ft;
    rc = residual(ctx, ctx->Ut, ctx->Un, ctx->Ft, &ft);
    S.ms_assemble += ms_since(t0);
    if (rc) return restore(rc);
    double dn;
    TRY(norm2(ctx, ctx->dU, &dn));
    eps = unorm > 0 ? dn / unorm : 0.0;
    S.eps_update = eps;
    if (verbose())
      std::fprintf(stderr, "[seird] t=%g picard %d |F| %.6e -> %.6e (f0 %.6e) gmres %d eps %.3e\n", ctx->t, its, f,
                   ft, f0, lits, eps);
    std::swap(ctx->U, ctx->Ut);
    std::swap(ctx->F, ctx->Ft);
    f = ft;
    ++its;
  }
  S.newton_its = its;
  S.res_final = f;
  ctx->t += ctx->opt.dt;
  S.ms_total = ms_since(t_begin);
  timing_collect(ctx, &S);
  if (st) *st = S;
  return SEIRD_OK;
}

int newton_step(seird_ctx* ctx, seird_stats* st) {
  Range rg_("seird step");
  if (ctx->opt.nonlinear == 1) return picard_step(ctx, st);
  using clk = std::chrono::steady_clock;
  const auto t_begin = clk::now();
  const int64_t len = vlen(ctx);
  const cudaStream_t s = ctx->stream;
  seird_stats S;
  std::memset(&S, 0, sizeof(S));
  timing_reset(ctx);
  CK(cudaMemcpyAsync(ctx->Un, ctx->U, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  auto t0 = clk::now();
  double f;
  int rc = SEIRD_OK;
  if (ctx->have_prev && ctx->Flast && !ctx->sched_on) {
    // F(u^n; u^n) = F(u^n; u^{n-1}) - M (u^n - u^{n-1}): the previous step's last residual
    // minus a mass product (same rates, same dt), instead of a full assembly
    launch_axpby(len, 1.0, ctx->Un, -1.0, ctx->Uprev, ctx->Ut, s);
    launch_mass(ctx->hs.n, ctx->hs.m, ctx->tri, ctx->xy, ctx->Ut, ctx->elem, ctx->node_inc_ptr, ctx->node_inc,
                ctx->F, ctx->partial, ctx->scal + 6, s);
    launch_axpby(len, 1.0, ctx->Flast, -1.0, ctx->F, ctx->F, s);
    CK(cudaGetLastError());
    TRY(norm2(ctx, ctx->F, &f));
  } else {
    rc = residual(ctx, ctx->U, ctx->Un, ctx->F, &f);
  }
  S.ms_assemble += ms_since(t0);
  if (rc) return rc;
  const double f0 = f;  // the stopping test is relative to ||F(u^n)||
  S.res0 = f0;
  if (ctx->opt.predictor >= 1 && ctx->have_prev && ctx->Uprev) {
    // first iterate: the polynomial through u^n and the earlier states held (up to
    // options.predictor of them) evaluated one step ahead: sum_k (-1)^k C(p+1, k+1) u^{n-k},
    // e.g. 2 u^n - u^{n-1} or 4 u^n - 6 u^{n-1} + 4 u^{n-2} - u^{n-3}; kept only if it is
    // admissible and lowers ||F||
    t0 = clk::now();
    const int deg = std::max(1, std::min<int>(ctx->opt.predictor, ctx->hist_depth));
    // coefficient of u^{n-k} in the degree-deg extrapolation: (-1)^k C(deg+1, k+1)
    auto coef = [deg](int k) {
      double c = 1.0;
      for (int i = 0; i < k + 1; ++i) c = c * (deg + 1 - i) / (i + 1);
      return (k % 2 ? -1.0 : 1.0) * c;
    };
    launch_axpby(len, coef(0), ctx->Un, coef(1), ctx->Uhist[0], ctx->Ut, s);
    for (int k = 2; k <= deg; ++k) launch_axpby(len, 1.0, ctx->Ut, coef(k), ctx->Uhist[k - 1], ctx->Ut, s);
    double fp = 0.0;
    rc = residual(ctx, ctx->Ut, ctx->Un, ctx->Ft, &fp);
    S.ms_assemble += ms_since(t0);
    if (rc == SEIRD_OK && fp < f) {
      std::swap(ctx->U, ctx->Ut);
      std::swap(ctx->F, ctx->Ft);
      f = fp;
    } else if (rc != SEIRD_OK && rc != SEIRD_ENONFINITE) {
      return rc;
    }
  }
  double unorm;
  TRY(norm2(ctx, ctx->Un, &unorm));
  int its = 0;
  double eta = ctx->opt.gmres_rtol, f_prev = f;
  auto restore = [&](int code) {
    cudaMemcpyAsync(ctx->U, ctx->Un, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    return code;
  };
  while (!(f <= ctx->opt.newton_rtol * f0 + ctx->opt.newton_atol)) {
    if (its >= ctx->opt.newton_maxit) return restore(fail(ctx, SEIRD_ENEWTON_MAXIT, "newton: iteration limit"));
    t0 = clk::now();
    rc = jacobian(ctx, ctx->U);
    if (rc) return restore(rc);
    CK(cudaStreamSynchronize(s));
    S.ms_assemble += ms_since(t0);
    const bool rebuild = !ctx->pc_ready || (its == 0 ? ctx->pc_age_steps > ctx->opt.pc_keep_steps
                                                     : its % std::max(1, ctx->opt.pc_lag) == 0);
    if (rebuild) {
      t0 = clk::now();
      rc = pc_setup(ctx);
      S.ms_setup += ms_since(t0);
      if (rc) return restore(rc);
      S.pc_setups++;
    }
    // J dU = -F
    launch_axpby(len, -1.0, ctx->F, 0.0, ctx->F, ctx->stage, s);
    if (ctx->opt.gmres_forcing == 1) {
      // Eisenstat-Walker choice 2 with the usual safeguard, capped at 0.5, and
      // no tighter than what brings ||F|| to the Newton target
      const double first = ctx->opt.forcing_first > 0.0 ? ctx->opt.forcing_first : 0.1;
      double e = its == 0 ? first : 0.9 * (f / f_prev) * (f / f_prev);
      if (its > 0 && 0.9 * eta * eta > 0.1) e = std::max(e, 0.9 * eta * eta);
      // near the Newton target, solve just far enough to finish in this iteration
      const double tgt = (ctx->opt.newton_rtol * f0 + ctx->opt.newton_atol) / f;
      if (e < 10.0 * tgt) e = 0.2 * tgt;
      e = std::max(e, 0.2 * tgt);
      eta = std::min(std::max(e, 1e-14), 0.5);
    } else {
      eta = ctx->opt.gmres_rtol;
    }
    f_prev = f;
    t0 = clk::now();
    int lits = 0;
    bool conv = false;
    rc = gmres(ctx, ctx->stage, ctx->dU, eta, &lits, &conv);
    S.ms_solve += ms_since(t0);
    S.gmres_its += lits;
    if (rc) return restore(rc);
    if (!conv && !rebuild) {  // the carried-over preconditioner fell short: rebuild it and solve again
      t0 = clk::now();
      rc = pc_setup(ctx);
      S.ms_setup += ms_since(t0);
      if (rc) return restore(rc);
      S.pc_setups++;
      t0 = clk::now();
      rc = gmres(ctx, ctx->stage, ctx->dU, eta, &lits, &conv);
      S.ms_solve += ms_since(t0);
      S.gmres_its += lits;
      if (rc) return restore(rc);
    }
    double lam = 1.0, ft = 0.0;
    t0 = clk::now();
    for (int ls = 0;; ++ls) {
      launch_axpby(len, 1.0, ctx->U, lam, ctx->dU, ctx->Ut, s);
      rc = residual(ctx, ctx->Ut, ctx->Un, ctx->Ft, &ft);
      if (rc == SEIRD_ENONFINITE && ls < ctx->opt.ls_maxit) {  // N <= 0 on the trial point: shorten the step
        lam *= 0.5;
        S.ls_halvings++;
        continue;
      }
      if (rc) return restore(rc);
      if (ft <= (1.0 - 1e-4 * lam) * f || ls >= ctx->opt.ls_maxit) break;
      lam *= 0.5;
      S.ls_halvings++;
    }
    S.ms_assemble += ms_since(t0);
    double dn;
    TRY(norm2(ctx, ctx->dU, &dn));
    S.eps_update = unorm > 0 ? lam * dn / unorm : 0.0;
    if (verbose())
      std::fprintf(stderr, "[seird] t=%g newton %d |F| %.6e -> %.6e (f0 %.6e) gmres %d (eta %.2e) conv %d lambda %g |dU| %.3e\n",
                   ctx->t, its, f, ft, f0, lits, eta, (int)conv, lam, dn);
    std::swap(ctx->U, ctx->Ut);
    std::swap(ctx->F, ctx->Ft);
    f = ft;
    ++its;
  }
  S.newton_its = its;
  S.res_final = f;
  ctx->t += ctx->opt.dt;
  ctx->pc_age_steps++;
  if (ctx->Uprev) {
    // the held states move one step back by rotating the buffers (u^{n-k} -> u^{n-k-1}, the oldest
    // buffer is reused for u^n -> u^{n-1}): one copy per step whatever the degree
    const int depth = ctx->have_prev ? ctx->hist_depth : 0;
    const int nh = ctx->n_hist;
    double* recycled = ctx->Uhist[nh - 1];
    for (int k = nh - 1; k > 0; --k) ctx->Uhist[k] = ctx->Uhist[k - 1];
    ctx->Uhist[0] = recycled;
    ctx->Uprev = recycled;
    ctx->hist_depth = std::min(depth + 1, std::max(1, (int)ctx->opt.predictor));
    CK(cudaMemcpyAsync(ctx->Uprev, ctx->Un, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ctx->Flast, ctx->F, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    ctx->have_prev = true;
  }
  S.ms_total = ms_since(t_begin);
  timing_collect(ctx, &S);
  if (st) *st = S;
  return SEIRD_OK;
}

// caller-numbered input -> internal vector dst
int to_internal(seird_ctx* ctx, const double* src, int on_device, double* dst) {
  const int64_t len = vlen(ctx);
  const double* dsrc = src;
  if (!on_device) {
    CK(cudaMemcpyAsync(ctx->stage, src, sizeof(double) * len, cudaMemcpyHostToDevice, ctx->stream));
    dsrc = ctx->stage;
  }
  launch_gather5(ctx->hs.n, ctx->perm, dsrc, dst, ctx->stream);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));  // stage is reused by the next call
  return SEIRD_OK;
}

int from_internal(seird_ctx* ctx, const double* src, double* dst, int on_device) {
  const int64_t len = vlen(ctx);
  if (on_device) {
    launch_scatter5(ctx->hs.n, ctx->perm, src, dst, ctx->stream);
    CK(cudaGetLastError());
    return SEIRD_OK;
  }
  launch_scatter5(ctx->hs.n, ctx->perm, src, ctx->stage, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(dst, ctx->stage, sizeof(double) * len, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return SEIRD_OK;
}

// Device buffers owned by one adjoint call (freed on every return path).
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  int get(seird_ctx* ctx, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(count, 1));
    if (e != cudaSuccess) return fail(ctx, SEIRD_ENOMEM, std::string("adjoint: cudaMalloc: ") + cudaGetErrorString(e));
    ptrs.push_back(*p);
    return SEIRD_OK;
  }
};

int adjoint_impl(seird_ctx* ctx, const seird_misfit* sp, double* jout, double* grad, double* gfield) {
  const HostSetup& hs = ctx->hs;
  const int64_t n = hs.n, len = 5 * n, nnzb = (int64_t)hs.col.size();
  const int N = sp->n_steps, C = sp->checkpoint_every;
  if (ctx->opt.precision != 0) return fail(ctx, SEIRD_EINVAL, "adjoint: FP64 contexts only");
  if (N < 1 || C < 1 || sp->n_obs_nodes < 1 || sp->n_obs_steps < 1 || !sp->obs_nodes || !sp->obs_steps ||
      !sp->I_hat || !sp->D_hat)
    return fail(ctx, SEIRD_EINVAL, "adjoint: bad misfit specification");
  std::vector<int32_t> obs_of_step(N + 1, -1);
  for (int r = 0; r < sp->n_obs_steps; ++r) {
    const int k = sp->obs_steps[r];
    if (k < 1 || k > N || (r > 0 && k <= sp->obs_steps[r - 1]))
      return fail(ctx, SEIRD_EINVAL, "adjoint: obs_steps must increase within 1..n_steps");
    obs_of_step[k] = r;
  }
  std::vector<int32_t> nodes(sp->n_obs_nodes);
  std::vector<char> seen(n, 0);
  for (int q = 0; q < sp->n_obs_nodes; ++q) {
    const int32_t i = sp->obs_nodes[q];
    if (i < 0 || i >= n || seen[i]) return fail(ctx, SEIRD_EINVAL, "adjoint: obs_nodes out of range or repeated");
    seen[i] = 1;
    nodes[q] = hs.iperm[i];
  }
  const double rtol = sp->lin_rtol > 0 ? sp->lin_rtol : 1e-10;
  const cudaStream_t s = ctx->stream;
  const int nseg = (N + C - 1) / C;
  Scratch S;
  double *ckpt, *seg, *lam, *lam_next, *rhs, *valT, *Ihat, *Dhat, *gacc, *gf, *jacc;
  int32_t* dnodes;
  TRY(S.get(ctx, &ckpt, (size_t)(nseg + 1) * len));
  TRY(S.get(ctx, &seg, (size_t)(C + 1) * len));
  TRY(S.get(ctx, &lam, len));
  TRY(S.get(ctx, &lam_next, len));
  TRY(S.get(ctx, &rhs, len));
  TRY(S.get(ctx, &valT, 25 * nnzb));
  TRY(S.get(ctx, &Ihat, (size_t)sp->n_obs_steps * sp->n_obs_nodes));
  TRY(S.get(ctx, &Dhat, (size_t)sp->n_obs_steps * sp->n_obs_nodes));
  const int B = ctx->n_samples;
  TRY(S.get(ctx, &gacc, 16 * (size_t)B));
  TRY(S.get(ctx, &gf, n));
  TRY(S.get(ctx, &jacc, 2));
  TRY(S.get(ctx, &dnodes, sp->n_obs_nodes));
  const size_t nobs_all = (size_t)sp->n_obs_steps * sp->n_obs_nodes;
  CK(cudaMemcpyAsync(Ihat, sp->I_hat, sizeof(double) * nobs_all, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Dhat, sp->D_hat, sizeof(double) * nobs_all, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dnodes, nodes.data(), sizeof(int32_t) * nodes.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(gacc, 0, sizeof(double) * 16 * B, s));
  CK(cudaMemsetAsync(gf, 0, sizeof(double) * n, s));
  CK(cudaMemsetAsync(jacc, 0, sizeof(double) * 2, s));
  CK(cudaMemsetAsync(lam_next, 0, sizeof(double) * len, s));
  const double t0 = ctx->t;
  CK(cudaMemcpyAsync(ckpt, ctx->U, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
  // every step of the run and of its recomputation builds its own preconditioner, so the
  // recomputed states are the forward ones bit for bit
  const int32_t keep = ctx->opt.pc_keep_steps, pred = ctx->opt.predictor;
  ctx->opt.pc_keep_steps = 0;
  ctx->opt.predictor = 0;
  auto restore = [&](int code) {
    cudaMemcpyAsync(ctx->U, ckpt, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    ctx->t = t0;
    ctx->opt.pc_keep_steps = keep;
    ctx->opt.predictor = pred;
    ctx->have_prev = false;
    return code;
  };
  const int nobs = sp->n_obs_nodes;
  // forward run: checkpoints and misfit
  for (int k = 1; k <= N; ++k) {
    ctx->have_prev = false;  // no step history: every step starts from its own u^n
    int rc = newton_step(ctx, nullptr);
    if (rc) return restore(rc);
    if (k % C == 0) CK(cudaMemcpyAsync(ckpt + (size_t)(k / C) * len, ctx->U, sizeof(double) * len,
                                       cudaMemcpyDeviceToDevice, s));
    if (obs_of_step[k] >= 0) {
      const int r = obs_of_step[k];
      launch_misfit(nobs, dnodes, Ihat + (size_t)r * nobs, Dhat + (size_t)r * nobs, ctx->U, nullptr, jacc, s);
    }
  }
  // reverse sweep, segment by segment from the checkpoints; the contraction
  // kernel's per-CTA partial sums use the red_grid x NV_STRIDE partial buffer
  const int grid = ctx->red_grid;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int k0 = sgi * C, k1 = std::min(N, (sgi + 1) * C);
    CK(cudaMemcpyAsync(ctx->U, ckpt + (size_t)sgi * len, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(seg, ctx->U, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    for (int k = k0 + 1; k <= k1; ++k) {
      ctx->have_prev = false;
      int rc = newton_step(ctx, nullptr);
      if (rc) return restore(rc);
      CK(cudaMemcpyAsync(seg + (size_t)(k - k0) * len, ctx->U, sizeof(double) * len, cudaMemcpyDeviceToDevice, s));
    }
    for (int k = k1; k > k0; --k) {
      const double* Uk = seg + (size_t)(k - k0) * len;
      // rhs = M lambda_{k+1} - dj/du^k
      launch_mass(n, hs.m, ctx->tri, ctx->xy, lam_next, ctx->elem, ctx->node_inc_ptr, ctx->node_inc, rhs,
                  ctx->partial, ctx->scal + 6, s);
      if (obs_of_step[k] >= 0) {
        const int r = obs_of_step[k];
        launch_misfit(nobs, dnodes, Ihat + (size_t)r * nobs, Dhat + (size_t)r * nobs, Uk, rhs, jacc + 1, s);
      }
      // J_k^T lambda_k = rhs with the step's FGMRES and a preconditioner built from J_k^T
      int rc = jacobian(ctx, Uk);
      if (rc) return restore(rc);
      launch_bsr_transpose(nnzb, ctx->tpos, ctx->val, valT, s);
      std::swap(ctx->val, valT);
      ctx->eager_cycles = true;  // a captured cycle holds the pointer of J, not of J^T
      rc = pc_setup(ctx);
      int lits = 0;
      bool conv = false;
      if (!rc) rc = gmres(ctx, rhs, lam, rtol, &lits, &conv);
      ctx->eager_cycles = false;
      std::swap(ctx->val, valT);
      ctx->pc_ready = false;  // the factors belong to J^T
      if (rc) return restore(rc);
      if (!conv) return restore(fail(ctx, SEIRD_EGMRES, "adjoint: transposed solve did not converge"));
      if (B == 1) {
        launch_param_contract(n, hs.m, ctx->tri, ctx->xy, Uk, lam, ctx->bfield, make_rates(ctx),
                              ctx->opt.quadrature, ctx->partial, grid, NV_STRIDE, ctx->elem, ctx->node_inc_ptr,
                              ctx->node_inc, gf, s);
        launch_reduce_cols(grid, 10, ctx->partial, gacc, 1, s);
      } else {  // an ensemble: each sample's rates get the contraction over its own triangles
        for (int b = 0; b < B; ++b) {
          const int64_t t0 = ctx->sample_tri_ptr[b], t1 = ctx->sample_tri_ptr[b + 1];
          launch_param_contract(n, t1 - t0, ctx->tri + 3 * t0, ctx->xy, Uk, lam, ctx->bfield, make_rates(ctx),
                                ctx->opt.quadrature, ctx->partial, grid, NV_STRIDE, ctx->elem + 3 * t0, nullptr,
                                nullptr, nullptr, s);
          launch_reduce_cols(grid, 10, ctx->partial, gacc + 16 * b, 1, s);
        }
        launch_field_gather(n, ctx->node_inc_ptr, ctx->node_inc, ctx->elem, gf, s);
      }
      CK(cudaGetLastError());
      std::swap(lam, lam_next);
    }
  }
  double jv = 0.0;
  std::vector<double> g(16 * (size_t)B);
  CK(cudaMemcpyAsync(&jv, jacc, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(g.data(), gacc, sizeof(double) * 16 * B, cudaMemcpyDeviceToHost, s));
  if (gfield) {
    std::vector<double> gi(n);
    CK(cudaMemcpyAsync(gi.data(), gf, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int64_t k = 0; k < n; ++k) gfield[hs.perm[k]] = gi[k];
  }
  CK(cudaStreamSynchronize(s));
  if (jout) *jout = jv;
  if (grad)
    for (int b = 0; b < B; ++b)
      for (int k = 0; k < 10; ++k) grad[10 * b + k] = g[16 * b + k];
  return restore(SEIRD_OK);
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

void seird_default_options(seird_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dt = 1.0;
  o->newton_rtol = 1e-8;
  o->newton_atol = 0.0;
  o->newton_maxit = 20;
  o->ls_maxit = 10;
  o->gmres_restart = 30;
  o->gmres_maxit = 200;
  o->gmres_rtol = 1e-5;
  o->gmres_atol = 1e-50;
  o->gmres_dtol = 1e5;
  o->n_subdomains = 4;
  o->overlap = 1;
  o->coarse = 0;
  o->precision = 0;
  o->quadrature = 0;
  o->pc_lag = 1;
  o->owner = nullptr;
  o->seed = 0;
  o->stream = nullptr;
}

const char* seird_last_error(const seird_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

int64_t seird_launch_count(void) { return launch_total(); }

void seird_destroy(seird_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  if (ctx->coarse_graph) cudaGraphExecDestroy(ctx->coarse_graph);
  if (ctx->cycle_exec) cudaGraphExecDestroy(ctx->cycle_exec);
  for (void* p : ctx->allocations) cudaFree(p);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->h_cyc) cudaFreeHost(ctx->h_cyc);
  if (ctx->h_flag) cudaFreeHost(ctx->h_flag);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static int create_impl(seird_ctx* ctx, const seird_mesh* mesh, const seird_params* params) {
  seird_options& o = ctx->opt;
  if (!(o.dt > 0) || o.gmres_restart < 1 || o.gmres_restart > MAX_RESTART || o.gmres_maxit < 1 ||
      o.newton_maxit < 0 || o.ls_maxit < 0 || o.overlap < 0 || o.coarse < 0 || o.coarse > 3 ||
      (o.quadrature != 0 && o.quadrature != 1) || (o.precision != 0 && o.precision != 1) ||
      (o.gmres_forcing != 0 && o.gmres_forcing != 1) || (o.nonlinear != 0 && o.nonlinear != 1) ||
      (o.gmres_one_pass != 0 && o.gmres_one_pass != 1) || o.pc_keep_steps < 0 ||
      (o.predictor < 0 || o.predictor > seird::MAX_PREDICTOR) || !(o.forcing_first >= 0.0 && o.forcing_first < 1.0) || (o.autotune != 0 && o.autotune != 1) || (o.graph != 0 && o.graph != 1) ||
      o.ilu_fill < 0 || o.ilu_fill > 8 || !(o.picard_tol >= 0))
    return fail(ctx, SEIRD_EINVAL, "invalid option value");
  std::string err;
  int rc = build_setup(mesh, &o, ctx->hs, err);
  if (rc) return fail(ctx, rc, err);
  HostSetup& hs = ctx->hs;
  if (o.coarse && 5 * (int64_t)hs.Pc * 8 > 200 * 1024)
    return fail(ctx, SEIRD_EINVAL, "coarse space supports at most 5120 coarse units (options.coarse_group)");
  // a stage of the subdomain solves must fit the factor ring (only a row with more blocks than
  // the ring, a node with hundreds of neighbours, can make one larger)
  if (solve_max_stage_blocks(ctx) > SOLVE_RING_FULL)
    return fail(ctx, SEIRD_EINVAL, "a subdomain row has more blocks than the solve's shared-memory ring holds (" +
                                       std::to_string(SOLVE_RING_FULL) + ")");
  if (o.stream) {
    ctx->stream = (cudaStream_t)o.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  CK(upload_quadrature());
  cgs_init();
  coarse_init();
  CK(cudaGetLastError());
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ctx->sms = std::max(1, sms);
  ctx->red_grid = ctx->sms * 3;
  const int64_t n = hs.n, m = hs.m, len = 5 * n;
  const int64_t nnzb = (int64_t)hs.col.size();
  const int R = o.gmres_restart;
  // mesh, patterns, maps
  TRY(upload(ctx, &ctx->xy, hs.xy));
  TRY(upload(ctx, &ctx->tri, hs.tri));
  TRY(upload(ctx, &ctx->perm, hs.perm));
  TRY(upload(ctx, &ctx->row_ptr, hs.row_ptr));
  TRY(upload(ctx, &ctx->col, hs.col));
  TRY(upload(ctx, &ctx->tpos, hs.tpos));
  TRY(upload(ctx, &ctx->node_inc_ptr, hs.node_inc_ptr));
  TRY(upload(ctx, &ctx->node_inc, hs.node_inc));
  TRY(upload(ctx, &ctx->blk_inc_ptr, hs.blk_inc_ptr));
  TRY(upload(ctx, &ctx->blk_inc, hs.blk_inc));
  if (params->beta_field) {
    std::vector<double> bf(n);
    for (int64_t k = 0; k < n; ++k) bf[k] = params->beta_field[hs.perm[k]];
    TRY(upload(ctx, &ctx->bfield, bf));
  }
  if (o.precision == 0) TRY(dalloc(ctx, &ctx->val, 25 * nnzb));
  TRY(dalloc(ctx, &ctx->elem, 15 * m));
  TRY(dalloc(ctx, &ctx->geo, 8 * m));
  launch_tri_geometry(m, ctx->tri, ctx->xy, ctx->geo, ctx->stream);
  CK(cudaGetLastError());
  TRY(dalloc(ctx, &ctx->nodebuf, 8 * (size_t)hs.n));
  TRY(dalloc(ctx, &ctx->rec, (size_t)REC * m));
  double** vecs[] = {&ctx->U, &ctx->Un, &ctx->F, &ctx->Ft, &ctx->dU, &ctx->Ut, &ctx->stage, &ctx->stage2, &ctx->w};
  for (double** v : vecs) TRY(dalloc(ctx, v, len));
  if (o.predictor >= 1) {
    ctx->n_hist = o.predictor;
    for (int k = 0; k < ctx->n_hist; ++k) TRY(dalloc(ctx, &ctx->Uhist[k], len));
    ctx->Uprev = ctx->Uhist[0];
    TRY(dalloc(ctx, &ctx->Flast, len));
  }
  const bool mix = o.precision == 1;
  TRY(dalloc(ctx, &ctx->V, (size_t)(R + 1) * len));
  if (mix) {
    TRY(dalloc(ctx, &ctx->Z32, (size_t)R * len));
    TRY(dalloc(ctx, &ctx->val32, 25 * nnzb));
  } else {
    TRY(dalloc(ctx, &ctx->Z, (size_t)R * len));
  }
  const int64_t npart = std::max<int64_t>((int64_t)ctx->sms * 6 * NV_STRIDE, (n + 255) / 256);  // up to 6 CTAs/SM
  if (o.autotune) TRY(dalloc(ctx, &ctx->tune_buf, len));
  TRY(dalloc(ctx, &ctx->partial, npart));
  TRY(dalloc(ctx, &ctx->hcol, 2 * NV_STRIDE));
  TRY(dalloc(ctx, &ctx->gm, (size_t)(R + 1) * R + 2 * R + (R + 1) + R));
  TRY(dalloc(ctx, &ctx->scal, 16));
  TRY(dalloc(ctx, &ctx->err, 1));
  CK(cudaMemset(ctx->err, 0, sizeof(int32_t)));
  CK(cudaMemset(ctx->U, 0, sizeof(double) * len));
  CK(cudaMemset(ctx->gm, 0, sizeof(double) * ((size_t)(R + 1) * R + 2 * R + (R + 1) + R)));
  CK(cudaMallocHost((void**)&ctx->h_scal, sizeof(double) * 16));
  if (o.graph) {
    TRY(dalloc(ctx, &ctx->cyc_ctl, 4));
    CK(cudaMallocHost((void**)&ctx->h_cyc, sizeof(int) * 8));
  }
  CK(cudaMallocHost((void**)&ctx->h_err, sizeof(int32_t)));
  *ctx->h_err = 0;
  TRY(dalloc(ctx, &ctx->dflag, 1));
  CK(cudaMallocHost((void**)&ctx->h_flag, sizeof(int)));
  // RAS
  TRY(upload(ctx, &ctx->sd_row0, hs.sd_row0));
  TRY(upload(ctx, &ctx->sd_node, hs.sd_node));
  TRY(upload(ctx, &ctx->l_row_ptr, hs.l_row_ptr));
  TRY(upload(ctx, &ctx->l_col, hs.l_col));
  TRY(upload(ctx, &ctx->l_gblk, hs.l_gblk));
  TRY(upload(ctx, &ctx->l_diag, hs.l_diag));
  TRY(upload(ctx, &ctx->upd_ptr, hs.upd_ptr));
  TRY(upload(ctx, &ctx->upd, hs.upd));
  TRY(upload(ctx, &ctx->fwd_order, hs.fwd_order));
  TRY(upload(ctx, &ctx->fwd_lev, hs.fwd_lev));
  TRY(upload(ctx, &ctx->sd_fwd_lev0, hs.sd_fwd_lev0));
  TRY(upload(ctx, &ctx->bwd_order, hs.bwd_order));
  TRY(upload(ctx, &ctx->bwd_lev, hs.bwd_lev));
  TRY(upload(ctx, &ctx->sd_bwd_lev0, hs.sd_bwd_lev0));
  TRY(upload(ctx, &ctx->own_ptr, hs.own_ptr));
  TRY(upload(ctx, &ctx->owner, hs.owner));
  TRY(upload(ctx, &ctx->sd_sched, hs.sd_sched));
  const int64_t NL = (int64_t)hs.sd_node.size();
  const int64_t NLB = (int64_t)hs.l_col.size();
  for (int dir = 0; dir < 2; ++dir) {
    const HostSetup::SolvePlan& sp = dir == 0 ? hs.sp_fwd : hs.sp_bwd;
    seird_ctx::PlanPtrs& q = dir == 0 ? ctx->pf : ctx->pb;
    TRY(upload(ctx, &q.row, sp.row));
    TRY(upload(ctx, &q.start, sp.start));
    TRY(upload(ctx, &q.cnt, sp.cnt));
    TRY(upload(ctx, &q.levpos, sp.levpos));
    TRY(upload(ctx, &q.levblk, sp.levblk));
    TRY(upload(ctx, &q.sd_lev0, sp.sd_lev0));
    TRY(upload(ctx, &q.src, sp.src));
    TRY(upload(ctx, &q.col, sp.col));
    TRY(upload(ctx, &q.info, sp.info));
    if (mix) TRY(dalloc(ctx, dir == 0 ? &ctx->fL32 : &ctx->bU32, (size_t)28 * std::max<size_t>(1, sp.src.size())));
    else TRY(dalloc(ctx, dir == 0 ? &ctx->fL : &ctx->bU, (size_t)26 * std::max<size_t>(1, sp.src.size())));
  }
  if (mix) {
    TRY(dalloc(ctx, &ctx->fval32, 25 * NLB));
    TRY(dalloc(ctx, &ctx->dinv32, 25 * NL));
    TRY(dalloc(ctx, &ctx->ywork32, 5 * NL));
    TRY(dalloc(ctx, &ctx->zwork32, 5 * NL));
  } else {
    TRY(dalloc(ctx, &ctx->fval, 25 * NLB));
    TRY(dalloc(ctx, &ctx->dinv, 25 * NL));
    TRY(dalloc(ctx, &ctx->ywork, 5 * NL));
    TRY(dalloc(ctx, &ctx->zwork, 5 * NL));
  }
  // coarse
  if (o.coarse >= 2) {
    TRY(dalloc(ctx, &ctx->pct, len));
    if (o.precision == 1) TRY(dalloc(ctx, &ctx->pcu32, len));
    else TRY(dalloc(ctx, &ctx->pcu, len));
    TRY(upload(ctx, &ctx->az_ptr, hs.az_ptr));
    TRY(upload(ctx, &ctx->az_unit, hs.az_unit));
    TRY(upload(ctx, &ctx->az_blk, hs.az_blk));
    if (o.precision == 1) TRY(dalloc(ctx, &ctx->azval32, 25 * hs.az_unit.size()));
    else TRY(dalloc(ctx, &ctx->azval, 25 * hs.az_unit.size()));
  }
  if (o.coarse) {
    TRY(upload(ctx, &ctx->cunit_ptr, hs.cunit_ptr));
    TRY(upload(ctx, &ctx->cunit, hs.cunit));
    TRY(upload(ctx, &ctx->cpos, hs.cpos));
    TRY(upload(ctx, &ctx->cseg_blk, hs.cseg_blk));
    TRY(upload(ctx, &ctx->cchunk_ptr, hs.cchunk_ptr));
    TRY(upload(ctx, &ctx->cdst_ptr, hs.cdst_ptr));
    TRY(upload(ctx, &ctx->cdst_idx, hs.cdst_idx));
    const int64_t nc = 5 * (int64_t)hs.Pc;
    const int64_t nchunk = (int64_t)hs.cchunk_ptr.size() - 1;
    const bool dense = nc <= DENSE_COARSE_MAX;
    TRY(dalloc(ctx, &ctx->cpart, std::max<int64_t>(25 * nchunk, dense ? ((nc + 63) / 64) * nc : 0)));
    TRY(dalloc(ctx, &ctx->cband, 25 * (size_t)hs.Pc * (2 * hs.cband + 1)));
    TRY(dalloc(ctx, &ctx->cdinv, 25 * (size_t)hs.Pc));
    TRY(dalloc(ctx, &ctx->crhs, 2 * nc));
    TRY(dalloc(ctx, &ctx->cy32, nc));
    if (dense) TRY(dalloc(ctx, &ctx->ainvT, (size_t)nc * nc));
  }
  CK(cudaDeviceSynchronize());
  return SEIRD_OK;
}

int seird_create(const seird_mesh* mesh, const seird_params* params, const seird_options* opt, seird_ctx** out) {
  if (!out) return fail(nullptr, SEIRD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !params) return fail(nullptr, SEIRD_EINVAL, "mesh and params must not be NULL");
  seird_ctx* ctx = new (std::nothrow) seird_ctx();
  if (!ctx) return fail(nullptr, SEIRD_ENOMEM, "host allocation failed");
  ctx->params = *params;
  ctx->params.beta_field = nullptr;  // copied to the device, never retained
  if (opt) ctx->opt = *opt;
  else seird_default_options(&ctx->opt);
  int rc = host_guard(ctx, [&]() -> int { return create_impl(ctx, mesh, params); });
  ctx->opt.owner = nullptr;  // read during create only, never retained
  if (rc) {
    g_create_error = ctx->last_error;
    seird_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return SEIRD_OK;
}

int seird_create_ensemble(const seird_mesh* mesh, int32_t n_samples, const seird_params* params,
                          const seird_options* opt, seird_ctx** out) {
  if (!out) return fail(nullptr, SEIRD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !params || !mesh->xy || !mesh->tri) return fail(nullptr, SEIRD_EINVAL, "mesh and params must not be NULL");
  if (n_samples < 1) return fail(nullptr, SEIRD_EINVAL, "n_samples must be >= 1");
  return host_guard(nullptr, [&]() -> int {
    seird_options o;
    if (opt) o = *opt;
    else seird_default_options(&o);
    const int64_t n = mesh->n_nodes, m = mesh->n_tris, B = n_samples;
    if (n < 3 || m < 1) return fail(nullptr, SEIRD_EINVAL, "mesh needs at least 3 nodes and 1 triangle");
    if (B * n > (int64_t)INT32_MAX / 8 || B * m > (int64_t)INT32_MAX / 9)
      return fail(nullptr, SEIRD_EINVAL, "ensemble too large for 32-bit element maps");
    // one partition of the mesh, repeated for every sample: sample k owns
    // subdomains [k P, (k+1) P), so its nodes are one contiguous internal range
    std::vector<int32_t> own;
    int32_t P = 0;
    std::string err;
    int rc = partition_nodes(mesh, &o, own, P, err);
    if (rc) return fail(nullptr, rc, err);
    std::vector<double> xy(2 * B * n);
    std::vector<int32_t> tri(3 * B * m), owner(B * n);
    for (int64_t k = 0; k < B; ++k) {
      std::copy(mesh->xy, mesh->xy + 2 * n, xy.begin() + 2 * k * n);
      for (int64_t q = 0; q < 3 * m; ++q) tri[3 * k * m + q] = (int32_t)(mesh->tri[q] + k * n);
      for (int64_t i = 0; i < n; ++i) owner[k * n + i] = (int32_t)(own[i] + k * P);
    }
    std::vector<double> bf;
    seird_params p0 = params[0];
    if (p0.beta_field) {
      bf.resize(B * n);
      for (int64_t k = 0; k < B; ++k) std::copy(p0.beta_field, p0.beta_field + n, bf.begin() + k * n);
      p0.beta_field = bf.data();
    }
    o.owner = owner.data();
    o.n_subdomains = (int32_t)(B * P);
    if (o.coarse_group == 0) {
      // coarse units must not span two samples: the group size divides the per-sample partition
      int32_t G = 1;
      auto fits = [&](int32_t g) {
        const int64_t units = B * (P / g);
        return 5 * units <= DENSE_COARSE_MAX && units <= COARSE_BLOCKCOL_MAX;
      };
      while (G < P && !(P % G == 0 && fits(G))) ++G;
      o.coarse_group = G;
    }
    seird_mesh um{B * n, B * m, xy.data(), tri.data()};
    seird_ctx* ctx = nullptr;
    rc = seird_create(&um, &p0, &o, &ctx);
    if (rc) return rc;
    std::unique_ptr<seird_ctx, void (*)(seird_ctx*)> hold(ctx, seird_destroy);  // destroyed unless completed
    std::vector<double> rows(RATE_ROW * B);
    for (int64_t k = 0; k < B; ++k) {
      const seird_params& q = params[k];
      const double v[RATE_ROW] = {q.A,     q.beta_i, q.beta_e, q.sigma, q.gamma_e, q.gamma_r, q.gamma_d,
                                  q.alpha, q.mu,     q.nu[0],  q.nu[1], q.nu[2],   q.nu[3]};
      std::copy(v, v + RATE_ROW, rows.begin() + RATE_ROW * k);
    }
    rc = upload(ctx, &ctx->rtab, rows);
    if (rc) {
      g_create_error = ctx->last_error;
      return rc;
    }
    ctx->n_samples = n_samples;
    ctx->n_per_sample = n;
    // internal triangles are ordered by their smallest node, so each sample's are one range
    ctx->sample_tri_ptr.assign(B + 1, 0);
    for (int64_t t = 0; t < B * m; ++t) {
      const int32_t* v = ctx->hs.tri.data() + 3 * t;
      ctx->sample_tri_ptr[std::min({v[0], v[1], v[2]}) / n + 1]++;
    }
    for (int64_t k = 0; k < B; ++k) ctx->sample_tri_ptr[k + 1] += ctx->sample_tri_ptr[k];
    *out = hold.release();
    return SEIRD_OK;
  });
}

int seird_set_state(seird_ctx* ctx, const double* u, int on_device, double t) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !u) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (ctx->have_prev && t == ctx->t) {
      // the state the context already holds, at its own time (a caller that round-trips the
      // state through its memory between steps): the step history stays valid
      TRY(to_internal(ctx, u, on_device, ctx->Ut));
      launch_differs(vlen(ctx), ctx->Ut, ctx->U, ctx->dflag, ctx->stream);
      CK(cudaMemcpyAsync(ctx->h_flag, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(ctx->U, ctx->Ut, sizeof(double) * vlen(ctx), cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      ctx->have_prev = *ctx->h_flag == 0;
      return SEIRD_OK;
    }
    TRY(to_internal(ctx, u, on_device, ctx->U));
    ctx->t = t;
    ctx->have_prev = false;
    return SEIRD_OK;
  });
}

int seird_get_state(const seird_ctx* cctx, double* u, int on_device, double* t) {
  return host_guard(const_cast<seird_ctx*>(cctx), [&]() -> int {
    seird_ctx* ctx = const_cast<seird_ctx*>(cctx);
    if (!ctx || !u) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    TRY(from_internal(ctx, ctx->U, u, on_device));
    if (t) *t = ctx->t;
    return SEIRD_OK;
  });
}

int seird_step(seird_ctx* ctx, seird_stats* stats) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx) return fail(nullptr, SEIRD_EINVAL, "NULL context");
    return newton_step(ctx, stats);
  });
}

int seird_run(seird_ctx* ctx, int32_t n_steps, seird_stats* per_step) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || n_steps < 0) return fail(ctx, SEIRD_EINVAL, "bad argument");
    for (int32_t k = 0; k < n_steps; ++k) TRY(newton_step(ctx, per_step ? per_step + k : nullptr));
    return SEIRD_OK;
  });
}

int seird_set_params(seird_ctx* ctx, const seird_params* params) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !params) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (ctx->rtab) return fail(ctx, SEIRD_EINVAL, "set_params: an ensemble's rates are fixed at creation");
    ctx->have_prev = false;  // the previous step's residual belongs to the old rates
    ctx->params = *params;
    ctx->params.beta_field = nullptr;
    if (params->beta_field) {
      const HostSetup& hs = ctx->hs;
      std::vector<double> bf(hs.n);
      for (int64_t k = 0; k < hs.n; ++k) bf[k] = params->beta_field[hs.perm[k]];
      if (!ctx->bfield) TRY(dalloc(ctx, &ctx->bfield, hs.n));
      CK(cudaMemcpy(ctx->bfield, bf.data(), sizeof(double) * hs.n, cudaMemcpyHostToDevice));
    }
    ctx->pc_ready = false;
    return SEIRD_OK;
  });
}

int seird_set_beta_schedule(seird_ctx* ctx, const seird_beta_schedule* sched) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx) return fail(ctx, SEIRD_EINVAL, "NULL context");
    if (ctx->rtab) return fail(ctx, SEIRD_EINVAL, "beta schedule: not available on an ensemble");
    ctx->have_prev = false;
    if (!sched) {
      ctx->sched_on = false;
      ctx->pc_ready = false;
      return SEIRD_OK;
    }
    const double v[10] = {sched->b0,        sched->b1,        sched->t_mid,     sched->beta_central, sched->beta_eastern,
                          sched->beta_western, sched->x_eastern, sched->x_western, sched->k_eastern,   sched->k_western};
    for (double x : v)
      if (!std::isfinite(x)) return fail(ctx, SEIRD_EINVAL, "beta schedule: non-finite value");
    if (!ctx->bsched) TRY(dalloc(ctx, &ctx->bsched, ctx->hs.n));
    launch_beta_field(ctx->hs.n, ctx->xy, *sched, ctx->bsched, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->sched = *sched;
    ctx->sched_on = true;
    ctx->pc_ready = false;
    return SEIRD_OK;
  });
}

int seird_adjoint(seird_ctx* ctx, const seird_misfit* spec, double* misfit, double* grad, double* grad_field) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !spec) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (ctx->sched_on) return fail(ctx, SEIRD_EINVAL, "adjoint: turn the beta schedule off first (constant rates only)");

    return adjoint_impl(ctx, spec, misfit, grad, grad_field);
  });
}

int seird_get_info(const seird_ctx* ctx, seird_info* info) {
  if (!ctx || !info) return SEIRD_EINVAL;
  info->n_nodes = ctx->hs.n;
  info->n_tris = ctx->hs.m;
  info->nnzb = (int64_t)ctx->hs.col.size();
  info->n_subdomains = ctx->hs.P;
  info->subdomain_rows = (int64_t)ctx->hs.sd_node.size();
  info->subdomain_blocks = (int64_t)ctx->hs.l_col.size();
  info->max_levels = ctx->hs.max_levels;
  info->coarse_band = ctx->hs.cband;
  info->device_bytes = ctx->device_bytes;
  info->coarse_units = ctx->hs.Pc;
  info->spmv_threads = ctx->spmv_tb;
  info->cgs_ctas = ctx->red_grid;
  info->cgs_tile = ctx->cgs_tile;
  info->ilu_batch = ctx->ilu_ch;
  info->ilu_warps = ctx->ilu_warps;
  info->ilu_ring = ctx->ilu_ring;
  return SEIRD_OK;
}

int seird_eval_residual(seird_ctx* ctx, const double* u, const double* u_prev, double* F, int on_device) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !u || !u_prev || !F) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    TRY(to_internal(ctx, u, on_device, ctx->Ut));
    TRY(to_internal(ctx, u_prev, on_device, ctx->stage2));
    double fn;
    TRY(residual(ctx, ctx->Ut, ctx->stage2, ctx->Ft, &fn));
    return from_internal(ctx, ctx->Ft, F, on_device);
  });
}

int seird_eval_jacobian(seird_ctx* ctx, const double* u, int on_device) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !u) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    TRY(to_internal(ctx, u, on_device, ctx->Ut));
    TRY(jacobian(ctx, ctx->Ut, ctx->opt.nonlinear == 1));
    return check_flags(ctx, "jacobian");
  });
}

int seird_get_jacobian(const seird_ctx* cctx, int32_t* row_ptr, int32_t* col, double* val) {
  return host_guard(const_cast<seird_ctx*>(cctx), [&]() -> int {
    seird_ctx* ctx = const_cast<seird_ctx*>(cctx);
    if (!ctx || !row_ptr || !col || !val) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (!ctx->jac_ready) return fail(ctx, SEIRD_EINVAL, "no Jacobian assembled");
    const HostSetup& hs = ctx->hs;
    const int64_t nnzb = (int64_t)hs.col.size();
    std::vector<double> v(25 * nnzb);
    CK(cudaStreamSynchronize(ctx->stream));
    if (mixed(ctx)) {  // the mixed path keeps only the FP32 copy
      std::vector<float> v32(25 * nnzb);
      CK(cudaMemcpy(v32.data(), ctx->val32, sizeof(float) * v32.size(), cudaMemcpyDeviceToHost));
      for (size_t q = 0; q < v.size(); ++q) v[q] = v32[q];
    } else {
      CK(cudaMemcpy(v.data(), ctx->val, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
    }
    row_ptr[0] = 0;
    std::vector<std::pair<int32_t, int32_t>> ent;
    int64_t pos = 0;
    for (int64_t i = 0; i < hs.n; ++i) {
      const int32_t k = hs.iperm[i];
      ent.clear();
      for (int32_t b = hs.row_ptr[k]; b < hs.row_ptr[k + 1]; ++b) ent.push_back({hs.perm[hs.col[b]], b});
      std::sort(ent.begin(), ent.end());
      for (auto& e : ent) {
        col[pos] = e.first;
        std::memcpy(val + 25 * pos, v.data() + 25 * (int64_t)e.second, 25 * sizeof(double));
        ++pos;
      }
      row_ptr[i + 1] = (int32_t)pos;
    }
    return SEIRD_OK;
  });
}

int seird_apply_jacobian(seird_ctx* ctx, const double* x, double* y, int on_device) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !x || !y) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (!ctx->jac_ready) return fail(ctx, SEIRD_EINVAL, "no Jacobian assembled");
    TRY(to_internal(ctx, x, on_device, ctx->stage2));
    TRY(spmv(ctx, ctx->stage2, ctx->Ft));
    return from_internal(ctx, ctx->Ft, y, on_device);
  });
}

int seird_precond_setup(seird_ctx* ctx) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx) return fail(nullptr, SEIRD_EINVAL, "NULL context");
    return pc_setup(ctx);
  });
}

int seird_precond_apply(seird_ctx* ctx, const double* r, double* z, int on_device) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !r || !z) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (!ctx->pc_ready) return fail(ctx, SEIRD_EINVAL, "preconditioner not set up");
    TRY(to_internal(ctx, r, on_device, ctx->stage2));
    TRY(pc_apply(ctx, ctx->stage2, ctx->Ft));
    TRY(check_flags(ctx, "preconditioner apply"));
    return from_internal(ctx, ctx->Ft, z, on_device);
  });
}

int seird_set_launch_shapes(seird_ctx* ctx, int32_t spmv_threads, int32_t cgs_ctas, int32_t cgs_tile,
                            int32_t ilu_batch, int32_t ilu_warps, int32_t ilu_ring) {
  if (!ctx) return SEIRD_EINVAL;
  if ((spmv_threads && spmv_threads != 128 && spmv_threads != 256 && spmv_threads != 512) || cgs_ctas < 0 ||
      cgs_ctas > 64 * ctx->sms || (cgs_tile && cgs_tile != 128 && cgs_tile != 256) || ilu_batch < 0 ||
      ilu_batch > 4 || (ilu_warps && ilu_warps != 3 && ilu_warps != 7) ||
      (ilu_ring && ilu_ring != SOLVE_RING_FULL && ilu_ring != SOLVE_RING_HALF))
    return fail(ctx, SEIRD_EINVAL, "set_launch_shapes: a shape outside its candidates");
  if (ilu_ring == SOLVE_RING_HALF && solve_max_stage_blocks(ctx) > SOLVE_RING_HALF)
    return fail(ctx, SEIRD_EINVAL, "set_launch_shapes: a solve stage is larger than a one-stage ring");
  if (ilu_ring) ctx->ilu_ring = ilu_ring;
  if (spmv_threads) ctx->spmv_tb = spmv_threads;
  if (cgs_ctas) ctx->red_grid = cgs_ctas;
  if (cgs_tile) ctx->cgs_tile = cgs_tile;
  if (ilu_batch) ctx->ilu_ch = ilu_batch;
  if (ilu_warps) ctx->ilu_warps = ilu_warps;
  ctx->tuned = true;  // the autotuner keeps these
  if (ctx->cycle_exec) {  // a captured restart cycle holds the old shapes
    cudaGraphExecDestroy(ctx->cycle_exec);
    ctx->cycle_exec = nullptr;
  }
  return SEIRD_OK;
}

int seird_set_wait_limit(seird_ctx* ctx, int32_t polls) {
  if (!ctx) return SEIRD_EINVAL;
  ctx->wait_polls = polls == 0 ? SOLVE_WAIT_POLLS_DEFAULT : std::max<int32_t>(polls, 0);
  if (ctx->cycle_exec) {  // a captured restart cycle holds the old limit in its kernel arguments
    cudaGraphExecDestroy(ctx->cycle_exec);
    ctx->cycle_exec = nullptr;
  }
  return SEIRD_OK;
}

int seird_linear_solve(seird_ctx* ctx, const double* b, double* x, int on_device, int32_t* its) {
  return host_guard(ctx, [&]() -> int {
    if (!ctx || !b || !x) return fail(ctx, SEIRD_EINVAL, "NULL argument");
    if (!ctx->pc_ready) return fail(ctx, SEIRD_EINVAL, "preconditioner not set up");
    TRY(to_internal(ctx, b, on_device, ctx->stage2));
    int k = 0;
    bool conv = false;
    TRY(gmres(ctx, ctx->stage2, ctx->dU, ctx->opt.gmres_rtol, &k, &conv));
    if (its) *its = k;
    TRY(from_internal(ctx, ctx->dU, x, on_device));
    return conv ? SEIRD_OK : fail(ctx, SEIRD_EGMRES, "gmres: iteration limit reached");
  });
}

int seird_bsr_spmv(int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val, const double* x,
                   double* y, void* stream) {
  if (n_rows < 0) return SEIRD_EINVAL;
  if (n_rows == 0) return SEIRD_OK;
  if (!row_ptr || !col || !val || !x || !y) return SEIRD_EINVAL;
  launch_spmv<double>(n_rows, row_ptr, col, val, x, y, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? SEIRD_OK : SEIRD_ECUDA;
}

int seird_bsr_spmv_f32val(int64_t n_rows, const int32_t* row_ptr, const int32_t* col, const float* val,
                          const double* x, double* y, void* stream) {
  if (n_rows < 0) return SEIRD_EINVAL;
  if (n_rows == 0) return SEIRD_OK;
  if (!row_ptr || !col || !val || !x || !y) return SEIRD_EINVAL;
  launch_spmv<float>(n_rows, row_ptr, col, val, x, y, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? SEIRD_OK : SEIRD_ECUDA;
}

}  // extern "C"
