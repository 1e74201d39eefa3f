// Device-side shared declarations: rate parameters, launch accounting, small
// reductions.  Included by the .cu files of the library only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/seird.h"

namespace seird {

// Rates of Eq. seird1-5 plus dt, packed for kernel arguments.
struct Rates {
  double A, bi, be, sigma, ge, gr, gd, alpha, mu;
  double nu[4];
  double dt;
  // ensembles: per-sample rows [A, bi, be, sigma, ge, gr, gd, alpha, mu, nu0..3] of a
  // device table, sample = internal node / nper (NULL: the scalars above for every node)
  const double* tab;
  int64_t nper;
};
constexpr int RATE_ROW = 13;

#ifdef __CUDACC__
// The rates that hold at internal node `node` (its sample's row of the table).
__device__ __forceinline__ Rates rates_at(const Rates& r, int64_t node) {
  if (!r.tab) return r;
  Rates q = r;
  const double* t = r.tab + RATE_ROW * (node / r.nper);
  q.A = t[0];
  q.bi = t[1];
  q.be = t[2];
  q.sigma = t[3];
  q.ge = t[4];
  q.gr = t[5];
  q.gd = t[6];
  q.alpha = t[7];
  q.mu = t[8];
  q.nu[0] = t[9];
  q.nu[1] = t[10];
  q.nu[2] = t[11];
  q.nu[3] = t[12];
  return q;
}
#endif

// Jacobian record of one triangle: area, N-weighted stiffness K_ab (6 pairs), pad,
// G_{c,a} = |T|/3 grad u_c . grad phi_a stored [a][c] (12), reaction moments P^k_ab
// stored [pair][k] (24).  The gather of block (a, b) reads G[a][0..3] and
// P[pair][0..3]: 32 consecutive bytes each, starting on 32-byte boundaries (FP64).
constexpr int REC = 44;
constexpr int REC_K = 1, REC_G = 8, REC_P = 20;

void count_launch();
void count_launches(int64_t k);
int64_t launch_total();
// message returned by seird_last_error(NULL) (per host thread)
void set_global_error(const std::string& msg);

// quadrature tables are uploaded once per process (degree-5 and vertex rules)
cudaError_t upload_quadrature();  // quadrature tables to constant memory (checked, synchronised)

// ---- launchers (defined in the .cu files) ----
// geo: per-triangle |T| and hat-function gradients (8 doubles each) from launch_tri_geometry,
// or NULL to compute them from xy; nd: 8 doubles per node of scratch (degree-5 rule)
void launch_tri_geometry(int64_t m, const int32_t* tri, const double* xy, double* geo, cudaStream_t s);
void launch_residual(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* geo, const double* U,
                     const double* Un, const double* bfield, const Rates& r, int rule, double* nd, double* elem,
                     const int32_t* inc_ptr, const int32_t* inc, double* F, double* partial, double* out_norm2,
                     int32_t* err, cudaStream_t s);
void launch_beta_field(int64_t n, const double* xy, const seird_beta_schedule& s, double* out, cudaStream_t st);
void launch_jacobian(int64_t nnzb, int64_t m, const int32_t* tri, const double* xy, const double* geo, const double* U,
                     const double* bfield, const Rates& r, int rule, void* rec, const int32_t* inc_ptr,
                     const int32_t* inc, void* val, bool fp32, bool picard, int32_t* err, cudaStream_t s);
// y = A x, or y = b - A x when b != NULL
template <class VT>
void launch_spmv(int64_t nrow, const int32_t* rp, const int32_t* col, const VT* val, const double* x, double* y,
                 cudaStream_t s, int tb = 256, const double* b = nullptr);

// vectors (length len, grid-stride)
void launch_norm2(int64_t len, const double* x, double* partial, int grid, double* out, cudaStream_t s);
void launch_mdot(int64_t len, int nv, const double* V, int64_t ld, const double* w, double* partial, int grid,
                 double* out, cudaStream_t s, int tile = 0);
void launch_update_mdot(int64_t len, int nv, const double* V, int64_t ld, const double* h, double* w,
                        double* partial, int grid, double* out_add, cudaStream_t s, int tile = 0);
void launch_update_norm(int64_t len, int nv, const double* V, int64_t ld, const double* h, double* w,
                        double* partial, int grid, double* out, cudaStream_t s);
void launch_scale(int64_t len, const double* x, const double* alpha_ptr, int invert, double* y, cudaStream_t s);
void launch_axpby(int64_t len, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);
void launch_multi_axpy(int64_t len, int nv, const double* Zs, int64_t ld, const double* coef, double* x,
                       cudaStream_t s);
// Convergence control of a GMRES restart cycle captured into a CUDA graph (see k_givens);
// all zero outside captures.
struct CycleCtl {
  int* ctl = nullptr;
  const double* tol = nullptr;
  cudaGraphConditionalHandle next = 0;
  int has_next = 0;
};
void launch_givens(int j, double* gm, const double* h1, const double* h2, const double* hnext, int ldh,
                   double* out_res, cudaStream_t s, const CycleCtl& cc = CycleCtl());
void launch_reduce_cols(int grid, int nv, const double* partial, double* out, int add, cudaStream_t s);
void cgs_init();
constexpr int NV_STRIDE = 65;  // row stride of the CGS partial-sum buffer
void launch_hsolve(int k, double* gm, int ldh, cudaStream_t s);
void launch_gather5(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t s);
void launch_scatter5(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t s);

// discrete adjoint
void launch_mass(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* V, double* elem,
                 const int32_t* inc_ptr, const int32_t* inc, double* out, double* partial, double* norm2,
                 cudaStream_t s);
void launch_field_gather(int64_t n, const int32_t* inc_ptr, const int32_t* inc, const double* fe, double* out,
                         cudaStream_t s);
void launch_param_contract(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* U,
                           const double* lam, const double* bfield, const Rates& r, int rule, double* partial,
                           int grid, int stride, double* fe, const int32_t* inc_ptr, const int32_t* inc,
                           double* field_out, cudaStream_t s);
void launch_misfit(int nobs, const int32_t* nodes, const double* Ihat, const double* Dhat, const double* U,
                   double* rhs, double* jacc, cudaStream_t s);
void launch_bsr_transpose(int64_t nnzb, const int32_t* tpos, const double* val, double* valT, cudaStream_t s);

// RAS and coarse space
constexpr int SOLVE_BUF_BLOCKS_DEV = 118;  // factor blocks per ILU-solve stage buffer
constexpr int SOLVE_BUF_ROWS_DEV = 128;    // rows per ILU-solve stage
struct SolvePlanDev {
  const int32_t* row;
  const int64_t* start;
  const int32_t* cnt;
  const int32_t* levpos;
  const int64_t* levblk;
  const int32_t* sd_lev0;
  const int4* info;  // per position: row, first block relative to its stage, block count, 0
};
struct RasDev {
  int32_t P;
  const int32_t* sd_sched;  // CTA b of a per-subdomain kernel works on subdomain sd_sched[b]
  const int32_t* sd_row0;
  const int32_t* sd_node;
  const int64_t* l_row_ptr;
  const int32_t* l_col;
  const int32_t* l_gblk;
  const int64_t* l_diag;
  const int64_t* upd_ptr;
  const int64_t* upd;
  const int32_t* fwd_order;
  const int32_t* fwd_lev;
  const int32_t* sd_fwd_lev0;
  const int32_t* bwd_order;
  const int32_t* bwd_lev;
  const int32_t* sd_bwd_lev0;
  const int32_t* own_ptr;
  double* fval;
  double* dinv;
  double* ywork;
  double* zwork;
  float* fval32;  // mixed-precision path
  float* dinv32;
  float* ywork32;
  float* zwork32;
  SolvePlanDev fwd, bwd;  // level-ordered solve copies of the factors
  double* fL;
  double* bU;
  float* fL32;
  float* bU32;
  // polls of each bounded wait on a stage's data or ring space in the solve (<= 0:
  // none, so every wait gives up at once); the final wait for issued copies to land
  // keeps the fixed bound SOLVE_DRAIN_POLLS
  int32_t wait_polls;
  // blocks whose solution entries a consumer row loads before their FMAs (1-4; the autotuner's
  // choice, 2 by default); every choice forms the same sums in the same order
  int32_t solve_ch;
  int32_t solve_warps;  // consumer warps per subdomain CTA: 7 (256 threads) or 3 (128 threads)
  int32_t solve_ring;   // blocks in the factor ring: SOLVE_RING_FULL (two stages) or SOLVE_RING_HALF (one)
};
constexpr int32_t SOLVE_RING_FULL = 2 * SOLVE_BUF_BLOCKS_DEV;
constexpr int32_t SOLVE_RING_HALF = SOLVE_BUF_BLOCKS_DEV;
constexpr int32_t SOLVE_WAIT_POLLS_DEFAULT = 1 << 20;
void launch_ilu_factor(const RasDev& d, const double* val, const float* val32, int32_t* err, bool fp32,
                       cudaStream_t s);
void launch_ilu_reorg(const RasDev& d, int64_t nfwd, int64_t nbwd, const int64_t* fsrc, const int32_t* fcol,
                      const int64_t* bsrc, const int32_t* bcol, bool fp32, cudaStream_t s);
void launch_ilu_solve(const RasDev& d, const double* r, double* z, int32_t* err, cudaStream_t s);
void launch_ilu_solve32(const RasDev& d, const double* r, float* z, int32_t* err, cudaStream_t s);
void launch_spmv32(int64_t nrow, const int32_t* rp, const int32_t* col, const float* val, const float* x, double* y,
                   cudaStream_t s, int tb = 256, const double* b = nullptr);
void launch_multi_axpy32(int64_t len, int nv, const float* Zs, int64_t ld, const double* coef, double* x,
                         cudaStream_t s);
void launch_f32_to_f64(int64_t n, const float* src, double* dst, cudaStream_t s);
void launch_add32(int64_t len, const float* u, float* z, cudaStream_t s);
// *flag = 1 if a and b differ in any bit pattern, else 0 (flag is cleared first)
void launch_differs(int64_t len, const double* a, const double* b, int* flag, cudaStream_t s);

struct CoarseDev {
  int32_t P, band;
  const int32_t* cpos;
  const int32_t* owner;
  const int32_t* own_ptr;
  const int32_t* cseg_blk;
  const int32_t* cchunk_ptr;
  int32_t nchunk;
  const int32_t* cdst_ptr;
  const int64_t* cdst_idx;
  int32_t ndst;
  double* cpart;   // chunk partial sums (assembly) and GEMV partials (apply)
  double* cband;
  double* cdinv;
  double* crhs;    // [2 * 5P]: Z^T r, then A_c^{-1} Z^T r
  double* ainvT;   // [5P][5P] explicit inverse, transposed (NULL: banded solve per apply)
  float* y32;      // [5P] FP32 copy of A_c^{-1} Z^T r for the mixed-precision path
};
void launch_coarse_assemble(const CoarseDev& c, const double* val, const float* val32, cudaStream_t s);
void launch_az_build(int64_t nseg, const int32_t* az_blk, const double* val, const float* val32, double* azval,
                     float* azval32, bool fp32, cudaStream_t s);
void launch_az_sub(const CoarseDev& c, int64_t n, const int64_t* az_ptr, const int32_t* az_unit,
                   const double* azval, const float* azval32, bool fp32, double* t, cudaStream_t s);
void launch_coarse_factor(const CoarseDev& c, int32_t* err, cudaStream_t s);
template <class TZ>
void launch_coarse_apply_add(const CoarseDev& c, int64_t n, const double* r, TZ* z, cudaStream_t s);
void launch_coarse_solve(const CoarseDev& c, const double* r, cudaStream_t s);
// mixed-precision path, after launch_coarse_solve: y32 = (float) y, then z += Z y32 in FP32,
// and t -= (J Z) y32 with FP32 products (accumulated in FP32, subtracted in FP64)
void launch_coarse_y32(const CoarseDev& c, cudaStream_t s);
void launch_coarse_prolong32(const CoarseDev& c, int64_t n, float* z, cudaStream_t s);
template <class TZ>
void launch_coarse_prolong(const CoarseDev& c, int64_t n, TZ* z, cudaStream_t s);

}  // namespace seird
