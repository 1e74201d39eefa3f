// Internal declarations of the SEIRD library: the context, the host-side setup
// products and the kernel launchers.  Everything here sits behind include/seird.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/seird.h"
#include "kernels.cuh"

namespace seird {

// Device error flags (bitmask written by kernels, read by the host after a phase).
enum : int {
  ERR_NONPOS_N = 1,    // N <= 0 at a quadrature point (1/N undefined)
  ERR_SINGULAR = 2,    // a 5x5 pivot block is singular
  ERR_NONFINITE = 4,   // a non-finite value in a reduction
  ERR_TIMEOUT = 8,     // a bounded wait gave up
};

constexpr int MAX_RESTART = 64;
constexpr int MAX_PREDICTOR = 6;  // highest degree of the Newton predictor's extrapolation
// coarse problems up to this many unknowns (5 x subdomains) keep an explicit
// inverse (applied as a GEMV); larger ones are solved through the band factors
constexpr int64_t DENSE_COARSE_MAX = 8192;
// coarse units whose explicit inverse is built five columns per CTA (25 doubles per unit in shared memory)
constexpr int32_t COARSE_BLOCKCOL_MAX = 1160;
// blocks per ILU-solve level buffer (two buffers of 24 KB in FP64 at 26 doubles per block)
constexpr int32_t SOLVE_BUF_BLOCKS = SOLVE_BUF_BLOCKS_DEV;
constexpr int32_t SOLVE_BUF_ROWS = SOLVE_BUF_ROWS_DEV;
// a stage of the subdomain solve costs about as much as this many blocks (its barrier and
// the latency of its first dependency loads), for the launch order of the subdomain CTAs
constexpr int64_t SOLVE_STAGE_WEIGHT = 40;
// solve work of subdomain q that orders the subdomain CTAs: blocks + SOLVE_STAGE_WEIGHT x stages
struct HostSetup;
int64_t solve_work(const HostSetup& hs, int32_t q);

// Host-side products of the setup phase (all indices in the internal numbering,
// where nodes are sorted by (subdomain, caller index)).
struct HostSetup {
  int64_t n = 0, m = 0;
  int32_t P = 0;
  std::vector<int32_t> perm;     // internal -> caller
  std::vector<int32_t> iperm;    // caller -> internal
  std::vector<int32_t> owner;    // internal node -> subdomain
  std::vector<int32_t> own_ptr;  // [P+1] owned nodes of p are [own_ptr[p], own_ptr[p+1])
  std::vector<double> xy;        // [n][2] internal order
  std::vector<int32_t> tri;      // [m][3] internal node ids (triangles sorted by min node)
  // global 5x5 BSR pattern
  std::vector<int32_t> row_ptr, col;  // [n+1], [nnzb]
  std::vector<int32_t> tpos;          // [nnzb] index of block (j,i) for block (i,j) (the pattern is symmetric)
  // residual gather: per node, list of (t*3 + a)
  std::vector<int32_t> node_inc_ptr, node_inc;
  // Jacobian gather: per block, list of (t*9 + a*3 + b)
  std::vector<int32_t> blk_inc_ptr, blk_inc;
  // subdomains (concatenated): local rows of subdomain p are [sd_row0[p], sd_row0[p+1])
  std::vector<int32_t> sd_row0;     // [P+1]
  std::vector<int32_t> sd_node;     // [NL] internal node of each local row
  std::vector<int64_t> l_row_ptr;   // [NL+1] absolute block offsets
  std::vector<int32_t> l_col;       // [NLB] local column (row index within the subdomain)
  std::vector<int32_t> l_gblk;      // [NLB] global J block of each local block
  std::vector<int64_t> l_diag;      // [NL] absolute index of the diagonal block
  std::vector<int64_t> upd_ptr;     // [NLB+1] ILU(0) update pairs of each lower block
  std::vector<int64_t> upd;         // [2*nupd] (destination block, source block) pairs
  std::vector<int32_t> fwd_order;   // [NL] local rows (relative) grouped by forward level
  std::vector<int32_t> fwd_lev;     // level boundaries (relative to the subdomain's rows)
  std::vector<int32_t> sd_fwd_lev0; // [P+1] offsets into fwd_lev (each subdomain has nlev+1 entries)
  std::vector<int32_t> bwd_order, bwd_lev, sd_bwd_lev0;
  int32_t max_levels = 0;
  int32_t max_sd_rows = 0;
  int32_t ilu_fill = 0;             // levels of fill of the subdomain factors (options.ilu_fill)
  // ILU(0) solve plans: the solve reads factor blocks from a copy laid out in
  // level order (forward: each row's strictly lower blocks; backward: each row's
  // inverted pivot block, then its upper blocks), so that every level is one
  // contiguous range that is prefetched into shared memory while the previous
  // level computes.  Levels are split so that a range fits the buffer.
  struct SolvePlan {
    std::vector<int32_t> row;     // [NL] local row at each position (per subdomain, level order)
    std::vector<int64_t> start;   // [NL] first block (absolute, in the solve copy) of each position
    std::vector<int32_t> cnt;     // [NL] blocks of each position
    std::vector<int32_t> levpos;  // per subdomain nlev+1 entries: position boundaries (relative)
    std::vector<int64_t> levblk;  // per subdomain nlev+1 entries: block boundaries (absolute)
    std::vector<int32_t> sd_lev0; // [P+1] offsets into levpos/levblk
    std::vector<int64_t> src;     // [nblocks] factor block (>= 0) or -1-R for the inverted pivot of row R
    std::vector<int32_t> col;     // [nblocks] sweep position of the entry each block multiplies (own for a pivot)
    std::vector<int32_t> info;    // [NL][4] per position: forward (node, first block in its stage, blocks, 0),
                                  // backward (forward position, first block, blocks, node if owned else -1)
    int32_t max_lev_blocks = 0;
  } sp_fwd, sp_bwd;
  // launch order of the per-subdomain kernels (factor and solve): subdomains by
  // descending solve work (blocks + SOLVE_STAGE_WEIGHT x stages, both sweeps), ties in
  // index order, so the longest start first and the grid's tail holds the short ones
  std::vector<int32_t> sd_sched;    // [P]
  // coarse space: subdomain p sits at block row cpos[p] of the banded coarse matrix
  // coarse units: groups of cG consecutive subdomains (cG = 1 unless the coarse matrix would be too
  // large for its explicit inverse); unit u owns the internal nodes [cunit_ptr[u], cunit_ptr[u+1])
  int32_t cG = 1, Pc = 0;
  std::vector<int32_t> cunit_ptr;   // [Pc+1]
  std::vector<int32_t> cunit;       // [n] unit of each internal node
  std::vector<int32_t> cpos;        // [Pc]
  // A Z (J seen through the coarse prolongation): in each BSR row the blocks of one coarse
  // unit are consecutive, one segment per (row, unit)
  std::vector<int64_t> az_ptr;      // [n+1] segments of each row
  std::vector<int32_t> az_unit;     // [nseg] coarse unit of each segment
  std::vector<int32_t> az_blk;      // [nseg+1] first block of each segment (the last entry is nnzb)
  int32_t cband = 0;                // half bandwidth in blocks
  std::vector<int32_t> cseg_blk;    // [nnzb] J block ids ordered by (cpos p, cpos q) then id
  std::vector<int32_t> cchunk_ptr;  // [nchunk+1] chunks of cseg_blk summed by one warp
  std::vector<int32_t> cdst_ptr;    // [ndst+1] chunk range of each coarse block
  std::vector<int64_t> cdst_idx;    // [ndst] block index in the band storage
};

int build_setup(const seird_mesh* mesh, const seird_options* opt, HostSetup& hs, std::string& err);
int64_t check_setup(const HostSetup& hs, std::string& first);
// Subdomain of every node: the caller's owner array (validated) or the seeded
// recursive coordinate bisection into opt->n_subdomains parts.
int partition_nodes(const seird_mesh* mesh, const seird_options* opt, std::vector<int32_t>& owner, int32_t& P,
                    std::string& err);

template <class T>
struct DevArray {
  T* p = nullptr;
  size_t n = 0;
};

struct Workspace;

}  // namespace seird

struct seird_ctx {
  seird::HostSetup hs;
  seird_params params{};
  seird_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double t = 0.0;
  std::string last_error;
  int64_t device_bytes = 0;
  std::vector<void*> allocations;
  // device mesh and patterns
  double* xy = nullptr;
  int32_t* tri = nullptr;
  double* bfield = nullptr;
  // ensembles (seird_create_ensemble): per-sample rate rows, samples of n_per_sample nodes
  int32_t n_samples = 1;
  int64_t n_per_sample = 0;
  double* rtab = nullptr;
  std::vector<int64_t> sample_tri_ptr;  // [n_samples+1] internal triangle range of each sample
  // the coarse factorisation's fixed launch sequence (two launches per block
  // column), captured once into a CUDA graph on a private stream and replayed
  cudaGraphExec_t coarse_graph = nullptr;
  int64_t coarse_graph_kernels = 0;
  // sigmoid transmission schedule (seird_set_beta_schedule): beta(x) at the nodes
  bool sched_on = false;
  seird_beta_schedule sched{};
  double* bsched = nullptr;
  int32_t* perm = nullptr;
  int32_t* cunit_ptr = nullptr;
  int32_t* cunit = nullptr;
  int64_t* az_ptr = nullptr;   // multiplicative two-grid: A Z segments and their 5x5 sums
  int32_t* az_unit = nullptr;
  int32_t* az_blk = nullptr;
  double* azval = nullptr;
  float* azval32 = nullptr;
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  int32_t* tpos = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  int32_t* node_inc_ptr = nullptr;
  int32_t* node_inc = nullptr;
  int32_t* blk_inc_ptr = nullptr;
  int32_t* blk_inc = nullptr;
  double* elem = nullptr;   // [m][15] residual element vectors
  double* rec = nullptr;    // [m][REC] Jacobian records
  // state and Newton vectors [n][5]
  double* U = nullptr;
  double* Un = nullptr;
  // earlier states for the predictor (options.predictor = p): Uhist[k] holds u^{n-1-k}, k < p, the
  // buffers rotating as steps complete; Uprev aliases Uhist[0] (u^{n-1})
  double* Uhist[seird::MAX_PREDICTOR] = {};
  int n_hist = 0;
  double* Uprev = nullptr;
  int hist_depth = 0;        // earlier states held (1: u^{n-1} ... p); valid while have_prev
  double* Flast = nullptr;  // F(u^n; u^{n-1}), the previous step's last residual
  bool have_prev = false;
  double* F = nullptr;
  double* Ft = nullptr;
  double* dU = nullptr;
  double* Ut = nullptr;
  double* stage = nullptr;  // staging for caller-numbered input/output
  double* stage2 = nullptr;
  // Krylov
  double* V = nullptr;      // [restart+1][5n]
  double* Z = nullptr;      // [restart][5n]
  double* w = nullptr;      // [5n]
  double* partial = nullptr;  // [grid][MAX_RESTART+1]
  double* hcol = nullptr;   // [MAX_RESTART+1] reduced dot products
  double* gm = nullptr;     // GMRES small state: H, cs, sn, g, y
  double* geo = nullptr;      // [m][8] |T| and hat-function gradients (set-up)
  double* nodebuf = nullptr;  // [n][8] node terms of the residual
  double* scal = nullptr;   // scalar outputs (norms)
  double* h_scal = nullptr; // pinned host mirror
  int32_t* err = nullptr;   // device error flags
  int32_t* h_err = nullptr; // pinned
  int* dflag = nullptr;      // device flag of seird_set_state's comparison with the held state
  int* h_flag = nullptr;     // pinned
  int red_grid = 0;
  // RAS
  int32_t* sd_row0 = nullptr;
  int32_t* sd_node = nullptr;
  int64_t* l_row_ptr = nullptr;
  int32_t* l_col = nullptr;
  int32_t* l_gblk = nullptr;
  int64_t* l_diag = nullptr;
  int64_t* upd_ptr = nullptr;
  int64_t* upd = nullptr;
  int32_t* fwd_order = nullptr;
  int32_t* fwd_lev = nullptr;
  int32_t* sd_fwd_lev0 = nullptr;
  int32_t* bwd_order = nullptr;
  int32_t* bwd_lev = nullptr;
  int32_t* sd_bwd_lev0 = nullptr;
  int32_t* own_ptr = nullptr;
  int32_t* owner = nullptr;
  int32_t* sd_sched = nullptr;
  double* fval = nullptr;   // [NLB][25] factor blocks
  float* fval32 = nullptr;
  double* dinv = nullptr;   // [NL][25] inverted U diagonal blocks
  float* dinv32 = nullptr;
  double* ywork = nullptr;  // [NL][5]
  double* zwork = nullptr;  // [NL][5]
  float* ywork32 = nullptr;  // mixed-precision path
  float* zwork32 = nullptr;
  struct PlanPtrs {
    int32_t* row = nullptr;
    int64_t* start = nullptr;
    int32_t* cnt = nullptr;
    int32_t* levpos = nullptr;
    int64_t* levblk = nullptr;
    int32_t* sd_lev0 = nullptr;
    int64_t* src = nullptr;
    int32_t* col = nullptr;
    int32_t* info = nullptr;
  } pf, pb;  // forward / backward solve plans
  double* fL = nullptr;  // level-ordered factor copies (FP64 path)
  double* bU = nullptr;
  float* fL32 = nullptr;  // (mixed path)
  float* bU32 = nullptr;
  float* Z32 = nullptr;      // [restart][5n] preconditioned basis in FP32
  double* pct = nullptr;     // [5n] residual between the steps of the multiplicative two-grid
  double* pcu = nullptr;     // [5n] FP64 post-smoothing correction
  float* pcu32 = nullptr;    // [5n] FP32 post-smoothing correction
  // coarse
  int32_t* cpos = nullptr;
  int32_t* cseg_blk = nullptr;
  int32_t* cchunk_ptr = nullptr;
  int32_t* cdst_ptr = nullptr;
  int64_t* cdst_idx = nullptr;
  double* cpart = nullptr;  // [nchunk][25]
  double* cband = nullptr;  // [P][2*cband+1][25] banded coarse matrix / factors
  double* cdinv = nullptr;  // [P][25]
  double* crhs = nullptr;   // [2][5P]
  float* cy32 = nullptr;    // [5P] FP32 copy of the coarse solution (mixed path)
  double* ainvT = nullptr;  // [5P][5P] explicit coarse inverse (transposed)
  bool pc_ready = false;
  int32_t wait_polls = seird::SOLVE_WAIT_POLLS_DEFAULT;  // seird_set_wait_limit
  // algorithmic bytes per kernel class since the step began (seird_stats.alg_bytes)
  double abytes[SEIRD_K_COUNT] = {};
  // launch shapes (options.autotune)
  int spmv_tb = 256, cgs_tile = 0, sms = 1;
  int ilu_ch = 2;     // dependency-load batch of the subdomain solves (options.autotune)
  int ilu_warps = 7;  // their consumer warps per CTA (7 or 3)
  int ilu_ring = seird::SOLVE_RING_FULL;  // and factor-ring blocks (two stages or one)
  bool tuned = false;
  double* tune_buf = nullptr;
  // GMRES restart cycle captured into a CUDA graph (options.graph)
  cudaGraphExec_t cycle_exec = nullptr;
  int cycle_m = 0;
  std::vector<int64_t> cycle_launches;  // kernels of the first j captured iterations, j <= m
  std::vector<double> cycle_bytes;      // [(m+1)][SEIRD_K_COUNT] their algorithmic bytes, cumulative
  int* cyc_ctl = nullptr;              // device [4]: iterations run, limit, outcome
  int* h_cyc = nullptr;                // pinned [8]: [0, 4) uploaded, [4, 8) read back
  bool eager_cycles = false;           // while the adjoint has J^T swapped in
  int32_t pc_age_steps = 0;  // time steps completed since the preconditioner was built
  bool jac_ready = false;
  // kernel-class timing (options.timing): (class, start event, end event) per launch group
  std::vector<cudaEvent_t> evpool;
  size_t ev_used = 0;
  std::vector<int> ev_class;
};
