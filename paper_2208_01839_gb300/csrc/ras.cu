// Restricted additive Schwarz preconditioner (Eq. RAS) with block-ILU(0)
// subdomain solves, and the coarse correction of Section 3.1 with the
// per-subdomain, per-compartment constant coarse space Z:
//   z = sum_p R_p^T D_p (L_p U_p)^{-1} R_p r  +  Z A_c^{-1} Z^T r,  A_c = Z^T J Z,
// applied additively or, as in Eq. RAS_2L, multiplicatively (the J Z blocks
// summed at set-up turn the second residual update into k_az_sub).
// One CTA per subdomain for the factorization and the solves; rows of one
// level of the ILU(0) dependency DAG are independent and run in parallel, with
// a barrier between stages, and the solve numbers a subdomain's solution
// entries by their position in the sweep.  The coarse matrix is block-banded
// (subdomains in reverse Cuthill-McKee order) and factored by block LU with 5x5
// pivot blocks inverted under partial pivoting, then inverted explicitly.
#include <cmath>

#include "kernels.cuh"

namespace seird {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

// |x| as an ordered integer key: for a value with its sign bit cleared, the
// bit pattern read as an integer grows with the magnitude (NaN above inf), so
// the pivot search runs on the integer pipe instead of GB300's narrow FP64 one.
__device__ __forceinline__ long long mag_key(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
__device__ __forceinline__ long long mag_key(float x) { return (long long)(__float_as_int(x) & 0x7fffffff); }
__device__ __forceinline__ bool key_ok(double, long long k) { return k != 0 && k <= 0x7ff0000000000000LL; }
__device__ __forceinline__ bool key_ok(float, long long k) { return k != 0 && k <= 0x7f800000LL; }

// Inverse of a 5x5 block by Gauss-Jordan with partial pivoting (largest |entry|
// of the column at or below the diagonal, ties to the lower row index), one
// warp: lane 5 r + c < 25 holds entry (r, c) of the block and of the identity
// it turns into the inverse, so each elimination step is two FP64 FMAs per
// lane.  Sets ERR_SINGULAR (2) on a zero (or NaN) pivot.
template <class T>
__device__ void warp_inv5(const T* __restrict__ D, T* __restrict__ out, int lane, int32_t* err) {
  const int r = lane / 5, c = lane - 5 * (lane / 5);
  const bool act = lane < 25;
  T a = act ? D[lane] : T(0);
  T b = (act && r == c) ? T(1) : T(0);
  bool sing = false;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    int piv = k;
    long long best = mag_key(__shfl_sync(FULL, a, 5 * k + k));
#pragma unroll
    for (int q = k + 1; q < 5; ++q) {
      const long long kq = mag_key(__shfl_sync(FULL, a, 5 * q + k));
      if (kq > best) {
        best = kq;
        piv = q;
      }
    }
    if (!key_ok(T(0), best)) sing = true;
    const int src = (r == k) ? 5 * piv + c : (r == piv ? 5 * k + c : lane);
    a = __shfl_sync(FULL, a, src & 31);
    b = __shfl_sync(FULL, b, src & 31);
    const T pinv = T(1) / __shfl_sync(FULL, a, 5 * k + k);
    if (r == k) {
      a *= pinv;
      b *= pinv;
    }
    const T f = __shfl_sync(FULL, a, (5 * r + k) & 31);
    const T pa = __shfl_sync(FULL, a, (5 * k + c) & 31);
    const T pb = __shfl_sync(FULL, b, (5 * k + c) & 31);
    if (act && r != k) {
      a = fmaT(-f, pa, a);
      b = fmaT(-f, pb, b);
    }
  }
  if (act) out[lane] = b;
  if (sing && lane == 0) atomicOr(err, 2);
}

template <class T>
__device__ __forceinline__ T* fvals(const RasDev& d);
template <>
__device__ __forceinline__ double* fvals<double>(const RasDev& d) { return d.fval; }
template <>
__device__ __forceinline__ float* fvals<float>(const RasDev& d) { return d.fval32; }
template <class T>
__device__ __forceinline__ T* dinvs(const RasDev& d);
template <>
__device__ __forceinline__ double* dinvs<double>(const RasDev& d) { return d.dinv; }
template <>
__device__ __forceinline__ float* dinvs<float>(const RasDev& d) { return d.dinv32; }
template <class T>
__device__ __forceinline__ T* ywk(const RasDev& d);
template <>
__device__ __forceinline__ double* ywk<double>(const RasDev& d) { return d.ywork; }
template <>
__device__ __forceinline__ float* ywk<float>(const RasDev& d) { return d.ywork32; }
template <class T>
__device__ __forceinline__ T* zwk(const RasDev& d);
template <>
__device__ __forceinline__ double* zwk<double>(const RasDev& d) { return d.zwork; }
template <>
__device__ __forceinline__ float* zwk<float>(const RasDev& d) { return d.zwork32; }

template <class T>
__device__ __forceinline__ const T* solve_fwd(const RasDev& d);
template <>
__device__ __forceinline__ const double* solve_fwd<double>(const RasDev& d) { return d.fL; }
template <>
__device__ __forceinline__ const float* solve_fwd<float>(const RasDev& d) { return d.fL32; }
template <class T>
__device__ __forceinline__ const T* solve_bwd(const RasDev& d);
template <>
__device__ __forceinline__ const double* solve_bwd<double>(const RasDev& d) { return d.bU; }
template <>
__device__ __forceinline__ const float* solve_bwd<float>(const RasDev& d) { return d.bU32; }

// Block ILU(k) of R_p J R_p^T on the set-up's pattern (ILU(0): the pattern of R_p J R_p^T;
// fill blocks start at zero), IKJ form, rows in forward-level order, in the arithmetic of T
// (FP64, or FP32 for the mixed-precision path).
template <class T, class TV>
__global__ void __launch_bounds__(256) k_ilu_factor(RasDev d, const TV* __restrict__ val, int32_t* err) {
  T* fval = fvals<T>(d);
  T* dinv = dinvs<T>(d);
  const int p = d.sd_sched[blockIdx.x];
  const int32_t r0 = d.sd_row0[p];
  const int32_t r1 = d.sd_row0[p + 1];
  const int64_t b0 = d.l_row_ptr[r0], b1 = d.l_row_ptr[r1];
  for (int64_t idx = threadIdx.x; idx < (b1 - b0) * 25; idx += blockDim.x) {
    const int64_t blk = b0 + idx / 25;
    const int e = (int)(idx % 25);
    const int32_t g = d.l_gblk[blk];  // -1: a fill block of ILU(k), zero before the factorisation
    fval[25 * blk + e] = g >= 0 ? (T)val[25 * (int64_t)g + e] : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int rr = lane / 5, cc = lane % 5;
  const int32_t L0 = d.sd_fwd_lev0[p];
  const int32_t nlev = d.sd_fwd_lev0[p + 1] - L0 - 1;
  for (int32_t lv = 0; lv < nlev; ++lv) {
    const int32_t s = d.fwd_lev[L0 + lv], e = d.fwd_lev[L0 + lv + 1];
    for (int32_t ri = s + warp; ri < e; ri += nw) {
      const int32_t i = d.fwd_order[r0 + ri];
      const int64_t R = (int64_t)r0 + i;
      const int64_t a0 = d.l_row_ptr[R], a1 = d.l_row_ptr[R + 1];
      for (int64_t a = a0; a < a1; ++a) {
        const int32_t k = d.l_col[a];
        if (k >= i) break;  // columns are sorted: the strictly lower blocks come first
        const T* Dk = dinv + 25 * ((int64_t)r0 + k);
        T* A = fval + 25 * a;
        T v = T(0);
        if (lane < 25) {
#pragma unroll
          for (int mm = 0; mm < 5; ++mm) v = fmaT(A[5 * rr + mm], Dk[5 * mm + cc], v);
        }
        __syncwarp();
        if (lane < 25) A[lane] = v;  // L_ik = A_ik U_kk^{-1}
        __syncwarp();
        for (int64_t u = d.upd_ptr[a]; u < d.upd_ptr[a + 1]; ++u) {
          const int64_t dst = d.upd[2 * u], src = d.upd[2 * u + 1];
          if (lane < 25) {  // A_ij -= L_ik U_kj, folded into the FMA chain
            T t = fval[25 * dst + lane];
#pragma unroll
            for (int mm = 0; mm < 5; ++mm) t = fmaT(-A[5 * rr + mm], fval[25 * src + 5 * mm + cc], t);
            fval[25 * dst + lane] = t;
          }
        }
        __syncwarp();
      }
      warp_inv5<T>(fval + 25 * d.l_diag[R], dinv + 25 * R, lane, err);
      __syncwarp();
    }
    __syncthreads();
  }
}

// ---- subdomain solves ---------------------------------------------------------
//
// The solve reads the factors from a copy in level order (SolvePlan): every
// level of the forward (then backward) sweep is one contiguous range of padded
// blocks (25 values and the block's local column in slot 25; 26 doubles or 28
// floats, so a block is a multiple of 16 bytes).  While a level computes, the
// next level's range is already in flight into the other half of a double
// buffer in shared memory (cp.async.bulk completing on an mbarrier), so the
// only global loads on a level's critical path are the solution entries of
// earlier levels.  Rows are mapped six to a warp (lane = 5 row + component), so
// the backward sweep's product with the inverted pivot block uses shuffles.

template <class T>
struct SolveBS;
template <>
struct SolveBS<double> {
  static constexpr int v = 26;
};
template <>
struct SolveBS<float> {
  static constexpr int v = 28;
};

__device__ __forceinline__ int col_of(double x) { return (int)__double_as_longlong(x); }
__device__ __forceinline__ int col_of(float x) { return __float_as_int(x); }
__device__ __forceinline__ void put_col(double* p, int c) { *p = __longlong_as_double((long long)c); }
__device__ __forceinline__ void put_col(float* p, int c) { *p = __int_as_float(c); }

template <class T>
__global__ void k_ilu_reorg(int64_t nblk, const int64_t* __restrict__ src, const int32_t* __restrict__ col,
                            const T* __restrict__ fval, const T* __restrict__ dinv, T* __restrict__ out) {
  constexpr int BS = SolveBS<T>::v;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nblk * BS;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g / BS;
    const int e = (int)(g - b * BS);
    if (e < 25) {
      const int64_t s = src[b];
      out[g] = s >= 0 ? fval[25 * s + e] : dinv[25 * (-1 - s) + e];
    } else if (e == 25) {
      put_col(out + g, col[b]);
    } else {
      out[g] = T(0);
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: gives up after `polls` polls (none when polls <= 0) and reports it
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int polls) {
  for (int it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// the wait for issued copies to land before a CTA exits: never shortened, so no bulk
// copy is in flight into the shared memory of a CTA that has left
constexpr int SOLVE_DRAIN_POLLS = 1 << 20;

// Stage data of one subdomain stream through two rings in shared memory: the
// factor blocks (SolveRing<T>::blocks) and the per-row records (SOLVE_RING_ROWS).
// Warp 7 is the producer: its lane 0 reads the level plan and issues the bulk
// copies of up to SOLVE_SLOTS stages ahead, as far as both rings have room;
// a stage's "full" mbarrier completes when its bytes have landed, and its
// "empty" mbarrier when the consumers are done with it.  Warps 0-6 consume
// the stages in order and meet at a named barrier after each one (the rows of
// a level depend on the rows of earlier levels).  A stage never wraps around a
// ring's end: the producer skips the tail.  Every wait is bounded; on a
// timeout the kernel sets bit 3 of *err, lets every issued copy land and
// returns.
// Ring of factor blocks: two stages (236 blocks: 49 KB in FP64, 26 KB in FP32) so that
// the next stage streams in while one is consumed, or one stage (118 blocks), which
// halves a CTA's shared memory so that more subdomains share an SM and hide each
// other's latency instead (SOLVE_RING_FULL / SOLVE_RING_HALF; a 354-block FP32 ring
// measured 6% slower).
constexpr int SOLVE_RING_ROWS = 2 * SOLVE_BUF_ROWS_DEV;
constexpr int SOLVE_SLOTS = 8;

__device__ __forceinline__ void mbar_init_count(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// named barrier 1 over the NCW consumer warps (the producer warp does not take part)
template <int NCW>
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * NCW) : "memory");
}

// NCW consumer warps (7 or 3) and one producer warp.  Seven consumers take up to 42
// rows of a stage in one round; three take 18, but their CTA of 128 threads needs half
// the registers, so where shared memory allows (the FP32 rings) twice as many
// subdomains run on an SM at once.  Every row's arithmetic is the same either way.
template <class T, class TZ, int CH, int NCW, int RB>
__global__ void __launch_bounds__(32 * (NCW + 1), NCW <= 3 ? 7 : 4)
    k_ilu_solve(RasDev d, const double* __restrict__ r, TZ* __restrict__ z, int32_t* err) {
  constexpr int BS = SolveBS<T>::v;
  constexpr int RR = SOLVE_RING_ROWS;
  constexpr int NS = SOLVE_SLOTS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[NS];
  __shared__ __align__(8) uint64_t empty[NS];
  __shared__ __align__(16) int4 info[RR];
  __shared__ int slot_vb[NS], slot_vr[NS], slot_n[NS];  // virtual ring starts and row count of a stage
  __shared__ int slot_k0[NS];                            // sweep position of a stage's first row
  __shared__ int abort_at;  // first stage at which a consumer warp's wait gave up (INT_MAX: none)
  T* ring = reinterpret_cast<T*>(smem_raw);
  const int p = d.sd_sched ? d.sd_sched[blockIdx.x] : (int)blockIdx.x;
  const int32_t r0 = d.sd_row0[p];
  T* y = ywk<T>(d) + 5 * (int64_t)r0;
  T* zz = zwk<T>(d) + 5 * (int64_t)r0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t LF = d.fwd.sd_lev0[p], nF = d.fwd.sd_lev0[p + 1] - LF - 1;
  const int32_t LB = d.bwd.sd_lev0[p], nB = d.bwd.sd_lev0[p + 1] - LB - 1;
  const int nstage = nF + nB;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init_count(&full[k], 1);
      mbar_init_count(&empty[k], 1);
    }
    abort_at = INT_MAX;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NCW) {
    // ---- producer: stage g < nF is forward level g, otherwise backward level
    // g - nF; it uses slot g % NS, whose barriers complete phase (g / NS) & 1 for it.
    if (lane != 0) return;
    const T* fL = solve_fwd<T>(d);
    const T* bU = solve_bwd<T>(d);
    int vb = 0, vr = 0, oldest = 0;  // ring heads (virtual, growing); oldest stage not known to be released
    int gi = 0;
    bool ok = true;
    for (; gi < nstage && ok; ++gi) {
      const bool fw = gi < nF;
      const SolvePlanDev& P = fw ? d.fwd : d.bwd;
      const int32_t lv = fw ? LF + gi : LB + gi - nF;
      const int32_t q0 = P.levpos[lv], q1 = P.levpos[lv + 1];
      const int64_t b0 = P.levblk[lv];
      const int nb = (int)(P.levblk[lv + 1] - b0), nr = q1 - q0;
      int sb = vb, sr = vr;
      if (sb % RB + nb > RB) sb += RB - sb % RB;
      if (sr % RR + nr > RR) sr += RR - sr % RR;
      // release stages (in order) until this one fits and its slot is free
      while (oldest < gi &&
             (gi - oldest >= NS || sb + nb - slot_vb[oldest % NS] > RB || sr + nr - slot_vr[oldest % NS] > RR)) {
        if (!mbar_wait(&empty[oldest % NS], (uint32_t)((oldest / NS) & 1), d.wait_polls) ||
            *(volatile int*)&abort_at != INT_MAX) {
          ok = false;
          break;
        }
        ++oldest;
      }
      if (!ok) break;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int sl = gi % NS;
      slot_vb[sl] = sb;
      slot_vr[sl] = sr;
      slot_n[sl] = nr;
      slot_k0[sl] = q0;
      const uint32_t bytes_b = (uint32_t)nb * BS * (uint32_t)sizeof(T);
      const uint32_t bytes_i = (uint32_t)nr * (uint32_t)sizeof(int4);
      mbar_arrive_tx(&full[sl], bytes_b + bytes_i);  // releases the slot fields above to the consumers
      if (bytes_b) bulk_g2s(ring + (size_t)(sb % RB) * BS, (fw ? fL : bU) + b0 * BS, bytes_b, &full[sl]);
      if (bytes_i) bulk_g2s(info + sr % RR, P.info + r0 + q0, bytes_i, &full[sl]);
      vb = sb + nb;
      vr = sr + nr;
    }
    if (!ok) atomicOr(err, 8);
    // every issued copy lands before the CTA can exit (the last stage issued on
    // each slot is the only one whose phase is still open)
    for (int k = gi - 1; k >= 0 && k >= gi - NS; --k)
      mbar_wait(&full[k % NS], (uint32_t)((k / NS) & 1), SOLVE_DRAIN_POLLS);
    return;
  }

  // ---- consumers (warps 0-6)
  // Solution entries are numbered by their position in the sweep: y (forward) and
  // z (backward) of position k live at 5 k in the subdomain's work arrays, so a
  // stage writes one contiguous run and reads the runs of earlier stages.  (A
  // shared-memory window of recent entries measured slower: the dependency loads
  // hit L1, and the window's shared memory comes out of L1.)
  const int rw = lane / 5, cpt = lane - 5 * rw;
  // A warp whose wait gives up skips the stage and records it; every consumer
  // reads abort_at after the named barrier that closes the stage, and only
  // values <= g (written before that barrier) end the loop at stage g, so all
  // consumer warps leave at the same stage.
  bool aborted = false;
  for (int g = 0; g < nstage; ++g) {
    const bool fw = g < nF;
    const int sl = g % NS;
    const bool landed = __all_sync(FULL, mbar_wait(&full[sl], (uint32_t)((g / NS) & 1), d.wait_polls));
    if (!landed && lane == 0) atomicMin(&abort_at, g);
    const T* B = ring + (size_t)(slot_vb[sl] % RB) * BS;
    const int4* inf = info + slot_vr[sl] % RR;
    const int nrows = landed ? slot_n[sl] : 0;
    const int k0 = slot_k0[sl];
    T* vec = fw ? y : zz;
    for (int qb = warp * 6; qb < nrows; qb += 6 * NCW) {
      const int q = qb + rw;
      const bool act = lane < 30 && q < nrows;
      int32_t st = 0, cn = 0, onode = -1;
      T acc = T(0), acc2 = T(0);
      if (act) {
        const int4 rec = inf[q];
        st = rec.y;
        cn = rec.z;
        onode = rec.w;
        // forward: r of the row's node; backward: the row's forward result
        acc = fw ? (T)r[5 * (int64_t)rec.x + cpt] : y[5 * rec.x + cpt];
      }
      // y_k -= sum L y_j (forward) or y_k - sum U z_j (backward, block 0 is the
      // inverted pivot).  The entries of CH blocks are loaded before any of their
      // FMAs, so a row waits for one memory latency per CH blocks, not per block.
      // A short row reloads its last block to fill the batch; a stage is bound by
      // its busiest warp's instruction chain, so the batch trades load rounds
      // against instructions (2.0M nodes: FP32 0.91 ms for 2 blocks against 0.96 /
      // 0.95 / 0.94 / 1.02 ms for 1 / 4 / 3 / 6; FP64 1.68 ms against 1.74 / 1.70 ms
      // for 1 / 3); the autotuner picks CH per context.  Block b of the row (counted
      // from its first product) goes to chain b % 2 whatever CH is: both chains
      // subtract, the slot of a batch's block u is fixed (u % 2), and after a batch
      // of odd size the two chains trade slots, so every CH gives the same sums in
      // the same order with no run-time choice of chain per FMA.
      const int32_t jb = fw ? 0 : 1;
      for (int32_t j = jb; j < cn; j += CH) {
        const int nb = min(CH, cn - j);
        T xv[CH][5];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const T* vk = vec + 5 * (int64_t)col_of(B[(st + j + min(u, nb - 1)) * BS + 25]);
#pragma unroll
          for (int mm = 0; mm < 5; ++mm) xv[u][mm] = vk[mm];
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          if (u < nb) {  // folded into two accumulator chains: no separate add per block
            const T* Lb = B + (st + j + u) * BS + 5 * cpt;
#pragma unroll
            for (int mm = 0; mm < 5; ++mm) {
              if (u & 1) acc2 = fmaT(-Lb[mm], xv[u][mm], acc2);
              else acc = fmaT(-Lb[mm], xv[u][mm], acc);
            }
          }
        }
        if (CH % 2 == 1) {  // the next batch starts on the other chain
          const T t = acc;
          acc = acc2;
          acc2 = t;
        }
      }
      // the chain that started from r (or y) and the other one; FP addition commutes, so
      // whichever register holds which chain the sum is the same (and -fma(a, b, c) =
      // fma(-a, b, -c) exactly, so this equals the r - sum_even - (sum_odd) of a chain that adds)
      acc += acc2;
      const int kq = k0 + q;  // this row's position
      T v = acc;
      if (!fw) {
        // z = U_kk^{-1} (...): the five partial results of the row sit in lanes 5 rw .. 5 rw + 4
        v = T(0);
        const T* Dv = B + st * BS + 5 * cpt;
#pragma unroll
        for (int mm = 0; mm < 5; ++mm) {
          const T am = __shfl_sync(FULL, acc, 5 * rw + mm);
          if (act) v = fmaT(Dv[mm], am, v);
        }
      }
      if (act) {
        vec[5 * (int64_t)kq + cpt] = v;
        if (!fw && onode >= 0) z[5 * (int64_t)onode + cpt] = (TZ)v;
      }
    }
    consumers_sync<NCW>();  // every row of this stage is written; the stage's ring space is free
    if (*(volatile int*)&abort_at <= g) {
      aborted = true;
      break;
    }
    if (tid == 0) mbar_arrive(&empty[sl]);
  }
  if (aborted && tid == 0) atomicOr(err, 8);
}

// ---- coarse space --------------------------------------------------------

// one warp per chunk of J blocks that belong to the same coarse block
template <class TV>
__global__ void k_coarse_chunks(int32_t nchunk, const int32_t* __restrict__ cptr, const int32_t* __restrict__ blk,
                                const TV* __restrict__ val, double* __restrict__ cpart) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= nchunk || lane >= 25) return;
  double s = 0.0;
  for (int32_t b = cptr[gw]; b < cptr[gw + 1]; ++b) s += (double)val[25 * (int64_t)blk[b] + lane];
  cpart[25 * gw + lane] = s;
}

__global__ void k_coarse_dst(int32_t ndst, const int32_t* __restrict__ dptr, const int64_t* __restrict__ didx,
                             const double* __restrict__ cpart, double* __restrict__ band) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 25 * (int64_t)ndst) return;
  const int64_t dd = g / 25;
  const int e = (int)(g - 25 * dd);
  double s = 0.0;
  for (int32_t c = dptr[dd]; c < dptr[dd + 1]; ++c) s += cpart[25 * (int64_t)c + e];
  band[25 * didx[dd] + e] = s;
}

__device__ __forceinline__ double* bblk(double* band, int bw, int ib, int jb) {
  return band + 25 * ((int64_t)ib * (2 * bw + 1) + (jb - ib + bw));
}

// block step kb: invert the pivot block, form the L column below it
__global__ void k_band_pivot(int P, int bw, int kb, double* band, double* cdinv, int32_t* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp == 0) warp_inv5<double>(bblk(band, bw, kb, kb), cdinv + 25 * (int64_t)kb, lane, err);
  __syncthreads();
  const double* Dk = cdinv + 25 * (int64_t)kb;
  const int rr = lane / 5, cc = lane % 5;
  const int last = min(P - 1, kb + bw);
  for (int ib = kb + 1 + warp; ib <= last; ib += nw) {
    double* A = bblk(band, bw, ib, kb);
    double v = 0.0;
    if (lane < 25) {
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) v = fma(A[5 * rr + mm], Dk[5 * mm + cc], v);
    }
    __syncwarp();
    if (lane < 25) A[lane] = v;
  }
}

// block step kb: trailing update A_ij -= L_ik A_kj for i, j in (kb, kb+bw]
__global__ void k_band_update(int P, int bw, int kb, double* band) {
  const int nb = min(bw, P - 1 - kb);
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t pair = g / 25;
  if (pair >= (int64_t)nb * nb) return;
  const int e = (int)(g - 25 * pair);
  const int ib = kb + 1 + (int)(pair / nb), jb = kb + 1 + (int)(pair % nb);
  const int rr = e / 5, cc = e % 5;
  const double* L = bblk(band, bw, ib, kb);
  const double* Ak = bblk(band, bw, kb, jb);
  double v = 0.0;
#pragma unroll
  for (int mm = 0; mm < 5; ++mm) v = fma(L[5 * rr + mm], Ak[5 * mm + cc], v);
  bblk(band, bw, ib, jb)[e] -= v;
}

// y <- A_c^{-1} y with the banded block LU factors (one CTA, y in shared memory).
// With unit != 0, CTA b solves for the unit vector e_b and writes row b of
// A_c^{-T} (= column b of A_c^{-1}) to yg + b*5P: the explicit inverse.
__global__ void k_band_solve(int P, int bw, const double* __restrict__ band, const double* __restrict__ cdinv,
                             double* __restrict__ yg, int unit) {
  extern __shared__ double ys[];
  const int tid = threadIdx.x, bd = blockDim.x;
  double* bandm = const_cast<double*>(band);
  if (unit) {
    for (int k = tid; k < 5 * P; k += bd) ys[k] = (k == (int)blockIdx.x) ? 1.0 : 0.0;
    yg += (int64_t)blockIdx.x * 5 * P;
  } else {
    for (int k = tid; k < 5 * P; k += bd) ys[k] = yg[k];
  }
  __syncthreads();
  for (int kb = unit ? (int)blockIdx.x / 5 : 0; kb < P; ++kb) {  // e_b is zero above block b/5
    const int nb = min(bw, P - 1 - kb);
    for (int t = tid; t < 5 * nb; t += bd) {
      const int ib = kb + 1 + t / 5, r = t % 5;
      const double* L = bblk(bandm, bw, ib, kb) + 5 * r;
      double v = 0.0;
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) v = fma(L[mm], ys[5 * kb + mm], v);
      ys[5 * ib + r] -= v;
    }
    __syncthreads();
  }
  for (int kb = P - 1; kb >= 0; --kb) {
    double tmp = 0.0;
    if (tid < 5) {
      const double* Dk = cdinv + 25 * (int64_t)kb + 5 * tid;
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) tmp = fma(Dk[mm], ys[5 * kb + mm], tmp);
    }
    __syncthreads();
    if (tid < 5) ys[5 * kb + tid] = tmp;
    __syncthreads();
    const int nb = min(bw, kb);
    for (int t = tid; t < 5 * nb; t += bd) {
      const int ib = kb - 1 - t / 5, r = t % 5;
      const double* Ub = bblk(bandm, bw, ib, kb) + 5 * r;
      double v = 0.0;
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) v = fma(Ub[mm], ys[5 * kb + mm], v);
      ys[5 * ib + r] -= v;
    }
    __syncthreads();
  }
  for (int k = tid; k < 5 * P; k += bd) yg[k] = ys[k];
}

// Explicit inverse, one CTA per block column b of the identity: L U X = E_b for
// its five columns at once (ys[row][c] in shared memory), so a step over one
// block row of the band is 25 independent dot products per band block.  X goes
// to rows 5b..5b+4 of AinvT (row j of AinvT = column j of A_c^{-1}).
__global__ void __launch_bounds__(256) k_band_inv(int P, int bw, const double* __restrict__ band,
                                                  const double* __restrict__ cdinv, double* __restrict__ ainvT) {
  extern __shared__ double ys[];
  const int tid = threadIdx.x, bd = blockDim.x;
  const int b = blockIdx.x;
  double* bandm = const_cast<double*>(band);
  for (int k = tid; k < 25 * P; k += bd) ys[k] = (k / 5 == 5 * b + k % 5) ? 1.0 : 0.0;
  __syncthreads();
  for (int kb = b; kb < P; ++kb) {  // E_b is zero above block row b
    const int nb = min(bw, P - 1 - kb);
    for (int t = tid; t < 25 * nb; t += bd) {
      const int ib = kb + 1 + t / 25, r = (t / 5) % 5, cc = t % 5;
      const double* L = bblk(bandm, bw, ib, kb) + 5 * r;
      double v = 0.0;
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) v = fma(L[mm], ys[5 * (5 * kb + mm) + cc], v);
      ys[5 * (5 * ib + r) + cc] -= v;
    }
    __syncthreads();
  }
  for (int kb = P - 1; kb >= 0; --kb) {
    double tmp = 0.0;
    if (tid < 25) {
      const double* Dk = cdinv + 25 * (int64_t)kb + 5 * (tid / 5);
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) tmp = fma(Dk[mm], ys[5 * (5 * kb + mm) + tid % 5], tmp);
    }
    __syncthreads();
    if (tid < 25) ys[5 * (5 * kb + tid / 5) + tid % 5] = tmp;
    __syncthreads();
    const int nb = min(bw, kb);
    for (int t = tid; t < 25 * nb; t += bd) {
      const int ib = kb - 1 - t / 25, r = (t / 5) % 5, cc = t % 5;
      const double* Ub = bblk(bandm, bw, ib, kb) + 5 * r;
      double v = 0.0;
#pragma unroll
      for (int mm = 0; mm < 5; ++mm) v = fma(Ub[mm], ys[5 * (5 * kb + mm) + cc], v);
      ys[5 * (5 * ib + r) + cc] -= v;
    }
    __syncthreads();
  }
  const int64_t nc = 5 * (int64_t)P;
  for (int k = tid; k < 25 * P; k += bd) ainvT[(5 * b + k % 5) * nc + k / 5] = ys[k];
}

// part[chunk][i] = sum_{j in chunk} AinvT[j][i] rc[j]  (AinvT row j = column j of A_c^{-1})
constexpr int GEMV_CHUNK = 64;
__global__ void k_coarse_gemv_part(int nc, const double* __restrict__ AinvT, const double* __restrict__ rc,
                                   double* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * GEMV_CHUNK;
  const int j1 = min(nc, j0 + GEMV_CHUNK);
  if (i >= nc) return;
  double s = 0.0;
  for (int j = j0; j < j1; ++j) s = fma(AinvT[(int64_t)j * nc + i], rc[j], s);
  part[(int64_t)blockIdx.y * nc + i] = s;
}

__global__ void k_coarse_gemv_sum(int nc, int nchunk, const double* __restrict__ part, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double s = 0.0;
  for (int q = 0; q < nchunk; ++q) s += part[(int64_t)q * nc + i];
  y[i] = s;
}

// crhs[cpos[p]] = Z^T r : sums of r over the nodes owned by p, per compartment
__global__ void __launch_bounds__(256) k_coarse_restrict(const int32_t* __restrict__ own_ptr,
                                                         const int32_t* __restrict__ cpos,
                                                         const double* __restrict__ r, double* __restrict__ crhs) {
  __shared__ double sh[5][8];
  const int p = blockIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  for (int32_t i = own_ptr[p] + threadIdx.x; i < own_ptr[p + 1]; i += blockDim.x)
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] += r[5 * (int64_t)i + c];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) sh[c][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    crhs[5 * (int64_t)cpos[p] + threadIdx.x] = v;
  }
}

// z += Z y : every node adds its subdomain's coarse value
template <class TZ>
__global__ void k_coarse_prolong_add(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ cpos,
                                     const double* __restrict__ y, TZ* __restrict__ z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 5 * n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g / 5;
    z[g] = (TZ)((double)z[g] + y[5 * (int64_t)cpos[owner[i]] + (g - 5 * i)]);
  }
}

// z += Z y in FP32 (mixed path): every node adds its unit's coarse value
__global__ void k_coarse_prolong_add32(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ cpos,
                                       const float* __restrict__ y, float* __restrict__ z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 5 * n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g / 5;
    z[g] += y[5 * (int64_t)cpos[owner[i]] + (g - 5 * i)];
  }
}

__global__ void k_coarse_to_f32(int n, const double* __restrict__ y, float* __restrict__ y32) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) y32[g] = (float)y[g];
}

}  // namespace

void launch_ilu_factor(const RasDev& d, const double* val, const float* val32, int32_t* err, bool fp32,
                       cudaStream_t s) {
  if (fp32) k_ilu_factor<float, float><<<d.P, 256, 0, s>>>(d, val32, err);
  else k_ilu_factor<double, double><<<d.P, 256, 0, s>>>(d, val, err);
  count_launch();
}

size_t solve_smem(bool fp32, int ring_blocks) {
  return fp32 ? (size_t)ring_blocks * SolveBS<float>::v * sizeof(float)
              : (size_t)ring_blocks * SolveBS<double>::v * sizeof(double);
}

void launch_ilu_reorg(const RasDev& d, int64_t nfwd, int64_t nbwd, const int64_t* fsrc, const int32_t* fcol,
                      const int64_t* bsrc, const int32_t* bcol, bool fp32, cudaStream_t s) {
  const int grid = 152 * 8;
  if (fp32) {
    k_ilu_reorg<float><<<grid, 256, 0, s>>>(nfwd, fsrc, fcol, d.fval32, d.dinv32, d.fL32);
    k_ilu_reorg<float><<<grid, 256, 0, s>>>(nbwd, bsrc, bcol, d.fval32, d.dinv32, d.bU32);
  } else {
    k_ilu_reorg<double><<<grid, 256, 0, s>>>(nfwd, fsrc, fcol, d.fval, d.dinv, d.fL);
    k_ilu_reorg<double><<<grid, 256, 0, s>>>(nbwd, bsrc, bcol, d.fval, d.dinv, d.bU);
  }
  count_launch();
  count_launch();
}

// CTAs of one solve variant that the GPU holds at once (SMs x resident CTAs per SM), found
// once per variant; 0 if the occupancy query fails (the launch order is then always used)
template <class T, int CH, int NCW, int RB>
int solve_slots(size_t sm) {
  static const int slots = [sm] {
    int dev = 0, nsm = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ilu_solve<T, T, CH, NCW, RB>, 32 * (NCW + 1), sm) !=
            cudaSuccess) {
      (void)cudaGetLastError();  // the query's own error: nothing was launched
      return 0;
    }
    return nsm * nb;
  }();
  return slots;
}

// The longest-first launch order pays when the subdomain CTAs come in several waves
// (18.4M nodes, 4096 subdomains: 7.5% off the solve).  When every CTA is resident from
// the start it only decides which CTAs share an SM, and the natural order measured
// slightly better (2.0M nodes, 512 subdomains: 2.5%), so a single wave keeps it.
template <class T, int CH, int NCW, int RB>
void launch_ilu_solve_c(const RasDev& d, const double* r, T* z, int32_t* err, cudaStream_t s) {
  const size_t sm = solve_smem(sizeof(T) == 4, RB);
  RasDev dl = d;
  if (d.P <= solve_slots<T, CH, NCW, RB>(sm)) dl.sd_sched = nullptr;
  k_ilu_solve<T, T, CH, NCW, RB><<<d.P, 32 * (NCW + 1), sm, s>>>(dl, r, z, err);
}

template <class T, int NCW, int RB>
void launch_ilu_solve_w(const RasDev& d, const double* r, T* z, int32_t* err, cudaStream_t s, int ch) {
  switch (ch) {
    case 1: launch_ilu_solve_c<T, 1, NCW, RB>(d, r, z, err, s); break;
    case 3: launch_ilu_solve_c<T, 3, NCW, RB>(d, r, z, err, s); break;
    case 4: launch_ilu_solve_c<T, 4, NCW, RB>(d, r, z, err, s); break;
    default: launch_ilu_solve_c<T, 2, NCW, RB>(d, r, z, err, s); break;
  }
  count_launch();
}

template <class T>
void launch_ilu_solve_t(const RasDev& d, const double* r, T* z, int32_t* err, cudaStream_t s) {
  const bool half = d.solve_ring == SOLVE_RING_HALF;
  if (d.solve_warps == 3) {
    if (half) launch_ilu_solve_w<T, 3, SOLVE_RING_HALF>(d, r, z, err, s, d.solve_ch);
    else launch_ilu_solve_w<T, 3, SOLVE_RING_FULL>(d, r, z, err, s, d.solve_ch);
  } else {
    if (half) launch_ilu_solve_w<T, 7, SOLVE_RING_HALF>(d, r, z, err, s, d.solve_ch);
    else launch_ilu_solve_w<T, 7, SOLVE_RING_FULL>(d, r, z, err, s, d.solve_ch);
  }
}

void launch_ilu_solve(const RasDev& d, const double* r, double* z, int32_t* err, cudaStream_t s) {
  launch_ilu_solve_t<double>(d, r, z, err, s);
}

void launch_ilu_solve32(const RasDev& d, const double* r, float* z, int32_t* err, cudaStream_t s) {
  launch_ilu_solve_t<float>(d, r, z, err, s);
}

template <class T, int NCW, int RB>
void solve_attrs() {
  const int smem = (int)solve_smem(sizeof(T) == 4, RB);
  cudaFuncSetAttribute(k_ilu_solve<T, T, 1, NCW, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_ilu_solve<T, T, 2, NCW, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_ilu_solve<T, T, 3, NCW, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_ilu_solve<T, T, 4, NCW, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  // the resident-CTA counts, found here (at context creation) rather than in a captured launch
  (void)solve_slots<T, 1, NCW, RB>(smem);
  (void)solve_slots<T, 2, NCW, RB>(smem);
  (void)solve_slots<T, 3, NCW, RB>(smem);
  (void)solve_slots<T, 4, NCW, RB>(smem);
}
template <class T>
void solve_attrs_all() {
  solve_attrs<T, 7, SOLVE_RING_FULL>();
  solve_attrs<T, 3, SOLVE_RING_FULL>();
  solve_attrs<T, 7, SOLVE_RING_HALF>();
  solve_attrs<T, 3, SOLVE_RING_HALF>();
}

void launch_coarse_assemble(const CoarseDev& c, const double* val, const float* val32, cudaStream_t s) {
  const int64_t W = 2 * (int64_t)c.band + 1;
  cudaMemsetAsync(c.cband, 0, sizeof(double) * 25 * W * c.P, s);
  const int g = (int)((32 * (int64_t)c.nchunk + 255) / 256);
  if (val) k_coarse_chunks<double><<<g, 256, 0, s>>>(c.nchunk, c.cchunk_ptr, c.cseg_blk, val, c.cpart);
  else k_coarse_chunks<float><<<g, 256, 0, s>>>(c.nchunk, c.cchunk_ptr, c.cseg_blk, val32, c.cpart);
  k_coarse_dst<<<(int)((25 * (int64_t)c.ndst + 255) / 256), 256, 0, s>>>(c.ndst, c.cdst_ptr, c.cdst_idx, c.cpart,
                                                                          c.cband);
  count_launch();
  count_launch();
}

void launch_coarse_factor(const CoarseDev& c, int32_t* err, cudaStream_t s) {
  for (int kb = 0; kb < c.P; ++kb) {
    k_band_pivot<<<1, 256, 0, s>>>(c.P, c.band, kb, c.cband, c.cdinv, err);
    count_launch();
    const int nb = std::min(c.band, c.P - 1 - kb);
    if (nb > 0) {
      const int64_t th = 25 * (int64_t)nb * nb;
      k_band_update<<<(int)((th + 255) / 256), 256, 0, s>>>(c.P, c.band, kb, c.cband);
      count_launch();
    }
  }
  if (c.ainvT) {  // explicit inverse through the banded factors
    if (25 * (size_t)c.P * sizeof(double) <= 227 * 1024) {  // a block column of five unit vectors per CTA
      k_band_inv<<<c.P, 256, 25 * sizeof(double) * c.P, s>>>(c.P, c.band, c.cband, c.cdinv, c.ainvT);
    } else {  // one unit vector per CTA
      k_band_solve<<<5 * c.P, 256, sizeof(double) * 5 * c.P, s>>>(c.P, c.band, c.cband, c.cdinv, c.ainvT, 1);
    }
    count_launch();
  }
}

// y = A_c^{-1} Z^T r (left in crhs + 5P with the explicit inverse, in crhs otherwise)
void launch_coarse_solve(const CoarseDev& c, const double* r, cudaStream_t s) {
  k_coarse_restrict<<<c.P, 256, 0, s>>>(c.own_ptr, c.cpos, r, c.crhs);
  count_launch();
  const int nc = 5 * c.P;
  if (c.ainvT) {
    const int nchunk = (nc + GEMV_CHUNK - 1) / GEMV_CHUNK;
    k_coarse_gemv_part<<<dim3((nc + 127) / 128, nchunk), 128, 0, s>>>(nc, c.ainvT, c.crhs, c.cpart);
    k_coarse_gemv_sum<<<(nc + 127) / 128, 128, 0, s>>>(nc, nchunk, c.cpart, c.crhs + nc);
    count_launch();
    count_launch();
  } else {
    k_band_solve<<<1, 512, sizeof(double) * nc, s>>>(c.P, c.band, c.cband, c.cdinv, c.crhs, 0);
    count_launch();
  }
}

// z += Z y for the y of the last launch_coarse_solve
template <class TZ>
void launch_coarse_prolong(const CoarseDev& c, int64_t n, TZ* z, cudaStream_t s) {
  const int nc = 5 * c.P;
  int64_t g = (5 * n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  k_coarse_prolong_add<TZ><<<(int)g, 256, 0, s>>>(n, c.owner, c.cpos, c.ainvT ? c.crhs + nc : c.crhs, z);
  count_launch();
}
template void launch_coarse_prolong<double>(const CoarseDev&, int64_t, double*, cudaStream_t);

void launch_coarse_y32(const CoarseDev& c, cudaStream_t s) {
  const int nc = 5 * c.P;
  k_coarse_to_f32<<<(nc + 255) / 256, 256, 0, s>>>(nc, c.ainvT ? c.crhs + nc : c.crhs, c.y32);
  count_launch();
}

void launch_coarse_prolong32(const CoarseDev& c, int64_t n, float* z, cudaStream_t s) {
  int64_t g = (5 * n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  k_coarse_prolong_add32<<<(int)g, 256, 0, s>>>(n, c.owner, c.cpos, c.y32, z);
  count_launch();
}

template <class TZ>
void launch_coarse_apply_add(const CoarseDev& c, int64_t n, const double* r, TZ* z, cudaStream_t s) {
  launch_coarse_solve(c, r, s);
  launch_coarse_prolong<TZ>(c, n, z, s);
}
template void launch_coarse_apply_add<double>(const CoarseDev&, int64_t, const double*, double*, cudaStream_t);

// A Z segments: azval[s] = sum of the J blocks of segment s (one thread per entry)
template <class TV, class TA>
__global__ void k_az_build(int64_t nseg, const int32_t* __restrict__ az_blk, const TV* __restrict__ val,
                           TA* __restrict__ azval) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 25 * nseg) return;
  const int64_t s = g / 25;
  const int e = (int)(g - 25 * s);
  double acc = 0.0;
  for (int32_t b = az_blk[s]; b < az_blk[s + 1]; ++b) acc += (double)val[25 * (int64_t)b + e];
  azval[g] = (TA)acc;
}

// t -= (A Z) y for the coarse solution y (cpos order): one thread per scalar row
template <class TA>
__global__ void k_az_sub(int64_t n, const int64_t* __restrict__ az_ptr, const int32_t* __restrict__ az_unit,
                         const int32_t* __restrict__ cpos, const TA* __restrict__ azval,
                         const double* __restrict__ y, double* __restrict__ t) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 5 * n) return;
  const int64_t i = g / 5;
  const int rr = (int)(g - 5 * i);
  double acc = 0.0;
  for (int64_t s = az_ptr[i]; s < az_ptr[i + 1]; ++s) {
    const TA* A = azval + 25 * s + 5 * rr;
    const double* ys = y + 5 * (int64_t)cpos[az_unit[s]];
#pragma unroll
    for (int mm = 0; mm < 5; ++mm) acc = fma((double)A[mm], ys[mm], acc);
  }
  t[g] -= acc;
}

// the same with FP32 products for the mixed path (its result feeds an FP32 subdomain solve)
__global__ void k_az_sub32(int64_t n, const int64_t* __restrict__ az_ptr, const int32_t* __restrict__ az_unit,
                           const int32_t* __restrict__ cpos, const float* __restrict__ azval,
                           const float* __restrict__ y, double* __restrict__ t) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 5 * n) return;
  const int64_t i = g / 5;
  const int rr = (int)(g - 5 * i);
  float acc = 0.0f;
  for (int64_t s = az_ptr[i]; s < az_ptr[i + 1]; ++s) {
    const float* A = azval + 25 * s + 5 * rr;
    const float* ys = y + 5 * (int64_t)cpos[az_unit[s]];
#pragma unroll
    for (int mm = 0; mm < 5; ++mm) acc = fmaf(A[mm], ys[mm], acc);
  }
  t[g] -= (double)acc;
}

void launch_az_build(int64_t nseg, const int32_t* az_blk, const double* val, const float* val32, double* azval,
                     float* azval32, bool fp32, cudaStream_t s) {
  const unsigned g = (unsigned)((25 * nseg + 255) / 256);
  if (fp32) k_az_build<float, float><<<g, 256, 0, s>>>(nseg, az_blk, val32, azval32);
  else k_az_build<double, double><<<g, 256, 0, s>>>(nseg, az_blk, val, azval);
  count_launch();
}

void launch_az_sub(const CoarseDev& c, int64_t n, const int64_t* az_ptr, const int32_t* az_unit,
                   const double* azval, const float* azval32, bool fp32, double* t, cudaStream_t s) {
  const double* y = c.ainvT ? c.crhs + 5 * (int64_t)c.P : c.crhs;
  const unsigned g = (unsigned)((5 * n + 255) / 256);
  if (fp32) k_az_sub32<<<g, 256, 0, s>>>(n, az_ptr, az_unit, c.cpos, azval32, c.y32, t);
  else k_az_sub<double><<<g, 256, 0, s>>>(n, az_ptr, az_unit, c.cpos, azval, y, t);
  count_launch();
}

void coarse_init() {
  cudaFuncSetAttribute(k_band_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_band_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  solve_attrs_all<double>();
  solve_attrs_all<float>();
}

}  // namespace seird
