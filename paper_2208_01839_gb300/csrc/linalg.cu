// BSR SpMV and the vector kernels of restarted right-preconditioned (F)GMRES
// with CGS2 orthogonalisation (Section 3.2: GMRES with right preconditioning;
// FGMRES when the preconditioner varies).  FP64 accumulation throughout;
// reductions are two-stage (per-CTA partials, then one CTA in fixed order), so
// every result is bitwise reproducible run to run.
#include <cmath>

#include "kernels.cuh"

namespace seird {

namespace {

constexpr int NVMAX = 65;  // restart <= 64 -> at most 65 basis vectors

__device__ __forceinline__ double ld_val(const double* p) { return __ldg(p); }
__device__ __forceinline__ double ld_val(const float* p) { return (double)__ldg(p); }

// y = A x (b == NULL) or y = b - A x, 5x5 blocks.  One thread per scalar output row (block
// row i, row r): all 32 lanes of every warp do useful FP64 work, 25 FMA per block per 5 threads.
template <class VT>
__global__ void __launch_bounds__(512) k_bsr_spmv(int64_t nrow, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                  const double* __restrict__ x, const double* __restrict__ b,
                                                  double* __restrict__ y) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 5 * nrow) return;
  const int64_t i = g / 5;
  const int r = (int)(g - 5 * i);
  const int32_t k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
  double acc = 0.0;
  for (int32_t k = k0; k < k1; ++k) {
    const int64_t j = __ldg(col + k);
    const VT* v = val + 25 * (int64_t)k + 5 * r;
    const double* xj = x + 5 * j;
    acc = fma(ld_val(v + 0), __ldg(xj + 0), acc);
    acc = fma(ld_val(v + 1), __ldg(xj + 1), acc);
    acc = fma(ld_val(v + 2), __ldg(xj + 2), acc);
    acc = fma(ld_val(v + 3), __ldg(xj + 3), acc);
    acc = fma(ld_val(v + 4), __ldg(xj + 4), acc);
  }
  y[g] = b ? b[g] - acc : acc;
}

// Mixed-precision SpMV: FP32 values and FP32 input, FP32 arithmetic, FP64 output (y = A x,
// or y = b - A x when b != NULL).
__global__ void __launch_bounds__(512) k_bsr_spmv32(int64_t nrow, const int32_t* __restrict__ rp,
                                                    const int32_t* __restrict__ col, const float* __restrict__ val,
                                                    const float* __restrict__ x, const double* __restrict__ b,
                                                    double* __restrict__ y) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= 5 * nrow) return;
  const int64_t i = g / 5;
  const int r = (int)(g - 5 * i);
  const int32_t k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
  float acc = 0.f;
  for (int32_t k = k0; k < k1; ++k) {
    const int64_t j = __ldg(col + k);
    const float* v = val + 25 * (int64_t)k + 5 * r;
    const float* xj = x + 5 * j;
#pragma unroll
    for (int c = 0; c < 5; ++c) acc = fmaf(__ldg(v + c), __ldg(xj + c), acc);
  }
  y[g] = b ? b[g] - (double)acc : (double)acc;
}

// x += sum_k coef[k] Z_k with FP32 Z: the sum is formed in FP32, added in FP64
__global__ void k_multi_axpy32(int64_t len, int nv, const float* __restrict__ Z, int64_t ld,
                               const double* __restrict__ coef, double* __restrict__ x) {
  __shared__ float cs[NVMAX];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = (float)coef[k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int k = 0; k < nv; ++k) v = fmaf(cs[k], Z[k * ld + i], v);
    x[i] += (double)v;
  }
}

// valT = J^T on the same (structurally symmetric) block pattern: block k = (i,j)
// of J^T is the transpose of block tpos[k] = (j,i) of J
__global__ void k_bsr_transpose(int64_t nnzb, const int32_t* __restrict__ tpos, const double* __restrict__ val,
                                double* __restrict__ valT) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 25 * nnzb;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = g / 25;
    const int e = (int)(g - 25 * k), rr = e / 5, cc = e % 5;
    valT[g] = val[25 * (int64_t)tpos[k] + 5 * cc + rr];
  }
}

// *flag |= 1 when a and b differ in any bit pattern (so NaNs and signed zeros count as they are stored)
__global__ void k_differs(int64_t len, const double* __restrict__ a, const double* __restrict__ b, int* flag) {
  bool d = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    d |= __double_as_longlong(a[i]) != __double_as_longlong(b[i]);
  if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_add32(int64_t len, const float* __restrict__ u, float* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += u[i];
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// partial[cta] = sum over the CTA's slice of x^2
__global__ void __launch_bounds__(256) k_norm2_partial(int64_t len, const double* __restrict__ x,
                                                       double* __restrict__ partial) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    s += v * v;
  }
  s = block_sum<256>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[k] (+)= sum_cta partial[cta * stride + k], k < nv; fixed order
__global__ void k_reduce_cols(int grid, int nv, int stride, const double* __restrict__ partial, double* out,
                              int add) {
  __shared__ double sh[8];
  for (int k = 0; k < nv; ++k) {
    double s = 0.0;
    for (int c = threadIdx.x; c < grid; c += blockDim.x) s += partial[(int64_t)c * stride + k];
    s = block_sum<256>(s, sh);
    if (threadIdx.x == 0) out[k] = add ? out[k] + s : s;
  }
}

constexpr int KPW = (NVMAX + 7) / 8;  // dot products per warp

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  const int n = valid ? 8 : 0;  // src-size 0: nothing is read, the destination is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// CGS passes with double-buffered tiles: while tile t is consumed from shared
// memory, the basis entries (and w) of tile t+1 stream in through cp.async, so
// the FP64 pipe does not wait for the loads.  T entries per tile (256, or 128
// when many basis vectors would not fit twice).
// mode 0: partial[cta][k] = sum V_k . w ; mode 1: w -= V h, then the dots with w_new
template <int MODE, int T>
__global__ void __launch_bounds__(256) k_cgs_db(int64_t len, int nv, const double* __restrict__ V, int64_t ld,
                                                const double* __restrict__ h, double* __restrict__ w,
                                                double* __restrict__ partial) {
  extern __shared__ double smem[];
  double* hs = smem;                 // [NVMAX + 7]
  double* wt = hs + NVMAX + 7;       // [T] current w tile (after the update)
  double* bufs = wt + T;             // [2][nv + 1][T]: basis tiles and the incoming w tile
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nvb = nv + 1;
  if (MODE == 1)
    for (int k = tid; k < nv; k += blockDim.x) hs[k] = h[k];
  double acc[KPW];
#pragma unroll
  for (int q = 0; q < KPW; ++q) acc[q] = 0.0;
  const int64_t ntile = (len + T - 1) / T;
  auto load = [&](int64_t tile, int b) {
    double* dst = bufs + (size_t)b * nvb * T;
    const int64_t base = tile * T;
    for (int idx = tid; idx < nvb * T; idx += blockDim.x) {
      const int k = idx / T, e = idx - k * T;
      const int64_t i = base + e;
      const bool ok = i < len;
      const double* src = (k < nv ? V + k * ld : w) + (ok ? i : 0);
      cp_async8(dst + idx, src, ok);
    }
  };
  int64_t tile = blockIdx.x;
  if (tile < ntile) load(tile, 0);
  cp_async_commit();
  for (int b = 0; tile < ntile; tile += gridDim.x, b ^= 1) {
    if (tile + gridDim.x < ntile) load(tile + gridDim.x, b ^ 1);
    cp_async_commit();
    cp_async_wait1();  // the current tile's group has landed (this thread's copies)
    __syncthreads();   // ... and everyone else's
    const double* Vt = bufs + (size_t)b * nvb * T;
    const double* wsrc = Vt + (size_t)nv * T;
    for (int e = tid; e < T; e += blockDim.x) {
      double wi = wsrc[e];
      if (MODE == 1) {
        for (int k = 0; k < nv; ++k) wi = fma(-hs[k], Vt[k * T + e], wi);
        const int64_t i = tile * T + e;
        if (i < len) w[i] = wi;
      }
      wt[e] = wi;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < KPW; ++q) {
      const int k = wp + 8 * q;
      if (k < nv) {
        double s = acc[q];
#pragma unroll
        for (int e = lane; e < T; e += 32) s = fma(Vt[k * T + e], wt[e], s);
        acc[q] = s;
      }
    }
    __syncthreads();  // buffer b is refilled two tiles later
  }
#pragma unroll
  for (int q = 0; q < KPW; ++q) {
    const int k = wp + 8 * q;
    double s = acc[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0 && k < nv) partial[blockIdx.x * (int64_t)NVMAX + k] = s;
  }
}

// tile entries per CTA step: the caller's choice (128 or 256; 0 = by depth), 128 whenever
// 256 would not fit twice in shared memory
inline int cgs_tile(int nv, int want = 0) {
  if (nv > 27) return 128;
  return want == 128 ? 128 : 256;
}
inline size_t cgs_db_smem(int nv, int T) { return sizeof(double) * (NVMAX + 7 + T + 2 * (size_t)(nv + 1) * T); }

// second CGS pass update and ||w||^2 without staging: every thread needs only its
// own entries of the basis vectors, so they go straight to registers
__global__ void __launch_bounds__(256) k_cgs_update_norm(int64_t len, int nv, const double* __restrict__ V,
                                                         int64_t ld, const double* __restrict__ h,
                                                         double* __restrict__ w, double* __restrict__ partial) {
  __shared__ double hs[NVMAX];
  __shared__ double sh[8];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  double nrm = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    double a0 = w[i], a1 = 0.0;
    int k = 0;
    for (; k + 1 < nv; k += 2) {
      a0 = fma(-hs[k], __ldg(V + k * ld + i), a0);
      a1 = fma(-hs[k + 1], __ldg(V + (k + 1) * ld + i), a1);
    }
    if (k < nv) a0 = fma(-hs[k], __ldg(V + k * ld + i), a0);
    const double wi = a0 + a1;
    w[i] = wi;
    nrm = fma(wi, wi, nrm);
  }
  nrm = block_sum<256>(nrm, sh);
  if (threadIdx.x == 0) partial[blockIdx.x * (int64_t)NVMAX] = nrm;
}

// y = x * a (invert: a := 1/a), a read from device memory; a == 0 gives y = 0
__global__ void k_scale(int64_t len, const double* __restrict__ x, const double* __restrict__ ap, int invert,
                        double* __restrict__ y) {
  double a = *ap;
  if (invert) a = a != 0.0 ? 1.0 / a : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void k_axpby(int64_t len, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

// x += sum_k coef[k] Z_k
__global__ void k_multi_axpy(int64_t len, int nv, const double* __restrict__ Z, int64_t ld,
                             const double* __restrict__ coef, double* __restrict__ x) {
  __shared__ double cs[NVMAX];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = coef[k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    double v = x[i];
    for (int k = 0; k < nv; ++k) v = fma(cs[k], Z[k * ld + i], v);
    x[i] = v;
  }
}

// GMRES small state layout in gm (ldh = restart+1):
//   H[ldh*restart] column-major (H[row + ldh*col]), cs[restart], sn[restart], g[ldh], y[restart]
// Column j of H gets hcol[0..j] and hnext; previous rotations are applied, a new
// rotation annihilates H[j+1, j]; |g[j+1]| (the residual norm) goes to *out_res.
// In a captured restart cycle (cc.ctl != NULL) the kernel also takes the convergence
// decision of the iteration: cc.ctl[0] = iterations run, cc.ctl[2] = outcome (0 go on,
// 1 converged or breakdown, 2 past dtol or not finite), cc.ctl[1] = iteration limit of
// the cycle; cc.tol = {tolerance, dtol * ||b||}.  It arms the conditional node of the
// next iteration (cc.next) only while the outcome is 0 and the limit is not reached.
__global__ void k_givens(int j, double* gm, const double* __restrict__ h1, const double* __restrict__ h2,
                         const double* __restrict__ hnext_sq, int ldh, double* out_res, CycleCtl cc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int restart = ldh - 1;
  double* H = gm;
  double* cs = H + (int64_t)ldh * restart;
  double* sn = cs + restart;
  double* g = sn + restart;
  double col[NVMAX];
  for (int k = 0; k <= j; ++k) col[k] = h1[k] + h2[k];  // CGS2: both passes' coefficients
  const double hn = sqrt(fmax(*hnext_sq, 0.0));
  col[j + 1] = hn;
  for (int k = 0; k < j; ++k) {
    const double a = col[k], b = col[k + 1];
    col[k] = cs[k] * a + sn[k] * b;
    col[k + 1] = -sn[k] * a + cs[k] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double rr = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (rr != 0.0) {
    c = a / rr;
    s = b / rr;
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = rr;
  col[j + 1] = 0.0;
  for (int k = 0; k <= j + 1; ++k) H[k + (int64_t)ldh * j] = col[k];
  const double gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -s * gj;
  out_res[0] = fabs(g[j + 1]);
  out_res[1] = hn;
  if (cc.ctl) {
    const double res = fabs(g[j + 1]);
    int outcome = 0;
    if (!(res <= cc.tol[1]) || !isfinite(res)) outcome = 2;
    else if (res <= cc.tol[0] || hn == 0.0) outcome = 1;
    cc.ctl[0] = j + 1;
    cc.ctl[2] = outcome;
    if (cc.has_next) cudaGraphSetConditional(cc.next, (outcome == 0 && j + 1 < cc.ctl[1]) ? 1u : 0u);
  }
}

// y = H(0:k,0:k)^{-1} g(0:k) by back substitution (one thread)
__global__ void k_hsolve(int k, double* gm, int ldh) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int restart = ldh - 1;
  double* H = gm;
  double* g = H + (int64_t)ldh * restart + 2 * restart;
  double* y = g + ldh;
  for (int i = k - 1; i >= 0; --i) {
    double v = g[i];
    for (int c = i + 1; c < k; ++c) v -= H[i + (int64_t)ldh * c] * y[c];
    const double d = H[i + (int64_t)ldh * i];
    y[i] = d != 0.0 ? v / d : 0.0;
  }
}

__global__ void k_gather5(int64_t n, const int32_t* __restrict__ idx, const double* __restrict__ src,
                          double* __restrict__ dst) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 5 * n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = g / 5;
    dst[g] = src[5 * (int64_t)idx[k] + (g - 5 * k)];
  }
}

__global__ void k_scatter5(int64_t n, const int32_t* __restrict__ idx, const double* __restrict__ src,
                           double* __restrict__ dst) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 5 * n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = g / 5;
    dst[5 * (int64_t)idx[k] + (g - 5 * k)] = src[g];
  }
}

inline int grid_for(int64_t len, int tb = 256, int cap = 152 * 8) {
  int64_t g = (len + tb - 1) / tb;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <class VT>
void launch_spmv(int64_t nrow, const int32_t* rp, const int32_t* col, const VT* val, const double* x, double* y,
                 cudaStream_t s, int tb, const double* b) {
  if (nrow <= 0) return;
  const int64_t g = (5 * nrow + tb - 1) / tb;
  k_bsr_spmv<VT><<<g, tb, 0, s>>>(nrow, rp, col, val, x, b, y);
  count_launch();
}
template void launch_spmv<double>(int64_t, const int32_t*, const int32_t*, const double*, const double*, double*,
                                  cudaStream_t, int, const double*);
template void launch_spmv<float>(int64_t, const int32_t*, const int32_t*, const float*, const double*, double*,
                                 cudaStream_t, int, const double*);

void launch_spmv32(int64_t nrow, const int32_t* rp, const int32_t* col, const float* val, const float* x, double* y,
                   cudaStream_t s, int tb, const double* b) {
  if (nrow <= 0) return;
  k_bsr_spmv32<<<(5 * nrow + tb - 1) / tb, tb, 0, s>>>(nrow, rp, col, val, x, b, y);
  count_launch();
}

void launch_multi_axpy32(int64_t len, int nv, const float* Zs, int64_t ld, const double* coef, double* x,
                         cudaStream_t s) {
  k_multi_axpy32<<<grid_for(len), 256, 0, s>>>(len, nv, Zs, ld, coef, x);
  count_launch();
}

void launch_bsr_transpose(int64_t nnzb, const int32_t* tpos, const double* val, double* valT, cudaStream_t s) {
  k_bsr_transpose<<<grid_for(25 * nnzb), 256, 0, s>>>(nnzb, tpos, val, valT);
  count_launch();
}

void launch_differs(int64_t len, const double* a, const double* b, int* flag, cudaStream_t s) {
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  k_differs<<<grid_for(len), 256, 0, s>>>(len, a, b, flag);
  count_launch();
}

void launch_add32(int64_t len, const float* u, float* z, cudaStream_t s) {
  k_add32<<<grid_for(len), 256, 0, s>>>(len, u, z);
  count_launch();
}

void launch_f32_to_f64(int64_t n, const float* src, double* dst, cudaStream_t s) {
  k_f32_to_f64<<<grid_for(n), 256, 0, s>>>(n, src, dst);
  count_launch();
}

void launch_norm2(int64_t len, const double* x, double* partial, int grid, double* out, cudaStream_t s) {
  k_norm2_partial<<<grid, 256, 0, s>>>(len, x, partial);
  k_reduce_cols<<<1, 256, 0, s>>>(grid, 1, 1, partial, out, 0);
  count_launch();
  count_launch();
}

void launch_mdot(int64_t len, int nv, const double* V, int64_t ld, const double* w, double* partial, int grid,
                 double* out, cudaStream_t s, int tile) {
  if (cgs_tile(nv, tile) == 256)
    k_cgs_db<0, 256><<<grid, 256, cgs_db_smem(nv, 256), s>>>(len, nv, V, ld, nullptr, const_cast<double*>(w),
                                                            partial);
  else
    k_cgs_db<0, 128><<<grid, 256, cgs_db_smem(nv, 128), s>>>(len, nv, V, ld, nullptr, const_cast<double*>(w),
                                                            partial);
  k_reduce_cols<<<1, 256, 0, s>>>(grid, nv, NVMAX, partial, out, 0);
  count_launch();
  count_launch();
}

// first CGS pass update fused with the second pass's dot products; the dots
// are added to out_add (which holds the first-pass coefficients h)
void launch_update_mdot(int64_t len, int nv, const double* V, int64_t ld, const double* h, double* w,
                        double* partial, int grid, double* out_add, cudaStream_t s, int tile) {
  if (cgs_tile(nv, tile) == 256)
    k_cgs_db<1, 256><<<grid, 256, cgs_db_smem(nv, 256), s>>>(len, nv, V, ld, h, w, partial);
  else
    k_cgs_db<1, 128><<<grid, 256, cgs_db_smem(nv, 128), s>>>(len, nv, V, ld, h, w, partial);
  count_launch();
  (void)out_add;
}

void launch_update_norm(int64_t len, int nv, const double* V, int64_t ld, const double* h, double* w,
                        double* partial, int grid, double* out, cudaStream_t s) {
  k_cgs_update_norm<<<grid, 256, 0, s>>>(len, nv, V, ld, h, w, partial);
  k_reduce_cols<<<1, 256, 0, s>>>(grid, 1, NVMAX, partial, out, 0);
  count_launch();
  count_launch();
}

void cgs_init() {
  const int mx = 227 * 1024;
  cudaFuncSetAttribute(k_cgs_db<0, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_cgs_db<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_cgs_db<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_cgs_db<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

void launch_reduce_cols(int grid, int nv, const double* partial, double* out, int add, cudaStream_t s) {
  k_reduce_cols<<<1, 256, 0, s>>>(grid, nv, NVMAX, partial, out, add);
  count_launch();
}

void launch_scale(int64_t len, const double* x, const double* alpha_ptr, int invert, double* y, cudaStream_t s) {
  k_scale<<<grid_for(len), 256, 0, s>>>(len, x, alpha_ptr, invert, y);
  count_launch();
}

void launch_axpby(int64_t len, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  k_axpby<<<grid_for(len), 256, 0, s>>>(len, a, x, b, y, out);
  count_launch();
}

void launch_multi_axpy(int64_t len, int nv, const double* Zs, int64_t ld, const double* coef, double* x,
                       cudaStream_t s) {
  k_multi_axpy<<<grid_for(len), 256, 0, s>>>(len, nv, Zs, ld, coef, x);
  count_launch();
}

void launch_givens(int j, double* gm, const double* h1, const double* h2, const double* hnext, int ldh,
                   double* out_res, cudaStream_t s, const CycleCtl& cc) {
  k_givens<<<1, 32, 0, s>>>(j, gm, h1, h2, hnext, ldh, out_res, cc);
  count_launch();
}

void launch_hsolve(int k, double* gm, int ldh, cudaStream_t s) {
  k_hsolve<<<1, 32, 0, s>>>(k, gm, ldh);
  count_launch();
}

void launch_gather5(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t s) {
  k_gather5<<<grid_for(5 * n), 256, 0, s>>>(n, idx, src, dst);
  count_launch();
}

void launch_scatter5(int64_t n, const int32_t* idx, const double* src, double* dst, cudaStream_t s) {
  k_scatter5<<<grid_for(5 * n), 256, 0, s>>>(n, idx, src, dst);
  count_launch();
}

}  // namespace seird
