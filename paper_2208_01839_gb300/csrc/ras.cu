// Restricted additive Schwarz preconditioner (Eq. RAS) with block-ILU(0)
// subdomain solves, and the additive coarse correction of Section 3.1 with the
// per-subdomain, per-compartment constant coarse space Z:
//   z = sum_p R_p^T D_p (L_p U_p)^{-1} R_p r  +  Z A_c^{-1} Z^T r,  A_c = Z^T J Z.
// One CTA per subdomain for the factorization and the solves; rows of one
// level of the ILU(0) dependency DAG are independent and run in parallel, with
// a CTA barrier between levels.  The coarse matrix is block-banded (subdomains
// in reverse Cuthill-McKee order) and factored by block LU with 5x5 pivot
// blocks inverted under partial pivoting.
#include <cmath>

#include "kernels.cuh"

namespace seird {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Inverse of a 5x5 block by Gauss-Jordan with partial pivoting, one warp
// (lanes 0..4 hold the rows).  Sets ERR_SINGULAR (2) on a zero pivot.
__device__ void warp_inv5(const double* __restrict__ D, double* __restrict__ out, int lane, int32_t* err) {
  double a[5], b[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    a[c] = lane < 5 ? D[5 * lane + c] : 0.0;
    b[c] = (lane == c) ? 1.0 : 0.0;
  }
  bool sing = false;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = (lane >= k && lane < 5) ? fabs(a[k]) : -1.0;
    int idx = lane;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const double v2 = __shfl_down_sync(FULL, v, o, 8);
      const int i2 = __shfl_down_sync(FULL, idx, o, 8);
      if (v2 > v || (v2 == v && i2 < idx)) {
        v = v2;
        idx = i2;
      }
    }
    const double vmax = __shfl_sync(FULL, v, 0);
    const int piv = __shfl_sync(FULL, idx, 0);
    if (!(vmax > 0.0)) sing = true;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double ak = __shfl_sync(FULL, a[c], k), ap = __shfl_sync(FULL, a[c], piv);
      const double bk = __shfl_sync(FULL, b[c], k), bp = __shfl_sync(FULL, b[c], piv);
      if (lane == k) {
        a[c] = ap;
        b[c] = bp;
      } else if (lane == piv) {
        a[c] = ak;
        b[c] = bk;
      }
    }
    const double pv = __shfl_sync(FULL, a[k], k);
    const double pinv = pv != 0.0 ? 1.0 / pv : 0.0;
    if (lane == k) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        a[c] *= pinv;
        b[c] *= pinv;
      }
    }
    double pr[5], pb[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      pr[c] = __shfl_sync(FULL, a[c], k);
      pb[c] = __shfl_sync(FULL, b[c], k);
    }
    if (lane < 5 && lane != k) {
      const double f = a[k];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        a[c] = fma(-f, pr[c], a[c]);
        b[c] = fma(-f, pb[c], b[c]);
      }
    }
  }
  if (lane < 5) {
#pragma unroll
    for (int c = 0; c < 5; ++c) out[5 * lane + c] = b[c];
  }
  if (sing && lane == 0) atomicOr(err, 2);
}

// Block ILU(0) of R_p J R_p^T (IKJ form), rows in forward-level order.
__global__ void __launch_bounds__(256) k_ilu_factor(RasDev d, const double* __restrict__ val, int32_t* err) {
  const int p = blockIdx.x;
  const int32_t r0 = d.sd_row0[p];
  const int32_t r1 = d.sd_row0[p + 1];
  const int64_t b0 = d.l_row_ptr[r0], b1 = d.l_row_ptr[r1];
  for (int64_t idx = threadIdx.x; idx < (b1 - b0) * 25; idx += blockDim.x) {
    const int64_t blk = b0 + idx / 25;
    const int e = (int)(idx % 25);
    d.fval[25 * blk + e] = val[25 * (int64_t)d.l_gblk[blk] + e];
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
        const double* Dk = d.dinv + 25 * ((int64_t)r0 + k);
        double* A = d.fval + 25 * a;
        double v = 0.0;
        if (lane < 25) {
#pragma unroll
          for (int mm = 0; mm < 5; ++mm) v = fma(A[5 * rr + mm], Dk[5 * mm + cc], v);
        }
        __syncwarp();
        if (lane < 25) A[lane] = v;  // L_ik = A_ik U_kk^{-1}
        __syncwarp();
        for (int64_t u = d.upd_ptr[a]; u < d.upd_ptr[a + 1]; ++u) {
          const int64_t dst = d.upd[2 * u], src = d.upd[2 * u + 1];
          if (lane < 25) {
            double t = 0.0;
#pragma unroll
            for (int mm = 0; mm < 5; ++mm) t = fma(A[5 * rr + mm], d.fval[25 * src + 5 * mm + cc], t);
            d.fval[25 * dst + lane] -= t;  // A_ij -= L_ik U_kj
          }
        }
        __syncwarp();
      }
      warp_inv5(d.fval + 25 * d.l_diag[R], d.dinv + 25 * R, lane, err);
      __syncwarp();
    }
    __syncthreads();
  }
}

// z_owned += (L_p U_p)^{-1} R_p r restricted to the owned rows (RAS).
__global__ void __launch_bounds__(256) k_ilu_solve(RasDev d, const double* __restrict__ r, double* __restrict__ z) {
  const int p = blockIdx.x;
  const int32_t r0 = d.sd_row0[p];
  const int32_t nl = d.sd_row0[p + 1] - r0;
  double* y = d.ywork + 5 * (int64_t)r0;
  double* zz = d.zwork + 5 * (int64_t)r0;
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int32_t idx = tid; idx < 5 * nl; idx += bd) {
    const int32_t l = idx / 5, c = idx - 5 * l;
    y[idx] = r[5 * (int64_t)d.sd_node[r0 + l] + c];
  }
  __syncthreads();
  // forward: y_i -= sum_{k<i} L_ik y_k
  {
    const int32_t L0 = d.sd_fwd_lev0[p];
    const int32_t nlev = d.sd_fwd_lev0[p + 1] - L0 - 1;
    for (int32_t lv = 0; lv < nlev; ++lv) {
      const int32_t s = d.fwd_lev[L0 + lv], e = d.fwd_lev[L0 + lv + 1];
      for (int32_t idx = tid; idx < 5 * (e - s); idx += bd) {
        const int32_t ri = s + idx / 5, c = idx % 5;
        const int32_t i = d.fwd_order[r0 + ri];
        const int64_t R = (int64_t)r0 + i;
        double acc = y[5 * i + c];
        for (int64_t a = d.l_row_ptr[R]; a < d.l_row_ptr[R + 1]; ++a) {
          const int32_t k = d.l_col[a];
          if (k >= i) break;
          const double* L = d.fval + 25 * a + 5 * c;
          const double* yk = y + 5 * k;
#pragma unroll
          for (int mm = 0; mm < 5; ++mm) acc = fma(-L[mm], yk[mm], acc);
        }
        y[5 * i + c] = acc;
      }
      __syncthreads();
    }
  }
  // backward: z_i = U_ii^{-1} (y_i - sum_{j>i} U_ij z_j)
  {
    const int32_t L0 = d.sd_bwd_lev0[p];
    const int32_t nlev = d.sd_bwd_lev0[p + 1] - L0 - 1;
    for (int32_t lv = 0; lv < nlev; ++lv) {
      const int32_t s = d.bwd_lev[L0 + lv], e = d.bwd_lev[L0 + lv + 1];
      for (int32_t idx = tid; idx < 5 * (e - s); idx += bd) {
        const int32_t ri = s + idx / 5, c = idx % 5;
        const int32_t i = d.bwd_order[r0 + ri];
        const int64_t R = (int64_t)r0 + i;
        double acc = y[5 * i + c];
        for (int64_t a = d.l_diag[R] + 1; a < d.l_row_ptr[R + 1]; ++a) {
          const int32_t j = d.l_col[a];
          const double* Ub = d.fval + 25 * a + 5 * c;
          const double* zj = zz + 5 * j;
#pragma unroll
          for (int mm = 0; mm < 5; ++mm) acc = fma(-Ub[mm], zj[mm], acc);
        }
        y[5 * i + c] = acc;
      }
      __syncthreads();
      for (int32_t idx = tid; idx < 5 * (e - s); idx += bd) {
        const int32_t ri = s + idx / 5, c = idx % 5;
        const int32_t i = d.bwd_order[r0 + ri];
        const double* Di = d.dinv + 25 * ((int64_t)r0 + i) + 5 * c;
        const double* yi = y + 5 * i;
        double v = 0.0;
#pragma unroll
        for (int mm = 0; mm < 5; ++mm) v = fma(Di[mm], yi[mm], v);
        zz[5 * i + c] = v;
      }
      __syncthreads();
    }
  }
  const int32_t own0 = d.own_ptr[p], own1 = d.own_ptr[p + 1];
  for (int32_t idx = tid; idx < 5 * nl; idx += bd) {
    const int32_t l = idx / 5, c = idx - 5 * l;
    const int32_t node = d.sd_node[r0 + l];
    if (node >= own0 && node < own1) z[5 * (int64_t)node + c] = zz[idx];
  }
}

// ---- coarse space --------------------------------------------------------

// one warp per chunk of J blocks that belong to the same coarse block
__global__ void k_coarse_chunks(int32_t nchunk, const int32_t* __restrict__ cptr, const int32_t* __restrict__ blk,
                                const double* __restrict__ val, double* __restrict__ cpart) {
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= nchunk || lane >= 25) return;
  double s = 0.0;
  for (int32_t b = cptr[gw]; b < cptr[gw + 1]; ++b) s += val[25 * (int64_t)blk[b] + lane];
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
  if (warp == 0) warp_inv5(bblk(band, bw, kb, kb), cdinv + 25 * (int64_t)kb, lane, err);
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

// y <- A_c^{-1} y with the banded block LU factors (one CTA, y in shared memory)
__global__ void k_band_solve(int P, int bw, const double* __restrict__ band, const double* __restrict__ cdinv,
                             double* __restrict__ yg) {
  extern __shared__ double ys[];
  const int tid = threadIdx.x, bd = blockDim.x;
  double* bandm = const_cast<double*>(band);
  for (int k = tid; k < 5 * P; k += bd) ys[k] = yg[k];
  __syncthreads();
  for (int kb = 0; kb < P; ++kb) {
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
__global__ void k_coarse_prolong_add(int64_t n, const int32_t* __restrict__ owner, const int32_t* __restrict__ cpos,
                                     const double* __restrict__ y, double* __restrict__ z) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < 5 * n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g / 5;
    z[g] += y[5 * (int64_t)cpos[owner[i]] + (g - 5 * i)];
  }
}

}  // namespace

void launch_ilu_factor(const RasDev& d, const double* val, int32_t* err, cudaStream_t s) {
  k_ilu_factor<<<d.P, 256, 0, s>>>(d, val, err);
  count_launch();
}

void launch_ilu_solve(const RasDev& d, const double* r, double* z, cudaStream_t s) {
  k_ilu_solve<<<d.P, 256, 0, s>>>(d, r, z);
  count_launch();
}

void launch_coarse_assemble(const CoarseDev& c, const double* val, cudaStream_t s) {
  const int64_t W = 2 * (int64_t)c.band + 1;
  cudaMemsetAsync(c.cband, 0, sizeof(double) * 25 * W * c.P, s);
  k_coarse_chunks<<<(int)((32 * (int64_t)c.nchunk + 255) / 256), 256, 0, s>>>(c.nchunk, c.cchunk_ptr, c.cseg_blk, val,
                                                                               c.cpart);
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
}

void launch_coarse_apply_add(const CoarseDev& c, int64_t n, const double* r, double* z, cudaStream_t s) {
  k_coarse_restrict<<<c.P, 256, 0, s>>>(c.own_ptr, c.cpos, r, c.crhs);
  k_band_solve<<<1, 512, sizeof(double) * 5 * c.P, s>>>(c.P, c.band, c.cband, c.cdinv, c.crhs);
  int64_t g = (5 * n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  k_coarse_prolong_add<<<(int)g, 256, 0, s>>>(n, c.owner, c.cpos, c.crhs, z);
  count_launch();
  count_launch();
  count_launch();
}

void coarse_init() {
  cudaFuncSetAttribute(k_band_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace seird
