// Residual and Jacobian assembly of the discrete system of Eq. weakform
// (P1 triangles, backward Euler, Eq. timediscrete; reaction rows of Eq.
// vec_component2).  Two phases each, atomic-free and deterministic:
//   element phase  (one thread per triangle): element vector / Jacobian record;
//   gather phase   (one thread per node / per 5x5 block): fixed-order sums over
//                  the incident triangles, lists built at setup.
// All arithmetic is FP64.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/seird.h"
#include "kernels.cuh"

namespace seird {

// Quadrature tables: rule 0 = Radon's degree-5 seven-point rule (barycentric
// points on the centroid and two three-point orbits at (6 -+ sqrt 15)/21,
// weights 9/40 and (155 -+ sqrt 15)/1200); rule 1 = three vertices, 1/3 each.
__constant__ double cQL[2][7][3];
__constant__ double cQW[2][7];
// w_q phi_a phi_b at point q for the pairs (0,0) (1,1) (2,2) (0,1) (0,2) (1,2)
__constant__ double cQC[2][7][6];
// The degree-5 rule by its symmetry orbits: the centroid (weight W0) and two
// three-point orbits o = 1, 2 whose point k has barycentric coordinate B_o at
// vertex k and A_o at the other two (D_o = B_o - A_o, weight W_o).  A point value
// of a P1 field x is then A_o sum(x) + D_o x_k, and sums over an orbit of
// w_q phi_a phi_b f(q) reduce to the orbit sum of f and single point values:
//   sum_k W L_a L_a f_k = W A^2 S + W (B^2 - A^2) f_a
//   sum_k W L_a L_b f_k = W A B S - W A D f_c      (a != b, c the third vertex)
//   sum_k W L_a f_k     = W A S + W D f_a.
// cORB: [0..2] A1 D1 W1, [3..5] A2 D2 W2, [6] W0, [7] W0/3, [8] W1 A1, [9] W2 A2,
// [10] W1 D1, [11] W2 D2, [12] W0/9, [13] W1 A1^2, [14] W1 (B1^2 - A1^2), [15] W1 A1 B1,
// [16] -W1 A1 D1, [17..20] the same for orbit 2.
__constant__ double cORB[21];
__constant__ float cORBf[21];  // the same in FP32 (FP32 Jacobian record)

cudaError_t upload_quadrature() {
  double L[2][7][3] = {};
  double W[2][7] = {};
  const double r = std::sqrt(15.0);
  const double a1 = (6.0 - r) / 21.0, b1 = (9.0 + 2.0 * r) / 21.0;
  const double a2 = (6.0 + r) / 21.0, b2 = (9.0 - 2.0 * r) / 21.0;
  const double pts[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
  const double w1 = (155.0 - r) / 1200.0, w2 = (155.0 + r) / 1200.0;
  const double wts[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
  for (int q = 0; q < 7; ++q) {
    for (int a = 0; a < 3; ++a) L[0][q][a] = pts[q][a];
    W[0][q] = wts[q];
  }
  for (int q = 0; q < 3; ++q) {
    L[1][q][q] = 1.0;
    W[1][q] = 1.0 / 3.0;
  }
  double Cw[2][7][6] = {};
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int rule = 0; rule < 2; ++rule)
    for (int q = 0; q < 7; ++q)
      for (int s = 0; s < 6; ++s) Cw[rule][q][s] = W[rule][q] * L[rule][q][pa[s]] * L[rule][q][pb[s]];
  cudaError_t e = cudaMemcpyToSymbol(cQL, L, sizeof(L));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(cQW, W, sizeof(W));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(cQC, Cw, sizeof(Cw));
  // orbit form of the same table: point 1 + k (4 + k) has its larger (smaller) coordinate at vertex k
  double O[21];
  const double A1 = L[0][1][1], B1 = L[0][1][0], A2 = L[0][4][1], B2 = L[0][4][0];
  const double W0 = W[0][0], W1 = W[0][1], W2 = W[0][4];
  const double D1 = B1 - A1, D2 = B2 - A2;
  const double orb[21] = {A1, D1, W1, A2, D2, W2, W0, W0 / 3.0, W1 * A1, W2 * A2, W1 * D1, W2 * D2, W0 / 9.0,
                          W1 * A1 * A1, W1 * (B1 * B1 - A1 * A1), W1 * A1 * B1, -W1 * A1 * D1,
                          W2 * A2 * A2, W2 * (B2 * B2 - A2 * A2), W2 * A2 * B2, -W2 * A2 * D2};
  float Of[21];
  for (int k = 0; k < 21; ++k) {
    O[k] = orb[k];
    Of[k] = (float)orb[k];
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(cORB, O, sizeof(O));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(cORBf, Of, sizeof(Of));
  // copies from pageable memory may return before their DMA has landed: a kernel on
  // a non-blocking stream is ordered after the tables only once the device is idle
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

namespace {

struct Tri {
  double area, gx[3], gy[3];
  int32_t v[3];
};

__device__ __forceinline__ Tri load_tri(const int32_t* __restrict__ tri, const double* __restrict__ xy, int64_t t) {
  Tri T;
  T.v[0] = tri[3 * t];
  T.v[1] = tri[3 * t + 1];
  T.v[2] = tri[3 * t + 2];
  const double x0 = xy[2 * (int64_t)T.v[0]], y0 = xy[2 * (int64_t)T.v[0] + 1];
  const double x1 = xy[2 * (int64_t)T.v[1]], y1 = xy[2 * (int64_t)T.v[1] + 1];
  const double x2 = xy[2 * (int64_t)T.v[2]], y2 = xy[2 * (int64_t)T.v[2] + 1];
  const double twoA = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
  const double inv = 1.0 / twoA;
  T.area = 0.5 * twoA;
  T.gx[0] = (y1 - y2) * inv;
  T.gy[0] = (x2 - x1) * inv;
  T.gx[1] = (y2 - y0) * inv;
  T.gy[1] = (x0 - x2) * inv;
  T.gx[2] = (y0 - y1) * inv;
  T.gy[2] = (x1 - x0) * inv;
  return T;
}

template <class T>
struct TriT {
  T area, gx[3], gy[3];
  int32_t v[3];
};

template <class T>
__device__ __forceinline__ T orb(int i) {
  if constexpr (sizeof(T) == 4) return cORBf[i];
  else return cORB[i];
}

// x > 0 and not NaN, from the bits (integer pipe): 0 < bits <= bits(+inf)
__device__ __forceinline__ bool positive(double x) {
  return (unsigned long long)(__double_as_longlong(x) - 1) < 0x7FF0000000000000ull;
}

// 1/N at the seven points of the degree-5 rule with one division (Montgomery's
// simultaneous inversion: prefix products, one reciprocal, back substitution).
// The point values of a P1 field lie within a factor 1/min(A2, B2) < 17 of each
// other, so when the full product is in [1e-280, 1e280] no prefix product left
// the normal range; otherwise the points are divided one by one.
__device__ __forceinline__ void reciprocals7(const double (&N)[7], double (&r)[7]) {
  double pre[7];
  pre[0] = N[0];
#pragma unroll
  for (int q = 1; q < 7; ++q) pre[q] = pre[q - 1] * N[q];
  if (pre[6] >= 1e-280 && pre[6] <= 1e280) {
    double inv = 1.0 / pre[6];
#pragma unroll
    for (int q = 6; q > 0; --q) {
      r[q] = inv * pre[q - 1];
      inv *= N[q];
    }
    r[0] = inv;
  } else {
#pragma unroll
    for (int q = 0; q < 7; ++q) r[q] = 1.0 / N[q];
  }
}

// Triangle t from the geometry table written at set-up (k_tri_geometry: |T| and the
// gradients of the three hat functions, 8 doubles per triangle), or from the
// coordinates when there is no table.
__device__ __forceinline__ Tri tri_of(const int32_t* __restrict__ tri, const double* __restrict__ xy,
                                      const double* __restrict__ geo, int64_t t) {
  if (!geo) return load_tri(tri, xy, t);
  Tri T;
  T.v[0] = tri[3 * t];
  T.v[1] = tri[3 * t + 1];
  T.v[2] = tri[3 * t + 2];
  const double2* g = reinterpret_cast<const double2*>(geo + 8 * t);
  const double2 g0 = g[0], g1 = g[1], g2 = g[2], g3 = g[3];
  T.area = g0.x;
  T.gx[0] = g0.y;
  T.gx[1] = g1.x;
  T.gx[2] = g1.y;
  T.gy[0] = g2.x;
  T.gy[1] = g2.y;
  T.gy[2] = g3.x;
  return T;
}

__global__ void __launch_bounds__(256) k_tri_geometry(int64_t m, const int32_t* __restrict__ tri,
                                                      const double* __restrict__ xy, double* __restrict__ geo) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Tri T = load_tri(tri, xy, t);
  double2* g = reinterpret_cast<double2*>(geo + 8 * t);
  g[0] = make_double2(T.area, T.gx[0]);
  g[1] = make_double2(T.gx[1], T.gx[2]);
  g[2] = make_double2(T.gy[0], T.gy[1]);
  g[3] = make_double2(T.gy[2], 0.0);
}

// Node terms of the degree-5 residual, 8 doubles per node: w = u - u^n - dt L u (L the
// linear part of the reaction of Eq. seird1-5), N = s + e + i + r + d and
// l = beta_I i + beta_E e.  The element phase reads them at its vertices.
__global__ void __launch_bounds__(256) k_residual_node(int64_t n, const double* __restrict__ U,
                                                       const double* __restrict__ Un, Rates rin,
                                                       double* __restrict__ nd) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Rates r = rates_at(rin, i);
  double u[5], du[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    u[c] = U[5 * i + c];
    du[c] = u[c] - Un[5 * i + c];
  }
  const double N = u[0] + u[1] + u[2] + u[3] + u[4];
  const double dt = r.dt;
  double2* o = reinterpret_cast<double2*>(nd + 8 * i);
  o[0] = make_double2(du[0] - dt * (r.alpha * N - r.mu * u[0]), du[1] + dt * (r.sigma + r.ge + r.mu) * u[1]);
  o[1] = make_double2(du[2] - dt * (r.sigma * u[1] - (r.gr + r.gd + r.mu) * u[2]),
                      du[3] - dt * (r.ge * u[1] + r.gr * u[2] - r.mu * u[3]));
  o[2] = make_double2(du[4] - dt * r.gd * u[2], N);
  o[3] = make_double2(r.bi * u[2] + r.be * u[1], 0.0);
}

// Element residual with the degree-5 rule: consistent mass, exact diffusion, and the
// reaction as the mass product M w of the node terms (the rule integrates the linear
// terms exactly) plus the transmission term through the rule's orbit form (cORB).
template <bool BF>
__global__ void __launch_bounds__(128) k_residual_elem5(int64_t m, const int32_t* __restrict__ tri,
                                                        const double* __restrict__ xy,
                                                        const double* __restrict__ geo,
                                                        const double* __restrict__ U, const double* __restrict__ nd,
                                                        const double* __restrict__ bfield, Rates rin,
                                                        double* __restrict__ elem, int32_t* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Tri T = tri_of(tri, xy, geo, t);
  const Rates r = rates_at(rin, T.v[0]);
  double u[3][4], w[3][5], Nv[3], l[3], Fe[3][5];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2* q = reinterpret_cast<const double2*>(nd + 8 * (int64_t)T.v[a]);
    const double2 q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    w[a][0] = q0.x;
    w[a][1] = q0.y;
    w[a][2] = q1.x;
    w[a][3] = q1.y;
    w[a][4] = q2.x;
    Nv[a] = q2.y;
    l[a] = q3.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) u[a][c] = U[5 * (int64_t)T.v[a] + c];
  }
  const double SN = Nv[0] + Nv[1] + Nv[2];
  const double Nbar = SN * (1.0 / 3.0);
  const double m12 = T.area * (1.0 / 12.0);  // (phi_a, phi_b) = |T| (1 + delta_ab) / 12
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const double msw = m12 * (w[0][c] + w[1][c] + w[2][c]);
#pragma unroll
    for (int a = 0; a < 3; ++a) Fe[a][c] = fma(m12, w[a][c], msw);
  }
  // diffusion: dt nubar_c |T| mean_T(N) grad u_c . grad phi_a  (nubar_D = 0)
  const double dNA = r.dt * Nbar * T.area;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double coef = dNA * r.nu[c];
    const double gux = coef * (u[0][c] * T.gx[0] + u[1][c] * T.gx[1] + u[2][c] * T.gx[2]);
    const double guy = coef * (u[0][c] * T.gy[0] + u[1][c] * T.gy[1] + u[2][c] * T.gy[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) Fe[a][c] = fma(gux, T.gx[a], fma(guy, T.gy[a], Fe[a][c]));
  }
  // transmission s -> e, kappa s (beta_I i + beta_E e) b, at the rule's points
  double bv[3] = {1.0, 1.0, 1.0};
  if (BF) {
#pragma unroll
    for (int a = 0; a < 3; ++a) bv[a] = bfield[T.v[a]];
  }
  const double A1 = cORB[0], D1 = cORB[1], A2 = cORB[3], D2 = cORB[4];
  const double Ss = u[0][0] + u[1][0] + u[2][0], Sl = l[0] + l[1] + l[2];
  const double Sb = BF ? bv[0] + bv[1] + bv[2] : 3.0;
  double Nq[7], rq[7];  // centroid, orbit 1, orbit 2
  Nq[0] = Nbar;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Nq[1 + k] = A1 * SN + D1 * Nv[k];
    Nq[4 + k] = A2 * SN + D2 * Nv[k];
  }
  bool bad = false;
#pragma unroll
  for (int q = 0; q < 7; ++q) bad |= !positive(Nq[q]);
  reciprocals7(Nq, rq);
  const double T0 = (1.0 - r.A * rq[0]) * (Ss * (1.0 / 3.0)) * (Sl * (1.0 / 3.0)) * (BF ? Sb * (1.0 / 3.0) : 1.0);
  double T1[3], T2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double s1 = A1 * Ss + D1 * u[k][0], l1 = A1 * Sl + D1 * l[k];
    const double s2 = A2 * Ss + D2 * u[k][0], l2 = A2 * Sl + D2 * l[k];
    T1[k] = (1.0 - r.A * rq[1 + k]) * s1 * l1 * (BF ? A1 * Sb + D1 * bv[k] : 1.0);
    T2[k] = (1.0 - r.A * rq[4 + k]) * s2 * l2 * (BF ? A2 * Sb + D2 * bv[k] : 1.0);
  }
  const double dA = r.dt * T.area;
  const double sh = dA * (cORB[7] * T0 + cORB[8] * (T1[0] + T1[1] + T1[2]) + cORB[9] * (T2[0] + T2[1] + T2[2]));
  const double e1 = dA * cORB[10], e2 = dA * cORB[11];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double v = fma(e1, T1[a], fma(e2, T2[a], sh));
    Fe[a][0] += v;
    Fe[a][1] -= v;
  }
  if (bad) atomicOr(err, 1);
  double* out = elem + 15 * t;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 5; ++c) out[5 * a + c] = Fe[a][c];
}

// Element residual with the three-vertex rule: consistent mass for the time
// difference, exact diffusion, the linear reaction terms lumped (|T|/3 at each
// vertex) and the transmission term at the vertices.
template <bool BF>
__global__ void __launch_bounds__(128) k_residual_elem_vertex(int64_t m, const int32_t* __restrict__ tri,
                                                              const double* __restrict__ xy,
                                                              const double* __restrict__ geo,
                                                              const double* __restrict__ U,
                                                              const double* __restrict__ Un,
                                                              const double* __restrict__ bfield, Rates rin,
                                                              double* __restrict__ elem, int32_t* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Tri T = tri_of(tri, xy, geo, t);
  const Rates r = rates_at(rin, T.v[0]);
  double u[3][5], Fe[3][5], Nv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int c = 0; c < 5; ++c) u[a][c] = U[5 * (int64_t)T.v[a] + c];
    Nv[a] = u[a][0] + u[a][1] + u[a][2] + u[a][3] + u[a][4];
  }
  const double Nbar = (Nv[0] + Nv[1] + Nv[2]) * (1.0 / 3.0);
  const double m12 = T.area * (1.0 / 12.0);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double du[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) du[a] = u[a][c] - Un[5 * (int64_t)T.v[a] + c];
    const double sdu = du[0] + du[1] + du[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) Fe[a][c] = m12 * (du[a] + sdu);
  }
  const double a3 = T.area / 3.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double Mu[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) Mu[c] = a3 * u[a][c];
    const double MN = Mu[0] + Mu[1] + Mu[2] + Mu[3] + Mu[4];
    Fe[a][0] -= r.dt * (r.alpha * MN - r.mu * Mu[0]);
    Fe[a][1] += r.dt * (r.sigma + r.ge + r.mu) * Mu[1];
    Fe[a][2] -= r.dt * (r.sigma * Mu[1] - (r.gr + r.gd + r.mu) * Mu[2]);
    Fe[a][3] -= r.dt * (r.ge * Mu[1] + r.gr * Mu[2] - r.mu * Mu[3]);
    Fe[a][4] -= r.dt * r.gd * Mu[2];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double gux = u[0][c] * T.gx[0] + u[1][c] * T.gx[1] + u[2][c] * T.gx[2];
    const double guy = u[0][c] * T.gy[0] + u[1][c] * T.gy[1] + u[2][c] * T.gy[2];
    const double coef = r.dt * r.nu[c] * Nbar * T.area;
#pragma unroll
    for (int a = 0; a < 3; ++a) Fe[a][c] += coef * (gux * T.gx[a] + guy * T.gy[a]);
  }
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {  // |T|/3 at vertex a
    const double N = Nv[a];
    const double bq = BF ? bfield[T.v[a]] : 1.0;
    bad |= !(N > 0.0);
    const double kappa = 1.0 - r.A / N;
    const double Tr = kappa * u[a][0] * (r.bi * u[a][2] + r.be * u[a][1]) * bq;
    const double wq = r.dt * a3 * Tr;
    Fe[a][0] += wq;
    Fe[a][1] -= wq;
  }
  if (bad) atomicOr(err, 1);
  double* out = elem + 15 * t;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 5; ++c) out[5 * a + c] = Fe[a][c];
}

// Node gather of element vectors (fixed order) plus per-CTA partial ||F||^2.
__global__ void __launch_bounds__(256) k_residual_gather(int64_t n, const int32_t* __restrict__ inc_ptr,
                                                         const int32_t* __restrict__ inc,
                                                         const double* __restrict__ elem, double* __restrict__ F,
                                                         double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double ss = 0.0;
  if (i < n) {
    double acc[5] = {0, 0, 0, 0, 0};
    for (int32_t k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
      const double* e = elem + 5 * (int64_t)inc[k];
#pragma unroll
      for (int c = 0; c < 5; ++c) acc[c] += e[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      F[5 * i + c] = acc[c];
      ss += acc[c] * acc[c];
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

// Fixed-order sum of per-CTA partials (one CTA).
__global__ void k_sum_partials(int64_t np, const double* __restrict__ partial, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int64_t k = threadIdx.x; k < np; k += blockDim.x) v += partial[k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (threadIdx.x == 0) *out = x;
  }
}

// symmetric pair index: (0,0) (1,1) (2,2) (0,1) (0,2) (1,2)
__device__ __forceinline__ int sym(int a, int b) {
  return a == b ? a : (a + b + 2);
}

// Jacobian record of a triangle.
// T is the arithmetic and storage type: FP64, or FP32 when the Jacobian only
// feeds the FP32 operator and FP32 factors of the mixed-precision path.
// PIC: the record of the Picard matrix of Eq. weak_vec_implicit instead (no
// derivative of N in the diffusion coefficient, and moment 0 holds the
// coefficient kappa beta_I i b of B(u)'s (E, S) entry instead of the Allee
// derivative).
template <int RULE, bool BF, class T, bool PIC>
__global__ void __launch_bounds__(128) k_jac_record(int64_t m, const int32_t* __restrict__ tri,
                                                    const double* __restrict__ xy, const double* __restrict__ geo,
                                                    const double* __restrict__ U,
                                                    const double* __restrict__ bfield, Rates rin,
                                                    T* __restrict__ rec, int32_t* err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // A, beta_I, beta_E, dt, nubar_S..R in type T (see rate_consts)
  constexpr bool kCTA = sizeof(T) == 4;
  __shared__ T srk[8];
  if (kCTA && !rin.tab) {
    if (threadIdx.x == 0) {
      srk[0] = (T)rin.A;
      srk[1] = (T)rin.bi;
      srk[2] = (T)rin.be;
      srk[3] = (T)rin.dt;
      for (int c = 0; c < 4; ++c) srk[4 + c] = (T)rin.nu[c];
    }
    __syncthreads();
  }
  if (t >= m) return;
  const Tri Tg = tri_of(tri, xy, geo, t);
  const Rates r = rates_at(rin, Tg.v[0]);
  const bool shr = kCTA && !rin.tab;
  TriT<T> Tt;
  Tt.area = (T)Tg.area;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Tt.gx[a] = (T)Tg.gx[a];
    Tt.gy[a] = (T)Tg.gy[a];
    Tt.v[a] = Tg.v[a];
  }
  T u[3][5];
  T Nbar = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      u[a][c] = (T)U[5 * (int64_t)Tt.v[a] + c];
      Nbar += u[a][c];
    }
  Nbar *= T(1.0 / 3.0);
  T* out = rec + (int64_t)REC * t;
  out[0] = Tt.area;
  // N-weighted stiffness dt |T| mean(N) grad phi_a . grad phi_b
  // the gather reads the sums below already scaled: K and P by dt, G_c by dt nu_c
  const T dtT = shr ? srk[3] : (T)r.dt;
  const T an = dtT * Tt.area * Nbar;
  out[REC_K + 0] = an * (Tt.gx[0] * Tt.gx[0] + Tt.gy[0] * Tt.gy[0]);
  out[REC_K + 1] = an * (Tt.gx[1] * Tt.gx[1] + Tt.gy[1] * Tt.gy[1]);
  out[REC_K + 2] = an * (Tt.gx[2] * Tt.gx[2] + Tt.gy[2] * Tt.gy[2]);
  out[REC_K + 3] = an * (Tt.gx[0] * Tt.gx[1] + Tt.gy[0] * Tt.gy[1]);
  out[REC_K + 4] = an * (Tt.gx[0] * Tt.gx[2] + Tt.gy[0] * Tt.gy[2]);
  out[REC_K + 5] = an * (Tt.gx[1] * Tt.gx[2] + Tt.gy[1] * Tt.gy[2]);
  // G_{c,a} = dt nubar_c |T|/3 grad u_c . grad phi_a (derivative of mean_T(N) by any u_{b,c'})
  const T a3 = Tt.area * T(1.0 / 3.0);
  if (!PIC) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T gux = u[0][c] * Tt.gx[0] + u[1][c] * Tt.gx[1] + u[2][c] * Tt.gx[2];
      const T guy = u[0][c] * Tt.gy[0] + u[1][c] * Tt.gy[1] + u[2][c] * Tt.gy[2];
      const T gsc = a3 * dtT * (shr ? srk[4 + c] : (T)r.nu[c]);
#pragma unroll
      for (int a = 0; a < 3; ++a) out[REC_G + 4 * a + c] = gsc * (gux * Tt.gx[a] + guy * Tt.gy[a]);
    }
  }
  // reaction moments P^k_ab = dt |T| sum_q w_q phi_a phi_b rho_k(x_q):
  //   rho_0 = A s lam / N^2 (d kappa/du_c' = A/N^2 for every c'), rho_1 = kappa lam,
  //   rho_2 = kappa s beta_E b, rho_3 = kappa s beta_I b.
  T P[4][6];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s) P[k][s] = T(0);
  T bv[3] = {T(1), T(1), T(1)};
  if (BF) {
#pragma unroll
    for (int a = 0; a < 3; ++a) bv[a] = (T)bfield[Tt.v[a]];
  }
  T Nv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) Nv[a] = u[a][0] + u[a][1] + u[a][2] + u[a][3] + u[a][4];
  const T A = shr ? srk[0] : (T)r.A, bi = shr ? srk[1] : (T)r.bi, be = shr ? srk[2] : (T)r.be;
  bool bad = false;
  if (RULE == 0 && !PIC) {
    // the degree-5 rule by its orbits (cORB): per moment, the centroid value, the two
    // orbit sums and the six point values give the six pair moments
    const T A1 = orb<T>(0), D1 = orb<T>(1), A2 = orb<T>(3), D2 = orb<T>(4);
    T l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) l[a] = bi * u[a][2] + be * u[a][1];
    const T Ss = u[0][0] + u[1][0] + u[2][0], Sl = l[0] + l[1] + l[2], SN = Nv[0] + Nv[1] + Nv[2];
    const T Sb = BF ? bv[0] + bv[1] + bv[2] : T(3);
    T Nq[7], rq[7];
    Nq[0] = Nbar;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Nq[1 + k] = A1 * SN + D1 * Nv[k];
      Nq[4 + k] = A2 * SN + D2 * Nv[k];
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      if constexpr (sizeof(T) == 8) bad |= !positive(Nq[q]);
      else bad |= !(Nq[q] > T(0));
    }
    if constexpr (sizeof(T) == 8) {
      reciprocals7(Nq, rq);
    } else {
#pragma unroll
      for (int q = 0; q < 7; ++q) rq[q] = T(1) / Nq[q];
    }
    // rho at point q from s, l, b there
    auto moments = [&](int q, T s, T lv, T b, T (&rho)[4]) {
      const T Ar = A * rq[q];
      const T kappa = T(1) - Ar;
      const T lam = lv * b;
      const T ksb = kappa * s * b;
      rho[0] = Ar * rq[q] * (s * lam);
      rho[1] = kappa * lam;
      rho[2] = ksb * be;
      rho[3] = ksb * bi;
    };
    T rc[4], S1[4] = {0, 0, 0, 0}, S2[4] = {0, 0, 0, 0};
    moments(0, Ss * T(1.0 / 3.0), Sl * T(1.0 / 3.0), BF ? Sb * T(1.0 / 3.0) : T(1), rc);
    // P[k][a] (a < 3, pair (a, a)) and P[k][3 + (2 - c)] (the pair opposite vertex c) take the
    // point values; the orbit sums and the centroid value are added to all pairs at the end
    const T ar = dtT * Tt.area;
    const T cdR1 = ar * orb<T>(14), coR1 = ar * orb<T>(16), cdR2 = ar * orb<T>(18), coR2 = ar * orb<T>(20);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T rho1[4], rho2[4];
      moments(1 + k, A1 * Ss + D1 * u[k][0], A1 * Sl + D1 * l[k], BF ? A1 * Sb + D1 * bv[k] : T(1), rho1);
      moments(4 + k, A2 * Ss + D2 * u[k][0], A2 * Sl + D2 * l[k], BF ? A2 * Sb + D2 * bv[k] : T(1), rho2);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        S1[j] += rho1[j];
        S2[j] += rho2[j];
        P[j][k] = cdR1 * rho1[j] + cdR2 * rho2[j];
        P[j][5 - k] = coR1 * rho1[j] + coR2 * rho2[j];  // pairs (1,2) (0,2) (0,1) at 5, 4, 3
      }
    }
    const T c0 = ar * orb<T>(12), cdS1 = ar * orb<T>(13), coS1 = ar * orb<T>(15);
    const T cdS2 = ar * orb<T>(17), coS2 = ar * orb<T>(19);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T base = c0 * rc[j];
      const T bd = base + cdS1 * S1[j] + cdS2 * S2[j];
      const T bo = base + coS1 * S1[j] + coS2 * S2[j];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        P[j][a] += bd;
        P[j][3 + a] += bo;
      }
    }
  } else {
    constexpr int NQ = RULE == 0 ? 7 : 3;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const T L0 = (T)cQL[RULE][q][0], L1 = (T)cQL[RULE][q][1], L2 = (T)cQL[RULE][q][2];
      const T sq = L0 * u[0][0] + L1 * u[1][0] + L2 * u[2][0];
      const T eq = L0 * u[0][1] + L1 * u[1][1] + L2 * u[2][1];
      const T iq = L0 * u[0][2] + L1 * u[1][2] + L2 * u[2][2];
      const T N = L0 * Nv[0] + L1 * Nv[1] + L2 * Nv[2];
      const T bq = BF ? L0 * bv[0] + L1 * bv[1] + L2 * bv[2] : T(1);
      bad |= !(N > T(0));
      const T invN = T(1) / N;
      const T kappa = T(1) - A * invN;
      const T lam = (bi * iq + be * eq) * bq;
      const T ksb = kappa * sq * bq;
      T rho[4];
      rho[0] = PIC ? kappa * bi * iq * bq : A * invN * invN * sq * lam;
      rho[1] = kappa * lam;
      rho[2] = ksb * be;
      rho[3] = ksb * bi;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const T cw = (T)cQC[RULE][q][s];  // w_q phi_a phi_b; the area multiplies once at the end
#pragma unroll
        for (int k = 0; k < 4; ++k) P[k][s] += cw * rho[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int s = 0; s < 6; ++s) P[k][s] *= dtT * Tt.area;
  }
  if (bad) atomicOr(err, 1);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int s = 0; s < 6; ++s) out[REC_P + 4 * s + k] = P[k][s];
  out[REC_K + 6] = T(0);
}

// dt, nubar_S..R, alpha, mu, sigma, gamma_E, gamma_R, gamma_D in type T.  FP32 kernels with one
// set of rates (no per-sample table) convert them once per CTA: GB300 converts FP64 to FP32
// at its FP64 rate, which per thread would cost as much as the block's arithmetic.  Every
// thread of the CTA calls it.
template <class T>
__device__ __forceinline__ void rate_consts(const Rates& rin, const Rates& r, T (&k)[11]) {
  auto fill = [](const Rates& q, T* o) {
    o[0] = (T)q.dt;
    for (int c = 0; c < 4; ++c) o[1 + c] = (T)q.nu[c];
    o[5] = (T)q.alpha;
    o[6] = (T)q.mu;
    o[7] = (T)q.sigma;
    o[8] = (T)q.ge;
    o[9] = (T)q.gr;
    o[10] = (T)q.gd;
  };
  if (sizeof(T) == 4 && !rin.tab) {
    __shared__ T sk[11];
    if (threadIdx.x == 0) fill(rin, sk);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 11; ++i) k[i] = sk[i];
  } else {
    fill(r, k);
  }
}

// Writes each thread's 5x5 block B to val[25 k ...] through shared memory, so that a
// warp stores its 32 consecutive blocks as contiguous 800-value runs (one thread per
// block would store 25 values 200 bytes apart per instruction).  Every thread of
// the CTA calls it; blocks k >= nnzb are not written.
template <class T>
__device__ __forceinline__ void stage_store25(const T (&B)[5][5], int64_t k, int64_t nnzb, T* __restrict__ val) {
  __shared__ T sm[128 * 25];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* ws = sm + warp * 32 * 25;
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) ws[lane * 25 + 5 * i + c] = B[i][c];
  __syncwarp();
  const int64_t k0 = k - lane;  // the warp's first block
  const int64_t nb = nnzb - k0 < 32 ? nnzb - k0 : 32;
  if (nb <= 0) return;
  T* dst = val + 25 * k0;
  for (int j = lane; j < 25 * nb; j += 32) dst[j] = ws[j];
}

// One thread per 5x5 block: fixed-order sums over the triangles sharing the
// node pair, then the block of dF_i/dU_j:
//   M delta + dt nubar_c (G_c + K delta) - dt int phi_i phi_j dR_c/du_c'.
// RULE: the reaction quadrature.  The degree-5 rule integrates the linear
// reaction terms exactly (consistent mass Mr = M); the vertex rule lumps them
// (Mr = |T|/3 on the diagonal pair only), and the Jacobian follows the residual.
template <class T, bool PIC, int RULE>
__global__ void __launch_bounds__(128) k_jac_gather(int64_t nnzb, const int32_t* __restrict__ inc_ptr,
                                                    const int32_t* __restrict__ inc, const T* __restrict__ rec,
                                                    const int32_t* __restrict__ tri, Rates rin,
                                                    T* __restrict__ val) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = k < nnzb;
  Rates r = rin;
  if (live && rin.tab) {  // the block row's node: row vertex of the first incident triangle
    const int32_t e = inc[inc_ptr[k]];
    r = rates_at(rin, tri[3 * (int64_t)(e / 9) + (e % 9) / 3]);
  }
  T M = 0, Mr = 0, K = 0, G[4] = {0, 0, 0, 0}, P[4] = {0, 0, 0, 0};
  const int32_t q0 = live ? inc_ptr[k] : 0, q1 = live ? inc_ptr[k + 1] : 0;
  for (int32_t q = q0; q < q1; ++q) {
    const int32_t e = inc[q];
    const int32_t t = e / 9, ab = e - 9 * t;
    const int a = ab / 3, b = ab - 3 * a;
    const T* R = rec + (int64_t)REC * t;
    const int s = sym(a, b);
    M += R[0] * (a == b ? T(2.0 / 12.0) : T(1.0 / 12.0));
    if (RULE == 1 && a == b) Mr += R[0] * T(1.0 / 3.0);
    K += R[REC_K + s];
    if (!PIC) {
#pragma unroll
      for (int c = 0; c < 4; ++c) G[c] += R[REC_G + 4 * a + c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) P[c] += R[REC_P + 4 * s + c];
  }
  if (RULE == 0) Mr = M;
  // K, G and P arrive scaled by dt (G_c by dt nubar_c), see k_jac_record
  T rk[11];
  rate_consts<T>(rin, r, rk);
  const T dt = rk[0];
  const T nu0 = rk[1], nu1 = rk[2], nu2 = rk[3], nu3 = rk[4];
  const T dMr = dt * Mr;
  const T alpha = rk[5], mu = rk[6], sigma = rk[7], ge = rk[8], gr = rk[9], gd = rk[10];
  T B[5][5];
#pragma unroll
  for (int i = 0; i < 5; ++i)
#pragma unroll
    for (int c = 0; c < 5; ++c) B[i][c] = T(0);
  if (PIC) {
    // Picard matrix: M + dt nubar_c K on the diagonal, minus dt int B_cc'(u^k) phi_i phi_j with
    // B of Eq. vec_component2 (P1 = kappa(beta_I i + beta_E e) b, P2 = kappa s beta_E b,
    // P0 = kappa beta_I i b here)
#pragma unroll
    for (int c = 1; c < 5; ++c) B[0][c] = -alpha * dMr;
    B[0][0] = M + nu0 * K + (mu - alpha) * dMr + P[1];
    B[1][0] = -P[0];
    B[1][1] = M + nu1 * K - P[2] + (sigma + ge + mu) * dMr;
  } else {
    // rows S, E: transmission derivative row  dT/du_c' = P0 + [S]P1 + [E]P2 + [I]P3
    const T rS = G[0] - alpha * dMr + P[0], rE = G[1] - P[0];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      B[0][c] = rS;
      B[1][c] = rE;
      B[2][c] = G[2];
      B[3][c] = G[3];
    }
    B[0][0] += M + nu0 * K + P[1] + mu * dMr;
    B[0][1] += P[2];
    B[0][2] += P[3];
    B[1][0] -= P[1];
    B[1][1] += M + nu1 * K - P[2] + (sigma + ge + mu) * dMr;
    B[1][2] -= P[3];
  }
  B[2][1] -= sigma * dMr;
  B[2][2] += M + nu2 * K + (gr + gd + mu) * dMr;
  B[3][1] -= ge * dMr;
  B[3][2] -= gr * dMr;
  B[3][3] += M + nu3 * K + mu * dMr;
  B[4][2] -= gd * dMr;
  B[4][4] += M;
  stage_store25<T>(B, k, nnzb, val);
}

// ---- discrete-adjoint terms ------------------------------------------------

// M V per compartment with the consistent mass: element vectors |T|/12 (V_a + sum_b V_b)
__global__ void __launch_bounds__(128) k_mass_elem(int64_t m, const int32_t* __restrict__ tri,
                                                   const double* __restrict__ xy, const double* __restrict__ V,
                                                   double* __restrict__ elem) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= m) return;
  const Tri T = load_tri(tri, xy, t);
  const double m12 = T.area * (1.0 / 12.0);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = V[5 * (int64_t)T.v[a] + c];
    const double s = v[0] + v[1] + v[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) elem[15 * t + 5 * a + c] = m12 * (v[a] + s);
  }
}

// lambda^T dF/dp for the ten rates, summed per CTA (partial[cta*stride + k]),
// and the transmission-field element terms fe[t][a] = lambda^T dF/db at corner a.
// F is linear in each rate, so dF/dp_k is read off the weak form:
//   nubar_c : dt |T| mean(N) grad u_c . grad lambda_c
//   rates in R: -dt |T| sum_q w_q sum_c lambda_c(x_q) dR_c/dp(x_q), with
//     beta_I: kappa s i b (lambda_E - lambda_S)   beta_E: kappa s e b (lambda_E - lambda_S)
//     sigma : e (lambda_I - lambda_E)             gamma_E: e (lambda_R - lambda_E)
//     gamma_R: i (lambda_R - lambda_I)            gamma_D: i (lambda_D - lambda_I)
//   field b_j: dt |T| sum_q w_q phi_j kappa s (beta_I i + beta_E e) (lambda_S - lambda_E).
template <int RULE, bool BF>
__global__ void __launch_bounds__(256) k_param_contract(int64_t m, const int32_t* __restrict__ tri,
                                                        const double* __restrict__ xy, const double* __restrict__ U,
                                                        const double* __restrict__ lam,
                                                        const double* __restrict__ bfield, Rates rin, int stride,
                                                        double* __restrict__ partial, double* __restrict__ fe) {
  __shared__ double sh[8];
  double acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
    const Tri T = load_tri(tri, xy, t);
    const Rates r = rates_at(rin, T.v[0]);
    double u[3][5], l[3][5];
    double Nbar = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        u[a][c] = U[5 * (int64_t)T.v[a] + c];
        l[a][c] = lam[5 * (int64_t)T.v[a] + c];
        Nbar += u[a][c];
      }
    Nbar *= (1.0 / 3.0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double gux = u[0][c] * T.gx[0] + u[1][c] * T.gx[1] + u[2][c] * T.gx[2];
      const double guy = u[0][c] * T.gy[0] + u[1][c] * T.gy[1] + u[2][c] * T.gy[2];
      const double glx = l[0][c] * T.gx[0] + l[1][c] * T.gx[1] + l[2][c] * T.gx[2];
      const double gly = l[0][c] * T.gy[0] + l[1][c] * T.gy[1] + l[2][c] * T.gy[2];
      acc[6 + c] += r.dt * T.area * Nbar * (gux * glx + guy * gly);
    }
    double bv[3] = {1.0, 1.0, 1.0};
    if (BF) {
#pragma unroll
      for (int a = 0; a < 3; ++a) bv[a] = bfield[T.v[a]];
    }
    double f3[3] = {0.0, 0.0, 0.0};
    constexpr int NQ = RULE == 0 ? 7 : 3;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double uq[5], lq[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        uq[c] = cQL[RULE][q][0] * u[0][c] + cQL[RULE][q][1] * u[1][c] + cQL[RULE][q][2] * u[2][c];
        lq[c] = cQL[RULE][q][0] * l[0][c] + cQL[RULE][q][1] * l[1][c] + cQL[RULE][q][2] * l[2][c];
      }
      const double bq = BF ? cQL[RULE][q][0] * bv[0] + cQL[RULE][q][1] * bv[1] + cQL[RULE][q][2] * bv[2] : 1.0;
      const double N = uq[0] + uq[1] + uq[2] + uq[3] + uq[4];
      const double kappa = 1.0 - r.A / N;
      const double wq = r.dt * T.area * cQW[RULE][q];
      const double ks = kappa * uq[0];
      const double dSE = lq[1] - lq[0];
      acc[0] -= wq * ks * uq[2] * bq * dSE;
      acc[1] -= wq * ks * uq[1] * bq * dSE;
      acc[2] -= wq * uq[1] * (lq[2] - lq[1]);
      acc[3] -= wq * uq[1] * (lq[3] - lq[1]);
      acc[4] -= wq * uq[2] * (lq[3] - lq[2]);
      acc[5] -= wq * uq[2] * (lq[4] - lq[2]);
      const double fb = -wq * ks * (r.bi * uq[2] + r.be * uq[1]) * dSE;
#pragma unroll
      for (int a = 0; a < 3; ++a) f3[a] += fb * cQL[RULE][q][a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) fe[3 * t + a] = f3[a];
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
      partial[(int64_t)blockIdx.x * stride + k] = s;
    }
    __syncthreads();
  }
}

// out[i] += sum over the node's incident (t, a) of fe[3 t + a]  (fixed order)
__global__ void k_gather_scalar_add(int64_t n, const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc,
                                    const double* __restrict__ fe, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int32_t k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) s += fe[inc[k]];
  out[i] += s;
}

// misfit of one observation step (one CTA, fixed-order sum): *jacc += sum (dI^2 + dD^2);
// with rhs != NULL also rhs -= dj/du = 2 (dI, dD) at the observed entries
__global__ void k_misfit(int nobs, const int32_t* __restrict__ nodes, const double* __restrict__ Ihat,
                         const double* __restrict__ Dhat, const double* __restrict__ U, double* rhs, double* jacc) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nobs; k += blockDim.x) {
    const int64_t i = nodes[k];
    const double dI = U[5 * i + 2] - Ihat[k], dD = U[5 * i + 4] - Dhat[k];
    s += dI * dI + dD * dD;
    if (rhs) {
      rhs[5 * i + 2] -= 2.0 * dI;
      rhs[5 * i + 4] -= 2.0 * dD;
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *jacc += t;
  }
}

}  // namespace

void launch_tri_geometry(int64_t m, const int32_t* tri, const double* xy, double* geo, cudaStream_t s) {
  if (m <= 0) return;
  k_tri_geometry<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, tri, xy, geo);
  count_launch();
}

void launch_residual(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* geo, const double* U,
                     const double* Un, const double* bfield, const Rates& r, int rule, double* nd, double* elem,
                     const int32_t* inc_ptr, const int32_t* inc, double* F, double* partial, double* out_norm2,
                     int32_t* err, cudaStream_t s) {
  const int tb = 128;
  const int64_t g = (m + tb - 1) / tb;
  if (rule == 0) {
    k_residual_node<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, U, Un, r, nd);
    count_launch();
    if (bfield) k_residual_elem5<true><<<g, tb, 0, s>>>(m, tri, xy, geo, U, nd, bfield, r, elem, err);
    else k_residual_elem5<false><<<g, tb, 0, s>>>(m, tri, xy, geo, U, nd, bfield, r, elem, err);
  } else {
    if (bfield) k_residual_elem_vertex<true><<<g, tb, 0, s>>>(m, tri, xy, geo, U, Un, bfield, r, elem, err);
    else k_residual_elem_vertex<false><<<g, tb, 0, s>>>(m, tri, xy, geo, U, Un, bfield, r, elem, err);
  }
  count_launch();
  const int64_t g2 = (n + 255) / 256;
  k_residual_gather<<<g2, 256, 0, s>>>(n, inc_ptr, inc, elem, F, partial);
  count_launch();
  k_sum_partials<<<1, 1024, 0, s>>>(g2, partial, out_norm2);
  count_launch();
}

// beta(x) of the sigmoid schedule (Eq. beta_x) at every node, x = first coordinate
__global__ void k_beta_field(int64_t n, const double* __restrict__ xy, seird_beta_schedule s, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = xy[2 * i];
  const double east = (s.beta_eastern - s.beta_central) / (1.0 + exp(-s.k_eastern * (x - s.x_eastern)));
  const double west = (s.beta_western - s.beta_central) / (1.0 + exp(s.k_western * (x - s.x_western)));
  out[i] = s.beta_central + east + west;
}

void launch_beta_field(int64_t n, const double* xy, const seird_beta_schedule& s, double* out, cudaStream_t st) {
  k_beta_field<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, xy, s, out);
  count_launch();
}

template <class T, bool PIC>
static void jacobian_kernels(int64_t nnzb, int64_t m, const int32_t* tri, const double* xy, const double* geo,
                             const double* U,
                             const double* bfield, const Rates& r, int rule, T* rc, const int32_t* inc_ptr,
                             const int32_t* inc, T* val, int32_t* err, cudaStream_t s) {
  const int tb = 128;  // k_jac_gather stages 128 blocks per CTA in shared memory
  const int64_t g = (m + tb - 1) / tb;
  const int64_t g2 = (nnzb + tb - 1) / tb;
  if (rule == 0) {
    if (bfield) k_jac_record<0, true, T, PIC><<<g, tb, 0, s>>>(m, tri, xy, geo, U, bfield, r, rc, err);
    else k_jac_record<0, false, T, PIC><<<g, tb, 0, s>>>(m, tri, xy, geo, U, bfield, r, rc, err);
  } else {
    if (bfield) k_jac_record<1, true, T, PIC><<<g, tb, 0, s>>>(m, tri, xy, geo, U, bfield, r, rc, err);
    else k_jac_record<1, false, T, PIC><<<g, tb, 0, s>>>(m, tri, xy, geo, U, bfield, r, rc, err);
  }
  if (rule == 0) k_jac_gather<T, PIC, 0><<<g2, tb, 0, s>>>(nnzb, inc_ptr, inc, rc, tri, r, val);
  else k_jac_gather<T, PIC, 1><<<g2, tb, 0, s>>>(nnzb, inc_ptr, inc, rc, tri, r, val);
}

void launch_jacobian(int64_t nnzb, int64_t m, const int32_t* tri, const double* xy, const double* geo, const double* U,
                     const double* bfield, const Rates& r, int rule, void* rec, const int32_t* inc_ptr,
                     const int32_t* inc, void* val, bool fp32, bool picard, int32_t* err, cudaStream_t s) {
  if (fp32) {
    float* rc = static_cast<float*>(rec);
    float* v = static_cast<float*>(val);
    if (picard) jacobian_kernels<float, true>(nnzb, m, tri, xy, geo, U, bfield, r, rule, rc, inc_ptr, inc, v, err, s);
    else jacobian_kernels<float, false>(nnzb, m, tri, xy, geo, U, bfield, r, rule, rc, inc_ptr, inc, v, err, s);
  } else {
    double* rc = static_cast<double*>(rec);
    double* v = static_cast<double*>(val);
    if (picard) jacobian_kernels<double, true>(nnzb, m, tri, xy, geo, U, bfield, r, rule, rc, inc_ptr, inc, v, err, s);
    else jacobian_kernels<double, false>(nnzb, m, tri, xy, geo, U, bfield, r, rule, rc, inc_ptr, inc, v, err, s);
  }
  count_launch();
  count_launch();
}

void launch_mass(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* V, double* elem,
                 const int32_t* inc_ptr, const int32_t* inc, double* out, double* partial, double* norm2,
                 cudaStream_t s) {
  k_mass_elem<<<(m + 127) / 128, 128, 0, s>>>(m, tri, xy, V, elem);
  const int64_t g2 = (n + 255) / 256;
  k_residual_gather<<<g2, 256, 0, s>>>(n, inc_ptr, inc, elem, out, partial);
  k_sum_partials<<<1, 1024, 0, s>>>(g2, partial, norm2);
  count_launch();
  count_launch();
  count_launch();
}

void launch_param_contract(int64_t n, int64_t m, const int32_t* tri, const double* xy, const double* U,
                           const double* lam, const double* bfield, const Rates& r, int rule, double* partial,
                           int grid, int stride, double* fe, const int32_t* inc_ptr, const int32_t* inc,
                           double* field_out, cudaStream_t s) {
  if (rule == 0) {
    if (bfield) k_param_contract<0, true><<<grid, 256, 0, s>>>(m, tri, xy, U, lam, bfield, r, stride, partial, fe);
    else k_param_contract<0, false><<<grid, 256, 0, s>>>(m, tri, xy, U, lam, bfield, r, stride, partial, fe);
  } else {
    if (bfield) k_param_contract<1, true><<<grid, 256, 0, s>>>(m, tri, xy, U, lam, bfield, r, stride, partial, fe);
    else k_param_contract<1, false><<<grid, 256, 0, s>>>(m, tri, xy, U, lam, bfield, r, stride, partial, fe);
  }
  count_launch();
  if (field_out) {
    k_gather_scalar_add<<<(n + 255) / 256, 256, 0, s>>>(n, inc_ptr, inc, fe, field_out);
    count_launch();
  }
}

void launch_field_gather(int64_t n, const int32_t* inc_ptr, const int32_t* inc, const double* fe, double* out,
                         cudaStream_t s) {
  k_gather_scalar_add<<<(n + 255) / 256, 256, 0, s>>>(n, inc_ptr, inc, fe, out);
  count_launch();
}

void launch_misfit(int nobs, const int32_t* nodes, const double* Ihat, const double* Dhat, const double* U,
                   double* rhs, double* jacc, cudaStream_t s) {
  k_misfit<<<1, 1024, 0, s>>>(nobs, nodes, Ihat, Dhat, U, rhs, jacc);
  count_launch();
}

// ---- allocation-free residual (seird_residual_noalloc) -----------------------
// Scratch for callers that cannot allocate: element vectors of up to
// SEIRD_NOALLOC_MAX_TRIS triangles, the per-CTA partial sums of the gather, and
// the error word.  Host code must not pass the symbol itself to a kernel (on the
// host it names a stand-in, not device memory); it looks up the device address
// with cudaGetSymbolAddress once per device.
// layout: [elements 15*MAX_TRIS][node terms 8*MAX_NODES][partials][norm slot][error word]
constexpr int64_t NOALLOC_PARTIALS = (SEIRD_NOALLOC_MAX_NODES + 255) / 256;
constexpr int64_t NOALLOC_WORDS =
    15 * (int64_t)SEIRD_NOALLOC_MAX_TRIS + 8 * (int64_t)SEIRD_NOALLOC_MAX_NODES + NOALLOC_PARTIALS + 2;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_WORDS];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};
}  // namespace

}  // namespace seird

extern "C" int seird_residual_noalloc(int64_t n_nodes, int64_t n_tris, const double* xy, const int32_t* tri,
                                      const int32_t* inc_ptr, const int32_t* inc, const seird_params* params,
                                      const double* beta_field_dev, double dt, int32_t quadrature, const double* u,
                                      const double* u_prev, double* F, double* norm2, void* stream) {
  using namespace seird;
  auto fail = [](int code, const std::string& m) {
    set_global_error(m);
    return code;
  };
  if (n_nodes < 3 || n_tris < 1 || !xy || !tri || !inc_ptr || !inc || !params || !u || !u_prev || !F)
    return fail(SEIRD_EINVAL, "seird_residual_noalloc: NULL argument or empty mesh");
  if (n_tris > SEIRD_NOALLOC_MAX_TRIS || n_nodes > SEIRD_NOALLOC_MAX_NODES)
    return fail(SEIRD_EINVAL, "seird_residual_noalloc: mesh exceeds the fixed scratch (at most " +
                                  std::to_string(SEIRD_NOALLOC_MAX_TRIS) + " triangles and " +
                                  std::to_string(SEIRD_NOALLOC_MAX_NODES) + " nodes)");
  if (!(dt >= 0) || (quadrature != 0 && quadrature != 1))
    return fail(SEIRD_EINVAL, "seird_residual_noalloc: bad dt or quadrature");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {  // one-time set-up on this device (the device is current)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: cudaGetSymbolAddress: ") +
                                     cudaGetErrorString(e));
      e = upload_quadrature();  // checked copies, then a device synchronisation
      if (e != cudaSuccess)
        return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: quadrature tables: ") +
                                     cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<double*>(p);  // cached only once both steps succeeded
    }
    base = g_noalloc_ptr[dev];
  }
  double* elem = base;
  double* nd = base + 15 * (int64_t)SEIRD_NOALLOC_MAX_TRIS;
  double* partial = nd + 8 * (int64_t)SEIRD_NOALLOC_MAX_NODES;
  double* nrm = norm2 ? norm2 : partial + NOALLOC_PARTIALS;  // own slot when the caller wants no norm
  int32_t* err = reinterpret_cast<int32_t*>(partial + NOALLOC_PARTIALS + 1);
  const cudaStream_t s = (cudaStream_t)stream;
  // the error word must start at zero; elements and partials are overwritten
  e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: ") + cudaGetErrorString(e));
  Rates r{};
  r.A = params->A;
  r.bi = params->beta_i;
  r.be = params->beta_e;
  r.sigma = params->sigma;
  r.ge = params->gamma_e;
  r.gr = params->gamma_r;
  r.gd = params->gamma_d;
  r.alpha = params->alpha;
  r.mu = params->mu;
  for (int c = 0; c < 4; ++c) r.nu[c] = params->nu[c];
  r.dt = dt;
  launch_residual(n_nodes, n_tris, tri, xy, nullptr, u, u_prev, beta_field_dev, r, quadrature, nd, elem, inc_ptr, inc,
                  F, partial, nrm, err, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: launch: ") + cudaGetErrorString(e));
  int32_t flags = 0;
  e = cudaMemcpyAsync(&flags, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(SEIRD_ECUDA, std::string("seird_residual_noalloc: ") + cudaGetErrorString(e));
  if (flags) return fail(SEIRD_ENONFINITE, "seird_residual_noalloc: N <= 0 at a quadrature point");
  return SEIRD_OK;
}
