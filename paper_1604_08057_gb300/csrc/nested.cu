// Nested Krylov approximation of the k x k sign, one level of nesting (Sec. 4.1,
// which runs the TSL nested once with an inner Krylov size of 100):
//
//   S = (T_k + T_k^{-1}) / 2,   sgn(S) = sgn(T_k)
//   S Q_m = Q_m H_m + h_{m+1,m} q_{m+1} e_m^T   (Arnoldi from q_1 = e_1)
//   y = beta_0 Q_m sgn(H_m) e_1
//
// The map z -> (z + 1/z)/2 keeps the sign of Re z, and S, unlike T_k, is dense,
// so its Krylov space from e_1 is not spanned by e_1 .. e_m.  Stages, for nb
// problems at once (problem p = blockIdx.y, or blockIdx.x for the one-block
// kernels):
//   1. k_nest_lu: LU factorisation of the tridiagonal T with partial pivoting
//      (row interchanges between neighbours), U with two superdiagonals, O(k),
//      one thread per problem.
//   2. k_nest_s: the dense S, one column j of T^{-1} per thread (forward
//      elimination of e_j with the recorded interchanges and multipliers,
//      back substitution), written as (T^{-1} + T)/2; O(k) per thread, rows
//      written coalesced across the threads of a warp.
//   3. per inner step j: k_nest_matvec (w = S q_j, one warp per row) and
//      k_nest_orth (one block per problem: classical Gram-Schmidt twice
//      against q_0 .. q_j, column j of H, normalisation; a vanishing residual
//      closes the Krylov space and sets m_eff = j + 1).
//   4. the m_eff x m_eff Hessenberg H goes through the library's scaled Newton
//      sign; k_nest_combine forms y = beta_0 Q sgn(H) e_1.
// Reductions are in a fixed order, so results do not depend on scheduling.
#include <algorithm>

#include "kernels.h"

namespace ov {

namespace {

inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

constexpr double kNestBreakdown = 1e-14;
constexpr int kOrthThreads = 1024;

OV_HD zd zrecip(zd a) { return zdiv(mk(1.0, 0.0), a); }
OV_HD bool zfinite(zd a) { return isfinite(a.re) && isfinite(a.im); }

// sum of |v_i|^2 over the block, valid in every thread (fixed order)
__device__ double block_norm2(const zd* __restrict__ v, int k, double* red) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) acc += norm2(v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < nw; ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

}  // namespace

// LU of T (alpha_j = T[j][j], beta_j = T[j-1][j], delta_j = T[j][j-1]) with
// partial pivoting.  Per problem, at lu + p * 4k: [1/u0 | u1 | u2 | l], piv at p * k.
// Step i eliminates T[i+1][i]: rows i and i+1 are exchanged when
// |T[i+1][i]| > |current pivot|, and l_i is the multiplier of row i+1.
__global__ void k_nest_lu(const zd* __restrict__ alpha, const zd* __restrict__ beta, const double* __restrict__ delta,
                          int k, zd* __restrict__ lu, int* __restrict__ piv, int* __restrict__ err) {
  if (threadIdx.x != 0) return;
  const int p = blockIdx.x;
  const zd* a = alpha + (int64_t)p * k;
  const zd* b = beta + (int64_t)p * k;
  const double* d = delta + (int64_t)p * k;
  zd* u0 = lu + (int64_t)p * 4 * k;
  zd* u1 = u0 + k;
  zd* u2 = u1 + k;
  zd* lm = u2 + k;
  int* pv = piv + (int64_t)p * k;
  const zd zero = mk(0.0, 0.0);
  zd dc = a[0];                          // diagonal and first superdiagonal of the current row i
  zd uc = k > 1 ? b[1] : zero;
  for (int i = 0; i + 1 < k; ++i) {
    const zd sub = mk(d[i + 1], 0.0);    // T[i+1][i]
    const zd dn = a[i + 1];              // T[i+1][i+1]
    const zd un = i + 2 < k ? b[i + 2] : zero;   // T[i+1][i+2]
    if (norm2(dc) >= norm2(sub)) {
      if (norm2(dc) == 0.0) {            // a zero column: T is singular
        atomicOr(err, 1);
        return;
      }
      const zd f = zdiv(sub, dc);
      u0[i] = zrecip(dc);
      u1[i] = uc;
      u2[i] = zero;
      lm[i] = f;
      pv[i] = 0;
      dc = dn - f * uc;
      uc = un;
    } else {
      const zd f = zdiv(dc, sub);
      u0[i] = zrecip(sub);
      u1[i] = dn;
      u2[i] = un;
      lm[i] = f;
      pv[i] = 1;
      dc = uc - f * dn;
      uc = zero - f * un;
    }
  }
  if (norm2(dc) == 0.0 || !zfinite(dc)) {
    atomicOr(err, 1);
    return;
  }
  u0[k - 1] = zrecip(dc);
  u1[k - 1] = zero;
  u2[k - 1] = zero;
  lm[k - 1] = zero;
  pv[k - 1] = 0;
}

// S = (T^{-1} + T)/2, row-major at s + p * k^2; thread j computes column j.
__global__ void k_nest_s(const zd* __restrict__ alpha, const zd* __restrict__ beta, const double* __restrict__ delta,
                         int k, const zd* __restrict__ lu, const int* __restrict__ piv, zd* __restrict__ s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (j >= k) return;
  const zd* u0 = lu + (int64_t)p * 4 * k;
  const zd* u1 = u0 + k;
  const zd* u2 = u1 + k;
  const zd* lm = u2 + k;
  const int* pv = piv + (int64_t)p * k;
  zd* S = s + (int64_t)p * k * k;
  const zd zero = mk(0.0, 0.0), one = mk(1.0, 0.0);
  // forward elimination of e_j: entries above j - 1 stay zero
  const int i0 = j > 0 ? j - 1 : 0;
  for (int i = 0; i < i0; ++i) S[(int64_t)i * k + j] = zero;
  zd c = i0 == j ? one : zero;
  for (int i = i0; i + 1 < k; ++i) {
    zd nx = i + 1 == j ? one : zero;
    if (pv[i]) {
      const zd t = c;
      c = nx;
      nx = t;
    }
    S[(int64_t)i * k + j] = c;
    c = nx - lm[i] * c;
  }
  S[(int64_t)(k - 1) * k + j] = c;
  // back substitution with U (diagonal, two superdiagonals); S entry (x_i + T[i][j]) / 2
  const zd* a = alpha + (int64_t)p * k;
  const zd* b = beta + (int64_t)p * k;
  const double* d = delta + (int64_t)p * k;
  zd x1 = zero, x2 = zero;               // x_{i+1}, x_{i+2}
  for (int i = k - 1; i >= 0; --i) {
    zd r = S[(int64_t)i * k + j];
    cmsub(r, u1[i], x1);
    cmsub(r, u2[i], x2);
    const zd xi = r * u0[i];
    zd t = zero;
    if (i == j) t = a[j];
    else if (i == j - 1) t = b[j];
    else if (i == j + 1) t = mk(d[i], 0.0);
    S[(int64_t)i * k + j] = 0.5 * (xi + t);
    x2 = x1;
    x1 = xi;
  }
}

// q_0 = e_1 and m_eff = m for every problem (q and h zeroed beforehand)
__global__ void k_nest_init(zd* q, int64_t qstride, int* meff, int m, int nb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  q[p * qstride] = mk(1.0, 0.0);
  meff[p] = m;
}

// w = S q_j: one warp per row
__global__ void k_nest_matvec(const zd* __restrict__ s, const zd* __restrict__ q, zd* __restrict__ w, int k, int m,
                              int j, const int* __restrict__ meff) {
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= k) return;
  const double2* row = reinterpret_cast<const double2*>(s + (int64_t)p * k * k + (int64_t)i * k);
  const double2* qj = reinterpret_cast<const double2*>(q + (int64_t)p * m * k + (int64_t)j * k);
  zd acc = mk(0.0, 0.0);
  for (int l = lane; l < k; l += 32) {
    const double2 a = __ldg(row + l);
    const double2 v = qj[l];
    cmac(acc, mk(a.x, a.y), mk(v.x, v.y));
  }
  acc = warp_sum(acc);
  if (lane == 0) w[(int64_t)p * k + i] = acc;
}

// Column j of H and q_{j+1}: classical Gram-Schmidt twice, one block per problem.
__global__ void __launch_bounds__(kOrthThreads) k_nest_orth(zd* __restrict__ q, zd* __restrict__ w, zd* __restrict__ h,
                                                            int k, int m, int j, int* __restrict__ meff,
                                                            int* __restrict__ err) {
  const int p = blockIdx.x;
  if (j >= meff[p]) return;
  extern __shared__ zd hs[];             // j + 1 Gram-Schmidt coefficients
  __shared__ double red[33];
  __shared__ int stop;
  zd* Q = q + (int64_t)p * m * k;
  zd* W = w + (int64_t)p * k;
  zd* H = h + (int64_t)p * m * m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double wn0 = block_norm2(W, k, red);
  for (int pass = 0; pass < 2; ++pass) {
    for (int c = warp; c <= j; c += nw) {
      zd acc = mk(0.0, 0.0);
      for (int i = lane; i < k; i += 32) cdotac(acc, Q[(int64_t)c * k + i], W[i]);
      acc = warp_sum(acc);
      if (lane == 0) hs[c] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      zd v = W[i];
      for (int c = 0; c <= j; ++c) cmsub(v, Q[(int64_t)c * k + i], hs[c]);
      W[i] = v;
    }
    for (int c = threadIdx.x; c <= j; c += blockDim.x) H[(int64_t)c * m + j] = H[(int64_t)c * m + j] + hs[c];
    __syncthreads();
  }
  if (j + 1 >= m) return;
  const double n2 = block_norm2(W, k, red);
  if (threadIdx.x == 0) {
    stop = 0;
    if (!isfinite(n2) || !isfinite(wn0)) {
      atomicOr(err, 1);
      stop = 1;
    } else if (!(sqrt(n2) > kNestBreakdown * sqrt(wn0))) {
      stop = 1;                          // the Krylov space of S is invariant: H_{j+1} is complete
    }
    if (stop) meff[p] = j + 1;
    else H[(int64_t)(j + 1) * m + j] = mk(sqrt(n2), 0.0);
  }
  __syncthreads();
  if (stop) return;
  const double inv = 1.0 / sqrt(n2);
  for (int i = threadIdx.x; i < k; i += blockDim.x) Q[(int64_t)(j + 1) * k + i] = inv * W[i];
}

// y = beta_0 sum_{c < me} q_c F[c][0] (F row-major with leading dimension ld)
__global__ void k_nest_combine(const zd* __restrict__ q, const zd* __restrict__ f, int ld, int k, int me, double beta0,
                               zd* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  zd acc = mk(0.0, 0.0);
  for (int c = 0; c < me; ++c) cmac(acc, q[(int64_t)c * k + i], f[(int64_t)c * ld]);
  y[i] = beta0 * acc;
}

int nested_prepare(const zd* alpha, const zd* beta, const double* delta, int k, int nb, int m, const NestWs& W,
                   int* err, cudaStream_t st) {
  k_nest_lu<<<nb, 32, 0, st>>>(alpha, beta, delta, k, W.lu, W.piv, err);
  k_nest_s<<<dim3(nblk(k, 128), nb), 128, 0, st>>>(alpha, beta, delta, k, W.lu, W.piv, W.s);
  cudaMemsetAsync(W.q, 0, sizeof(zd) * (size_t)nb * m * k, st);
  cudaMemsetAsync(W.h, 0, sizeof(zd) * (size_t)nb * m * m, st);
  k_nest_init<<<nblk(nb, 32), 32, 0, st>>>(W.q, (int64_t)m * k, W.meff, m, nb);
  return 3;
}

int nested_arnoldi(int k, int nb, int m, const NestWs& W, int* err, cudaStream_t st) {
  const size_t smem = sizeof(zd) * (size_t)m;
  for (int j = 0; j < m; ++j) {
    k_nest_matvec<<<dim3(nblk(k, 8), nb), 256, 0, st>>>(W.s, W.q, W.w, k, m, j, W.meff);
    k_nest_orth<<<nb, kOrthThreads, smem, st>>>(W.q, W.w, W.h, k, m, j, W.meff, err);
  }
  return 2 * m;
}

void nested_combine(const zd* q, const zd* f, int ld, int k, int me, double beta0, zd* y, cudaStream_t st) {
  k_nest_combine<<<nblk(k, 128), 128, 0, st>>>(q, f, ld, k, me, beta0, y);
}

}  // namespace ov
