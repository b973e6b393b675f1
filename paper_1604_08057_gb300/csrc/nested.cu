// Nested Krylov approximation of the k x k sign, one nesting level (Sec. 4.1,
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
//      (row interchanges between neighbours), U with two superdiagonals, O(k):
//      one warp per problem stages chunks of the coefficients in shared
//      memory, lane 0 runs the elimination chain on them, the warp writes the
//      factors back.
//   2. k_nest_s: the dense S, one column j of T^{-1} per thread (forward
//      elimination of e_j with the recorded interchanges and multipliers,
//      back substitution), written as (T^{-1} + T)/2; O(k) per thread, the
//      factors staged per chunk of rows in shared memory, rows of S written
//      coalesced across the threads of a warp.
//   3. per inner step j: k_nest_matvec (w = S q_j, one warp per row), then
//      classical Gram-Schmidt twice against q_0 .. q_j, each pass as
//      k_nest_dots (one block per coefficient) and k_nest_update (tiles of 32
//      rows, eight warps splitting the sum over the basis), and
//      k_nest_normalize (the norm, column j of H, q_{j+1}; a vanishing
//      residual closes the Krylov space and sets m_eff = j + 1).  The whole
//      sequence is replayed as one CUDA graph when a call repeats its shape.
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
// |T[i+1][i]| > |current pivot|, and l_i is the multiplier of row i+1.  One warp
// per problem: the coefficients of rows [c0 + 1, c0 + kLuChunk] are staged in
// shared memory, lane 0 runs the chunk's steps, the warp writes the factors out.
constexpr int kLuChunk = 256;
__global__ void __launch_bounds__(32) k_nest_lu(const zd* __restrict__ alpha, const zd* __restrict__ beta,
                                                const double* __restrict__ delta, int k, zd* __restrict__ lu,
                                                int* __restrict__ piv, int* __restrict__ err) {
  __shared__ zd sa[kLuChunk], sb[kLuChunk], o0[kLuChunk], o1[kLuChunk], o2[kLuChunk], ol[kLuChunk];
  __shared__ double sd[kLuChunk];
  __shared__ int op[kLuChunk];
  __shared__ zd carry[2];
  __shared__ int bad;
  const int p = blockIdx.x, lane = threadIdx.x;
  const zd* a = alpha + (int64_t)p * k;
  const zd* b = beta + (int64_t)p * k;
  const double* d = delta + (int64_t)p * k;
  zd* u0 = lu + (int64_t)p * 4 * k;
  zd* u1 = u0 + k;
  zd* u2 = u1 + k;
  zd* lm = u2 + k;
  int* pv = piv + (int64_t)p * k;
  const zd zero = mk(0.0, 0.0);
  if (lane == 0) {
    carry[0] = a[0];                       // diagonal and first superdiagonal of the current row
    carry[1] = k > 1 ? b[1] : zero;
    bad = 0;
  }
  for (int c0 = 0; c0 + 1 < k; c0 += kLuChunk) {
    const int n = min(kLuChunk, k - 1 - c0);   // steps i = c0 .. c0 + n - 1
    // row i+1 of step i: T[i+1][i] = delta_{i+1}, T[i+1][i+1] = alpha_{i+1}, T[i+1][i+2] = beta_{i+2}
    for (int t = lane; t < n; t += 32) {
      const int i = c0 + t;
      sd[t] = d[i + 1];
      sa[t] = a[i + 1];
      sb[t] = i + 2 < k ? b[i + 2] : zero;
    }
    __syncwarp();
    if (lane == 0 && !bad) {
      zd dc = carry[0], uc = carry[1];
      for (int t = 0; t < n; ++t) {
        const zd sub = mk(sd[t], 0.0), dn = sa[t], un = sb[t];
        if (norm2(dc) >= norm2(sub)) {
          if (norm2(dc) == 0.0) {          // a zero column: T is singular
            bad = 1;
            break;
          }
          const zd inv = zrecip(dc);
          const zd f = sub * inv;
          o0[t] = inv;
          o1[t] = uc;
          o2[t] = zero;
          ol[t] = f;
          op[t] = 0;
          dc = dn - f * uc;
          uc = un;
        } else {
          const zd inv = zrecip(sub);
          const zd f = dc * inv;
          o0[t] = inv;
          o1[t] = dn;
          o2[t] = un;
          ol[t] = f;
          op[t] = 1;
          dc = uc - f * dn;
          uc = zero - f * un;
        }
      }
      carry[0] = dc;
      carry[1] = uc;
    }
    __syncwarp();
    if (bad) break;
    for (int t = lane; t < n; t += 32) {
      const int i = c0 + t;
      u0[i] = o0[t];
      u1[i] = o1[t];
      u2[i] = o2[t];
      lm[i] = ol[t];
      pv[i] = op[t];
    }
    __syncwarp();
  }
  if (lane != 0) return;
  const zd dc = carry[0];
  if (bad || norm2(dc) == 0.0 || !zfinite(dc)) {
    atomicOr(err, 1);
    return;
  }
  u0[k - 1] = zrecip(dc);
  u1[k - 1] = zero;
  u2[k - 1] = zero;
  lm[k - 1] = zero;
  pv[k - 1] = 0;
}

// S = (T^{-1} + T)/2, row-major at s + p * k^2; thread j computes column j.  The
// factors of rows [r0, r0 + kSChunk) are staged in shared memory by the block;
// the forward pass runs over the chunks in ascending order, the back
// substitution in descending order.
constexpr int kSThreads = 128;
constexpr int kSChunk = 128;
__global__ void __launch_bounds__(kSThreads) k_nest_s(const zd* __restrict__ alpha, const zd* __restrict__ beta,
                                                      const double* __restrict__ delta, int k,
                                                      const zd* __restrict__ lu, const int* __restrict__ piv,
                                                      zd* __restrict__ s) {
  __shared__ zd f0[kSChunk], f1[kSChunk], f2[kSChunk], fl[kSChunk];
  __shared__ int fp[kSChunk];
  const int j = blockIdx.x * kSThreads + threadIdx.x;
  const int p = blockIdx.y;
  const bool live = j < k;
  const zd* u0 = lu + (int64_t)p * 4 * k;
  const zd* u1 = u0 + k;
  const zd* u2 = u1 + k;
  const zd* lm = u2 + k;
  const int* pv = piv + (int64_t)p * k;
  zd* S = s + (int64_t)p * k * k;
  const zd zero = mk(0.0, 0.0), one = mk(1.0, 0.0);
  // forward elimination of e_j: entries above j - 1 stay zero
  const int i0 = j > 0 ? j - 1 : 0;
  if (live)
    for (int i = 0; i < i0 && i < k; ++i) S[(int64_t)i * k + j] = zero;
  zd c = i0 == j ? one : zero;
  for (int r0 = 0; r0 + 1 < k; r0 += kSChunk) {
    const int n = min(kSChunk, k - 1 - r0);      // steps i = r0 .. r0 + n - 1
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kSThreads) {
      fl[t] = lm[r0 + t];
      fp[t] = pv[r0 + t];
    }
    __syncthreads();
    if (!live) continue;
    for (int t = max(0, i0 - r0); t < n; ++t) {
      const int i = r0 + t;
      zd nx = i + 1 == j ? one : zero;
      if (fp[t]) {
        const zd tmp = c;
        c = nx;
        nx = tmp;
      }
      S[(int64_t)i * k + j] = c;
      c = nx - fl[t] * c;
    }
  }
  if (live) S[(int64_t)(k - 1) * k + j] = c;
  // back substitution with U (diagonal, two superdiagonals); S entry (x_i + T[i][j]) / 2
  const zd* a = alpha + (int64_t)p * k;
  const zd* b = beta + (int64_t)p * k;
  const double* d = delta + (int64_t)p * k;
  zd x1 = zero, x2 = zero;               // x_{i+1}, x_{i+2}
  for (int hi = k; hi > 0; hi -= kSChunk) {
    const int lo = max(0, hi - kSChunk);   // rows [lo, hi)
    __syncthreads();
    for (int t = threadIdx.x; t < hi - lo; t += kSThreads) {
      f0[t] = u0[lo + t];
      f1[t] = u1[lo + t];
      f2[t] = u2[lo + t];
    }
    __syncthreads();
    if (!live) continue;
    constexpr int PF = 8;                // column entries loaded ahead of the chain
    for (int i = hi - 1; i >= lo; i -= PF) {
      zd r[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) r[u] = i - u >= lo ? S[(int64_t)(i - u) * k + j] : zero;
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int ii = i - u;
        if (ii < lo) break;
        const int t = ii - lo;
        zd v = r[u];
        cmsub(v, f1[t], x1);
        cmsub(v, f2[t], x2);
        const zd xi = v * f0[t];
        zd tt = zero;
        if (ii == j) tt = a[j];
        else if (ii == j - 1) tt = b[j];
        else if (ii == j + 1) tt = mk(d[ii], 0.0);
        S[(int64_t)ii * k + j] = 0.5 * (xi + tt);
        x2 = x1;
        x1 = xi;
      }
    }
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

// h_c = q_c^dag w for c <= j (block c) and, when wn is given, ||w||^2 (block j + 1)
constexpr int kDotThreads = 256;
__global__ void __launch_bounds__(kDotThreads) k_nest_dots(const zd* __restrict__ q, const zd* __restrict__ w,
                                                           zd* __restrict__ hb, double* __restrict__ wn, int k, int m,
                                                           int j, const int* __restrict__ meff) {
  __shared__ zd red[32];
  const int p = blockIdx.y, c = blockIdx.x;
  if (j >= meff[p]) return;
  const zd* W = w + (int64_t)p * k;
  zd v[1] = {mk(0.0, 0.0)};
  if (c <= j) {
    const zd* Q = q + (int64_t)p * m * k + (int64_t)c * k;
    for (int i = threadIdx.x; i < k; i += kDotThreads) cdotac(v[0], Q[i], W[i]);
  } else {
    for (int i = threadIdx.x; i < k; i += kDotThreads) v[0].re += norm2(W[i]);
  }
  block_sum<1>(v, red);
  if (threadIdx.x == 0) {
    if (c <= j) hb[(int64_t)p * m + c] = v[0];
    else wn[p] = v[0].re;
  }
}

// w -= sum_{c <= j} q_c h_c over tiles of 32 rows (eight warps split the sum over
// c, combined in warp order), and H[c][j] += h_c (block 0)
constexpr int kUpdRows = 32;
constexpr int kUpdGroups = 8;
__global__ void __launch_bounds__(kUpdRows* kUpdGroups) k_nest_update(const zd* __restrict__ q, zd* __restrict__ w,
                                                                      const zd* __restrict__ hb, zd* __restrict__ h,
                                                                      int k, int m, int j,
                                                                      const int* __restrict__ meff) {
  extern __shared__ zd hs[];             // j + 1 coefficients
  __shared__ zd part[kUpdGroups][kUpdRows];
  const int p = blockIdx.y;
  if (j >= meff[p]) return;
  const int r = threadIdx.x & 31, g = threadIdx.x >> 5;
  for (int c = threadIdx.x; c <= j; c += kUpdRows * kUpdGroups) hs[c] = hb[(int64_t)p * m + c];
  __syncthreads();
  const int i = blockIdx.x * kUpdRows + r;
  const zd* Q = q + (int64_t)p * m * k;
  zd acc = mk(0.0, 0.0);
  if (i < k)
    for (int c = g; c <= j; c += kUpdGroups) cmac(acc, Q[(int64_t)c * k + i], hs[c]);
  part[g][r] = acc;
  __syncthreads();
  if (g == 0 && i < k) {
    zd t = part[0][r];
#pragma unroll
    for (int gg = 1; gg < kUpdGroups; ++gg) t = t + part[gg][r];
    zd* W = w + (int64_t)p * k;
    W[i] = W[i] - t;
  }
  if (blockIdx.x == 0) {
    zd* H = h + (int64_t)p * m * m;
    for (int c = threadIdx.x; c <= j; c += kUpdRows * kUpdGroups) H[(int64_t)c * m + j] = H[(int64_t)c * m + j] + hs[c];
  }
}

// ||w||, the breakdown test against ||S q_j|| (wn0 = its square), H[j+1][j] and
// q_{j+1} = w / ||w||; one block per problem (j + 1 < m)
__global__ void __launch_bounds__(kOrthThreads) k_nest_normalize(zd* __restrict__ q, const zd* __restrict__ w,
                                                                 zd* __restrict__ h, const double* __restrict__ wn0,
                                                                 int k, int m, int j, int* __restrict__ meff,
                                                                 int* __restrict__ err) {
  __shared__ double red[33];
  __shared__ int stop;
  const int p = blockIdx.x;
  if (j >= meff[p]) return;
  const zd* W = w + (int64_t)p * k;
  const double n2 = block_norm2(W, k, red);
  if (threadIdx.x == 0) {
    const double w0 = wn0[p];
    stop = 0;
    if (!isfinite(n2) || !isfinite(w0)) {
      atomicOr(err, 1);
      stop = 1;
    } else if (!(sqrt(n2) > kNestBreakdown * sqrt(w0))) {
      stop = 1;                          // the Krylov space of S is invariant: H_{j+1} is complete
    }
    if (stop) meff[p] = j + 1;
    else h[(int64_t)p * m * m + (int64_t)(j + 1) * m + j] = mk(sqrt(n2), 0.0);
  }
  __syncthreads();
  if (stop) return;
  const double inv = 1.0 / sqrt(n2);
  zd* Q = q + (int64_t)p * m * k + (int64_t)(j + 1) * k;
  for (int i = threadIdx.x; i < k; i += blockDim.x) Q[i] = inv * W[i];
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
  k_nest_s<<<dim3(nblk(k, kSThreads), nb), kSThreads, 0, st>>>(alpha, beta, delta, k, W.lu, W.piv, W.s);
  cudaMemsetAsync(W.q, 0, sizeof(zd) * (size_t)nb * m * k, st);
  cudaMemsetAsync(W.h, 0, sizeof(zd) * (size_t)nb * m * m, st);
  k_nest_init<<<nblk(nb, 32), 32, 0, st>>>(W.q, (int64_t)m * k, W.meff, m, nb);
  return 3;
}

int nested_arnoldi(int k, int nb, int m, const NestWs& W, int* err, cudaStream_t st) {
  int launches = 0;
  for (int j = 0; j < m; ++j) {
    const size_t smem = sizeof(zd) * (size_t)(j + 1);
    k_nest_matvec<<<dim3(nblk(k, 8), nb), 256, 0, st>>>(W.s, W.q, W.w, k, m, j, W.meff);
    for (int pass = 0; pass < 2; ++pass) {
      k_nest_dots<<<dim3(j + 1 + (pass == 0 ? 1 : 0), nb), kDotThreads, 0, st>>>(W.q, W.w, W.hb, pass == 0 ? W.wn : nullptr,
                                                                                k, m, j, W.meff);
      k_nest_update<<<dim3(nblk(k, kUpdRows), nb), kUpdRows * kUpdGroups, smem, st>>>(W.q, W.w, W.hb, W.h, k, m, j,
                                                                                       W.meff);
    }
    launches += 5;
    if (j + 1 < m) {
      k_nest_normalize<<<nb, kOrthThreads, 0, st>>>(W.q, W.w, W.h, W.wn, k, m, j, W.meff, err);
      ++launches;
    }
  }
  return launches;
}

void nested_combine(const zd* q, const zd* f, int ld, int k, int me, double beta0, zd* y, cudaStream_t st) {
  k_nest_combine<<<nblk(k, 128), 128, 0, st>>>(q, f, ld, k, me, beta0, y);
}

}  // namespace ov
