// Dense FP64 complex k x k kernels for the matrix sign of the tridiagonal
// T_k and the Frechet adjoint from the Theorem-1 block matrix (Sec. 2):
// in-place Gauss-Jordan inversion with partial pivoting, GEMM, and the
// scaled Newton update X <- (g X + s X^{-1}/g)/2 with deterministic norms.
// Matrices are row-major, element (i, j) at i*k + j.
#include "kernels.h"

namespace ov {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__global__ void k_zero(zd* a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = mk(0.0, 0.0);
}
__global__ void k_copy(const zd* __restrict__ a, zd* __restrict__ b, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
__global__ void k_adjoint(const zd* __restrict__ a, zd* __restrict__ b, int k) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * k) return;
  const int i = (int)(t / k), j = (int)(t % k);
  b[(int64_t)i * k + j] = conj(a[(int64_t)j * k + i]);
}
// T[j][j] = alpha_j, T[j-1][j] = beta_j, T[j][j-1] = delta_j
__global__ void k_build_t(const zd* __restrict__ alpha, const zd* __restrict__ beta,
                          const double* __restrict__ delta, int k, zd* __restrict__ t) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  t[(int64_t)j * k + j] = alpha[j];
  if (j > 0) {
    t[(int64_t)(j - 1) * k + j] = beta[j];
    t[(int64_t)j * k + j - 1] = mk(delta[j], 0.0);
  }
}
__global__ void k_set_column0(zd* e, const zd* __restrict__ gy, int64_t stride, double beta0, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const zd g = gy[(int64_t)i * stride];
  e[(int64_t)i * k] = mk(beta0 * g.re, beta0 * g.im);
}
__global__ void k_extract_y(const zd* __restrict__ f, double beta0, int k, zd* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const zd v = f[(int64_t)i * k];
  y[i] = mk(beta0 * v.re, beta0 * v.im);
}
__global__ void k_extract_tri(const zd* __restrict__ e, int k, zd* ga, zd* gb, double* gd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  ga[j] = e[(int64_t)j * k + j];
  gb[j] = j > 0 ? e[(int64_t)(j - 1) * k + j] : mk(0.0, 0.0);
  gd[j] = j > 0 ? e[(int64_t)j * k + j - 1].re : 0.0;
}

void dense_zero(zd* a, int64_t n, cudaStream_t st) { k_zero<<<nblk(n, 256), 256, 0, st>>>(a, n); }
void dense_copy(const zd* a, zd* b, int64_t n, cudaStream_t st) { k_copy<<<nblk(n, 256), 256, 0, st>>>(a, b, n); }
void dense_adjoint(const zd* a, zd* b, int k, cudaStream_t st) {
  k_adjoint<<<nblk((int64_t)k * k, 256), 256, 0, st>>>(a, b, k);
}
void dense_build_t(const zd* alpha, const zd* beta, const double* delta, int k, zd* t, cudaStream_t st) {
  dense_zero(t, (int64_t)k * k, st);
  k_build_t<<<nblk(k, 128), 128, 0, st>>>(alpha, beta, delta, k, t);
}
void dense_set_column0(zd* e, const zd* gy, int64_t stride, double beta0, int k, cudaStream_t st) {
  dense_zero(e, (int64_t)k * k, st);
  k_set_column0<<<nblk(k, 128), 128, 0, st>>>(e, gy, stride, beta0, k);
}
void dense_extract_y(const zd* f, double beta0, int k, zd* y, cudaStream_t st) {
  k_extract_y<<<nblk(k, 128), 128, 0, st>>>(f, beta0, k, y);
}
void dense_extract_tri(const zd* e, int k, zd* ga, zd* gb, double* gd, cudaStream_t st) {
  k_extract_tri<<<nblk(k, 128), 128, 0, st>>>(e, k, ga, gb, gd);
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion in place, partial pivoting by row swaps; the column
// order is restored at the end in reverse pivot order.
// ---------------------------------------------------------------------------
constexpr int PIV_THREADS = 1024;

__global__ void __launch_bounds__(PIV_THREADS) k_gj_pivot(zd* x, int k, int kk, int* ipiv, zd* prow, zd* col,
                                                          double* logdet, int* err) {
  __shared__ double sv[PIV_THREADS / 32];
  __shared__ int si[PIV_THREADS / 32];
  __shared__ int sp;
  __shared__ zd spiv;
  // argmax |x[i][kk]|, i >= kk (ties to the smaller index)
  double best = -1.0;
  int bi = kk;
  for (int i = kk + threadIdx.x; i < k; i += blockDim.x) {
    const double a = norm2(x[(int64_t)i * k + kk]);
    if (a > best) { best = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sv[w] > sv[0] || (sv[w] == sv[0] && si[w] < si[0])) { sv[0] = sv[w]; si[0] = si[w]; }
    sp = si[0];
    ipiv[kk] = sp;
  }
  __syncthreads();
  const int p = sp;
  if (p != kk) {
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      const zd a = x[(int64_t)kk * k + c];
      x[(int64_t)kk * k + c] = x[(int64_t)p * k + c];
      x[(int64_t)p * k + c] = a;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    spiv = x[(int64_t)kk * k + kk];
    const double a = sqrt(norm2(spiv));
    if (!(a > 0.0) || !isfinite(a)) *err |= ERRB_SINGULAR;
    *logdet += log(a);
  }
  __syncthreads();
  const zd inv = zdiv(mk(1.0, 0.0), spiv);
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const zd v = (c == kk) ? inv : x[(int64_t)kk * k + c] * inv;
    prow[c] = v;
    x[(int64_t)kk * k + c] = v;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (i != kk) col[i] = x[(int64_t)i * k + kk];
}

__global__ void k_gj_elim(zd* x, int k, int kk, const zd* __restrict__ prow, const zd* __restrict__ col) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= k || c >= k || i == kk) return;
  const zd f = col[i];
  const int64_t o = (int64_t)i * k + c;
  if (c == kk) x[o] = -(f * prow[kk]);
  else x[o] = x[o] - f * prow[c];
}

__global__ void k_gj_unscramble(zd* x, int k, const int* __restrict__ ipiv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  for (int kk = k - 1; kk >= 0; --kk) {
    const int p = ipiv[kk];
    if (p != kk) {
      const zd a = x[(int64_t)i * k + kk];
      x[(int64_t)i * k + kk] = x[(int64_t)i * k + p];
      x[(int64_t)i * k + p] = a;
    }
  }
}

void dense_inverse(zd* x, int k, int* ipiv, zd* prow, zd* col, double* logdet, int* err, cudaStream_t st) {
  const dim3 eb(32, 8);
  const dim3 eg(nblk(k, 32), nblk(k, 8));
  for (int kk = 0; kk < k; ++kk) {
    k_gj_pivot<<<1, PIV_THREADS, 0, st>>>(x, k, kk, ipiv, prow, col, logdet, err);
    k_gj_elim<<<eg, eb, 0, st>>>(x, k, kk, prow, col);
  }
  k_gj_unscramble<<<nblk(k, 128), 128, 0, st>>>(x, k, ipiv);
}

// ---------------------------------------------------------------------------
// C = A B, complex FP64, 32 x 32 tiles, 2 x 2 outputs per thread
// ---------------------------------------------------------------------------
constexpr int GT = 32, GK = 16;
__global__ void __launch_bounds__(256) k_gemm(const zd* __restrict__ a, const zd* __restrict__ b,
                                              zd* __restrict__ c, int k) {
  __shared__ zd as[GT][GK + 1];
  __shared__ zd bs[GK][GT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  zd acc[2][2];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 2; ++q) acc[r][q] = mk(0.0, 0.0);
  for (int k0 = 0; k0 < k; k0 += GK) {
    for (int t = threadIdx.x; t < GT * GK; t += 256) {
      const int r = t / GK, q = t % GK;
      const int gi = row0 + r, gk = k0 + q;
      as[r][q] = (gi < k && gk < k) ? a[(int64_t)gi * k + gk] : mk(0.0, 0.0);
      const int r2 = t / GT, q2 = t % GT;
      const int gk2 = k0 + r2, gj = col0 + q2;
      bs[r2][q2] = (gk2 < k && gj < k) ? b[(int64_t)gk2 * k + gj] : mk(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      const zd a0 = as[ty * 2][q], a1 = as[ty * 2 + 1][q];
      const zd b0 = bs[q][tx * 2], b1 = bs[q][tx * 2 + 1];
      cmac(acc[0][0], a0, b0);
      cmac(acc[0][1], a0, b1);
      cmac(acc[1][0], a1, b0);
      cmac(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 2; ++q) {
      const int gi = row0 + ty * 2 + r, gj = col0 + tx * 2 + q;
      if (gi < k && gj < k) c[(int64_t)gi * k + gj] = acc[r][q];
    }
}
void dense_gemm(const zd* a, const zd* b, zd* c, int k, cudaStream_t st) {
  k_gemm<<<dim3(nblk(k, GT), nblk(k, GT)), 256, 0, st>>>(a, b, c, k);
}

// Xn = 0.5 (g X + s Xi / g);  stats += w * (|Xn - X|^2, |Xn|^2)
__global__ void __launch_bounds__(256) k_newton_combine(const zd* __restrict__ x, const zd* __restrict__ xi,
                                                        zd* __restrict__ xn, int64_t n, int k,
                                                        const double* __restrict__ logdet, int scaling,
                                                        double s, double w, double* stats, zd* part,
                                                        unsigned* cnt) {
  __shared__ zd scratch[32];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  zd v[1] = {mk(0.0, 0.0)};
  const double g = scaling ? exp(-(*logdet) / k) : 1.0;
  if (i < n) {
    const zd a = x[i], b = xi[i];
    const double h = 0.5 * s / g;
    const zd o = mk(0.5 * g * a.re + h * b.re, 0.5 * g * a.im + h * b.im);
    xn[i] = o;
    v[0] = mk(norm2(o - a), norm2(o));
  }
  block_sum<1>(v, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (arrive_last(cnt, gridDim.x)) {
    zd t = mk(0.0, 0.0);
    if (threadIdx.x == 0) {
      for (unsigned b = 0; b < gridDim.x; ++b) t = t + ld_cg(part + b);
      stats[0] += w * t.re;
      stats[1] += w * t.im;
    }
  }
}
void dense_newton_combine(const zd* x, const zd* xi, zd* xn, int k, const double* logdet, int scaling,
                          double s, double w, double* stats, zd* part, unsigned* cnt, cudaStream_t st) {
  const int64_t n = (int64_t)k * k;
  k_newton_combine<<<nblk(n, 256), 256, 0, st>>>(x, xi, xn, n, k, logdet, scaling, s, w, stats, part, cnt);
}

}  // namespace ov
