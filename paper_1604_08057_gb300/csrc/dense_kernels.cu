// Dense FP64 complex k x k kernels for the matrix sign of the tridiagonal
// T_k and the Frechet adjoint from the Theorem-1 block matrix (Sec. 2):
// in-place Gauss-Jordan inversion with partial pivoting, GEMM, and the
// scaled Newton update X <- (g X + s X^{-1}/g)/2 with deterministic norms.
// Matrices are row-major, element (i, j) at i*k + j.
#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace ov {

static inline unsigned nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__global__ void k_zero(zd* a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = mk(0.0, 0.0);
}
// batched: problem p (blockIdx.y) at a + p * sa, b + p * sb; act (may be null) switches problems off
__global__ void k_copy(const zd* __restrict__ a, int64_t sa, zd* __restrict__ b, int64_t sb, int64_t n,
                       const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[p * sb + i] = a[p * sa + i];
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
void dense_copy(const zd* a, zd* b, int64_t n, cudaStream_t st) {
  k_copy<<<nblk(n, 256), 256, 0, st>>>(a, 0, b, 0, n, nullptr);
}
void dense_copy_batch(const zd* a, int64_t sa, zd* b, int64_t sb, int64_t n, int nb, const int* act,
                      cudaStream_t st) {
  k_copy<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(a, sa, b, sb, n, act);
}
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
// Gauss-Jordan inversion with partial pivoting and no row swaps: at step kk
// the pivot is the unused row p_kk with the largest |X[p][kk]|; row p_kk is
// normalised and column kk is eliminated from every other row (the inverse is
// built in place, column kk receiving -X[i][kk]/pivot).  One launch per step,
// one block per row, reading X_in and writing X_out (ping-pong), so no block
// sees a row that another block has already rewritten.  Each thread owns a
// fixed set of columns and reads only those entries of its row and of the
// pivot row: no shared memory, no block-wide barrier.  The pivot of step kk+1
// is chosen during step kk by a 64-bit atomicMax over packed keys
//   (top 52 bits of the FP64 |X[i][kk+1]|^2) << 12 | (4095 - i),
// so the largest modulus wins and, among keys equal in those bits, the lowest
// row; the maximum does not depend on the order of arrival.  At the end
//   inv(A)[i][j] = X[p_i][q_j],  q = p^{-1}.
// ---------------------------------------------------------------------------
constexpr int GJ_THREADS = 128;
constexpr int GJ_JPT = 8;   // columns per thread held in registers (k <= 1024)

// The inversion's products with explicit roundings, so that every kernel form
// (one launch per step, or one cooperative launch) rounds them identically,
// whatever the compiler would contract on its own.
__device__ __forceinline__ double gj_nrm(zd a) { return fma(a.re, a.re, a.im * a.im); }
__device__ __forceinline__ zd gj_mul(zd a, zd b) {
  return mk(fma(a.re, b.re, -(a.im * b.im)), fma(a.re, b.im, a.im * b.re));
}
__device__ __forceinline__ zd gj_recip(zd b) {
  const double d = gj_nrm(b);
  return mk(b.re / d, -b.im / d);
}

__device__ __forceinline__ unsigned long long gj_key(double nrm, int i) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(nrm);
  return ((b >> 12) << 12) | (unsigned long long)(4095 - i);
}
__device__ __forceinline__ void gj_offer(unsigned long long* key, double nrm, int i, int* err) {
  if (!(nrm >= 0.0)) {   // NaN entry: no pivot can be trusted
    atomicOr(err, ERRB_SINGULAR);
    return;
  }
  atomicMax(key, gj_key(nrm, i));
}

// Batched over problems p = blockIdx.y (matrices at stride k*k, row flags and
// pivots at stride k, keys at stride k + 1); act (may be null) switches problems off.
// used-row flags cleared and the candidates of column 0 offered (keys zeroed beforehand)
__global__ void k_gj_init(const zd* __restrict__ x, int k, unsigned long long* keys, int* used, int* err,
                          const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  used[(int64_t)p * k + i] = 0;
  gj_offer(keys + (int64_t)p * (k + 1), gj_nrm(x[(int64_t)p * k * k + (int64_t)i * k]), i, err);
}

template <int JPT>
__global__ void __launch_bounds__(GJ_THREADS, 6) k_gj_step(const zd* __restrict__ xin, zd* __restrict__ xout, int k,
                                                        int kk, unsigned long long* keys, int* used, int* prows,
                                                        double* logdet, int ld_stride, int* err,
                                                        const int* __restrict__ act) {
  const int pb = blockIdx.y;   // the problem
  if (act && !act[pb]) return;
  {
    const int64_t n = (int64_t)k * k;
    xin += pb * n;
    xout += pb * n;
    keys += (int64_t)pb * (k + 1);
    used += (int64_t)pb * k;
    prows += (int64_t)pb * k;
    if (logdet) logdet += (int64_t)pb * ld_stride;
  }
  const int i = blockIdx.x;   // the block's row
  const zd* xr = xin + (int64_t)i * k;
  zd* yr = xout + (int64_t)i * k;
  // the row's own entries do not depend on the pivot: issue them first
  zd xv[JPT > 0 ? JPT : 1];
  if (JPT > 0) {
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = threadIdx.x + q * GJ_THREADS;
      xv[q] = j < k ? xr[j] : mk(0.0, 0.0);
    }
  }
  const zd fr = xr[kk];
  const int row_used = used[i];
  const unsigned long long key = keys[kk];
  const int cand = 4095 - (int)(key & 4095ull);
  const bool bad = key == 0ull || cand < 0 || cand >= k;
  const int p = bad ? kk : cand;
  const zd* pr = xin + (int64_t)p * k;
  const zd piv = pr[kk];
  // 1/pivot and the row factor m = X[i][kk]/pivot, once per warp
  zd inv = mk(0.0, 0.0), m = mk(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) {
    inv = gj_recip(piv);
    m = gj_mul(fr, inv);
  }
  inv.re = __shfl_sync(0xffffffffu, inv.re, 0);
  inv.im = __shfl_sync(0xffffffffu, inv.im, 0);
  m.re = __shfl_sync(0xffffffffu, m.re, 0);
  m.im = __shfl_sync(0xffffffffu, m.im, 0);
  const bool offer = i != p && !row_used && kk + 1 < k;
  if (JPT > 0) {
    zd pv[JPT > 0 ? JPT : 1];
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = threadIdx.x + q * GJ_THREADS;
      pv[q] = j < k ? pr[j] : mk(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = threadIdx.x + q * GJ_THREADS;
      if (j >= k) break;
      zd v;
      if (i == p) {
        v = (j == kk) ? inv : gj_mul(pv[q], inv);
      } else if (j == kk) {
        v = mk(-m.re, -m.im);
      } else {
        v = xv[q];
        cmsub(v, m, pv[q]);
      }
      yr[j] = v;
      if (j == kk + 1 && offer) gj_offer(keys + kk + 1, gj_nrm(v), i, err);
    }
  } else {
    for (int j = threadIdx.x; j < k; j += GJ_THREADS) {
      zd v;
      if (i == p) {
        v = (j == kk) ? inv : gj_mul(pr[j], inv);
      } else if (j == kk) {
        v = mk(-m.re, -m.im);
      } else {
        v = xr[j];
        cmsub(v, m, pr[j]);
      }
      yr[j] = v;
      if (j == kk + 1 && offer) gj_offer(keys + kk + 1, gj_nrm(v), i, err);
    }
  }
  if (threadIdx.x == 0) {
    if (bad && i == 0) atomicOr(err, ERRB_SINGULAR);
    if (i == p) {
      const double nrm = gj_nrm(piv);   // |pivot| = sqrt(nrm) is positive and finite iff nrm is
      if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(err, ERRB_SINGULAR);
      if (logdet) *logdet += log(sqrt(nrm));
      prows[kk] = p;
      used[p] = 1;
    }
  }
}

__global__ void k_gj_invperm(const int* __restrict__ prows, int* q, int k, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k) q[(int64_t)p * k + prows[(int64_t)p * k + c]] = c;
}
__global__ void k_gj_gather(const zd* __restrict__ x, zd* __restrict__ out, const int* __restrict__ prows,
                            const int* __restrict__ q, int k, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = (int64_t)k * k;
  if (t >= n) return;
  const int i = (int)(t / k), j = (int)(t % k);
  out[p * n + t] = x[p * n + (int64_t)prows[(int64_t)p * k + i] * k + q[(int64_t)p * k + j]];
}

static void gj_launch_all(const zd* a, zd* ainv, zd* w0, zd* w1, int k, int nb, const int* act, int* ipiv,
                          int* used, unsigned long long* keys, double* logdet, int ld_stride, int* err,
                          cudaStream_t st) {
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)(k + 1) * nb, st);
  k_gj_init<<<dim3(nblk(k, 128), nb), 128, 0, st>>>(a, k, keys, used, err, act);
  const zd* in = a;
  zd* bufs[2] = {w0, w1};
  for (int kk = 0; kk < k; ++kk) {
    zd* out = bufs[kk & 1];
    if (k <= GJ_THREADS * GJ_JPT)
      k_gj_step<GJ_JPT><<<dim3(k, nb), GJ_THREADS, 0, st>>>(in, out, k, kk, keys, used, ipiv, logdet, ld_stride,
                                                            err, act);
    else
      k_gj_step<0><<<dim3(k, nb), GJ_THREADS, 0, st>>>(in, out, k, kk, keys, used, ipiv, logdet, ld_stride, err,
                                                       act);
    in = out;
  }
  int* q = used;   // the flags are no longer needed
  k_gj_invperm<<<dim3(nblk(k, 128), nb), 128, 0, st>>>(ipiv, q, k, act);
  k_gj_gather<<<dim3(nblk((int64_t)k * k, 256), nb), 256, 0, st>>>(in, ainv, ipiv, q, k, act);
}

// ---------------------------------------------------------------------------
// The same Gauss-Jordan inversion as one cooperative launch per inversion.
// Problem p owns blocks (0..bp-1, p); block b keeps rows [b*R, b*R + R) of its
// matrix in shared memory for all k steps, so the matrix is read once and the
// inverse written once.  Step kk needs the pivot row p_kk as it stood after
// step kk-1; every block therefore publishes, during step kk-1, its own best
// candidate row for column kk (fully updated, to a double-buffered row slot in
// global memory), then its key (plus one; 1 = no candidate) to its own word of
// step kk's key slots with a release store.  A block's wait for step kk is a
// warp reading all bp key words of the step until none is zero; their maximum
// is the pivot, so the wait and the pivot search are one round of loads.  The
// candidate row is updated and published before the bulk of the block's rows,
// so the other blocks' progress overlaps that update.  The arithmetic of every
// entry, the pivot keys and the order of the log|det| sum are those of
// k_gj_step, so both forms give identical results.  Waits are bounded by a
// time limit: a warp that runs out sets ERRB_TIMEOUT, and every block of
// every problem leaves at its next wait.
// ---------------------------------------------------------------------------
constexpr int GJP_THREADS = 256;
constexpr int GJP_RMAX = 32;                       // rows per block (one warp ranks them)
constexpr unsigned long long GJP_WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
// One full warp waits until the n words at slots are all non-zero and returns
// their maximum (in every lane), or 0 when another block gave up or the limit
// passed (then ERRB_TIMEOUT is set).
__device__ unsigned long long warp_wait_slots(const unsigned long long* slots, int n, int* err,
                                              unsigned long long limit_ns) {
  const int lane = threadIdx.x & 31;
  const unsigned long long t0 = gtimer();
  for (unsigned spin = 0;; ++spin) {
    bool all = true;
    unsigned long long m = 0ull;
    for (int q = lane; q < n; q += 32) {
      const unsigned long long v = ld_acquire_u64(slots + q);
      all = all && v != 0ull;
      m = v > m ? v : m;
    }
    if (__all_sync(0xffffffffu, all)) return warp_max_u64(m);
    if ((spin & 63u) == 63u) {
      int stop = 0;
      if (lane == 0) {
        if (*(volatile int*)err & ERRB_TIMEOUT) {
          stop = 1;
        } else if (gtimer() - t0 > limit_ns || spin > (1u << 22)) {
          atomicOr(err, ERRB_TIMEOUT);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return 0ull;
    }
  }
}

// 16-byte asynchronous copy global -> shared (bypassing L1), and its completion
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// JPT: columns per thread (k <= JPT * GJP_THREADS); the pivot row's entries of
// the thread's columns are held in registers for the bulk update.  While a step's
// bulk update runs, warp 0 looks once (without waiting) whether every block has
// published its candidate for the next step; if so, the next pivot row is copied
// into shared memory in the background, and the next step starts from it instead
// of waiting for the keys and loading the row.
template <int JPT>
__global__ void __launch_bounds__(GJP_THREADS) k_gj_persist(const zd* __restrict__ a, zd* __restrict__ ainv, int k,
                                                          int R, int bp, zd* pub0, zd* pub1,
                                                          unsigned long long* slots, int* ipiv, double* logdet,
                                                          int ld_stride, int* err, const int* __restrict__ act,
                                                          unsigned long long limit_ns) {
  extern __shared__ double2 gjp_smem[];
  zd* xs = reinterpret_cast<zd*>(gjp_smem);   // R rows x k
  zd* pv = xs + (int64_t)R * k;               // the step's pivot row as it stood before the step
  int* prow = reinterpret_cast<int*>(pv + k); // pivot row of each step
  int* qs = prow + k;                         // inverse permutation (at the end)
  double* pn = reinterpret_cast<double*>(qs + k);   // |pivot|^2 of each step (block 0, for log|det|)
  zd* pvn = reinterpret_cast<zd*>(pn + k);          // the next step's pivot row, prefetched
  __shared__ zd ms[GJP_RMAX];                 // row factors X[i][kk] / pivot
  __shared__ int used_s[GJP_RMAX];
  __shared__ unsigned long long best_s, key_s, pre_s;
  const int pb = blockIdx.y;
  if (act && !act[pb]) return;
  const int b = blockIdx.x, t = threadIdx.x;
  const int r0 = b * R, nr = min(R, k - r0);
  const int64_t n = (int64_t)k * k;
  a += pb * n;
  ainv += pb * n;
  slots += (int64_t)pb * (k + 1) * GJ_KEY_SLOTS;
  ipiv += (int64_t)pb * k;
  if (logdet) logdet += (int64_t)pb * ld_stride;
  pub0 += (int64_t)pb * bp * k;
  pub1 += (int64_t)pb * bp * k;

  for (int64_t e = t; e < (int64_t)nr * k; e += GJP_THREADS) xs[e] = a[(int64_t)r0 * k + e];
  if (t < GJP_RMAX) used_s[t] = 0;
  if (t == 0) pre_s = 0ull;
  __syncthreads();
  // offers for column 0: the rows as loaded
  if (t < 32) {
    unsigned long long key = 0ull;
    if (t < nr) {
      const double nrm = gj_nrm(xs[(int64_t)t * k]);
      if (!(nrm >= 0.0)) atomicOr(err, ERRB_SINGULAR);
      else key = gj_key(nrm, r0 + t);
    }
    key = warp_max_u64(key);
    if (t == 0) best_s = key;
  }
  __syncthreads();
  if (best_s) {
    const int lr = 4095 - (int)(best_s & 4095ull) - r0;
    for (int j = t; j < k; j += GJP_THREADS) pub0[(int64_t)b * k + j] = xs[(int64_t)lr * k + j];
  }
  __syncthreads();
  if (t == 0) st_release_u64(slots + b, best_s + 1ull);

  for (int kk = 0; kk < k; ++kk) {
    const unsigned long long pre = pre_s;   // key of this step when its pivot row was prefetched
    if (t < 32) {
      if (pre) {
        cp_async_wait_all();   // the lanes' copies of the row into pvn
        if (t == 0) key_s = pre;
      } else {
        const unsigned long long mx = warp_wait_slots(slots + (int64_t)kk * GJ_KEY_SLOTS, bp, err, limit_ns);
        if (t == 0) key_s = mx;
      }
    }
    __syncthreads();
    if (t == 0) pre_s = 0ull;
    const unsigned long long mx = key_s;
    if (mx == 0ull) return;                   // a wait gave up: every block leaves
    const unsigned long long key = mx - 1ull;
    const int p = 4095 - (int)(key & 4095ull);
    if (key == 0ull || p < 0 || p >= k) {     // every block sees the same key and leaves
      if (b == 0 && t == 0) atomicOr(err, ERRB_SINGULAR);
      return;
    }
    const zd* prg = ((kk & 1) ? pub1 : pub0) + (int64_t)(p / R) * k;
    zd pvr[JPT];
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = t + q * GJP_THREADS;
      pvr[q] = j < k ? (pre ? pvn[j] : ld_cg(prg + j)) : mk(0.0, 0.0);
      if (j < k) pv[j] = pvr[q];
    }
    const zd piv = pre ? pvn[kk] : ld_cg(prg + kk);
    const zd inv = gj_recip(piv);
    const int lp = p - r0;   // local index of the pivot row (in range only in its owner)
    if (t < nr) ms[t] = gj_mul(xs[(int64_t)t * k + kk], inv);
    if (t == 0) {
      prow[kk] = p;
      if (lp >= 0 && lp < nr) used_s[lp] = 1;
      if (b == 0) {
        // |pivot| = sqrt(nrm) is positive and finite iff nrm is; its logarithm is
        // summed after the loop, off the steps' latency chain
        const double nrm = gj_nrm(piv);
        if (!(nrm > 0.0) || !isfinite(nrm)) atomicOr(err, ERRB_SINGULAR);
        pn[kk] = nrm;
      }
    }
    __syncthreads();
    int skip = -1;
    if (kk + 1 < k) {
      // rank this block's candidates for column kk+1 by their updated entries
      if (t < 32) {
        unsigned long long kb = 0ull;
        if (t < nr && !used_s[t]) {
          zd v = xs[(int64_t)t * k + kk + 1];
          cmsub(v, ms[t], pv[kk + 1]);
          const double nrm = gj_nrm(v);
          if (!(nrm >= 0.0)) atomicOr(err, ERRB_SINGULAR);
          else kb = gj_key(nrm, r0 + t);
        }
        kb = warp_max_u64(kb);
        if (t == 0) best_s = kb;
      }
      __syncthreads();
      const unsigned long long bk = best_s;
      if (bk) {
        // update and publish the best candidate first
        skip = 4095 - (int)(bk & 4095ull) - r0;
        const zd m = ms[skip];
        zd* out = ((kk & 1) ? pub0 : pub1) + (int64_t)b * k;
        zd* row = xs + (int64_t)skip * k;
#pragma unroll
        for (int q = 0; q < JPT; ++q) {
          const int j = t + q * GJP_THREADS;
          if (j < k) {
            zd v;
            if (j == kk) {
              v = mk(-m.re, -m.im);
            } else {
              v = row[j];
              cmsub(v, m, pvr[q]);
            }
            row[j] = v;
            out[j] = v;
          }
        }
      }
      __syncthreads();
      if (t == 0) st_release_u64(slots + (int64_t)(kk + 1) * GJ_KEY_SLOTS + b, bk + 1ull);
    }
    // the rest of the block's rows: X[i][j] -= m_i X[p][j] ...
    for (int r = 0; r < nr; ++r) {
      if (r == (nr >> 1) && t < 32 && kk + 1 < k) {
        // halfway: are all of the next step's candidates published?  (one look, no wait)
        const unsigned long long* sl = slots + (int64_t)(kk + 1) * GJ_KEY_SLOTS;
        bool all = true;
        unsigned long long m1 = 0ull;
        for (int q = t; q < bp; q += 32) {
          const unsigned long long v = ld_acquire_u64(sl + q);
          all = all && v != 0ull;
          m1 = v > m1 ? v : m1;
        }
        if (__all_sync(0xffffffffu, all)) {
          m1 = warp_max_u64(m1);
          const unsigned long long key1 = m1 - 1ull;
          const int p1 = 4095 - (int)(key1 & 4095ull);
          if (key1 != 0ull && p1 >= 0 && p1 < k) {   // else the next step takes the waiting path
            __syncwarp();   // orders the lanes' acquires before every lane's copies
            const zd* src = (((kk + 1) & 1) ? pub1 : pub0) + (int64_t)(p1 / R) * k;
            for (int j = t; j < k; j += 32) cp_async16(pvn + j, src + j);
            cp_async_commit();
            if (t == 0) pre_s = m1;
          }
        }
      }
      if (r == skip || r == lp) continue;
      const zd m = ms[r];
      zd* row = xs + (int64_t)r * k;
#pragma unroll
      for (int q = 0; q < JPT; ++q) {
        const int j = t + q * GJP_THREADS;
        if (j < k) {
          zd v = row[j];
          cmsub(v, m, pvr[q]);
          row[j] = v;
        }
      }
    }
    // ... except column kk, which receives -m_i (same thread: after its own write) ...
    if (t == kk % GJP_THREADS) {
      for (int r = 0; r < nr; ++r) {
        if (r == skip || r == lp) continue;
        const zd m = ms[r];
        xs[(int64_t)r * k + kk] = mk(-m.re, -m.im);
      }
    }
    // ... and the pivot row, which is normalised
    if (lp >= 0 && lp < nr) {
      zd* row = xs + (int64_t)lp * k;
#pragma unroll
      for (int q = 0; q < JPT; ++q) {
        const int j = t + q * GJP_THREADS;
        if (j < k) row[j] = (j == kk) ? inv : gj_mul(pvr[q], inv);
      }
    }
    __syncthreads();
  }
  // inv(A)[i][j] = X[p_i][q_j] with q = p^{-1}: this block's row g goes to row q_g
  for (int c = t; c < k; c += GJP_THREADS) qs[prow[c]] = c;
  __syncthreads();
  for (int r = 0; r < nr; ++r) {
    zd* dst = ainv + (int64_t)qs[r0 + r] * k;
    const zd* src = xs + (int64_t)r * k;
    for (int j = t; j < k; j += GJP_THREADS) dst[j] = src[qs[j]];
  }
  if (b == 0) {
    for (int c = t; c < k; c += GJP_THREADS) ipiv[c] = prow[c];
    if (logdet) {
      // log|det| = sum over the steps, in step order, of log |pivot| (the terms in
      // parallel, the sum by one thread: the same operations as the step form)
      for (int c = t; c < k; c += GJP_THREADS) pn[c] = log(sqrt(pn[c]));
      __syncthreads();
      if (t == 0) {
        double ld = *logdet;
        for (int c = 0; c < k; ++c) ld += pn[c];
        *logdet = ld;
      }
    }
  }
}

// Self-test of the bounded wait: block 0's warp waits (limit_ns) on a key word
// that nothing writes and gives up; block 1's, with a 100x longer limit, must
// leave through block 0's ERRB_TIMEOUT.  how[b] = 1 when block b gave up.
__global__ void k_wait_probe(const unsigned long long* slot, int* err, int* how, unsigned long long limit_ns) {
  const unsigned long long mx = warp_wait_slots(slot, 1, err, blockIdx.x == 0 ? limit_ns : 100ull * limit_ns);
  if (threadIdx.x == 0) how[blockIdx.x] = mx == 0ull ? 1 : 0;
}
void dense_wait_probe(unsigned long long* slot, int* err, int* how, unsigned long long limit_ns, cudaStream_t st) {
  k_wait_probe<<<2, 32, 0, st>>>(slot, err, how, limit_ns);
}

// Launch shape of the persistent form for (k, nb), or false where it does not
// fit: rows per block R <= 32, the block's rows in shared memory, and all
// nb * bp blocks resident at once (a cooperative launch checks this too).
typedef void (*GjpKernel)(const zd*, zd*, int, int, int, zd*, zd*, unsigned long long*, int*, double*, int, int*,
                          const int*, unsigned long long);
static GjpKernel gjp_kernel(int k) {
  if (k <= 2 * GJP_THREADS) return k_gj_persist<2>;
  if (k <= 4 * GJP_THREADS) return k_gj_persist<4>;
  if (k <= 6 * GJP_THREADS) return k_gj_persist<6>;
  return nullptr;
}

static bool gjp_shape(int k, int nb, int* R_out, int* bp_out, size_t* smem_out) {
  int dev = 0, nsm = 0, smem_optin = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return false;
  }
  const GjpKernel kern = gjp_kernel(k);
  if (nsm <= 0 || k < 2 || !kern || nb < 1) return false;
  const int per = std::max(1, nsm / nb);
  const int R = (k + per - 1) / per;
  if (R > GJP_RMAX) return false;
  const int bp = (k + R - 1) / R;
  if (bp > GJ_KEY_SLOTS) return false;
  const size_t smem =
      ((size_t)R * k + 2 * (size_t)k) * sizeof(zd) + 2 * (size_t)k * sizeof(int) + (size_t)k * sizeof(double);
  if (smem + 2048 > (size_t)smem_optin) return false;
  // one value for every caller (worker threads may race here)
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - 2048) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GJP_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if ((int64_t)per_sm * nsm < (int64_t)bp * nb) return false;
  *R_out = R;
  *bp_out = bp;
  *smem_out = smem;
  return true;
}

// Cooperative inversions issued from different streams (the worker contexts of
// a batch) are chained through one event per device, so that no two of them
// are ever partly resident at once, each waiting for blocks that the other
// holds the room for.
namespace {
struct CoopChain {
  int dev;
  cudaEvent_t ev;
};
std::mutex g_coop_mutex;
std::vector<CoopChain> g_coop;
}  // namespace

static bool gj_persist_launch(const zd* a, zd* ainv, zd* w0, zd* w1, int k, int nb, const int* act, int* ipiv,
                              int* used, unsigned long long* keys, double* logdet, int ld_stride, int* err,
                              cudaStream_t st) {
  int R = 0, bp = 0;
  size_t smem = 0;
  if (!gjp_shape(k, nb, &R, &bp, &smem)) return false;
  // the key slots: (k + 1) steps x GJ_KEY_SLOTS words per problem, all zero at the start
  if (cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (size_t)(k + 1) * GJ_KEY_SLOTS * nb, st) != cudaSuccess)
    return false;
  unsigned long long limit = GJP_WAIT_NS;
  void* args[] = {(void*)&a,      (void*)&ainv, (void*)&k,         (void*)&R,   (void*)&bp,
                  (void*)&w0,     (void*)&w1,   (void*)&keys,      (void*)&ipiv, (void*)&logdet,
                  (void*)&ld_stride, (void*)&err, (void*)&act, (void*)&limit};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_coop_mutex);
  cudaEvent_t ev = nullptr;
  for (const CoopChain& c : g_coop)
    if (c.dev == dev) ev = c.ev;
  if (!ev) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    g_coop.push_back({dev, ev});
  }
  if (cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaLaunchCooperativeKernel((const void*)gjp_kernel(k), dim3(bp, nb), dim3(GJP_THREADS), args, smem, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaEventRecord(ev, st);
  return true;
}

// The k + 4 launches of one inversion are captured once per (k, buffers) as a
// CUDA graph and replayed on the caller's stream: the steps are short, so the
// per-launch overhead of k back-to-back launches is a large part of their time.
namespace {
struct GjGraph {
  const void* ptrs[11];
  int k, nb, ld_stride, dev;
  cudaGraphExec_t exec;
};
std::mutex g_gj_mutex;
std::vector<GjGraph> g_gj_graphs;
}  // namespace

int dense_inverse(const zd* a, zd* ainv, zd* w0, zd* w1, int k, int nb, const int* act, int* ipiv, int* used,
                  unsigned long long* keys, double* logdet, int ld_stride, int* err, int mode, cudaStream_t st) {
  if (mode != GJ_STEPS && gj_persist_launch(a, ainv, w0, w1, k, nb, act, ipiv, used, keys, logdet, ld_stride, err, st))
    return 1;
  const void* ptrs[11] = {a, ainv, w0, w1, ipiv, used, keys, logdet, err, act, nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_gj_mutex);
  for (const GjGraph& g : g_gj_graphs) {
    if (g.k == k && g.nb == nb && g.ld_stride == ld_stride && g.dev == dev && std::equal(ptrs, ptrs + 11, g.ptrs)) {
      cudaGraphLaunch(g.exec, st);
      return k + 3;
    }
  }
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    gj_launch_all(a, ainv, w0, w1, k, nb, act, ipiv, used, keys, logdet, ld_stride, err, cap);
    ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess && graph &&
         cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  }
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  if (!ok) {   // capture unavailable: launch directly
    cudaGetLastError();
    gj_launch_all(a, ainv, w0, w1, k, nb, act, ipiv, used, keys, logdet, ld_stride, err, st);
    return k + 3;
  }
  if (g_gj_graphs.size() >= 64) {
    cudaGraphExecDestroy(g_gj_graphs.front().exec);
    g_gj_graphs.erase(g_gj_graphs.begin());
  }
  GjGraph g;
  std::copy(ptrs, ptrs + 11, g.ptrs);
  g.k = k;
  g.nb = nb;
  g.ld_stride = ld_stride;
  g.dev = dev;
  g.exec = exec;
  g_gj_graphs.push_back(g);
  cudaGraphLaunch(exec, st);
  return k + 3;
}

// ---------------------------------------------------------------------------
// C = A B, complex FP64, 32 x 32 tiles, 2 x 2 outputs per thread
// ---------------------------------------------------------------------------
constexpr int GT = 32, GK = 16;
// C = op(A) op(B); op = identity (0) or conjugate transpose (1)
// C (M x N) = op(A) (M x K) op(B) (K x N), row-major with leading dimensions
// lda, ldb, ldc (op = H: the operand is stored transposed and conjugated).
// Batched over problems p = blockIdx.z: A at a + p * sa, B at b + p * sb, C at c + p * sc.
__global__ void __launch_bounds__(256) k_gemm(const zd* __restrict__ a, int64_t sa, int lda, const zd* __restrict__ b,
                                              int64_t sb, int ldb, zd* __restrict__ c, int64_t sc, int ldc, int M,
                                              int N, int K, int ha, int hb, const int* __restrict__ act) {
  __shared__ zd as[GT][GK + 1];
  __shared__ zd bs[GK][GT + 1];
  const int pz = blockIdx.z;
  if (act && !act[pz]) return;
  a += pz * sa;
  b += pz * sb;
  c += pz * sc;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  zd acc[2][2];
  for (int r = 0; r < 2; ++r)
    for (int q = 0; q < 2; ++q) acc[r][q] = mk(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int t = threadIdx.x; t < GT * GK; t += 256) {
      // op(A)[gi][gk]: row-major read along gk, or (conjugated) along gi for the adjoint
      const int r = ha ? t % GT : t / GK, q = ha ? t / GT : t % GK;
      const int gi = row0 + r, gk = k0 + q;
      zd av = mk(0.0, 0.0);
      if (gi < M && gk < K) av = ha ? conj(a[(int64_t)gk * lda + gi]) : a[(int64_t)gi * lda + gk];
      as[r][q] = av;
      const int r2 = hb ? t % GK : t / GT, q2 = hb ? t / GK : t % GT;
      const int gk2 = k0 + r2, gj = col0 + q2;
      zd bv = mk(0.0, 0.0);
      if (gk2 < K && gj < N) bv = hb ? conj(b[(int64_t)gj * ldb + gk2]) : b[(int64_t)gk2 * ldb + gj];
      bs[r2][q2] = bv;
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
      if (gi < M && gj < N) c[(int64_t)gi * ldc + gj] = acc[r][q];
    }
}
void dense_gemm(const zd* a, const zd* b, zd* c, int k, cudaStream_t st) {
  k_gemm<<<dim3(nblk(k, GT), nblk(k, GT)), 256, 0, st>>>(a, 0, k, b, 0, k, c, 0, k, k, k, k, 0, 0, nullptr);
}
void dense_gemm_op(const zd* a, int ha, const zd* b, int hb, zd* c, int k, cudaStream_t st) {
  k_gemm<<<dim3(nblk(k, GT), nblk(k, GT)), 256, 0, st>>>(a, 0, k, b, 0, k, c, 0, k, k, k, k, ha, hb, nullptr);
}
void dense_gemm_batch(const zd* a, int64_t sa, int ha, const zd* b, int64_t sb, int hb, zd* c, int64_t sc, int k,
                      int nb, const int* act, cudaStream_t st) {
  k_gemm<<<dim3(nblk(k, GT), nblk(k, GT), nb), 256, 0, st>>>(a, sa, k, b, sb, k, c, sc, k, k, k, k, ha, hb, act);
}
void dense_gemm_rect_batch(const zd* a, int64_t sa, int lda, int ha, const zd* b, int64_t sb, int ldb, int hb, zd* c,
                           int64_t sc, int ldc, int M, int N, int K, int nb, const int* act, cudaStream_t st) {
  k_gemm<<<dim3(nblk(N, GT), nblk(M, GT), nb), 256, 0, st>>>(a, sa, lda, b, sb, ldb, c, sc, ldc, M, N, K, ha, hb,
                                                             act);
}

// Low-rank start of the Frechet adjoint: E_0 = beta0_p g_p e_1^T = A B^H with
// A[:, 0] = beta0_p g_p (g at gy + p * gy_pstride, element i at i * gy_stride),
// B[:, 0] = e_1; factors are k x ld row-major, problem p at p * k * ld (zeroed first)
__global__ void k_lr_init(zd* fa, zd* fb, int k, int ld, const zd* __restrict__ gy, int64_t gy_pstride,
                          int64_t gy_stride, const double* __restrict__ beta0) {
  const int p = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const zd g = gy[p * gy_pstride + (int64_t)i * gy_stride];
  const double b0 = beta0[p];
  fa[(int64_t)p * k * ld + (int64_t)i * ld] = mk(b0 * g.re, b0 * g.im);
  fb[(int64_t)p * k * ld + (int64_t)i * ld] = mk(i == 0 ? 1.0 : 0.0, 0.0);
}
// A[:, 0:r] *= g/2,  A[:, r:2r] *= -1/(2g),  g = |det X_i|^(-1/k) when scaling, else 1
__global__ void k_lr_scale(zd* fa, int k, int ld, int r, const double* __restrict__ logdet, int ld_stride,
                           const int* __restrict__ scal, int scal_stride, const int* __restrict__ act) {
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * 2 * r) return;
  const int i = (int)(t / (2 * r)), j = (int)(t % (2 * r));
  const double g = scal[(int64_t)p * scal_stride] ? exp(-logdet[(int64_t)p * ld_stride] / k) : 1.0;
  const double f = j < r ? 0.5 * g : -0.5 / g;
  zd& v = fa[(int64_t)p * k * ld + (int64_t)i * ld + j];
  v = mk(f * v.re, f * v.im);
}
void dense_lr_init(zd* fa, zd* fb, int k, int ld, const zd* gy, int64_t gy_pstride, int64_t gy_stride,
                   const double* beta0, int nb, cudaStream_t st) {
  cudaMemsetAsync(fa, 0, sizeof(zd) * (size_t)k * ld * nb, st);
  cudaMemsetAsync(fb, 0, sizeof(zd) * (size_t)k * ld * nb, st);
  k_lr_init<<<dim3(nblk(k, 128), nb), 128, 0, st>>>(fa, fb, k, ld, gy, gy_pstride, gy_stride, beta0);
}
void dense_lr_scale(zd* fa, int k, int ld, int r, const double* logdet, int ld_stride, const int* scal,
                    int scal_stride, int nb, const int* act, cudaStream_t st) {
  k_lr_scale<<<dim3(nblk((int64_t)k * 2 * r, 256), nb), 256, 0, st>>>(fa, k, ld, r, logdet, ld_stride, scal,
                                                                      scal_stride, act);
}

// Xn = 0.5 (g X + s Xi / g);  stats += w * (|Xn - X|^2, |Xn|^2)
// Batched over problems p = blockIdx.y: matrices at stride n, log|det| at
// logdet + p * ld_stride, scaling flag scal[p * scal_stride] (or `scaling` for
// all when scal is null), stats at stats + 4 p, partials and ticket per problem.
__global__ void __launch_bounds__(256) k_newton_combine(const zd* __restrict__ x, const zd* __restrict__ xi,
                                                        zd* __restrict__ xn, int64_t n, int k,
                                                        const double* __restrict__ logdet, int ld_stride,
                                                        const int* __restrict__ scal, int scal_stride, int scaling,
                                                        double s, double w, double* stats, zd* part,
                                                        int64_t part_stride, unsigned* cnt,
                                                        const int* __restrict__ act) {
  __shared__ zd scratch[32];
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  x += p * n;
  xi += p * n;
  xn += p * n;
  stats += 4 * p;
  part += p * part_stride;
  cnt += 4 * p;
  const int sc = scal ? scal[(int64_t)p * scal_stride] : scaling;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  zd v[1] = {mk(0.0, 0.0)};
  const double g = sc ? exp(-logdet[(int64_t)p * ld_stride] / k) : 1.0;
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
    // the last block sums the partials: thread t takes blocks t, t + 256, ... in
    // order, then the fixed tree of block_sum (the same order on every run; one
    // thread alone would be a chain of k^2 / 256 dependent FP64 additions)
    zd t = mk(0.0, 0.0);
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t = t + ld_cg(part + b);
    zd tv[1] = {t};
    block_sum<1>(tv, scratch);
    if (threadIdx.x == 0) {
      stats[0] += w * tv[0].re;
      stats[1] += w * tv[0].im;
    }
  }
}
// Frobenius-norm scaling of the Newton step (Higham, "Functions of Matrices",
// ch. 5): g = (||X^{-1}||_F / ||X||_F)^{1/2}.  The combine kernel takes its scale
// as exp(-ld / k) (the determinant form), so the norm form is written as the
// equivalent ld = -(k / 4) log(||X^{-1}||_F^2 / ||X||_F^2).  Per problem p
// (blockIdx.y): NSB blocks sum |x|^2 and |xi|^2 over strided entries, the last
// block to arrive adds the partials in block order (deterministic).
constexpr int NSB = 64;
__global__ void __launch_bounds__(256) k_norm_scale(const zd* __restrict__ x, const zd* __restrict__ xi, int64_t n,
                                                    int k, double* ld, int ld_stride, zd* part, unsigned* cnt,
                                                    const int* __restrict__ act) {
  __shared__ zd scratch[32];
  const int p = blockIdx.y;
  if (act && !act[p]) return;
  x += p * n;
  xi += p * n;
  part += (int64_t)p * NSB;
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a += norm2(x[i]);
    b += norm2(xi[i]);
  }
  zd v[1] = {mk(a, b)};
  block_sum<1>(v, scratch);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (arrive_last(cnt + p, gridDim.x)) {
    if (threadIdx.x == 0) {
      zd t = mk(0.0, 0.0);
      for (unsigned q = 0; q < gridDim.x; ++q) t = t + ld_cg(part + q);
      ld[(int64_t)p * ld_stride] = -0.25 * k * log(t.im / t.re);
    }
  }
}
void dense_norm_scale(const zd* x, const zd* xi, int k, int nb, const int* act, double* ld, int ld_stride, zd* part,
                      unsigned* cnt, cudaStream_t st) {
  const int64_t n = (int64_t)k * k;
  const unsigned g = std::min<unsigned>(NSB, nblk(n, 256));
  k_norm_scale<<<dim3(g, nb), 256, 0, st>>>(x, xi, n, k, ld, ld_stride, part, cnt, act);
}

void dense_newton_combine(const zd* x, const zd* xi, zd* xn, int k, const double* logdet, int scaling,
                          double s, double w, double* stats, zd* part, unsigned* cnt, cudaStream_t st) {
  const int64_t n = (int64_t)k * k;
  k_newton_combine<<<nblk(n, 256), 256, 0, st>>>(x, xi, xn, n, k, logdet, 0, nullptr, 0, scaling, s, w, stats, part,
                                                 0, cnt, nullptr);
}
void dense_newton_combine_batch(const zd* x, const zd* xi, zd* xn, int k, int nb, const int* act,
                                const double* logdet, int ld_stride, const int* scal, int scal_stride, double s,
                                double w, double* stats, zd* part, int64_t part_stride, unsigned* cnt,
                                cudaStream_t st) {
  const int64_t n = (int64_t)k * k;
  k_newton_combine<<<dim3(nblk(n, 256), nb), 256, 0, st>>>(x, xi, xn, n, k, logdet, ld_stride, scal, scal_stride, 0,
                                                           s, w, stats, part, part_stride, cnt, act);
}

}  // namespace ov
