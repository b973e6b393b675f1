// FP64-accurate complex k x k products on the BF16 tensor cores, for the k x k
// iteration of the Frechet adjoint (Theorem 1), by an exact splitting of FP64
// operands into small-integer digits in the manner of Ozaki, Ogita, Oishi and
// Rump, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59
// (2012), with the digit products summed exactly in integers.
//
// C = op(A) op(B), op = identity or conjugate transpose.  Write L = op(A),
// R = op(B).  Each real plane of L is scaled per row, of R per column, by a power
// of two 2^e with every entry of the line below 2^e in magnitude, and written as
// ten base-128 digits (truncation; every digit carries the entry's sign):
//   L_il = 2^{e_i} (sum_{p=1..10} d_p,il 2^{-7p} + rho_il 2^{-70}),  |d| <= 127, |rho| < 1.
// The digits are integers, exact in BF16.  The product of two digit matrices has
// integer entries below k 127^2 < 2^24 for k <= 1024, so the tensor cores' FP32
// accumulation is exact in any order.  The 55 products with p + q <= 11 are
// formed; those with p + q >= 12 and the remainders rho are below ~12 k 2^{-70}
// of the line scales.  70 bits below the line's largest entry keep the 53 bits
// of every entry within 2^-17 of it and FP64 accuracy of the product for rows
// and columns spanning up to ~2^17 .. 2^30 (eight digits, 56 bits, measurably
// lost accuracy on the Newton iterates' inverses, whose rows span 1e7 .. 1e9).
// For each output entry the digit products are summed exactly in integer
// arithmetic by weight 2^{-7(p+q)}, converted to FP64 with at most two
// roundings, and scaled back by 2^{e_i + e_j}.  A complex product is four real
// ones, arranged so that one GEMM per left digit p covers both real planes of
// each side and every right digit q <= 11 - p: ten library BF16 GEMMs (cuBLAS,
// FP32 accumulation) per complex product; the splitting and the exact
// accumulation are the kernels below.
#include <cuda_bf16.h>
#include <cublas_v2.h>

#include <climits>

#include "kernels.h"

namespace ov {

constexpr int OZ_DIGITS = 10;           // base-128 digits per entry
constexpr int OZ_BAD = INT_MIN;         // scale marker of a line holding a non-finite entry

static inline unsigned oz_blocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// entry (a, b) of a real plane of op(M): M[a][b], or conj(M[b][a]) when h is set
__device__ __forceinline__ double oz_entry(const zd* M, int k, int h, int plane, int a, int b) {
  const zd v = h ? M[(int64_t)b * k + a] : M[(int64_t)a * k + b];
  return plane == 0 ? v.re : (h ? -v.im : v.im);
}

// The digits of r = x 2^{-e} (|x| < 2^e): d_p = sgn(x) (floor(|r| 2^{7p}) mod 128),
// p = 1 .. D, the base-128 expansion of |r| truncated after D digits (the same digits
// as repeating r <- 128 r, d = trunc(r), r <- r - d, each step of which is exact).
// Read off the binary representation in integer arithmetic: |x| = m 2^{E - 1075}
// with m the 53-bit significand (52 bits and E = 1 for subnormals), so digit p is
// bits [-sh, 7 - sh) of m with sh = E - 1075 - e + 7p.
__device__ __forceinline__ void oz_digits(double x, int e, float d[OZ_DIGITS]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const bool neg = (bits >> 63) != 0ull;
  const int E = (int)((bits >> 52) & 0x7ffull);
  const unsigned long long frac = bits & ((1ull << 52) - 1ull);
  const unsigned long long m = E ? (frac | (1ull << 52)) : frac;
  const int s0 = (E ? E : 1) - 1075 - e;
#pragma unroll
  for (int p = 0; p < OZ_DIGITS; ++p) {
    const int sh = s0 + 7 * (p + 1);
    unsigned long long v = 0ull;
    if (sh >= 0) {
      if (sh < 7) v = (m << sh) & 127ull;   // only the low 7 bits matter
    } else if (sh > -64) {
      v = (m >> (-sh)) & 127ull;
    }
    const float f = (float)(unsigned)v;
    d[p] = neg ? -f : f;
  }
}

// block-wide max of |entries| of one line and whether any entry is not finite;
// returns the line's scale exponent (or OZ_BAD) to every thread
__device__ int oz_line_scale(double m, int bad, double* red, int* redb) {
  red[threadIdx.x] = m;
  redb[threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
      redb[threadIdx.x] |= redb[threadIdx.x + s];
    }
    __syncthreads();
  }
  int e = 0;
  if (redb[0]) return OZ_BAD;
  if (red[0] > 0.0) frexp(red[0], &e);   // max = f 2^e with f in [0.5, 1)
  return e;
}

// Left factor: block a holds row a of op(M); both planes' scales, then the digits
// into dl[(p * 2 + plane) * k * k + a * k + b] (p < OZ_DIGITS).
__global__ void __launch_bounds__(256) k_oz_split_rows(const zd* __restrict__ M, int k, int h,
                                                       __nv_bfloat16* __restrict__ dl, int* __restrict__ expo) {
  __shared__ double red[256];
  __shared__ int redb[256];
  const int a = blockIdx.x;
  int e[2];
  for (int plane = 0; plane < 2; ++plane) {
    double m = 0.0;
    int bad = 0;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
      const double x = oz_entry(M, k, h, plane, a, b);
      bad |= !isfinite(x);
      m = fmax(m, fabs(x));
    }
    e[plane] = oz_line_scale(m, bad, red, redb);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    expo[a] = e[0];
    expo[k + a] = e[1];
  }
  const int64_t kk = (int64_t)k * k;
  for (int b = threadIdx.x; b < k; b += blockDim.x)
    for (int plane = 0; plane < 2; ++plane) {
      float d[OZ_DIGITS];
      oz_digits(e[plane] == OZ_BAD ? 0.0 : oz_entry(M, k, h, plane, a, b), e[plane] == OZ_BAD ? 0 : e[plane], d);
#pragma unroll
      for (int p = 0; p < OZ_DIGITS; ++p) dl[(p * 2 + plane) * kk + (int64_t)a * k + b] = __float2bfloat16(d[p]);
    }
}

// Right factor, pass 1: block b finds the scales of column b of op(M), both planes
__global__ void __launch_bounds__(256) k_oz_col_scale(const zd* __restrict__ M, int k, int h, int* __restrict__ expo) {
  __shared__ double red[256];
  __shared__ int redb[256];
  const int b = blockIdx.x;
  for (int plane = 0; plane < 2; ++plane) {
    double m = 0.0;
    int bad = 0;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
      const double x = oz_entry(M, k, h, plane, a, b);
      bad |= !isfinite(x);
      m = fmax(m, fabs(x));
    }
    const int e = oz_line_scale(m, bad, red, redb);
    if (threadIdx.x == 0) expo[plane * k + b] = e;
    __syncthreads();
  }
}

// Right factor, pass 2: digits of entry (a, b) into dr[a * 2Dk + (q * 2 + plane) * k + b]
// (row a of the k x 2Dk matrix whose column blocks are (digit q, plane); D = OZ_DIGITS)
__global__ void __launch_bounds__(256) k_oz_split_cols(const zd* __restrict__ M, int k, int h,
                                                       const int* __restrict__ expo, __nv_bfloat16* __restrict__ dr) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * k) return;
  const int a = (int)(t / k), b = (int)(t % k);
  for (int plane = 0; plane < 2; ++plane) {
    const int e = expo[plane * k + b];
    float d[OZ_DIGITS];
    oz_digits(e == OZ_BAD ? 0.0 : oz_entry(M, k, h, plane, a, b), e == OZ_BAD ? 0 : e, d);
#pragma unroll
    for (int q = 0; q < OZ_DIGITS; ++q)
      dr[(int64_t)a * 2 * OZ_DIGITS * k + (q * 2 + plane) * k + b] = __float2bfloat16(d[q]);
  }
}

// Offset (in floats) of the product block of left digit p (0-based): blocks of
// 2 (D - p) k x 2k floats, p = 0 .. D - 1 (D = OZ_DIGITS)
__host__ __device__ inline int64_t oz_prod_offset(int p, int k) {
  int64_t s = 0;
  for (int u = 0; u < p; ++u) s += (int64_t)4 * (OZ_DIGITS - u) * k * k;
  return s;
}

// The exact digit sum of one real product at output (i, j): S_t = sum_{p+q=t} P_pq
// (t = 2..11, integers below 10 * 2^24 < 2^28), then
//   sum_t S_t 2^{-7t} = hi 2^{-35} + mid 2^{-63} + lo 2^{-77}
// with hi (t = 2..5), mid (t = 6..9), lo (t = 10, 11) integers below 2^53.
__device__ __forceinline__ double oz_real_product(const float* __restrict__ prod, int k, int ap, int bp, int i,
                                                  int j) {
  int s[OZ_DIGITS] = {};   // s[t - 2]
#pragma unroll
  for (int p = 0; p < OZ_DIGITS; ++p) {
    const int nq = OZ_DIGITS - p;                 // right digits q = 0 .. nq - 1 (0-based p + q < D)
    const int64_t m = (int64_t)2 * nq * k;        // row length of this product block
    const float* blk = prod + oz_prod_offset(p, k) + ((int64_t)ap * k + i) * m + (int64_t)bp * k + j;
#pragma unroll
    for (int q = 0; q < nq; ++q) s[p + q] += __float2int_rn(blk[(int64_t)q * 2 * k]);
  }
  static_assert(OZ_DIGITS == 10, "the grouping below is for ten digits");
  const long long hi = ((long long)s[0] << 21) + ((long long)s[1] << 14) + ((long long)s[2] << 7) + s[3];
  const long long mid = ((long long)s[4] << 21) + ((long long)s[5] << 14) + ((long long)s[6] << 7) + s[7];
  const long long lo = ((long long)s[8] << 7) + s[9];
  return fma((double)hi, 0x1p-35, fma((double)mid, 0x1p-63, (double)lo * 0x1p-77));
}

__global__ void __launch_bounds__(256) k_oz_accum(const float* __restrict__ prod, int k, const int* __restrict__ el,
                                                  const int* __restrict__ er, zd* __restrict__ C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)k * k) return;
  const int i = (int)(t / k), j = (int)(t % k);
  const int lr = el[i], li = el[k + i], rr = er[j], ri = er[k + j];
  if (lr == OZ_BAD || li == OZ_BAD || rr == OZ_BAD || ri == OZ_BAD) {
    C[t] = mk(nan(""), nan(""));
    return;
  }
  const double re_re = ldexp(oz_real_product(prod, k, 0, 0, i, j), lr + rr);
  const double im_im = ldexp(oz_real_product(prod, k, 1, 1, i, j), li + ri);
  const double re_im = ldexp(oz_real_product(prod, k, 0, 1, i, j), lr + ri);
  const double im_re = ldexp(oz_real_product(prod, k, 1, 0, i, j), li + rr);
  C[t] = mk(re_re - im_im, re_im + im_re);
}

size_t oz_workspace_bytes(int k) {
  const size_t kk = (size_t)k * k;
  return 2 * 2 * OZ_DIGITS * kk * sizeof(__nv_bfloat16)          // digits of L and of R
         + (size_t)oz_prod_offset(OZ_DIGITS, k) * sizeof(float)   // digit products, 220 k^2
         + 4 * (size_t)k * sizeof(int) + 256;           // line scales
}

int oz_zgemm(void* handle, const zd* A, int hA, const zd* B, int hB, zd* C, int k, void* ws, cudaStream_t st) {
  if (k < 1 || k > OZ_MAX_K) return -1;
  cublasHandle_t h = static_cast<cublasHandle_t>(handle);
  const size_t kk = (size_t)k * k;
  __nv_bfloat16* dl = static_cast<__nv_bfloat16*>(ws);   // [p][plane][k][k]
  __nv_bfloat16* dr = dl + 2 * OZ_DIGITS * kk;             // [k][q][plane][k]
  float* prod = reinterpret_cast<float*>(dr + 2 * OZ_DIGITS * kk);
  int* el = reinterpret_cast<int*>(prod + oz_prod_offset(OZ_DIGITS, k));
  int* er = el + 2 * k;
  k_oz_split_rows<<<k, 256, 0, st>>>(A, k, hA, dl, el);
  k_oz_col_scale<<<k, 256, 0, st>>>(B, k, hB, er);
  k_oz_split_cols<<<oz_blocks((int64_t)kk, 256), 256, 0, st>>>(B, k, hB, er, dr);
  if (cudaGetLastError() != cudaSuccess) return -2;
  if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return -3;
  const float one = 1.f, zero = 0.f;
  // column-major view: P_p^T (2 nq k x 2k) = Dr^T (first 2 nq k rows, ld 2Dk) x Dl_p^T (k x 2k, ld k)
  for (int p = 0; p < OZ_DIGITS; ++p) {
    const int m = 2 * (OZ_DIGITS - p) * k;
    const cublasStatus_t cs =
        cublasGemmEx(h, CUBLAS_OP_N, CUBLAS_OP_N, m, 2 * k, k, &one, dr, CUDA_R_16BF, 2 * OZ_DIGITS * k,
                     dl + (size_t)p * 2 * kk, CUDA_R_16BF, k, &zero, prod + oz_prod_offset(p, k), CUDA_R_32F, m,
                     CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (cs != CUBLAS_STATUS_SUCCESS) return -3;
  }
  k_oz_accum<<<oz_blocks((int64_t)kk, 256), 256, 0, st>>>(prod, k, el, er, C);
  if (cudaGetLastError() != cudaSuccess) return -2;
  return 4;   // own kernel launches
}

void* oz_create_handle() {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return nullptr;
  // FP32 accumulation without reduced-precision split-K reductions: the digit
  // products must stay exact integers
  cublasSetMathMode(h, (cublasMath_t)(CUBLAS_DEFAULT_MATH | CUBLAS_MATH_DISALLOW_REDUCED_PRECISION_REDUCTION));
  return h;
}
void oz_destroy_handle(void* h) {
  if (h) cublasDestroy(static_cast<cublasHandle_t>(h));
}

}  // namespace ov
