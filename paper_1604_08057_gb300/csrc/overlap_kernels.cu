// Vector kernels of the overlap operator D_ov = 1 + gamma5 sgn(H) (Sec. 1, Eq.
// overlap), its Krylov solver, and the U(1) current estimator (Sec. 4.3).  They
// work on the user layout, interleaved complex128 spinors [V][4][3] (spin
// index (e % 12) / 3 of complex element e), so the solver's vectors need no
// conversion.  Reductions are deterministic: fixed per-thread strides, a fixed
// block tree, partials summed in block order.
#include <algorithm>

#include "kernels.h"

namespace ov {

static inline unsigned ov_nblk(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// gamma5 in the chiral basis: +1 on spins 0, 1 and -1 on spins 2, 3
__device__ __forceinline__ double g5_sign(int64_t e) { return (e % 12) < 6 ? 1.0 : -1.0; }

// out = b + gamma5 x  (g5 != 0)  or  out = b + x
__global__ void k_ov_combine(const double2* __restrict__ b, const double2* __restrict__ x, double2* __restrict__ out,
                             int64_t n, int g5) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double s = g5 ? g5_sign(e) : 1.0;
  const double2 a = b[e], c = x[e];
  out[e] = make_double2(a.x + s * c.x, a.y + s * c.y);
}
void ov_combine(const double* b, const double* x, double* out, int64_t n, int g5, cudaStream_t st) {
  k_ov_combine<<<ov_nblk(n, 256), 256, 0, st>>>(reinterpret_cast<const double2*>(b),
                                                reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(out),
                                                n, g5);
}

// out = f gamma5 in (f complex)
__global__ void k_gamma5_scale(const double2* __restrict__ in, double2* __restrict__ out, int64_t n, double fr,
                               double fi) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double s = g5_sign(e);
  const double2 a = in[e];
  out[e] = make_double2(s * (fr * a.x - fi * a.y), s * (fr * a.y + fi * a.x));
}
void gamma5_scale(const double* in, double* out, int64_t n, double fr, double fi, cudaStream_t st) {
  k_gamma5_scale<<<ov_nblk(n, 256), 256, 0, st>>>(reinterpret_cast<const double2*>(in),
                                                  reinterpret_cast<double2*>(out), n, fr, fi);
}

// partial[i][blk] = sum over the block's strided elements of conj(basis_i) w
constexpr int VD_THREADS = 256;
constexpr int VD_BLOCKS = 152;
__global__ void __launch_bounds__(VD_THREADS) k_vec_dots(const double2* __restrict__ basis, int64_t stride,
                                                         const double2* __restrict__ w, int64_t n,
                                                         zd* __restrict__ partial) {
  __shared__ zd scratch[32];
  const int i = blockIdx.y;
  const double2* bi = basis + (int64_t)i * stride;
  zd acc = mk(0.0, 0.0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = bi[e], c = w[e];
    cdotac(acc, mk(a.x, a.y), mk(c.x, c.y));
  }
  zd v[1] = {acc};
  block_sum<1>(v, scratch);
  if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = v[0];
}
__global__ void k_vec_dots_final(const zd* __restrict__ partial, int nblk, int nvec, zd* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvec) return;
  zd s = mk(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = s + partial[(int64_t)i * nblk + b];
  out[i] = s;
}
void vec_dots(const double* basis, int64_t stride, int nvec, const double* w, int64_t n, zd* out, zd* partial,
              cudaStream_t st) {
  const unsigned nb = std::min<unsigned>(VD_BLOCKS, ov_nblk(n, VD_THREADS));
  k_vec_dots<<<dim3(nb, nvec), VD_THREADS, 0, st>>>(reinterpret_cast<const double2*>(basis), stride / 2,
                                                     reinterpret_cast<const double2*>(w), n, partial);
  k_vec_dots_final<<<ov_nblk(nvec, 64), 64, 0, st>>>(partial, (int)nb, nvec, out);
}

// w += s sum_i coef_i basis_i   (coefficients on the device)
__global__ void k_vec_update(double2* __restrict__ w, const double2* __restrict__ basis, int64_t stride, int nvec,
                             const zd* __restrict__ coef, double s, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  zd acc = mk(0.0, 0.0);
  for (int i = 0; i < nvec; ++i) {
    const double2 a = basis[(int64_t)i * stride + e];
    cmac(acc, coef[i], mk(a.x, a.y));
  }
  const double2 o = w[e];
  w[e] = make_double2(o.x + s * acc.re, o.y + s * acc.im);
}
void vec_update(double* w, const double* basis, int64_t stride, int nvec, const zd* coef, double s, int64_t n,
                cudaStream_t st) {
  k_vec_update<<<ov_nblk(n, 256), 256, 0, st>>>(reinterpret_cast<double2*>(w),
                                                reinterpret_cast<const double2*>(basis), stride / 2, nvec, coef, s,
                                                n);
}

__global__ void k_coef_sign(const zd* __restrict__ in, const double* __restrict__ sg, zd* __restrict__ out, int l,
                            int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double s = sg[t % l];
  out[t] = mk(s * in[t].re, s * in[t].im);
}
void coef_sign(const zd* in, const double* sg, zd* out, int l, int np, cudaStream_t st) {
  const int n = l * np;
  if (n > 0) k_coef_sign<<<ov_nblk(n, 128), 128, 0, st>>>(in, sg, out, l, n);
}

// out = f in  (f complex, in and out may coincide)
__global__ void k_vec_scale(const double2* in, double2* out, double fr, double fi, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double2 a = in[e];
  out[e] = make_double2(fr * a.x - fi * a.y, fr * a.y + fi * a.x);
}
void vec_scale(const double* in, double* out, double fr, double fi, int64_t n, cudaStream_t st) {
  k_vec_scale<<<ov_nblk(n, 256), 256, 0, st>>>(reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out),
                                               fr, fi, n);
}

// out = a - b
__global__ void k_vec_sub(const double2* a, const double2* b, double2* out, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  out[e] = make_double2(a[e].x - b[e].x, a[e].y - b[e].y);
}
void vec_sub(const double* a, const double* b, double* out, int64_t n, cudaStream_t st) {
  k_vec_sub<<<ov_nblk(n, 256), 256, 0, st>>>(reinterpret_cast<const double2*>(a), reinterpret_cast<const double2*>(b),
                                             reinterpret_cast<double2*>(out), n);
}

// U(1) current from two link gradients (Sec. 4.3): with dU = i U dTheta,
//   dL/dTheta_{x,nu} = Re sum_ab conj(g_ab) i U_ab = -Im sum_ab conj(g_ab) U_ab;
// j[x][nu] (+)= scale * (dL_re/dTheta + i dL_im/dTheta).  Links and gradients in
// the user layout [V][4][3][3], j as [V][4] complex.
__global__ void k_theta_current(const double2* __restrict__ u, const double2* __restrict__ g_re,
                                const double2* __restrict__ g_im, double2* __restrict__ j, int64_t nlinks,
                                double scale, int accumulate) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  zd a = mk(0.0, 0.0), b = mk(0.0, 0.0);
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double2 ue = u[l * 9 + e], g1 = g_re[l * 9 + e], g2 = g_im[l * 9 + e];
    cdotac(a, mk(g1.x, g1.y), mk(ue.x, ue.y));
    cdotac(b, mk(g2.x, g2.y), mk(ue.x, ue.y));
  }
  double2 o = accumulate ? j[l] : make_double2(0.0, 0.0);
  o.x += scale * (-a.im);
  o.y += scale * (-b.im);
  j[l] = o;
}
void theta_current(const double* u, const double* g_re, const double* g_im, double* j, int64_t nlinks, double scale,
                   int accumulate, cudaStream_t st) {
  k_theta_current<<<ov_nblk(nlinks, 128), 128, 0, st>>>(
      reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(g_re),
      reinterpret_cast<const double2*>(g_im), reinterpret_cast<double2*>(j), nlinks, scale, accumulate);
}

}  // namespace ov
