// Shared device-side definitions: complex arithmetic, internal field layouts,
// deterministic block reductions and compensated FP32 dot products.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define OV_HD __host__ __device__ __forceinline__

namespace ov {

// ---------------------------------------------------------------------------
// complex numbers (plain struct, no library types)
// ---------------------------------------------------------------------------
template <typename R>
struct cplx {
  R re, im;
};

template <typename R> OV_HD cplx<R> mk(R a, R b) { cplx<R> z; z.re = a; z.im = b; return z; }
template <typename R> OV_HD cplx<R> operator+(cplx<R> a, cplx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R> OV_HD cplx<R> operator-(cplx<R> a, cplx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R> OV_HD cplx<R> operator-(cplx<R> a) { return mk(-a.re, -a.im); }
template <typename R> OV_HD cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> OV_HD cplx<R> operator*(R s, cplx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R> OV_HD cplx<R> conj(cplx<R> a) { return mk(a.re, -a.im); }
template <typename R> OV_HD cplx<R> times_i(cplx<R> a) { return mk(-a.im, a.re); }      // i a
template <typename R> OV_HD cplx<R> times_mi(cplx<R> a) { return mk(a.im, -a.re); }     // -i a
template <typename R> OV_HD R norm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// conj(a) * b
template <typename R> OV_HD cplx<R> cdot(cplx<R> a, cplx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
OV_HD double fma_(double a, double b, double c) { return fma(a, b, c); }
OV_HD float fma_(float a, float b, float c) { return fmaf(a, b, c); }
// acc += a * b, as four fused multiply-adds
template <typename R> OV_HD void cmac(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma_(a.re, b.re, acc.re);
  acc.re = fma_(-a.im, b.im, acc.re);
  acc.im = fma_(a.re, b.im, acc.im);
  acc.im = fma_(a.im, b.re, acc.im);
}
// acc -= a * b
template <typename R> OV_HD void cmsub(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma_(-a.re, b.re, acc.re);
  acc.re = fma_(a.im, b.im, acc.re);
  acc.im = fma_(-a.re, b.im, acc.im);
  acc.im = fma_(-a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> OV_HD void cdotac(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma_(a.re, b.re, acc.re);
  acc.re = fma_(a.im, b.im, acc.re);
  acc.im = fma_(a.re, b.im, acc.im);
  acc.im = fma_(-a.im, b.re, acc.im);
}
template <typename R> OV_HD cplx<R> czero() { return mk<R>(0, 0); }

typedef cplx<double> zd;

OV_HD zd zdiv(zd a, zd b) {
  double d = b.re * b.re + b.im * b.im;
  return mk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
template <typename R> OV_HD cplx<R> cast(zd a) { return mk<R>((R)a.re, (R)a.im); }

// ---------------------------------------------------------------------------
// Internal layouts (site-major structure of arrays, 16-byte chunks)
//   spinor, FP64: 12 chunks (one complex each):  chunk c of site s at c*V + s
//   spinor, FP32:  6 chunks (two complex each):  chunk c of site s at c*V + s
//   a spinor field occupies 24*V reals in both precisions.
//   links: 36 complex per site, entry e = nu*9 + a*3 + b at e*V + s.
// Component index of a spinor: spin*3 + colour.
// ---------------------------------------------------------------------------
template <typename R> struct Spinor { cplx<R> c[12]; };

// read-only loads go through the non-coherent path on the device
template <typename T> OV_HD T ldro(const T* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

OV_HD void load_spinor(const double* f, int64_t V, int64_t s, Spinor<double>& o) {
  const double2* p = reinterpret_cast<const double2*>(f);
#pragma unroll
  for (int c = 0; c < 12; ++c) { double2 t = p[c * V + s]; o.c[c] = mk(t.x, t.y); }
}
OV_HD void load_spinor(const float* f, int64_t V, int64_t s, Spinor<float>& o) {
  const float4* p = reinterpret_cast<const float4*>(f);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float4 t = p[c * V + s];
    o.c[2 * c] = mk(t.x, t.y);
    o.c[2 * c + 1] = mk(t.z, t.w);
  }
}
// the same through the read-only path (only for fields no kernel thread writes)
OV_HD void load_spinor_ro(const double* f, int64_t V, int64_t s, Spinor<double>& o) {
  const double2* p = reinterpret_cast<const double2*>(f);
#pragma unroll
  for (int c = 0; c < 12; ++c) { double2 t = ldro(p + c * V + s); o.c[c] = mk(t.x, t.y); }
}
OV_HD void load_spinor_ro(const float* f, int64_t V, int64_t s, Spinor<float>& o) {
  const float4* p = reinterpret_cast<const float4*>(f);
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float4 t = ldro(p + c * V + s);
    o.c[2 * c] = mk(t.x, t.y);
    o.c[2 * c + 1] = mk(t.z, t.w);
  }
}
OV_HD void store_spinor(double* f, int64_t V, int64_t s, const Spinor<double>& o) {
  double2* p = reinterpret_cast<double2*>(f);
#pragma unroll
  for (int c = 0; c < 12; ++c) p[c * V + s] = make_double2(o.c[c].re, o.c[c].im);
}
OV_HD void store_spinor(float* f, int64_t V, int64_t s, const Spinor<float>& o) {
  float4* p = reinterpret_cast<float4*>(f);
#pragma unroll
  for (int c = 0; c < 6; ++c)
    p[c * V + s] = make_float4(o.c[2 * c].re, o.c[2 * c].im, o.c[2 * c + 1].re, o.c[2 * c + 1].im);
}

// Links, FP64: 36 complex per site, entry e = nu*9 + a*3 + b at e*V + s (double2).
// Links, FP32: each direction's 9 complex padded to 10 and stored as 5 float4
// chunks (two complex each), chunk q of direction nu at (5*nu + q)*V + s, so a
// link is 5 sixteen-byte loads.  80 V floats per field.
constexpr int kLinkRealsF32 = 80;
constexpr int kLinkRealsF64 = 72;
template <typename R> constexpr int link_reals() { return sizeof(R) == 4 ? kLinkRealsF32 : kLinkRealsF64; }

OV_HD cplx<double> load_link_entry(const double* u, int64_t V, int64_t s, int e) {
  const double2 t = ldro(reinterpret_cast<const double2*>(u) + e * V + s);
  return mk(t.x, t.y);
}
OV_HD cplx<float> load_link_entry(const float* u, int64_t V, int64_t s, int e) {
  const int nu = e / 9, r = e % 9;
  const float4 t = ldro(reinterpret_cast<const float4*>(u) + (5 * nu + r / 2) * V + s);
  return (r & 1) ? mk(t.z, t.w) : mk(t.x, t.y);
}
template <typename R> struct Mat3 { cplx<R> m[9]; };
OV_HD void load_link(const double* u, int64_t V, int64_t s, int nu, Mat3<double>& o) {
#pragma unroll
  for (int e = 0; e < 9; ++e) o.m[e] = load_link_entry(u, V, s, nu * 9 + e);
}
OV_HD void load_link(const float* u, int64_t V, int64_t s, int nu, Mat3<float>& o) {
  const float4* p = reinterpret_cast<const float4*>(u) + (int64_t)5 * nu * V + s;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const float4 t = ldro(p + q * V);
    o.m[2 * q] = mk(t.x, t.y);
    if (q < 4) o.m[2 * q + 1] = mk(t.z, t.w);
  }
}

template <typename R> OV_HD void spinor_zero(Spinor<R>& a) {
#pragma unroll
  for (int c = 0; c < 12; ++c) a.c[c] = czero<R>();
}

// ---------------------------------------------------------------------------
// Lattice geometry
// ---------------------------------------------------------------------------
struct Geom {
  int nx, ny, nz, nt;
  int64_t V;
};

OV_HD void site_coords(const Geom& g, int64_t s, int c[4]) {
  c[0] = (int)(s % g.nx); s /= g.nx;
  c[1] = (int)(s % g.ny); s /= g.ny;
  c[2] = (int)(s % g.nz); s /= g.nz;
  c[3] = (int)s;
}
OV_HD int64_t site_index(const Geom& g, const int c[4]) {
  return (((int64_t)c[3] * g.nz + c[2]) * g.ny + c[1]) * g.nx + c[0];
}
// neighbour of site s in direction nu (0..3 = x,y,z,t), dir = +1 or -1, periodic
OV_HD int64_t neighbour(const Geom& g, int64_t s, const int c[4], int nu, int dir) {
  const int n[4] = {g.nx, g.ny, g.nz, g.nt};
  const int64_t stride[4] = {1, (int64_t)g.nx, (int64_t)g.nx * g.ny, (int64_t)g.nx * g.ny * g.nz};
  if (dir > 0) return (c[nu] == n[nu] - 1) ? s - (int64_t)(n[nu] - 1) * stride[nu] : s + stride[nu];
  return (c[nu] == 0) ? s + (int64_t)(n[nu] - 1) * stride[nu] : s - stride[nu];
}

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005): TwoSum and FMA-based TwoProduct).
// ---------------------------------------------------------------------------
struct Dot2f {
  float s, c;  // running sum and accumulated error
};
OV_HD void dot2_add_prod(Dot2f& a, float x, float y) {
  float p = x * y;
#ifdef __CUDA_ARCH__
  float ep = __fmaf_rn(x, y, -p);
#else
  float ep = fmaf(x, y, -p);
#endif
  float t = a.s + p;
  float z = t - a.s;
  float es = (a.s - (t - z)) + (p - z);
  a.s = t;
  a.c += es + ep;
}
// complex accumulator for sum conj(a) * b
struct ZDot2f {
  Dot2f re, im;
};
OV_HD void zdot2_zero(ZDot2f& z) { z.re.s = z.re.c = z.im.s = z.im.c = 0.f; }
OV_HD void zdot2_add(ZDot2f& z, cplx<float> a, cplx<float> b) {
  dot2_add_prod(z.re, a.re, b.re);
  dot2_add_prod(z.re, a.im, b.im);
  dot2_add_prod(z.im, a.re, b.im);
  dot2_add_prod(z.im, -a.im, b.re);
}
OV_HD zd zdot2_value(const ZDot2f& z) {
  return mk((double)z.re.s + (double)z.re.c, (double)z.im.s + (double)z.im.c);
}

// Per-thread accumulator of sum conj(a_i) b_i over one site's components:
// FP64 for double fields, Dot2 FP32 for float fields; result in FP64.
template <typename R> struct SiteDot;
template <> struct SiteDot<double> {
  zd acc;
  OV_HD void zero() { acc = mk(0.0, 0.0); }
  OV_HD void add(cplx<double> a, cplx<double> b) { cdotac(acc, a, b); }
  OV_HD zd value() const { return acc; }
};
template <> struct SiteDot<float> {
  ZDot2f acc;
  OV_HD void zero() { zdot2_zero(acc); }
  OV_HD void add(cplx<float> a, cplx<float> b) { zdot2_add(acc, a, b); }
  OV_HD zd value() const { return zdot2_value(acc); }
};

template <typename R>
OV_HD zd spinor_dot(const Spinor<R>& a, const Spinor<R>& b) {
  SiteDot<R> d;
  d.zero();
#pragma unroll
  for (int c = 0; c < 12; ++c) d.add(a.c[c], b.c[c]);
  return d.value();
}

// ---------------------------------------------------------------------------
// Deterministic reductions: fixed shuffle tree inside a warp, fixed order
// across warps, per-block partials summed in block order by the last block.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ zd warp_sum(zd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_down_sync(0xffffffffu, v.re, o);
    v.im += __shfl_down_sync(0xffffffffu, v.im, o);
  }
  return v;
}

// Sum over the block of NV complex values per thread; result valid in thread 0.
// scratch: shared array of at least NV * 32 zd.  blockDim.x must be a multiple of 32.
template <int NV>
__device__ __forceinline__ void block_sum(zd (&v)[NV], zd* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * 32 + warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      zd t = scratch[i * 32];
      for (int w = 1; w < nw; ++w) t = t + scratch[i * 32 + w];
      v[i] = t;
    }
  }
  __syncthreads();
}

// Returns true in every thread of the last block (of `total`) to arrive.
// The counter is reset by that block.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned total) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == total - 1);
    if (last) *counter = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ zd ld_cg(const zd* p) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(t.x, t.y);
}
#endif

}  // namespace ov
