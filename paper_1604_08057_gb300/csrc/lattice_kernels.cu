// Lattice-vector kernels: layout conversion, H / H^dagger application, the
// two-sided Lanczos step (stencil pair + biorthogonality dots, three-term
// update), classical Gram-Schmidt re-biorthogonalisation, basis combination,
// and the reverse sweep with the gauge-force contraction.
//
// Thread mapping: one thread per lattice site (blockIdx.y = source) unless a
// kernel says otherwise.  All reductions are deterministic: per-block partials
// are summed in block order by the last block to finish.
#include <algorithm>
#include <type_traits>

#include "dslash.cuh"
#include "kernels.h"

namespace ov {

constexpr int BS = 128;   // threads per block for site kernels
constexpr int NB = 8;     // basis vectors per block in the projection dots

static inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Threads per block of the per-step site kernels: a lattice with fewer than 152
// blocks of 128 sites would leave most SMs idle (the FP64 work per site keeps a
// block busy for ~100 us on the 4x4^3 workload), so below that it runs one warp
// per block and spreads over four times as many SMs.  The per-source partial-sum
// buffer (Lat::part) is sized for 32-thread blocks.
constexpr int64_t kSmallV = 152 * 128;
static inline int site_bs(int64_t V) { return V < kSmallV ? 32 : BS; }

// Site of this thread.  MAP 0: consecutive sites.  MAP 1 ("plane" tiles): block b
// owns the whole x-y plane b (Nx*Ny sites), so the +-x and +-y neighbours and their
// links are read by threads of the same block and are served by L1.
template <int MAP>
__device__ __forceinline__ int64_t thread_site(const Geom& g) {
  if (MAP == 0) return blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int plane = g.nx * g.ny;
  return threadIdx.x < plane ? (int64_t)blockIdx.x * plane + threadIdx.x : g.V;
}
static inline bool plane_ok(const Geom& g, int max_threads) {
  const int plane = g.nx * g.ny;
  return plane >= 64 && (plane + 31) / 32 * 32 <= max_threads;
}
static inline unsigned plane_threads(const Geom& g) { return (unsigned)((g.nx * g.ny + 31) / 32 * 32); }

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_pack_spinors(const double* __restrict__ aos, R* __restrict__ dst, int64_t V, int64_t vs) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  if (x >= V) return;
  const double2* in = reinterpret_cast<const double2*>(aos) + ((int64_t)src * V + x) * 12;
  Spinor<R> o;
#pragma unroll
  for (int c = 0; c < 12; ++c) { double2 t = in[c]; o.c[c] = mk<R>((R)t.x, (R)t.y); }
  store_spinor(dst + src * vs, V, x, o);
}

// Block start of the Theorem-1 TSL: r = (t, l) and s = (t + l, l) for every
// source, in 2V-site fields (upper half at sites 0..V-1).  t may be null (zero).
template <typename R>
__global__ void k_pack_block_start(const double* __restrict__ top, const double* __restrict__ bot,
                                   R* __restrict__ r, R* __restrict__ s, int64_t V, int64_t vs) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  if (x >= V) return;
  const int64_t Vf = 2 * V;
  const double2* lb = reinterpret_cast<const double2*>(bot) + ((int64_t)src * V + x) * 12;
  const double2* tp = top ? reinterpret_cast<const double2*>(top) + ((int64_t)src * V + x) * 12 : nullptr;
  Spinor<R> rt, st, lo;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const double2 l = lb[c];
    const double2 t = tp ? tp[c] : make_double2(0.0, 0.0);
    lo.c[c] = mk<R>((R)l.x, (R)l.y);
    rt.c[c] = mk<R>((R)t.x, (R)t.y);
    st.c[c] = mk<R>((R)(t.x + l.x), (R)(t.y + l.y));
  }
  store_spinor(r + src * vs, Vf, x, rt);
  store_spinor(r + src * vs, Vf, V + x, lo);
  store_spinor(s + src * vs, Vf, x, st);
  store_spinor(s + src * vs, Vf, V + x, lo);
}

template <typename R>
__global__ void k_unpack_spinors(const R* __restrict__ f, double* __restrict__ aos, int64_t V, int64_t vs) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  if (x >= V) return;
  Spinor<R> o;
  load_spinor(f + src * vs, V, x, o);
  double2* out = reinterpret_cast<double2*>(aos) + ((int64_t)src * V + x) * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) out[c] = make_double2((double)o.c[c].re, (double)o.c[c].im);
}

template <typename R>
__global__ void k_pack_links(const double* __restrict__ aos, R* __restrict__ u, int64_t V) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= V) return;
  const double2* in = reinterpret_cast<const double2*>(aos) + x * 36;
  if constexpr (sizeof(R) == 8) {
    for (int e = 0; e < 36; ++e) {
      double2 t = in[e];
      u[2 * (e * V + x)] = t.x;
      u[2 * (e * V + x) + 1] = t.y;
    }
  } else {
    float4* o = reinterpret_cast<float4*>(u);
    for (int nu = 0; nu < 4; ++nu)
      for (int q = 0; q < 5; ++q) {
        const double2 a = in[nu * 9 + 2 * q];
        const double2 b = q < 4 ? in[nu * 9 + 2 * q + 1] : make_double2(0.0, 0.0);
        o[(5 * nu + q) * V + x] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
      }
  }
}

__global__ void k_unpack_force(const double* __restrict__ f, double* __restrict__ du, int64_t V) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= V) return;
  double2* out = reinterpret_cast<double2*>(du) + x * 36;
  const double2* in = reinterpret_cast<const double2*>(f);
  for (int e = 0; e < 36; ++e) out[e] = in[e * V + x];
}

template <typename R>
void pack_spinors(const double* aos, R* dst, int nsrc, int64_t V, int64_t vs, cudaStream_t st) {
  k_pack_spinors<R><<<dim3(nblocks(V, BS), nsrc), BS, 0, st>>>(aos, dst, V, vs);
}
template <typename R>
void pack_block_start(const double* top, const double* bot, R* r, R* s, int nsrc, int64_t V, int64_t vs,
                      cudaStream_t st) {
  k_pack_block_start<R><<<dim3(nblocks(V, BS), nsrc), BS, 0, st>>>(top, bot, r, s, V, vs);
}
template <typename R>
void unpack_spinors(const R* f, double* aos, int nsrc, int64_t V, int64_t vs, cudaStream_t st) {
  k_unpack_spinors<R><<<dim3(nblocks(V, BS), nsrc), BS, 0, st>>>(f, aos, V, vs);
}
template <typename R>
void pack_links(const double* aos, R* u, int64_t V, cudaStream_t st) {
  k_pack_links<R><<<nblocks(V, BS), BS, 0, st>>>(aos, u, V);
}
void unpack_force(const double* f, double* du, int64_t V, cudaStream_t st) {
  k_unpack_force<<<nblocks(V, BS), BS, 0, st>>>(f, du, V);
}

// ---------------------------------------------------------------------------
// H and H^dagger
// ---------------------------------------------------------------------------
// NS sources per thread share every link load; blockIdx.y indexes groups of NS sources
template <typename R, int NS, int BSZ, int MAP>
__global__ void __launch_bounds__(BSZ) k_apply_h(Lat<R> L, const R* __restrict__ in, R* __restrict__ out,
                                                 int dagger, int nsrc) {
  const int64_t x = thread_site<MAP>(L.g);
  const int s0 = blockIdx.y * NS;
  if (x >= L.g.V) return;
  const R f = dagger ? L.efinv : L.ef, fi = dagger ? L.ef : L.efinv;
  FieldLoad<R> ld[NS];
  R ft[NS], fti[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    ld[i] = FieldLoad<R>{in + (int64_t)min(s0 + i, nsrc - 1) * L.vs, L.g.V};
    ft[i] = f;
    fti[i] = fi;
  }
  Spinor<R> o[NS];
  h_site_multi<NS>(ld, L.u, L.g, x, L.kappa, ft, fti, o);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (s0 + i < nsrc) store_spinor(out + (int64_t)(s0 + i) * L.vs, L.g.V, x, o[i]);
}

// out = dH in (dagger = 0) or dH^dag in (dagger = 1) for every source, dH along the
// links L.ue (may be null) and L.mdir (App. A, Eq. WD_op is affine in the links;
// the adjoint exchanges the temporal factors and negates m)
template <typename R>
__global__ void __launch_bounds__(BS) k_apply_dh(Lat<R> L, const R* __restrict__ in, R* __restrict__ out,
                                                 int dagger) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  if (x >= L.g.V) return;
  const FieldLoad<R> ld{in + src * L.vs, L.g.V};
  Spinor<R> o;
  if (dagger)
    dh_site_ld(ld, L.ue, L.u, L.g, x, L.kappa, L.efinv, L.ef, -L.mdir, o);
  else
    dh_site_ld(ld, L.ue, L.u, L.g, x, L.kappa, L.ef, L.efinv, L.mdir, o);
  store_spinor(out + src * L.vs, L.g.V, x, o);
}
template <typename R>
void apply_dh(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st) {
  k_apply_dh<R><<<dim3(nblocks(L.g.V, BS), L.nsrc), BS, 0, st>>>(L, in, out, dagger);
}

// Sources interleaved innermost (variant APPLY_IL, FP32): component pair cp of site x
// for source src is the float4 at (x * 6 + cp) * nsrc + src.  The per-site arithmetic
// is h_site_ld's, operation for operation, so the results equal variant 0's.
struct FieldLoadIL {
  const float4* f;
  int64_t ns;
  int src;
  OV_HD void operator()(int64_t s, Spinor<float>& o) const {
    const float4* p = f + s * 6 * ns + src;
#pragma unroll
    for (int cp = 0; cp < 6; ++cp) {
      const float4 t = ldro(p + cp * ns);
      o.c[2 * cp] = mk(t.x, t.y);
      o.c[2 * cp + 1] = mk(t.z, t.w);
    }
  }
};

__global__ void __launch_bounds__(256) k_apply_h_il(Lat<float> L, const float4* __restrict__ in,
                                                    float4* __restrict__ out, int dagger) {
  const int64_t ns = L.nsrc;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= L.g.V * ns) return;
  const int64_t x = t / ns;
  const int src = (int)(t - x * ns);
  const float f = dagger ? L.efinv : L.ef, fi = dagger ? L.ef : L.efinv;
  Spinor<float> o;
  h_site_ld(FieldLoadIL{in, ns, src}, L.u, L.g, x, L.kappa, f, fi, o);
  float4* po = out + x * 6 * ns + src;
#pragma unroll
  for (int cp = 0; cp < 6; ++cp)
    po[cp * ns] = make_float4(o.c[2 * cp].re, o.c[2 * cp].im, o.c[2 * cp + 1].re, o.c[2 * cp + 1].im);
}
void apply_h_il(const Lat<float>& L, const float* in, float* out, int dagger, cudaStream_t st) {
  const int64_t n = L.g.V * L.nsrc;
  k_apply_h_il<<<nblocks(n, 256), 256, 0, st>>>(L, reinterpret_cast<const float4*>(in),
                                                reinterpret_cast<float4*>(out), dagger);
}

// user spinors [src][site][12] complex128 <-> the interleaved FP32 layout (one thread
// per (site, source), sources fastest)
__global__ void k_pack_spinors_il(const double* __restrict__ aos, float4* __restrict__ dst, int64_t V, int64_t ns) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= V * ns) return;
  const int64_t x = t / ns, src = t - x * ns;
  const double2* in = reinterpret_cast<const double2*>(aos) + (src * V + x) * 12;
  float4* o = dst + x * 6 * ns + src;
#pragma unroll
  for (int cp = 0; cp < 6; ++cp) {
    const double2 a = in[2 * cp], b = in[2 * cp + 1];
    o[cp * ns] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}
__global__ void k_unpack_spinors_il(const float4* __restrict__ f, double* __restrict__ aos, int64_t V, int64_t ns) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= V * ns) return;
  const int64_t x = t / ns, src = t - x * ns;
  const float4* p = f + x * 6 * ns + src;
  double2* out = reinterpret_cast<double2*>(aos) + (src * V + x) * 12;
#pragma unroll
  for (int cp = 0; cp < 6; ++cp) {
    const float4 v = p[cp * ns];
    out[2 * cp] = make_double2((double)v.x, (double)v.y);
    out[2 * cp + 1] = make_double2((double)v.z, (double)v.w);
  }
}
void pack_spinors_il(const double* aos, float* dst, int nsrc, int64_t V, cudaStream_t st) {
  k_pack_spinors_il<<<nblocks(V * nsrc, 256), 256, 0, st>>>(aos, reinterpret_cast<float4*>(dst), V, nsrc);
}
void unpack_spinors_il(const float* f, double* aos, int nsrc, int64_t V, cudaStream_t st) {
  k_unpack_spinors_il<<<nblocks(V * nsrc, 256), 256, 0, st>>>(reinterpret_cast<const float4*>(f), aos, V, nsrc);
}

// launch variants (sources per thread, threads per block, site map); 0 is the default.
// Plane variants fall back to consecutive sites when an x-y plane has fewer than
// 64 sites or more than the variant's thread bound.
// Variants 9, 10, 11 (FP32 only; others run variant 0) stage 1, 2 or 4 z-planes of
// the input in shared memory (k_apply_h_staged, below); variant 12 (FP32 only)
// sweeps runs of z-planes through a ring of plane slots (k_apply_h_sweep); variant
// 13 (APPLY_IL, FP32, its own field layout) is k_apply_h_il above.
static const int kApplyVariants[][3] = {{1, 128, 0}, {1, 64, 0}, {1, 256, 0}, {2, 64, 0}, {2, 128, 0},
                                        {4, 64, 0}, {4, 128, 0}, {1, 512, 1}, {2, 256, 1},
                                        {1, 1, 2},   {1, 2, 2},   {1, 4, 2},   {1, 0, 3},
                                        {1, 256, 4}};
int apply_h_variants() { return (int)(sizeof(kApplyVariants) / sizeof(kApplyVariants[0])); }

template <typename R, int NS, int BSZ, int MAP>
static void launch_apply(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st) {
  if (MAP == 1 && !plane_ok(L.g, BSZ)) {
    launch_apply<R, NS, 128, 0>(L, in, out, dagger, st);
    return;
  }
  const unsigned bs = MAP == 1 ? plane_threads(L.g) : BSZ;
  const unsigned gx = MAP == 1 ? (unsigned)(L.g.V / (L.g.nx * L.g.ny)) : nblocks(L.g.V, BSZ);
  const int ns = L.nsrc < NS ? 1 : NS;   // a lone source never needs the wider variant
  if (ns == 1)
    k_apply_h<R, 1, BSZ, MAP><<<dim3(gx, L.nsrc), bs, 0, st>>>(L, in, out, dagger, L.nsrc);
  else
    k_apply_h<R, NS, BSZ, MAP><<<dim3(gx, (L.nsrc + NS - 1) / NS), bs, 0, st>>>(L, in, out, dagger, L.nsrc);
}

// ---------------------------------------------------------------------------
// FP32 H psi with the x-y-z neighbourhood staged in shared memory.
// A block owns tz consecutive z-planes (whole x-y planes) of one time slice and
// one source.  Those planes and the two z-halo planes (periodic) of all six
// float4 chunks of the input field are copied into shared memory by bulk
// asynchronous copies (cp.async.bulk, one per chunk and plane: a contiguous run
// of Nx*Ny 16-byte chunks at a 16-byte-aligned address, completing on one
// mbarrier), so each staged spinor crosses from global memory once and every
// x, y and z neighbour is read from shared memory at conflict-free consecutive
// addresses; the t neighbours and the links are loaded directly.  One thread
// per site of the owned planes, at most 512 per block (tz is reduced until the
// planes fit, and the form is not used where one x-y plane has more sites).  The wait on the copies is bounded (2 s): a
// block that runs out sets ERRB_TIMEOUT in *err, waits once more (bounded) for
// its copies, and writes nothing.
// ---------------------------------------------------------------------------
constexpr unsigned long long kStageWaitNs = 2000000000ull;
constexpr int kStageMaxSmem = 227 * 1024;

__device__ __forceinline__ unsigned long long stage_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool stage_wait(uint32_t mb, unsigned long long limit_ns) {
  const unsigned long long t0 = stage_clock();
  for (;;) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mb), "r"(0u)
        : "memory");
    if (done) return true;
    if (stage_clock() - t0 > limit_ns) return false;
  }
}

// psi(s) from the staged planes when s lies in them, else from global memory
struct StagedLoad {
  const float4* stg;     // [6][tz + 2][P]
  const float* f;        // the field (global)
  int64_t V;
  int P, nz, t, zlo, np, stride;   // stride = (tz + 2) * P
  __device__ void operator()(int64_t s, Spinor<float>& o) const {
    const int64_t tz_site = s / P;             // t * nz + z
    const int tt = (int)(tz_site / nz), zz = (int)(tz_site % nz);
    int i = zz - zlo;
    if (i < 0) i += nz;
    if (tt == t && i < np) {
      const float4* q = stg + (int64_t)i * P + (s - tz_site * P);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float4 v = q[(int64_t)c * stride];
        o.c[2 * c] = mk(v.x, v.y);
        o.c[2 * c + 1] = mk(v.z, v.w);
      }
      return;
    }
    load_spinor_ro(f, V, s, o);
  }
};

__global__ void __launch_bounds__(512) k_apply_h_staged(Lat<float> L, const float* __restrict__ in,
                                                         float* __restrict__ out, int dagger, int tz, int* err) {
  extern __shared__ __align__(128) float4 stg[];
  __shared__ __align__(8) unsigned long long mbar;
  const Geom& g = L.g;
  const int P = g.nx * g.ny;
  const int nzb = (g.nz + tz - 1) / tz;
  const int t = blockIdx.x / nzb, z0 = (blockIdx.x % nzb) * tz;
  const int src = blockIdx.y;
  const int tzb = min(tz, g.nz - z0);      // planes this block owns
  const int np = tzb + 2;                   // planes staged (owned + two halo planes)
  const int stride = (tz + 2) * P;
  const float* f = in + (int64_t)src * L.vs;
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)P * 16u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes * 6u * (uint32_t)np)
                 : "memory");
    const float4* f4 = reinterpret_cast<const float4*>(f);
    for (int c = 0; c < 6; ++c)
      for (int i = 0; i < np; ++i) {
        int z = z0 - 1 + i;
        z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
        const float4* sp = f4 + (int64_t)c * g.V + ((int64_t)t * g.nz + z) * P;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stg + (int64_t)c * stride + (int64_t)i * P);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         dst),
                     "l"(sp), "r"(bytes), "r"(mb)
                     : "memory");
      }
  }
  const bool ok = stage_wait(mb, kStageWaitNs);
  if (!ok) {
    if (threadIdx.x == 0 && err) atomicOr(err, ERRB_TIMEOUT);
    stage_wait(mb, kStageWaitNs);   // the copies still target this block's shared memory
    return;
  }
  const int zi = threadIdx.x / P, p = threadIdx.x - zi * P;
  if (zi >= tzb) return;
  const int64_t s = ((int64_t)t * g.nz + z0 + zi) * P + p;
  int zlo = z0 - 1;
  if (zlo < 0) zlo += g.nz;
  const StagedLoad ld{stg, f, g.V, P, g.nz, t, zlo, np, stride};
  Spinor<float> o;
  const float ft = dagger ? L.efinv : L.ef, fti = dagger ? L.ef : L.efinv;
  h_site_ld(ld, L.u, g, s, L.kappa, ft, fti, o);
  store_spinor(out + (int64_t)src * L.vs, g.V, s, o);
}

// ---------------------------------------------------------------------------
// FP32 H psi by a pipelined sweep along z.  A block owns a run of z-planes
// [zb, ze) of one time slice and one source and walks it plane by plane,
// keeping a ring of four plane slots in shared memory: planes z-1, z, z+1 are
// resident while plane z is computed and plane z+2 is in flight, so each plane
// is copied once per run (bulk asynchronous copies, one per chunk, completing
// on the slot's mbarrier) and the copies overlap the arithmetic.  One thread
// per site of a plane (planes of at most 256 sites; three blocks per SM).  x, y and z neighbours come from shared memory, t
// neighbours and links from global memory.  Every wait is bounded (2 s); on a
// timeout the block flags ERRB_TIMEOUT, waits (bounded) for the copies it has
// in flight, and stops.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;

struct SweepLoad {
  const float4* stg;       // [kRing][6][P]
  const float* f;
  int64_t V;
  int P, nz, t, z, sm, s0, sp;   // current plane z; slots of planes z-1, z, z+1
  __device__ void operator()(int64_t s, Spinor<float>& o) const {
    const int64_t tz_site = s / P;
    const int tt = (int)(tz_site / nz), zz = (int)(tz_site % nz);
    int slot = -1;
    if (tt == t) {
      if (zz == z) slot = s0;
      else if (zz == (z + 1 == nz ? 0 : z + 1)) slot = sp;
      else if (zz == (z == 0 ? nz - 1 : z - 1)) slot = sm;
    }
    if (slot >= 0) {
      const float4* q = stg + (int64_t)slot * 6 * P + (s - tz_site * P);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float4 v = q[(int64_t)c * P];
        o.c[2 * c] = mk(v.x, v.y);
        o.c[2 * c + 1] = mk(v.z, v.w);
      }
      return;
    }
    load_spinor_ro(f, V, s, o);
  }
};

__global__ void __launch_bounds__(256, 3) k_apply_h_sweep(Lat<float> L, const float* __restrict__ in,
                                                       float* __restrict__ out, int dagger, int nzc, int* err) {
  extern __shared__ __align__(128) float4 ring[];
  __shared__ __align__(8) unsigned long long mbar[kRing];
  const Geom& g = L.g;
  const int P = g.nx * g.ny;
  const int zc = blockIdx.x % nzc, t = blockIdx.x / nzc;
  const int zb = (int)((int64_t)zc * g.nz / nzc), ze = (int)((int64_t)(zc + 1) * g.nz / nzc);
  const int src = blockIdx.y;
  const float* f = in + (int64_t)src * L.vs;
  const float4* f4 = reinterpret_cast<const float4*>(f);
  if (threadIdx.x == 0) {
    for (int q = 0; q < kRing; ++q) {
      const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[q]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // plane index i = zg - (zb - 1) for zg in [zb - 1, ze]; slot i % kRing, fill (i / kRing)
  const int nplanes = ze - zb + 2;
  auto issue = [&](int i) {   // thread 0 only
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[i % kRing]);
    const uint32_t bytes = (uint32_t)P * 16u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes * 6u) : "memory");
    int zg = zb - 1 + i;
    zg = zg < 0 ? zg + g.nz : (zg >= g.nz ? zg - g.nz : zg);
    const float4* sp = f4 + ((int64_t)t * g.nz + zg) * P;
    float4* dst = ring + (int64_t)(i % kRing) * 6 * P;
    for (int c = 0; c < 6; ++c) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + (int64_t)c * P);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                   "l"(sp + (int64_t)c * g.V), "r"(bytes), "r"(mb)
                   : "memory");
    }
  };
  int issued = min(kRing, nplanes);
  if (threadIdx.x == 0)
    for (int i = 0; i < issued; ++i) issue(i);
  int waited = 0;   // planes 0 .. waited-1 have been observed complete by every thread
  auto wait_plane = [&](int i) -> bool {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar[i % kRing]);
    const uint32_t parity = (uint32_t)((i / kRing) & 1);
    const unsigned long long t0 = stage_clock();
    for (;;) {
      uint32_t done = 0;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(mb), "r"(parity)
          : "memory");
      if (done) return true;
      if (stage_clock() - t0 > kStageWaitNs) return false;
    }
  };
  bool ok = true;
  const float ft = dagger ? L.efinv : L.ef, fti = dagger ? L.ef : L.efinv;
  for (int z = zb; z < ze; ++z) {
    const int i0 = z - zb + 1;   // plane index of z
    bool okw = true;
    for (; waited <= i0 + 1; ++waited)
      if (okw) okw = wait_plane(waited);
    ok = __syncthreads_and(okw) != 0;   // one decision for the whole block
    if (!ok) break;
    if (threadIdx.x < P) {
      const int64_t s = ((int64_t)t * g.nz + z) * P + threadIdx.x;
      const SweepLoad ld{ring, f, g.V, P, g.nz, t, z, (i0 - 1) % kRing, i0 % kRing, (i0 + 1) % kRing};
      Spinor<float> o;
      h_site_ld(ld, L.u, g, s, L.kappa, ft, fti, o);
      store_spinor(out + (int64_t)src * L.vs, g.V, s, o);
    }
    __syncthreads();   // the slot of plane z - 1 is free again
    if (threadIdx.x == 0 && issued < nplanes) issue(issued);
    ++issued;
  }
  if (!ok) {
    if (threadIdx.x == 0 && err) atomicOr(err, ERRB_TIMEOUT);
    // copies still in flight target this block's shared memory: only the latest fill of
    // each slot can be pending (a slot is refilled only after its previous fill was
    // observed), so wait (bounded) for those
    const int last = min(issued, nplanes);
    for (int i = max(0, last - kRing); i < last; ++i) wait_plane(i);
  }
}

// planes per block of the staged variants; 0 when the lattice does not fit the form
static int stage_planes(const Geom& g, int want) {
  const int P = g.nx * g.ny;
  int tz = std::min(want, g.nz);
  while (tz > 1 && ((int64_t)P * tz > 512 || (int64_t)6 * (tz + 2) * P * 16 > kStageMaxSmem)) --tz;
  if ((int64_t)P * tz > 512 || (int64_t)6 * (tz + 2) * P * 16 > kStageMaxSmem) return 0;
  return tz;
}
template <typename R>
static void launch_apply_staged(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st, int want,
                                int* err) {
  if constexpr (std::is_same<R, float>::value) {
    const int tz = stage_planes(L.g, want);
    int dev = 0, optin = 0;
    if (tz > 0 && !L.block && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess) {
      const int P = L.g.nx * L.g.ny;
      const size_t smem = (size_t)6 * (tz + 2) * P * 16;
      // the opt-in limit covers the dynamic part plus the kernel's own 8-byte mbarrier
      bool fits = smem + 64 <= (size_t)optin;
      if (fits && smem > 48 * 1024 &&
          cudaFuncSetAttribute(k_apply_h_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess) {
        cudaGetLastError();
        fits = false;
      }
      if (fits) {
        const unsigned threads = (unsigned)((P * tz + 31) / 32 * 32);
        const unsigned gx = (unsigned)(L.g.nt * ((L.g.nz + tz - 1) / tz));
        k_apply_h_staged<<<dim3(gx, L.nsrc), threads, smem, st>>>(L, in, out, dagger, tz, err);
        return;
      }
    }
    cudaGetLastError();
  }
  launch_apply<R, 1, 128, 0>(L, in, out, dagger, st);
}

template <typename R>
static void launch_apply_sweep(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st, int* err) {
  if constexpr (std::is_same<R, float>::value) {
    const int P = L.g.nx * L.g.ny;
    const size_t smem = (size_t)kRing * 6 * P * 16;
    int dev = 0, optin = 0;
    if (!L.block && P <= 256 && L.g.nz >= 1 && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        smem + 128 <= (size_t)optin) {
      bool fits = true;
      if (smem > 48 * 1024 &&
          cudaFuncSetAttribute(k_apply_h_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess)
        fits = false;
      if (fits)
        cudaFuncSetAttribute(k_apply_h_sweep, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaGetLastError();
      if (fits) {
        // z runs per (t, source) row: about three blocks per SM in all, as few runs (as
        // long a pipeline) as that allows, each run at least two planes
        const int64_t rows = (int64_t)L.g.nt * L.nsrc;
        int nzc = (int)std::min<int64_t>((3 * 152 + rows / 2) / rows, std::max(1, L.g.nz / 2));
        if (nzc < 1) nzc = 1;
        const unsigned threads = (unsigned)((P + 31) / 32 * 32);
        k_apply_h_sweep<<<dim3((unsigned)(L.g.nt * nzc), L.nsrc), threads, smem, st>>>(L, in, out, dagger, nzc, err);
        return;
      }
    }
  }
  launch_apply<R, 1, 128, 0>(L, in, out, dagger, st);
}

template <typename R>
void apply_h(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st, int variant, int* err) {
  switch (variant) {
    case 12: launch_apply_sweep<R>(L, in, out, dagger, st, err); break;
    case 9: launch_apply_staged<R>(L, in, out, dagger, st, 1, err); break;
    case 10: launch_apply_staged<R>(L, in, out, dagger, st, 2, err); break;
    case 11: launch_apply_staged<R>(L, in, out, dagger, st, 4, err); break;
    case 1: launch_apply<R, 1, 64, 0>(L, in, out, dagger, st); break;
    case 2: launch_apply<R, 1, 256, 0>(L, in, out, dagger, st); break;
    case 3: launch_apply<R, 2, 64, 0>(L, in, out, dagger, st); break;
    case 4: launch_apply<R, 2, 128, 0>(L, in, out, dagger, st); break;
    case 5: launch_apply<R, 4, 64, 0>(L, in, out, dagger, st); break;
    case 6: launch_apply<R, 4, 128, 0>(L, in, out, dagger, st); break;
    case 7: launch_apply<R, 1, 512, 1>(L, in, out, dagger, st); break;
    case 8: launch_apply<R, 2, 256, 1>(L, in, out, dagger, st); break;
    default: launch_apply<R, 1, 128, 0>(L, in, out, dagger, st); break;
  }
}

// ---------------------------------------------------------------------------
// helpers for the recurrence scalars
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool finite_z(zd a) { return isfinite(a.re) && isfinite(a.im); }

__device__ __forceinline__ void flag_error(SrcScal& sc, int bit, int step) {
  if (sc.err == 0) sc.err_step = step;
  sc.err |= bit;
}

// Sum NV partial slots of this source (fixed block order); thread 0 gets the result.
template <int NV>
__device__ __forceinline__ void sum_partials(const zd* part, int nblk, zd (&out)[NV], zd* scratch) {
  zd v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = mk(0.0, 0.0);
  // each thread takes a contiguous range of blocks, so the order is fixed
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = v[i] + ld_cg(part + i * nblk + b);
  }
  block_sum<NV>(v, scratch);
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = v[i];
}

// omega = s^dag r, rr = r^dag r, ss = s^dag s  ->  delta_{j+1}, beta_{j+1} and the next scales
template <typename R>
__device__ void omega_finalize(const Lat<R>& L, int src, int j, zd om, double rr, double ss) {
  SrcScal& sc = L.sc[src];
  const double aom = sqrt(om.re * om.re + om.im * om.im);
  if (!finite_z(om) || !isfinite(rr) || !isfinite(ss)) {
    flag_error(sc, ERRB_NONFINITE, j + 1);
    return;
  }
  if (aom <= 1e-14 * sqrt(rr * ss)) {
    flag_error(sc, ERRB_BREAKDOWN, j + 1);
    return;
  }
  const double d = sqrt(aom);
  const zd bt = mk(om.re / d, om.im / d);
  L.beta[(int64_t)src * L.k + j + 1] = bt;
  L.delta[(int64_t)src * L.k + j + 1] = d;
  sc.sv = mk(1.0 / d, 0.0);
  sc.sw = zdiv(mk(1.0, 0.0), conj(bt));
}

// ---------------------------------------------------------------------------
// TSL forward: initialisation (beta_0 = ||b||)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(BS) k_tsl_init(Lat<R> L) {
  __shared__ zd scratch[2 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  zd v[2] = {mk(0.0, 0.0), mk(0.0, 0.0)};
  if (x < L.g.V) {
    Spinor<R> b;
    load_spinor(L.r + src * L.vs, L.g.V, x, b);
    v[0] = spinor_dot(b, b);
    if (L.block) {
      Spinor<R> a;
      load_spinor(L.s + src * L.vs, L.g.V, x, a);
      v[1] = spinor_dot(a, b);
    }
  }
  block_sum<2>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (arrive_last(L.cnt + src * 16 + 0, gridDim.x)) {
    zd s[2];
    sum_partials<2>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0) {
      SrcScal& sc = L.sc[src];
      sc.err = 0;
      sc.err_step = -1;
      const double b0 = sqrt(s[0].re);
      sc.beta0 = b0;
      if (!(b0 > 0.0) || !isfinite(b0)) flag_error(sc, ERRB_NONFINITE, 0);
      sc.sv = mk(1.0 / b0, 0.0);
      // w_1 = s sw with w_1^dag v_1 = 1: sw = beta_0 / conj(s^dag r); s = r in plain mode
      sc.sw = L.block ? zdiv(mk(b0, 0.0), conj(s[1])) : mk(1.0 / b0, 0.0);
      L.beta[(int64_t)src * L.k] = mk(0.0, 0.0);
      L.delta[(int64_t)src * L.k] = 0.0;
    }
  }
}
template <typename R>
void tsl_init(const Lat<R>& L, cudaStream_t st) {
  k_tsl_init<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L);
}

// ---------------------------------------------------------------------------
// TSL step j: v_j = sv r_{j-1}, w_j = sw s_{j-1} stored in the bases;
// p = H v_j, q = H^dag w_j; alpha_j = w_j^dag p.
// ---------------------------------------------------------------------------
template <typename R, int PAIR, int BSZ, int MAP>
__global__ void __launch_bounds__(BSZ) k_tsl_stencil(Lat<R> L, int j, int need_q) {
  __shared__ zd scratch[32];
  const int64_t x = thread_site<MAP>(L.g);
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  const R* rp = L.r + src * L.vs;
  const R* sp = L.s + src * L.vs;
  zd v[1] = {mk(0.0, 0.0)};
  if (x < V && L.sc[src].err == 0) {
    const cplx<R> sv = cast<R>(L.sc[src].sv), sw = cast<R>(L.sc[src].sw);
    Spinor<R> a, w, o;
    load_spinor(rp, V, x, a);
#pragma unroll
    for (int c = 0; c < 12; ++c) a.c[c] = sv * a.c[c];
    store_spinor(L.basis_v(src, j), V, x, a);
    load_spinor(sp, V, x, w);
#pragma unroll
    for (int c = 0; c < 12; ++c) w.c[c] = sw * w.c[c];
    store_spinor(L.basis_w(src, j), V, x, w);
    if (need_q && PAIR) {
      // H r and H^dag s share every link load
      const FieldLoad<R> ld[2] = {FieldLoad<R>{rp, V}, FieldLoad<R>{sp, V}};
      const R ft[2] = {L.ef, L.efinv}, fti[2] = {L.efinv, L.ef};
      Spinor<R> hh[2];
      h_site_multi<2>(ld, L.u, L.g, x, L.kappa, ft, fti, hh);
#pragma unroll
      for (int c = 0; c < 12; ++c) o.c[c] = sv * hh[0].c[c];
      store_spinor(L.p + src * L.vs, V, x, o);
      v[0] = spinor_dot(w, o);
#pragma unroll
      for (int c = 0; c < 12; ++c) o.c[c] = sw * hh[1].c[c];
      store_spinor(L.q + src * L.vs, V, x, o);
    } else {
      h_site(rp, L.u, L.g, x, L.kappa, L.ef, L.efinv, o);
#pragma unroll
      for (int c = 0; c < 12; ++c) o.c[c] = sv * o.c[c];
      store_spinor(L.p + src * L.vs, V, x, o);
      v[0] = spinor_dot(w, o);
      if (need_q) {
        h_site(sp, L.u, L.g, x, L.kappa, L.efinv, L.ef, o);
#pragma unroll
        for (int c = 0; c < 12; ++c) o.c[c] = sw * o.c[c];
        store_spinor(L.q + src * L.vs, V, x, o);
      }
    }
  }
  block_sum<1>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (arrive_last(L.cnt + src * 16 + 1, gridDim.x)) {
    zd s[1];
    sum_partials<1>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0) {
      SrcScal& sc = L.sc[src];
      if (!finite_z(s[0])) flag_error(sc, ERRB_NONFINITE, j);
      L.alpha[(int64_t)src * L.k + j] = s[0];
    }
  }
}
// Block TSL step (Theorem 1): with r = (r_u, r_l), s = (s_u, s_l) in 2V-site fields,
//   v_j = sv r, w_j = sw s,
//   p = sv (H r_u + dH r_l, H r_l),   q = sw (H^dag s_u, dH^dag s_u + H^dag s_l),
//   alpha_j = w_j^dag p  (over both halves).  One thread per lattice site.
template <typename R>
__global__ void __launch_bounds__(BS) k_tsl_stencil_block(Lat<R> L, int j, int need_q) {
  __shared__ zd scratch[32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t Vr = L.gl.V, Vf = L.g.V;
  const R* rp = L.r + src * L.vs;
  const R* sp = L.s + src * L.vs;
  zd v[1] = {mk(0.0, 0.0)};
  if (x < Vr && L.sc[src].err == 0) {
    const cplx<R> sv = cast<R>(L.sc[src].sv), sw = cast<R>(L.sc[src].sw);
    Spinor<R> a;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      load_spinor(rp, Vf, hf * Vr + x, a);
#pragma unroll
      for (int c = 0; c < 12; ++c) a.c[c] = sv * a.c[c];
      store_spinor(L.basis_v(src, j), Vf, hf * Vr + x, a);
      load_spinor(sp, Vf, hf * Vr + x, a);
#pragma unroll
      for (int c = 0; c < 12; ++c) a.c[c] = sw * a.c[c];
      store_spinor(L.basis_w(src, j), Vf, hf * Vr + x, a);
    }
    {
      const FieldLoadOff<R> ld[2] = {FieldLoadOff<R>{rp, Vf, 0}, FieldLoadOff<R>{rp, Vf, Vr}};
      const R ft[2] = {L.ef, L.ef}, fti[2] = {L.efinv, L.efinv};
      Spinor<R> hh[2], d;
      h_site_multi<2>(ld, L.u, L.gl, x, L.kappa, ft, fti, hh);
      dh_site_ld(ld[1], L.ue, L.u, L.gl, x, L.kappa, L.ef, L.efinv, L.mdir, d);
#pragma unroll
      for (int c = 0; c < 12; ++c) hh[0].c[c] = sv * (hh[0].c[c] + d.c[c]);
#pragma unroll
      for (int c = 0; c < 12; ++c) hh[1].c[c] = sv * hh[1].c[c];
      store_spinor(L.p + src * L.vs, Vf, x, hh[0]);
      store_spinor(L.p + src * L.vs, Vf, Vr + x, hh[1]);
      load_spinor(L.basis_w(src, j), Vf, x, a);
      v[0] = spinor_dot(a, hh[0]);
      load_spinor(L.basis_w(src, j), Vf, Vr + x, a);
      v[0] = v[0] + spinor_dot(a, hh[1]);
    }
    if (need_q) {
      const FieldLoadOff<R> ld[2] = {FieldLoadOff<R>{sp, Vf, 0}, FieldLoadOff<R>{sp, Vf, Vr}};
      const R ft[2] = {L.efinv, L.efinv}, fti[2] = {L.ef, L.ef};
      Spinor<R> hh[2], d;
      h_site_multi<2>(ld, L.u, L.gl, x, L.kappa, ft, fti, hh);
      dh_site_ld(ld[0], L.ue, L.u, L.gl, x, L.kappa, L.efinv, L.ef, -L.mdir, d);
#pragma unroll
      for (int c = 0; c < 12; ++c) hh[0].c[c] = sw * hh[0].c[c];
#pragma unroll
      for (int c = 0; c < 12; ++c) hh[1].c[c] = sw * (hh[1].c[c] + d.c[c]);
      store_spinor(L.q + src * L.vs, Vf, x, hh[0]);
      store_spinor(L.q + src * L.vs, Vf, Vr + x, hh[1]);
    }
  }
  block_sum<1>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
  if (arrive_last(L.cnt + src * 16 + 1, gridDim.x)) {
    zd s1[1];
    sum_partials<1>(part, gridDim.x, s1, scratch);
    if (threadIdx.x == 0) {
      SrcScal& sc = L.sc[src];
      if (!finite_z(s1[0])) flag_error(sc, ERRB_NONFINITE, j);
      L.alpha[(int64_t)src * L.k + j] = s1[0];
    }
  }
}

static const int kPairVariants[][3] = {{1, 128, 0}, {1, 64, 0}, {0, 128, 0}, {0, 64, 0}, {0, 256, 0},
                                       {1, 256, 1}, {0, 512, 1}};
int tsl_stencil_variants() { return (int)(sizeof(kPairVariants) / sizeof(kPairVariants[0])); }

template <typename R, int PAIR, int BSZ, int MAP>
static void launch_pair(const Lat<R>& L, int j, int q, cudaStream_t st) {
  if (MAP == 1 && !plane_ok(L.g, BSZ)) {
    launch_pair<R, PAIR, 128, 0>(L, j, q, st);
    return;
  }
  const unsigned bs = MAP == 1 ? plane_threads(L.g) : (unsigned)std::min(BSZ, site_bs(L.g.V));
  const unsigned gx = MAP == 1 ? (unsigned)(L.g.V / (L.g.nx * L.g.ny)) : nblocks(L.g.V, (int)bs);
  k_tsl_stencil<R, PAIR, BSZ, MAP><<<dim3(gx, L.nsrc), bs, 0, st>>>(L, j, q);
}

template <typename R>
void tsl_stencil(const Lat<R>& L, int j, bool need_q, cudaStream_t st, int variant) {
  const int q = need_q ? 1 : 0;
  if (L.block) {
    k_tsl_stencil_block<R><<<dim3(nblocks(L.gl.V, BS), L.nsrc), BS, 0, st>>>(L, j, q);
    return;
  }
  switch (variant) {
    case 1: launch_pair<R, 1, 64, 0>(L, j, q, st); break;
    case 2: launch_pair<R, 0, 128, 0>(L, j, q, st); break;
    case 3: launch_pair<R, 0, 64, 0>(L, j, q, st); break;
    case 4: launch_pair<R, 0, 256, 0>(L, j, q, st); break;
    case 5: launch_pair<R, 1, 256, 1>(L, j, q, st); break;
    case 6: launch_pair<R, 0, 512, 1>(L, j, q, st); break;
    default: launch_pair<R, 1, 128, 0>(L, j, q, st); break;
  }
}

// r = p - alpha_j v_j - beta_j v_{j-1};  s = q - conj(alpha_j) w_j - delta_j w_{j-1}
template <typename R>
__global__ void __launch_bounds__(BS) k_tsl_update(Lat<R> L, int j, int finalize) {
  __shared__ zd scratch[3 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  zd v[3] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
  if (x < V && L.sc[src].err == 0) {
    const cplx<R> al = cast<R>(L.alpha[(int64_t)src * L.k + j]);
    const cplx<R> alc = conj(al);
    Spinor<R> r, s, t;
    load_spinor(L.p + src * L.vs, V, x, r);
    load_spinor(L.q + src * L.vs, V, x, s);
    load_spinor(L.basis_v(src, j), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmsub(r.c[c], al, t.c[c]);
    load_spinor(L.basis_w(src, j), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmsub(s.c[c], alc, t.c[c]);
    if (j > 0) {
      const cplx<R> bt = cast<R>(L.beta[(int64_t)src * L.k + j]);
      const R dl = (R)L.delta[(int64_t)src * L.k + j];
      load_spinor(L.basis_v(src, j - 1), V, x, t);
#pragma unroll
      for (int c = 0; c < 12; ++c) cmsub(r.c[c], bt, t.c[c]);
      load_spinor(L.basis_w(src, j - 1), V, x, t);
#pragma unroll
      for (int c = 0; c < 12; ++c) s.c[c] = s.c[c] - dl * t.c[c];
    }
    store_spinor(L.r + src * L.vs, V, x, r);
    store_spinor(L.s + src * L.vs, V, x, s);
    if (finalize) {
      v[0] = spinor_dot(s, r);
      v[1] = spinor_dot(r, r);
      v[2] = spinor_dot(s, s);
    }
  }
  if (!finalize) return;   // uniform across the grid
  block_sum<3>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) part[i * gridDim.x + blockIdx.x] = v[i];
  }
  if (arrive_last(L.cnt + src * 16 + 2, gridDim.x)) {
    zd s[3];
    sum_partials<3>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0 && L.sc[src].err == 0) omega_finalize(L, src, j, s[0], s[1].re, s[2].re);
  }
}
template <typename R>
void tsl_update(const Lat<R>& L, int j, bool finalize, cudaStream_t st) {
  k_tsl_update<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, j, finalize ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt against the stored bases (basis indices 0..j).
//   side A: coefA_i = DA_i^dag a,  a -= sum_i coefA_i UA_i
//   side B: coefB_i = DB_i^dag b,  b -= sum_i coefB_i UB_i
// mode 0 (forward):  DA = W, UA = V, DB = V, UB = W   (a = r, b = s)
// mode 1 (adjoint):  DA = V, UA = W, DB = W, UB = V   (a = g_r, b = g_s)
// coef layout: [src][2*i + side];  cpart: [src][2*i + side][site block]
// ---------------------------------------------------------------------------
// sites per thread of the projection dots: 4 once there are enough basis
// vectors to fill the GPU with site blocks x basis blocks, else 1
static inline int proj_spt(int nb) { return nb >= NB ? 4 : 1; }

// Each thread accumulates `spt` sites (strided by the block size, so loads stay
// coalesced) before the block reduction, which then costs 1/spt per site.
template <typename R>
__global__ void __launch_bounds__(BS) k_proj_dots(Lat<R> L, int nb, int mode, const R* __restrict__ a,
                                                   const R* __restrict__ b, int64_t ab_stride,
                                                   zd* __restrict__ cpart, int64_t cp_stride, int spt, int ioff) {
  __shared__ zd scratch[2 * NB * 32];
  const int src = blockIdx.z;
  const int i0 = blockIdx.y * NB;
  const int64_t V = L.g.V;
  SiteDot<R> acc[2 * NB];
#pragma unroll
  for (int t = 0; t < 2 * NB; ++t) acc[t].zero();
  for (int q = 0; q < spt; ++q) {
    const int64_t x = (blockIdx.x * (int64_t)spt + q) * blockDim.x + threadIdx.x;
    if (x >= V) break;
    Spinor<R> va, vb, e;
    load_spinor(a + src * ab_stride, V, x, va);
    if (b) load_spinor(b + src * ab_stride, V, x, vb);
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int i = i0 + t;
      if (i < nb) {
        const R* da = mode == 0 ? L.basis_w(src, ioff + i) : L.basis_v(src, ioff + i);
        load_spinor(da, V, x, e);
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[2 * t].add(e.c[c], va.c[c]);
        if (b) {
          const R* db = mode == 0 ? L.basis_v(src, ioff + i) : L.basis_w(src, ioff + i);
          load_spinor(db, V, x, e);
#pragma unroll
          for (int c = 0; c < 12; ++c) acc[2 * t + 1].add(e.c[c], vb.c[c]);
        }
      }
    }
  }
  zd v[2 * NB];
#pragma unroll
  for (int t = 0; t < 2 * NB; ++t) v[t] = acc[t].value();
  block_sum<2 * NB>(v, scratch);
  if (threadIdx.x == 0) {
    zd* cp = cpart + src * cp_stride;
#pragma unroll
    for (int t = 0; t < 2 * NB; ++t) {
      const int i = i0 + t / 2;
      if (i < nb) cp[(int64_t)(2 * i + (t & 1)) * gridDim.x + blockIdx.x] = v[t];
    }
  }
}

__global__ void k_proj_reduce(const zd* __restrict__ cpart, int64_t cp_stride, int nsb, int nb,
                              zd* __restrict__ coef, int64_t coef_stride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;   // 2*i + side
  const int src = blockIdx.y;
  if (t >= 2 * nb) return;
  const zd* cp = cpart + src * cp_stride + (int64_t)t * nsb;
  zd s = mk(0.0, 0.0);
  for (int b = 0; b < nsb; ++b) s = s + cp[b];
  coef[src * coef_stride + t] = s;
}

// SMALL: the coefficients are at rounding level relative to a and b (the second
// Gram-Schmidt pass, whose input is already biorthogonal to working precision),
// so the correction sum_i c_i u_i is formed in FP32 arithmetic; its rounding is
// ~6e-8 of a correction that is itself ~1e-12 or less of a, far below FP64
// rounding of a.  FP64 fields are still read in full.
template <typename T, typename R> OV_HD void spinor_cast(const Spinor<R>& in, Spinor<T>& out) {
#pragma unroll
  for (int c = 0; c < 12; ++c) out.c[c] = mk<T>((T)in.c[c].re, (T)in.c[c].im);
}

template <typename R, bool SMALL>
__global__ void __launch_bounds__(BS) k_proj_update(Lat<R> L, int nb, int mode, R* __restrict__ a,
                                                     R* __restrict__ b, int64_t ab_stride,
                                                     const zd* __restrict__ coef, int64_t coef_stride,
                                                     int j, int finalize) {
  using A = typename std::conditional<SMALL, float, R>::type;   // accumulation type
  __shared__ zd cs[2 * 64];
  __shared__ zd scratch[3 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  const bool active = x < V;
  Spinor<A> ca, cb;
  Spinor<R> e;
  spinor_zero(ca);
  spinor_zero(cb);
  const zd* cf = coef + src * coef_stride;
  for (int i0 = 0; i0 < nb; i0 += 64) {
    const int n = min(64, nb - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) cs[t] = cf[2 * i0 + t];
    __syncthreads();
    if (active) {
      for (int t = 0; t < n; ++t) {
        const int i = i0 + t;
        const R* ua = mode == 0 ? L.basis_v(src, i) : L.basis_w(src, i);
        const cplx<A> c0 = cast<A>(cs[2 * t]);
        load_spinor(ua, V, x, e);
#pragma unroll
        for (int c = 0; c < 12; ++c) cmac(ca.c[c], c0, mk<A>((A)e.c[c].re, (A)e.c[c].im));
        if (b) {
          const R* ub = mode == 0 ? L.basis_w(src, i) : L.basis_v(src, i);
          const cplx<A> c1 = cast<A>(cs[2 * t + 1]);
          load_spinor(ub, V, x, e);
#pragma unroll
          for (int c = 0; c < 12; ++c) cmac(cb.c[c], c1, mk<A>((A)e.c[c].re, (A)e.c[c].im));
        }
      }
    }
  }
  zd v[3] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
  if (active) {
    Spinor<R> r, s;
    load_spinor(a + src * ab_stride, V, x, r);
#pragma unroll
    for (int c = 0; c < 12; ++c) r.c[c] = r.c[c] - mk<R>((R)ca.c[c].re, (R)ca.c[c].im);
    store_spinor(a + src * ab_stride, V, x, r);
    if (b) {
      load_spinor(b + src * ab_stride, V, x, s);
#pragma unroll
      for (int c = 0; c < 12; ++c) s.c[c] = s.c[c] - mk<R>((R)cb.c[c].re, (R)cb.c[c].im);
      store_spinor(b + src * ab_stride, V, x, s);
      if (finalize) {
        v[0] = spinor_dot(s, r);
        v[1] = spinor_dot(r, r);
        v[2] = spinor_dot(s, s);
      }
    }
  }
  if (!finalize) return;
  block_sum<3>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) part[i * gridDim.x + blockIdx.x] = v[i];
  }
  if (arrive_last(L.cnt + src * 16 + 3, gridDim.x)) {
    zd s3[3];
    sum_partials<3>(part, gridDim.x, s3, scratch);
    if (threadIdx.x == 0 && L.sc[src].err == 0) omega_finalize(L, src, j, s3[0], s3[1].re, s3[2].re);
  }
}

template <typename R>
void proj_dots(const Lat<R>& L, int j, int mode, const R* a, const R* b, int64_t ab_stride, zd* coef,
               zd* cpart, cudaStream_t st) {
  const int nb = j + 1;
  const int spt = proj_spt(nb);
  const unsigned nsb = nblocks(L.g.V, BS * spt);
  const int64_t cp_stride = (int64_t)2 * L.k * nsb;
  k_proj_dots<R><<<dim3(nsb, nblocks(nb, NB), L.nsrc), BS, 0, st>>>(L, nb, mode, a, b, ab_stride, cpart,
                                                                     cp_stride, spt, 0);
  k_proj_reduce<<<dim3(nblocks(2 * nb, 128), L.nsrc), 128, 0, st>>>(cpart, cp_stride, nsb, nb, coef,
                                                                      2 * (int64_t)L.k);
}
template <typename R>
void proj_update(const Lat<R>& L, int j, int mode, R* a, R* b, int64_t ab_stride, const zd* coef, bool finalize,
                 cudaStream_t st, bool small) {
  const int bs = site_bs(L.g.V);
  const dim3 grid(nblocks(L.g.V, bs), L.nsrc);
  if (small && sizeof(R) == 8)
    k_proj_update<R, true><<<grid, bs, 0, st>>>(L, j + 1, mode, a, b, ab_stride, coef, 2 * (int64_t)L.k, j,
                                                finalize ? 1 : 0);
  else
    k_proj_update<R, false><<<grid, bs, 0, st>>>(L, j + 1, mode, a, b, ab_stride, coef, 2 * (int64_t)L.k, j,
                                                 finalize ? 1 : 0);
}

// out[src][i] = v_i^dag x  for i < nvec (dots of the V basis with one vector per source)
template <typename R>
void basis_dots_range(const Lat<R>& L, int j0, int nvec, const R* x, int64_t x_stride, zd* out, zd* cpart,
                      cudaStream_t st) {
  const int spt = proj_spt(nvec);
  const unsigned nsb = nblocks(L.g.V, BS * spt);
  const int64_t cp_stride = (int64_t)2 * L.k * nsb;
  // mode 1 makes side A dot the V basis
  k_proj_dots<R><<<dim3(nsb, nblocks(nvec, NB), L.nsrc), BS, 0, st>>>(L, nvec, 1, x, nullptr, x_stride,
                                                                       cpart, cp_stride, spt, j0);
  k_proj_reduce<<<dim3(nblocks(2 * nvec, 128), L.nsrc), 128, 0, st>>>(cpart, cp_stride, nsb, nvec, out,
                                                                        2 * (int64_t)L.k);
}
template <typename R>
void basis_dots(const Lat<R>& L, int nvec, const R* x, int64_t x_stride, zd* out, zd* cpart, cudaStream_t st) {
  basis_dots_range(L, 0, nvec, x, x_stride, out, cpart, st);
}

// x[src] = sum_i y_i v_i, written as interleaved complex128 [src][V][12]
template <typename R>
__global__ void __launch_bounds__(BS) k_combine(Lat<R> L, int j0, int nvec, const zd* __restrict__ y,
                                                 double* __restrict__ out, int accumulate) {
  __shared__ zd ys[64];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  double2* o = reinterpret_cast<double2*>(out) + ((int64_t)src * V + x) * 12;
  zd acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = mk(0.0, 0.0);
  if (accumulate && x < V) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = mk(o[c].x, o[c].y);
  }
  for (int i0 = 0; i0 < nvec; i0 += 32) {
    const int n = min(32, nvec - i0);
    __syncthreads();
    if (threadIdx.x < n) ys[threadIdx.x] = y[(int64_t)src * L.k + j0 + i0 + threadIdx.x];
    __syncthreads();
    if (x < V) {
      Spinor<R> part, e;
      spinor_zero(part);
      for (int t = 0; t < n; ++t) {
        load_spinor(L.basis_v(src, j0 + i0 + t), V, x, e);
        const cplx<R> yc = cast<R>(ys[t]);
#pragma unroll
        for (int c = 0; c < 12; ++c) cmac(part.c[c], yc, e.c[c]);
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[c] = acc[c] + mk((double)part.c[c].re, (double)part.c[c].im);
    }
  }
  if (x < V) {
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = make_double2(acc[c].re, acc[c].im);
  }
}
// out = sum_{j < nvec} y_j u_j for one source, u = V (side 0) or W (side 1): a Ritz
// vector of the TSL (right V_k y, left W_k z), written in the user layout
template <typename R>
__global__ void __launch_bounds__(BS) k_ritz_combine(Lat<R> L, int src, int side, int nvec, const zd* __restrict__ y,
                                                     double* __restrict__ out) {
  __shared__ zd ys[32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t V = L.g.V;
  zd acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = mk(0.0, 0.0);
  for (int i0 = 0; i0 < nvec; i0 += 32) {
    const int n = min(32, nvec - i0);
    __syncthreads();
    if (threadIdx.x < n) ys[threadIdx.x] = y[i0 + threadIdx.x];
    __syncthreads();
    if (x < V) {
      Spinor<R> e;
      for (int t = 0; t < n; ++t) {
        load_spinor(side ? L.basis_w(src, i0 + t) : L.basis_v(src, i0 + t), V, x, e);
#pragma unroll
        for (int c = 0; c < 12; ++c) cmac(acc[c], ys[t], mk((double)e.c[c].re, (double)e.c[c].im));
      }
    }
  }
  if (x < V) {
    double2* o = reinterpret_cast<double2*>(out) + x * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = make_double2(acc[c].re, acc[c].im);
  }
}
template <typename R>
void ritz_combine(const Lat<R>& L, int src, int side, int nvec, const zd* y, double* out, cudaStream_t st) {
  k_ritz_combine<R><<<nblocks(L.g.V, BS), BS, 0, st>>>(L, src, side, nvec, y, out);
}

template <typename R>
void combine_range(const Lat<R>& L, int j0, int nvec, const zd* y, double* out, bool acc, cudaStream_t st) {
  k_combine<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, j0, nvec, y, out, acc ? 1 : 0);
}
template <typename R>
void combine(const Lat<R>& L, int nvec, const zd* y, double* out, cudaStream_t st) {
  combine_range(L, 0, nvec, y, out, false, st);
}

// ---------------------------------------------------------------------------
// Reverse sweep
// ---------------------------------------------------------------------------
// R1: A1 = v_{j+1}^dag Gv, A2 = w_{j+1}^dag Gw  ->  g_delta, g_beta, g_omega and the
// coefficients of g_r = Gv/delta + conj(beta) g_omega w_{j+1},  g_s = Gw/beta + delta conj(g_omega) v_{j+1}
template <typename R>
__global__ void __launch_bounds__(BS) k_rev_dots(Lat<R> L, Rev<R> B, int j) {
  __shared__ zd scratch[2 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  zd v[2] = {mk(0.0, 0.0), mk(0.0, 0.0)};
  if (x < V) {
    Spinor<R> a, g;
    load_spinor(L.basis_v(src, j + 1), V, x, a);
    load_spinor(B.gv + src * L.vs, V, x, g);
    v[0] = spinor_dot(a, g);
    load_spinor(L.basis_w(src, j + 1), V, x, a);
    load_spinor(B.gw + src * L.vs, V, x, g);
    v[1] = spinor_dot(a, g);
  }
  block_sum<2>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
  if (arrive_last(L.cnt + src * 16 + 4, gridDim.x)) {
    zd s[2];
    sum_partials<2>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0) {
      SrcScal& sc = L.sc[src];
      const int64_t o = (int64_t)src * L.k + j + 1;
      const double d = L.delta[o];
      const zd bt = L.beta[o];
      const zd om = mk(bt.re * d, bt.im * d);
      const double aom = d * d;
      double g_d = B.gdT[o] + sc.carry_delta - s[0].re / d;
      zd g_b = B.gbT[o] + sc.carry_beta - zdiv(conj(s[1]), conj(bt));
      zd g_w = mk(g_b.re / d, g_b.im / d);
      g_d -= (om.re * g_b.re + om.im * g_b.im) / (d * d);      // Re(conj(om) g_b)
      const double f = g_d / (2.0 * d * aom);
      g_w = g_w + mk(f * om.re, f * om.im);
      sc.cr1 = mk(1.0 / d, 0.0);
      sc.cr2 = conj(bt) * g_w;
      sc.cs1 = zdiv(mk(1.0, 0.0), bt);
      sc.cs2 = mk(d * g_w.re, -d * g_w.im);
      if (!finite_z(sc.cr2) || !finite_z(sc.cs2)) flag_error(sc, ERRB_NONFINITE, j);
    }
  }
}
template <typename R>
void rev_dots(const Lat<R>& L, const Rev<R>& B, int j, cudaStream_t st) {
  k_rev_dots<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, B, j);
}

// D1 = v_j^dag g_r, D2 = w_j^dag g_s, D3 = v_{j-1}^dag g_r, D4 = w_{j-1}^dag g_s -> g_alpha, carries
template <typename R>
__device__ void alpha_epilogue(const Lat<R>& L, const Rev<R>& B, int src, int j, const zd (&s)[4]) {
  SrcScal& sc = L.sc[src];
  const int64_t o = (int64_t)src * L.k + j;
  sc.g_alpha = B.gaT[o] - s[0] - conj(s[1]);
  if (j > 0) {
    sc.carry_beta = -s[2];
    sc.carry_delta = -s[3].re;
  } else {
    sc.carry_beta = mk(0.0, 0.0);
    sc.carry_delta = 0.0;
  }
}

template <typename R>
__device__ void alpha_dots_site(const Lat<R>& L, int src, int j, int64_t x, const Spinor<R>& gr,
                                const Spinor<R>& gs, zd (&v)[4]) {
  Spinor<R> e;
  load_spinor(L.basis_v(src, j), L.g.V, x, e);
  v[0] = spinor_dot(e, gr);
  load_spinor(L.basis_w(src, j), L.g.V, x, e);
  v[1] = spinor_dot(e, gs);
  if (j > 0) {
    load_spinor(L.basis_v(src, j - 1), L.g.V, x, e);
    v[2] = spinor_dot(e, gr);
    load_spinor(L.basis_w(src, j - 1), L.g.V, x, e);
    v[3] = spinor_dot(e, gs);
  }
}

// R2: g_r, g_s into the ring slot; optionally the four dots for g_alpha
template <typename R>
__global__ void __launch_bounds__(BS) k_rev_form(Lat<R> L, Rev<R> B, int j, int slot, int with_dots) {
  __shared__ zd scratch[4 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  zd v[4] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
  if (x < V) {
    const SrcScal& sc = L.sc[src];
    const cplx<R> cr1 = cast<R>(sc.cr1), cr2 = cast<R>(sc.cr2), cs1 = cast<R>(sc.cs1), cs2 = cast<R>(sc.cs2);
    Spinor<R> gr, gs, e;
    load_spinor(B.gv + src * L.vs, V, x, gr);
    load_spinor(L.basis_w(src, j + 1), V, x, e);
#pragma unroll
    for (int c = 0; c < 12; ++c) gr.c[c] = cr1 * gr.c[c] + cr2 * e.c[c];
    load_spinor(B.gw + src * L.vs, V, x, gs);
    load_spinor(L.basis_v(src, j + 1), V, x, e);
#pragma unroll
    for (int c = 0; c < 12; ++c) gs.c[c] = cs1 * gs.c[c] + cs2 * e.c[c];
    store_spinor(B.ring(B.gr_ring, slot, src), V, x, gr);
    store_spinor(B.ring(B.gs_ring, slot, src), V, x, gs);
    if (with_dots) alpha_dots_site(L, src, j, x, gr, gs, v);
  }
  if (!with_dots) return;
  block_sum<4>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) part[i * gridDim.x + blockIdx.x] = v[i];
  }
  if (arrive_last(L.cnt + src * 16 + 5, gridDim.x)) {
    zd s[4];
    sum_partials<4>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0) alpha_epilogue(L, B, src, j, s);
  }
}
template <typename R>
void rev_form(const Lat<R>& L, const Rev<R>& B, int j, int slot, bool with_dots, cudaStream_t st) {
  k_rev_form<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, B, j, slot,
                                                                                   with_dots ? 1 : 0);
}

// the four dots after the projection adjoint has been applied to g_r, g_s
template <typename R>
__global__ void __launch_bounds__(BS) k_rev_alpha_dots(Lat<R> L, Rev<R> B, int j, int slot) {
  __shared__ zd scratch[4 * 32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  zd v[4] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
  if (x < V) {
    Spinor<R> gr, gs;
    load_spinor(B.ring(B.gr_ring, slot, src), V, x, gr);
    load_spinor(B.ring(B.gs_ring, slot, src), V, x, gs);
    alpha_dots_site(L, src, j, x, gr, gs, v);
  }
  block_sum<4>(v, scratch);
  zd* part = L.part + src * L.part_stride;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) part[i * gridDim.x + blockIdx.x] = v[i];
  }
  if (arrive_last(L.cnt + src * 16 + 6, gridDim.x)) {
    zd s[4];
    sum_partials<4>(part, gridDim.x, s, scratch);
    if (threadIdx.x == 0) alpha_epilogue(L, B, src, j, s);
  }
}
template <typename R>
void rev_alpha_dots(const Lat<R>& L, const Rev<R>& B, int j, int slot, cudaStream_t st) {
  k_rev_alpha_dots<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, B, j, slot);
}

// Lazy projection-adjoint coefficients of recorded projection m (at step j):
//   acc_v[i] += -conj(beta_{j+1}) conj(e_s,i) w_{j+1},  acc_w[i] += -delta_{j+1} conj(e_r,i) v_{j+1}
__global__ void k_rev_proj_record(zd* ev, zd* ew, int64_t e_stride, int k, int m, int j, const zd* __restrict__ coef,
                                  int64_t coef_stride, const zd* __restrict__ beta, const double* __restrict__ delta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  if (i > j) return;
  const zd bt = beta[(int64_t)src * k + j + 1];
  const double d = delta[(int64_t)src * k + j + 1];
  const zd er = coef[src * coef_stride + 2 * i];
  const zd es = coef[src * coef_stride + 2 * i + 1];
  const int64_t o = src * e_stride + (int64_t)m * k + i;
  ev[o] = ev[o] - conj(bt) * conj(es);
  ew[o] = ew[o] - d * conj(er);
}
template <typename R>
void rev_proj_record(const Lat<R>& L, const Rev<R>& B, int j, int m, const zd* coef, cudaStream_t st) {
  k_rev_proj_record<<<dim3(nblocks(j + 1, 128), L.nsrc), 128, 0, st>>>(
      B.ev, B.ew, (int64_t)B.nreb_max * L.k, L.k, m, j, coef, 2 * (int64_t)L.k, L.beta, L.delta);
}

// reverse sweep start: g_alpha of the last step comes from G_T alone; no carries yet
__global__ void k_rev_init(SrcScal* sc, const zd* __restrict__ gaT, int k, int nsrc) {
  const int src = blockIdx.x * blockDim.x + threadIdx.x;
  if (src >= nsrc) return;
  sc[src].g_alpha = gaT[(int64_t)src * k + k - 1];
  sc[src].carry_beta = mk(0.0, 0.0);
  sc[src].carry_delta = 0.0;
}
template <typename R>
void rev_init(const Lat<R>& L, const Rev<R>& B, cudaStream_t st) {
  k_rev_init<<<nblocks(L.nsrc, 32), 32, 0, st>>>(L.sc, B.gaT, L.k, L.nsrc);
}

// R3a: the two stencil inputs of step j, formed once per site
//   g_p = g_r + g_alpha w_j  (into the ring, for the force too),   h_in = conj(g_alpha) v_j + g_s
// (g_r, g_s are absent at the last step j = k - 1).
template <typename R>
__global__ void __launch_bounds__(BS) k_rev_combine(Lat<R> L, Rev<R> B, int j, int slot) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  if (x >= V) return;
  const cplx<R> ga = cast<R>(L.sc[src].g_alpha);
  const bool carry = j < L.k - 1;
  Spinor<R> a, e;
  load_spinor(L.basis_w(src, j), V, x, e);
  if (carry) {
    load_spinor(B.ring(B.gr_ring, slot, src), V, x, a);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(a.c[c], ga, e.c[c]);
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) a.c[c] = ga * e.c[c];
  }
  store_spinor(B.ring(B.gp_ring, slot, src), V, x, a);
  const cplx<R> gac = conj(ga);
  load_spinor(L.basis_v(src, j), V, x, e);
  if (carry) {
    load_spinor(B.ring(B.gs_ring, slot, src), V, x, a);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(a.c[c], gac, e.c[c]);
  } else {
#pragma unroll
    for (int c = 0; c < 12; ++c) a.c[c] = gac * e.c[c];
  }
  store_spinor(B.hin + src * L.vs, V, x, a);
}
template <typename R>
void rev_combine(const Lat<R>& L, const Rev<R>& B, int j, int slot, cudaStream_t st) {
  k_rev_combine<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, B, j, slot);
}

// R3b: complete gradients of v_j and w_j
//   Gv_j = -conj(beta_{j+1}) g_r' - conj(alpha_j) g_r + conj(y_j) xbar + H^dag g_p + acc_v
//   Gw_j = -delta_{j+1} g_s' - alpha_j g_s + H h_in + acc_w
// (primes: the previous step's g_r, g_s; g_p and h_in from R3a).
template <typename R>
__global__ void __launch_bounds__(BS) k_rev_stencil(Lat<R> L, Rev<R> B, int j, int slot, int prev_slot,
                                                     int nrec) {
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int src = blockIdx.y;
  const int64_t V = L.g.V;
  if (x >= V) return;
  const int64_t o = (int64_t)src * L.k + j;
  const cplx<R> al = cast<R>(L.alpha[o]);
  const cplx<R> yj = cast<R>(B.y[(int64_t)src * L.k + j]);
  const R* gr = slot >= 0 && j < L.k - 1 ? B.ring(B.gr_ring, slot, src) : nullptr;
  const R* gs = slot >= 0 && j < L.k - 1 ? B.ring(B.gs_ring, slot, src) : nullptr;
  Spinor<R> hv, hw, t;
  h_site_ld(FieldLoad<R>{B.ring(B.gp_ring, slot, src), V}, L.u, L.g, x, L.kappa, L.efinv, L.ef, hv);
  h_site_ld(FieldLoad<R>{B.hin + src * L.vs, V}, L.u, L.g, x, L.kappa, L.ef, L.efinv, hw);
  load_spinor(B.xbar + src * L.vs, V, x, t);
#pragma unroll
  for (int c = 0; c < 12; ++c) cmac(hv.c[c], conj(yj), t.c[c]);
  if (gr) {
    load_spinor(gr, V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(hv.c[c], -conj(al), t.c[c]);
    load_spinor(gs, V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(hw.c[c], -al, t.c[c]);
  }
  if (prev_slot >= 0 && j + 1 < L.k - 1) {
    const cplx<R> bn = cast<R>(L.beta[o + 1]);
    const R dn = (R)L.delta[o + 1];
    load_spinor(B.ring(B.gr_ring, prev_slot, src), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(hv.c[c], -conj(bn), t.c[c]);
    load_spinor(B.ring(B.gs_ring, prev_slot, src), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) hw.c[c] = hw.c[c] - dn * t.c[c];
  }
  for (int m = 0; m < nrec; ++m) {
    const int jm = B.reb_steps[m];
    const int64_t eo = src * (int64_t)B.nreb_max * L.k + (int64_t)m * L.k + j;
    const cplx<R> cv = cast<R>(B.ev[eo]), cw = cast<R>(B.ew[eo]);
    load_spinor(L.basis_w(src, jm + 1), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(hv.c[c], cv, t.c[c]);
    load_spinor(L.basis_v(src, jm + 1), V, x, t);
#pragma unroll
    for (int c = 0; c < 12; ++c) cmac(hw.c[c], cw, t.c[c]);
  }
  store_spinor(B.gv_new + src * L.vs, V, x, hv);
  store_spinor(B.gw_new + src * L.vs, V, x, hw);
}
template <typename R>
void rev_stencil(const Lat<R>& L, const Rev<R>& B, int j, int slot, int prev_slot, int nrec, cudaStream_t st) {
  k_rev_stencil<R><<<dim3(nblocks(L.g.V, site_bs(L.g.V)), L.nsrc), site_bs(L.g.V), 0, st>>>(L, B, j, slot,
                                                                                      prev_slot, nrec);
}

// ---------------------------------------------------------------------------
// Force: g_H = sum_t (g_p,t v_t^dag + w_t g_q,t^dag) contracted into dU (FP64
// accumulator, layout e*V + x with e = nu*9 + a*3 + b) and dmu.  One thread per
// (site, direction); terms of ring slots 0..nterms-1 have steps j0, j0-1, ...
//   forward hop:  G[c][c'] += sum_s a(x)_{s,c} conj((C+ b(x+nu))_{s,c'})
//   backward hop: G[c][c'] += sum_s conj(a(x+nu)_{s,c'}) (C- b(x))_{s,c}
//   C+ = -kappa f gamma5 (1+gamma_nu),  C- = -kappa f^-1 gamma5 (1-gamma_nu)
//   dmu += Re <G_fwd - G_bwd, U_t(x)>  on temporal links.
// ---------------------------------------------------------------------------
template <int NU, typename R>
__device__ void force_term(const Lat<R>& L, int64_t x, int64_t xf, const R* a, const R* b, cplx<R> (&G)[9],
                           cplx<R> (&Gd)[9]) {
  const int64_t V = L.g.V;
  const R ff = NU == 3 ? L.ef : R(1), fb = NU == 3 ? L.efinv : R(1);
  Spinor<R> sa, sb;
  load_spinor(a, V, x, sa);
  load_spinor(b, V, xf, sb);
  force_half_fwd<NU>(sa, sb, -L.kappa * ff, G, Gd, NU == 3);
  load_spinor(a, V, xf, sa);
  load_spinor(b, V, x, sb);
  force_half_bwd<NU>(sa, sb, -L.kappa * fb, G, Gd, NU == 3);
}

template <int NU, typename R>
__device__ void force_dir(const Lat<R>& L, const Rev<R>& B, int64_t x, int nterms, int j0, int i0, int i1,
                          double* part, zd* dmu_site) {
  // items i0 .. i1-1 of the (source, term) pairs, source outer
  int c[4];
  site_coords(L.g, x, c);
  const int64_t xf = neighbour(L.g, x, c, NU, +1);
  zd acc[9];
  zd accd[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) acc[e] = accd[e] = mk(0.0, 0.0);
  for (int src = i0 / nterms; src * nterms < i1; ++src) {
    const int t0 = max(i0 - src * nterms, 0), t1 = min(i1 - src * nterms, nterms);
    if constexpr (sizeof(R) == 8) {
      // FP64 fields: accumulate straight into the FP64 sums
      for (int t = t0; t < t1; ++t) {
        const int j = j0 - t;
        force_term<NU>(L, x, xf, B.ring(B.gp_ring, t, src), L.basis_v(src, j), acc, accd);
        if (j < L.k - 1) force_term<NU>(L, x, xf, L.basis_w(src, j), B.ring(B.gs_ring, t, src), acc, accd);
      }
    } else {
      // FP32 fields: FP32 partial sums over one ring of terms, then FP64
      cplx<R> G[9], Gd[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) G[e] = Gd[e] = czero<R>();
      for (int t = t0; t < t1; ++t) {
        const int j = j0 - t;
        force_term<NU>(L, x, xf, B.ring(B.gp_ring, t, src), L.basis_v(src, j), G, Gd);
        if (j < L.k - 1) force_term<NU>(L, x, xf, L.basis_w(src, j), B.ring(B.gs_ring, t, src), G, Gd);
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        acc[e] = acc[e] + mk((double)G[e].re, (double)G[e].im);
        accd[e] = accd[e] + mk((double)Gd[e].re, (double)Gd[e].im);
      }
    }
  }
  if (part) {   // a split of the items: its own partial sum, added in split order later
    double2* f = reinterpret_cast<double2*>(part);
#pragma unroll
    for (int e = 0; e < 9; ++e) f[(int64_t)(NU * 9 + e) * L.g.V + x] = make_double2(acc[e].re, acc[e].im);
  } else {
    double2* f = reinterpret_cast<double2*>(B.force);
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      double2 o = f[(int64_t)(NU * 9 + e) * L.g.V + x];
      o.x += acc[e].re;
      o.y += acc[e].im;
      f[(int64_t)(NU * 9 + e) * L.g.V + x] = o;
    }
  }
  if (NU == 3) {
    double dm = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const cplx<R> u = load_link_entry(L.u, L.g.V, x, 27 + e);
      dm += accd[e].re * (double)u.re + accd[e].im * (double)u.im;     // Re(conj(Gd) u)
    }
    dmu_site->re = dm;
  }
}

// One launch per direction (smaller register footprint); on small lattices the
// (source, term) items are split over blockIdx.y, each split writing its own
// partial force, added in split order by k_force_reduce.  dmu comes from NU = 3.
template <int NU, typename R>
__global__ void __launch_bounds__(BS) k_force(Lat<R> L, Rev<R> B, int nterms, int j0, int nsplit, double* parts) {
  __shared__ zd scratch[32];
  const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int split = blockIdx.y, nitems = L.nsrc * nterms;
  const int i0 = (int)((int64_t)split * nitems / nsplit), i1 = (int)((int64_t)(split + 1) * nitems / nsplit);
  double* part = nsplit > 1 ? parts + (int64_t)split * 72 * L.g.V : nullptr;
  zd v[1] = {mk(0.0, 0.0)};
  if (x < L.g.V) force_dir<NU>(L, B, x, nterms, j0, i0, i1, part, &v[0]);
  if (NU != 3) return;
  block_sum<1>(v, scratch);
  if (threadIdx.x == 0) B.dmu_part[split * gridDim.x + blockIdx.x] = v[0];
  if (arrive_last(B.dmu_cnt, gridDim.x * gridDim.y)) {
    zd s[1];
    sum_partials<1>(B.dmu_part, gridDim.x * gridDim.y, s, scratch);
    if (threadIdx.x == 0) *B.dmu += s[0].re;
  }
}
__global__ void k_force_reduce(double* __restrict__ force, const double* __restrict__ parts, int nsplit, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = force[i];
  for (int sp = 0; sp < nsplit; ++sp) a += parts[sp * n + i];
  force[i] = a;
}
int force_splits(int64_t V) {
  const int64_t blocks = (V + BS - 1) / BS;
  if (blocks >= 152) return 1;
  const int64_t want = (2 * 152 + blocks - 1) / blocks;
  return (int)(want < kForceSplitMax ? want : kForceSplitMax);
}
template <typename R>
void force_flush(const Lat<R>& L, const Rev<R>& B, const int* /*unused*/, int nterms, int j0, cudaStream_t st) {
  if (nterms <= 0) return;
  const unsigned nb = nblocks(L.g.V, BS);
  int nsplit = B.force_parts ? force_splits(L.g.V) : 1;
  if (nsplit > L.nsrc * nterms) nsplit = L.nsrc * nterms;
  k_force<0, R><<<dim3(nb, nsplit), BS, 0, st>>>(L, B, nterms, j0, nsplit, B.force_parts);
  k_force<1, R><<<dim3(nb, nsplit), BS, 0, st>>>(L, B, nterms, j0, nsplit, B.force_parts);
  k_force<2, R><<<dim3(nb, nsplit), BS, 0, st>>>(L, B, nterms, j0, nsplit, B.force_parts);
  k_force<3, R><<<dim3(nb, nsplit), BS, 0, st>>>(L, B, nterms, j0, nsplit, B.force_parts);
  if (nsplit > 1) {
    const int64_t n = 72 * L.g.V;
    k_force_reduce<<<nblocks(n, 256), 256, 0, st>>>(B.force, B.force_parts, nsplit, n);
  }
}

// explicit instantiations
// ---------------------------------------------------------------------------
// Error estimates (Sec. 4.1, Eqs. error_est and bA_error_est): per source
//   out[3 src + 0] = ||a_top||^2,  out[3 src + 1] = ||a_bot - b||^2,  out[3 src + 2] = ||b||^2
// over interleaved complex128 fields of n doubles per source (a_top may be null).
// One block per source, fixed strides and tree: deterministic.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_eps_norms(const double* __restrict__ a_top, const double* __restrict__ a_bot,
                                                   const double* __restrict__ b, int64_t n, double* __restrict__ out) {
  __shared__ zd scratch[2 * 32];
  const int src = blockIdx.x;
  const double* at = a_top ? a_top + (int64_t)src * n : nullptr;
  const double* ab = a_bot + (int64_t)src * n;
  const double* bb = b + (int64_t)src * n;
  zd v[2] = {mk(0.0, 0.0), mk(0.0, 0.0)};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double t = at ? at[i] : 0.0, d = ab[i] - bb[i], q = bb[i];
    v[0].re = fma(t, t, v[0].re);
    v[0].im = fma(d, d, v[0].im);
    v[1].re = fma(q, q, v[1].re);
  }
  block_sum<2>(v, scratch);
  if (threadIdx.x == 0) {
    out[3 * src + 0] = v[0].re;
    out[3 * src + 1] = v[0].im;
    out[3 * src + 2] = v[1].re;
  }
}
void eps_norms(const double* a_top, const double* a_bot, const double* b, int nsrc, int64_t n, double* out,
               cudaStream_t st) {
  k_eps_norms<<<nsrc, 512, 0, st>>>(a_top, a_bot, b, n, out);
}

#define OV_INST(R)                                                                                        \
  template void ritz_combine<R>(const Lat<R>&, int, int, int, const zd*, double*, cudaStream_t);        \
  template void apply_dh<R>(const Lat<R>&, const R*, R*, int, cudaStream_t);                             \
  template void pack_spinors<R>(const double*, R*, int, int64_t, int64_t, cudaStream_t);                 \
  template void pack_block_start<R>(const double*, const double*, R*, R*, int, int64_t, int64_t,          \
                                    cudaStream_t);                                                       \
  template void unpack_spinors<R>(const R*, double*, int, int64_t, int64_t, cudaStream_t);               \
  template void pack_links<R>(const double*, R*, int64_t, cudaStream_t);                                 \
  template void apply_h<R>(const Lat<R>&, const R*, R*, int, cudaStream_t, int, int*);                   \
  template void tsl_init<R>(const Lat<R>&, cudaStream_t);                                                \
  template void tsl_stencil<R>(const Lat<R>&, int, bool, cudaStream_t, int);                             \
  template void tsl_update<R>(const Lat<R>&, int, bool, cudaStream_t);                                   \
  template void proj_dots<R>(const Lat<R>&, int, int, const R*, const R*, int64_t, zd*, zd*, cudaStream_t); \
  template void proj_update<R>(const Lat<R>&, int, int, R*, R*, int64_t, const zd*, bool, cudaStream_t, \
                               bool);                                                                   \
  template void basis_dots<R>(const Lat<R>&, int, const R*, int64_t, zd*, zd*, cudaStream_t);            \
  template void combine<R>(const Lat<R>&, int, const zd*, double*, cudaStream_t);                        \
  template void combine_range<R>(const Lat<R>&, int, int, const zd*, double*, bool, cudaStream_t);       \
  template void basis_dots_range<R>(const Lat<R>&, int, int, const R*, int64_t, zd*, zd*, cudaStream_t); \
  template void rev_init<R>(const Lat<R>&, const Rev<R>&, cudaStream_t);                                 \
  template void rev_dots<R>(const Lat<R>&, const Rev<R>&, int, cudaStream_t);                            \
  template void rev_form<R>(const Lat<R>&, const Rev<R>&, int, int, bool, cudaStream_t);                 \
  template void rev_proj_record<R>(const Lat<R>&, const Rev<R>&, int, int, const zd*, cudaStream_t);     \
  template void rev_alpha_dots<R>(const Lat<R>&, const Rev<R>&, int, int, cudaStream_t);                 \
  template void rev_combine<R>(const Lat<R>&, const Rev<R>&, int, int, cudaStream_t);                    \
  template void rev_stencil<R>(const Lat<R>&, const Rev<R>&, int, int, int, int, cudaStream_t);          \
  template void force_flush<R>(const Lat<R>&, const Rev<R>&, const int*, int, int, cudaStream_t);

OV_INST(double)
OV_INST(float)

}  // namespace ov
