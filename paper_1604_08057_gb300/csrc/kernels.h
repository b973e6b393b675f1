// Host-visible declarations of the kernel launchers and the device-side
// per-source state shared by the forward recurrence and the reverse sweep.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ov {

// error bits written by kernels into SrcScal::err
enum : int { ERRB_BREAKDOWN = 1, ERRB_NONFINITE = 2, ERRB_SINGULAR = 4, ERRB_TIMEOUT = 8 };

// Per-source scalars kept in device memory for the whole call.
struct SrcScal {
  double beta0;          // ||b||
  zd sv, sw;             // v_j = sv * r_{j-1},  w_j = sw * s_{j-1}
  int err;               // ERRB_* bits
  int err_step;          // first step that set an error bit
  // reverse sweep
  zd g_alpha;            // gradient of alpha_j of the current step
  zd carry_beta;         // gradient of beta_{j} carried from step j (for step j-1)
  double carry_delta;
  zd cr1, cr2, cs1, cs2; // g_r = cr1 Gv_{j+1} + cr2 w_{j+1};  g_s = cs1 Gw_{j+1} + cs2 v_{j+1}
};

// Everything a lattice kernel needs, passed by value.
template <typename R>
struct Lat {
  Geom g;
  R kappa, ef, efinv;        // kappa, e^{mu}, e^{-mu}
  const R* u;                // internal links (link_reals<R>() * V reals)
  int nsrc, k;
  int64_t vs;                // reals per lattice vector (padded)
  R* bv;                     // basis V: [src][kcap][vs]
  R* bw;                     // basis W: [src][kcap][vs]
  R* p; R* q; R* r; R* s;    // per-source scratch vectors [src][vs]
  SrcScal* sc;               // [src]
  zd* alpha;                 // [src][k]
  zd* beta;                  // [src][k]  (index j couples j-1 and j)
  double* delta;             // [src][k]
  zd* part;                  // reduction partials
  unsigned* cnt;             // last-block counters [src][16]
  int64_t part_stride;       // zd per source in `part`
  // block mode (Theorem-1 block matrix [[H, dH], [0, H]]): every field holds the
  // upper half at sites [0, V) and the lower half at [V, 2V) of a 2V-site field;
  // g.V is then 2V (element-wise kernels), gl is the lattice itself.
  int block;
  Geom gl;
  const R* ue;               // links of the direction E (internal layout) or null
  R mdir;                    // mu direction
  // basis window: vectors jbase .. jbase + kcap - 1 (all k from 0 unless segments are replayed)
  int kcap, jbase;
  OV_HD R* basis_v(int src, int j) const { return bv + ((int64_t)src * kcap + (j - jbase)) * vs; }
  OV_HD R* basis_w(int src, int j) const { return bw + ((int64_t)src * kcap + (j - jbase)) * vs; }
};

// reverse-sweep buffers
template <typename R>
struct Rev {
  R* gv; R* gw;              // complete gradients of v_{j+1}, w_{j+1}: [src][vs]
  R* gv_new; R* gw_new;      // gradients being formed for v_j, w_j
  R* gr_ring; R* gs_ring; R* gp_ring;   // [m][src][vs]
  R* hin;                    // conj(g_alpha) v_j + g_s of the current step: [src][vs]
  int m;                     // ring length
  const R* xbar;             // [src][vs]
  const zd* y;               // [src][k]
  const zd* gaT; const zd* gbT; const double* gdT;   // [src][k] gradients of T entries
  zd* ev; zd* ew;            // lazy projection-adjoint coefficients [src][nreb_max][k]
  int* reb_steps;            // [nreb_max] step of each recorded projection (host-ordered)
  int nreb_max;
  double* force;             // FP64 accumulator, 36 complex * V  (zd, layout e*V + x)
  double* force_parts;       // small lattices: force_splits(V) partial forces (72 V doubles each), or null
  double* dmu;               // single accumulator
  zd* dmu_part;              // partials for dmu
  unsigned* dmu_cnt;
  int nsrc;
  int64_t vs;
  OV_HD R* ring(R* base, int slot, int src) const { return base + ((int64_t)slot * nsrc + src) * vs; }
};

// ---- lattice launchers (precision R = double or float) ----
template <typename R> void pack_spinors(const double* src_aos, R* dst, int nsrc, int64_t V, int64_t vs, cudaStream_t st);
// Theorem-1 block start: r = (top, bot), s = (top + bot, bot) in fields of 2V sites (top may be null)
template <typename R> void pack_block_start(const double* top_aos, const double* bot_aos, R* r, R* s, int nsrc,
                                            int64_t V, int64_t vs, cudaStream_t st);
template <typename R> void unpack_spinors(const R* src, double* dst_aos, int nsrc, int64_t V, int64_t vs, cudaStream_t st);
template <typename R> void pack_links(const double* src_aos, R* dst, int64_t V, cudaStream_t st);
// launch variants of the two stencil kernels (chosen by the autotuner; 0 = default)
int apply_h_variants();
int tsl_stencil_variants();
// err (may be null): the staged variants set ERRB_TIMEOUT there when their bounded
// wait on the shared-memory copies runs out
template <typename R> void apply_h(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st,
                                   int variant = 0, int* err = nullptr);
// Variant APPLY_IL of the multi-source FP32 operator: fields with the sources
// interleaved innermost, float4 (two complex components) at ((x * 6 + cp) * nsrc + src),
// one thread per (site, source), a warp reading one site's component pair for 32
// sources as 512 contiguous bytes and its links as one broadcast.  apply_h runs
// variant 0 for APPLY_IL (its fields are per-source); apply_h_il, pack_spinors_il and
// unpack_spinors_il are the interleaved form.
constexpr int APPLY_IL = 13;
// out = dH in (dagger 0) or dH^dag in (dagger 1), dH along L.ue (may be null) and L.mdir
template <typename R> void apply_dh(const Lat<R>& L, const R* in, R* out, int dagger, cudaStream_t st);
void apply_h_il(const Lat<float>& L, const float* in, float* out, int dagger, cudaStream_t st);
void pack_spinors_il(const double* aos, float* dst, int nsrc, int64_t V, cudaStream_t st);
void unpack_spinors_il(const float* f, double* aos, int nsrc, int64_t V, cudaStream_t st);

template <typename R> void tsl_init(const Lat<R>& L, cudaStream_t st);
template <typename R> void tsl_stencil(const Lat<R>& L, int j, bool need_q, cudaStream_t st, int variant = 0);
template <typename R> void tsl_update(const Lat<R>& L, int j, bool finalize, cudaStream_t st);
// projection of (r, s) against bases (A: dots with `a` vector, B: dots with `b` vector).
// mode 0 (forward):  c = W^dag r, d = V^dag s;  r -= V c, s -= W d
// mode 1 (adjoint):  e_r = V^dag g_r, e_s = W^dag g_s;  g_r -= W e_r, g_s -= V e_s
template <typename R> void proj_dots(const Lat<R>& L, int j, int mode, const R* a, const R* b,
                                     int64_t ab_src_stride, zd* coef, zd* cpart, cudaStream_t st);
// small: the coefficients are at rounding level (a second Gram-Schmidt pass): FP32 accumulation
template <typename R> void proj_update(const Lat<R>& L, int j, int mode, R* a, R* b, int64_t ab_src_stride,
                                       const zd* coef, bool finalize_omega, cudaStream_t st, bool small);
template <typename R> void basis_dots(const Lat<R>& L, int nvec, const R* x, int64_t x_src_stride, zd* out,
                                      zd* cpart, cudaStream_t st);
// out[src][2 (j - j0)] = v_j^dag x  for j0 <= j < j0 + nvec
template <typename R> void basis_dots_range(const Lat<R>& L, int j0, int nvec, const R* x, int64_t x_src_stride,
                                            zd* out, zd* cpart, cudaStream_t st);
template <typename R> void combine(const Lat<R>& L, int nvec, const zd* y, double* out_aos, cudaStream_t st);
// out_aos (one field, user layout) = sum_{j < nvec} y_j u_j of source src, u = V (side 0) or W (side 1)
template <typename R> void ritz_combine(const Lat<R>& L, int src, int side, int nvec, const zd* y, double* out_aos,
                                       cudaStream_t st);
// out (+)= sum_{j0 <= j < j0 + nvec} y_j v_j  (accumulate when acc is set)
template <typename R> void combine_range(const Lat<R>& L, int j0, int nvec, const zd* y, double* out_aos, bool acc,
                                         cudaStream_t st);
void eps_norms(const double* a_top, const double* a_bot, const double* b, int nsrc, int64_t n, double* out,
               cudaStream_t st);

// reverse sweep
template <typename R> void rev_init(const Lat<R>& L, const Rev<R>& B, cudaStream_t st);
template <typename R> void rev_dots(const Lat<R>& L, const Rev<R>& B, int j, cudaStream_t st);
template <typename R> void rev_form(const Lat<R>& L, const Rev<R>& B, int j, int slot, bool with_dots, cudaStream_t st);
template <typename R> void rev_proj_record(const Lat<R>& L, const Rev<R>& B, int j, int m_index, const zd* coef, cudaStream_t st);
template <typename R> void rev_alpha_dots(const Lat<R>& L, const Rev<R>& B, int j, int slot, cudaStream_t st);
template <typename R> void rev_combine(const Lat<R>& L, const Rev<R>& B, int j, int slot, cudaStream_t st);
template <typename R> void rev_stencil(const Lat<R>& L, const Rev<R>& B, int j, int slot, int prev_slot,
                                       int nrec, cudaStream_t st);
// splits of the force contraction's (source, term) items: 1 unless the lattice has
// too few sites to fill the GPU, at most kForceSplitMax
constexpr int kForceSplitMax = 8;
int force_splits(int64_t V);
template <typename R> void force_flush(const Lat<R>& L, const Rev<R>& B, const int* steps_dev, int nterms,
                                       int first_slot, cudaStream_t st);
void unpack_force(const double* force, double* du_aos, int64_t V, cudaStream_t st);

// ---- dense FP64 k x k (row-major, complex) ----
void dense_build_t(const zd* alpha, const zd* beta, const double* delta, int k, zd* T, cudaStream_t st);
void dense_adjoint(const zd* A, zd* B, int k, cudaStream_t st);
void dense_copy(const zd* A, zd* B, int64_t n, cudaStream_t st);
void dense_zero(zd* A, int64_t n, cudaStream_t st);
// Batched forms: nb problems, problem p at A + p * sA (etc.); act (device, may be
// null = all) switches problems off, so each problem can stop on its own.
void dense_copy_batch(const zd* A, int64_t sA, zd* B, int64_t sB, int64_t n, int nb, const int* act,
                      cudaStream_t st);
// Ainv = A^{-1} by Gauss-Jordan with partial pivoting for nb problems (matrices
// at stride k*k; A is not modified; w0, w1 work matrices; ipiv, used: k ints and
// keys: (k + 1) * GJ_KEY_SLOTS words per problem); logdet[p * ld_stride] += log|det A_p|.
// mode GJ_AUTO: one cooperative launch per inversion where the rows fit in
// shared memory, else (and with GJ_STEPS) one launch per elimination step,
// replayed as a CUDA graph.  Both give identical results.  Returns the number
// of kernels launched.
enum : int { GJ_AUTO = 0, GJ_STEPS = 1 };
constexpr int GJ_KEY_SLOTS = 160;   // pivot-key words per step and problem (>= blocks per problem)
int dense_inverse(const zd* A, zd* Ainv, zd* w0, zd* w1, int k, int nb, const int* act, int* ipiv, int* used,
                  unsigned long long* keys, double* logdet, int ld_stride, int* err, int mode, cudaStream_t st);
// the bounded inter-block wait of the cooperative inversion, made to run out
void dense_wait_probe(unsigned long long* slot, int* err, int* how, unsigned long long limit_ns, cudaStream_t st);
void dense_gemm(const zd* A, const zd* B, zd* C, int k, cudaStream_t st);   // C = A B
// C = op(A) op(B), op = conjugate transpose when the flag is set
void dense_gemm_op(const zd* A, int hA, const zd* B, int hB, zd* C, int k, cudaStream_t st);
void dense_gemm_batch(const zd* A, int64_t sA, int hA, const zd* B, int64_t sB, int hB, zd* C, int64_t sC, int k,
                      int nb, const int* act, cudaStream_t st);
// C = op(A) op(B) for one k x k problem on the BF16 tensor cores by the exact digit
// splitting of ozaki.cu (k <= OZ_MAX_K); ws holds oz_workspace_bytes(k) device bytes,
// handle is a cuBLAS handle from oz_create_handle.  Returns the number of own kernels
// launched, or < 0 (-1 k out of range, -2 launch error, -3 cuBLAS error).
constexpr int OZ_MAX_K = 1024;
size_t oz_workspace_bytes(int k);
int oz_zgemm(void* handle, const zd* A, int hA, const zd* B, int hB, zd* C, int k, void* ws, cudaStream_t st);
void* oz_create_handle();
void oz_destroy_handle(void* handle);
// C (M x N) = op(A) op(B) with leading dimensions (op = conjugate transpose when the flag is set)
void dense_gemm_rect_batch(const zd* A, int64_t sA, int lda, int hA, const zd* B, int64_t sB, int ldb, int hB, zd* C,
                           int64_t sC, int ldc, int M, int N, int K, int nb, const int* act, cudaStream_t st);
// low-rank Frechet adjoint: factors A, B (k x ld each per problem) of E = A B^H
void dense_lr_init(zd* A, zd* B, int k, int ld, const zd* gy, int64_t gy_pstride, int64_t gy_stride,
                   const double* beta0, int nb, cudaStream_t st);
void dense_lr_scale(zd* A, int k, int ld, int r, const double* logdet, int ld_stride, const int* scal,
                    int scal_stride, int nb, const int* act, cudaStream_t st);
// Xn = 0.5 (g X + s Xi / g) with g = |det|^(-1/k) from *logdet when scaling, else 1;
// stats[0] += w |Xn - X|^2, stats[1] += w |Xn|^2 (deterministic order)
void dense_newton_combine(const zd* X, const zd* Xi, zd* Xn, int k, const double* logdet, int scaling,
                          double s, double w, double* stats, zd* part, unsigned* cnt, cudaStream_t st);
// batched: log|det| at logdet[p * ld_stride], scaling flag scal[p * scal_stride],
// stats at stats + 4 p, partials at part + p * part_stride, tickets at cnt + 4 p
void dense_newton_combine_batch(const zd* X, const zd* Xi, zd* Xn, int k, int nb, const int* act,
                                const double* logdet, int ld_stride, const int* scal, int scal_stride, double s,
                                double w, double* stats, zd* part, int64_t part_stride, unsigned* cnt,
                                cudaStream_t st);
// ---- overlap operator, its Krylov solver and the U(1) current (user layout, complex128) ----
// out = b + gamma5 x (g5 != 0) or b + x, n complex elements (12 per site)
void ov_combine(const double* b, const double* x, double* out, int64_t n, int g5, cudaStream_t st);
// out = f gamma5 in, f = fr + i fi
void gamma5_scale(const double* in, double* out, int64_t n, double fr, double fi, cudaStream_t st);
// out[i] = basis_i^dag w for i < nvec (basis_i at basis + i * stride doubles); partial: 152 * nvec zd
void vec_dots(const double* basis, int64_t stride, int nvec, const double* w, int64_t n, zd* out, zd* partial,
              cudaStream_t st);
// w += s sum_i coef_i basis_i (coef on the device)
void vec_update(double* w, const double* basis, int64_t stride, int nvec, const zd* coef, double s, int64_t n,
                cudaStream_t st);
void vec_scale(const double* in, double* out, double fr, double fi, int64_t n, cudaStream_t st);
// out[p * l + i] = sg[i] in[p * l + i] for p < np, i < l (deflation: the exact part's coefficients)
void coef_sign(const zd* in, const double* sg, zd* out, int l, int np, cudaStream_t st);
void vec_sub(const double* a, const double* b, double* out, int64_t n, cudaStream_t st);
// j[l] (+)= scale (-Im sum conj(g_re) U + i (-Im sum conj(g_im) U)) per link l < nlinks (9 entries each)
void theta_current(const double* u, const double* g_re, const double* g_im, double* j, int64_t nlinks, double scale,
                   int accumulate, cudaStream_t st);

// Frobenius-norm Newton scaling g = (||Xi||_F / ||X||_F)^{1/2} written as the equivalent
// ld[p * ld_stride] = -(k/4) log(||Xi||_F^2 / ||X||_F^2) (so that exp(-ld / k) = g), for
// nb problems at stride k*k; part: 64 zd and cnt: one ticket (zero) per problem.
void dense_norm_scale(const zd* X, const zd* Xi, int k, int nb, const int* act, double* ld, int ld_stride, zd* part,
                      unsigned* cnt, cudaStream_t st);
void dense_set_column0(zd* E, const zd* gy, int64_t gy_stride, double beta0, int k, cudaStream_t st);
void dense_extract_y(const zd* F, double beta0, int k, zd* y, cudaStream_t st);
void dense_extract_tri(const zd* E, int k, zd* ga, zd* gb, double* gd, cudaStream_t st);

// ---- nested Krylov sign of T_k (Sec. 4.1, one nesting level; nested.cu) ----
// Workspace for nb problems: lu [nb][4k], piv [nb][k], s [nb][k][k] (S = (T + T^{-1})/2),
// q [nb][m][k] (inner basis), w [nb][k], h [nb][m][m] (Hessenberg H_m), meff [nb],
// hb [nb][m] (one step's Gram-Schmidt coefficients), wn [nb] (||S q_j||^2).
struct NestWs {
  zd* lu;
  int* piv;
  zd* s;
  zd* q;
  zd* w;
  zd* h;
  int* meff;
  zd* hb;
  double* wn;
};
// LU of every T, S, q_0 = e_1, h = 0, meff = m; sets *err on a singular T.  Returns launches.
int nested_prepare(const zd* alpha, const zd* beta, const double* delta, int k, int nb, int m, const NestWs& W,
                   int* err, cudaStream_t st);
// m Arnoldi steps on S from e_1 (two launches per step); meff[p] drops below m when
// problem p's Krylov space closes.  Returns launches.
int nested_arnoldi(int k, int nb, int m, const NestWs& W, int* err, cudaStream_t st);
// y = beta0 sum_{c < me} q_c F[c][0]; q one problem's basis, F its sign (leading dimension ld)
void nested_combine(const zd* q, const zd* F, int ld, int k, int me, double beta0, zd* y, cudaStream_t st);

}  // namespace ov
