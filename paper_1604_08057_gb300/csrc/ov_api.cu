// C ABI of the library (include/ov.h): argument checks, workspace, and the
// host-side driver that enqueues the kernels of the forward two-sided Lanczos
// recurrence, the k x k sign, the reverse sweep and the force contraction.
#include <cmath>
#include <complex>
#include <cstddef>
#include <algorithm>
#include <atomic>
#include <thread>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ov.h"
#include "kernels.h"

using namespace ov;

namespace {

enum BufId {
  B_LINKS, B_BV, B_BW, B_P, B_Q, B_R, B_S, B_SC, B_ALPHA, B_BETA, B_DELTA, B_PART, B_CNT, B_COEF, B_CPART,
  B_T, B_X, B_XI, B_XN, B_E, B_EN, B_TMP1, B_TMP2, B_IPIV, B_PROW, B_COL, B_DSTAT, B_DPART, B_DCNT, B_DERR,
  B_Y, B_GY, B_GA, B_GB, B_GD, B_XBAR, B_GV, B_GW, B_GV2, B_GW2, B_GR, B_GS, B_GP, B_EV, B_EW, B_REB,
  B_FORCE, B_DMU, B_DMUPART, B_DMUCNT, B_W0, B_W1, B_REC, B_RECLD, B_ELINKS, B_BLOCKOUT, B_HIN, B_CKR, B_CKS, B_CKV, B_CKW, B_CKSC, B_FSIGN, B_ACT, B_SCAL, B_RSCAL, B_FPARTS, B_LRA, B_LRB, B_BETA0, B_EPS1T, B_EPS1B, B_EPS2T, B_EPS2B, B_EPSN, B_NSPART, B_NSCNT, B_OVX, B_OVB, B_GMV, B_GMW, B_GMR, B_GMH, B_GMP, B_CHI, B_CURX1, B_CURX2, B_CURG1, B_CURG2, B_AERR, B_OZ, B_DFA, B_DFC, B_DFSA, B_DFSC, B_DFPART, B_DFTOP, B_DFBOT, B_DFSG, B_RZY, B_RZF, B_RZH, B_RZD, B_EDT1, B_EDT2, B_EDX, B_EDC, B_CGY, B_CGR, B_CGP, B_CGQ, B_CGT, B_CGC, B_SIQ, B_SILT, B_SIT1, B_SIC, B_SIP, B_NLU, B_NPIV, B_NS, B_NQ, B_NW, B_NH, B_NHN, B_NMEFF, B_NHC, B_NHCN, B_NTA, B_NTB, B_NTD, B_NTY, B_NHB, B_NWN, NBUF
};

struct Status {
  int code;
};

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      std::fprintf(stderr, "ov: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), \
                   __FILE__, __LINE__);                                            \
      throw Status{OV_ERR_CUDA};                                                   \
    }                                                                              \
  } while (0)

inline void launch_check() { CK(cudaGetLastError()); }

int rebiorth_at(int step, int period) {
  if (period <= 0) return 0;
  if (period == 1) return 1;
  const int m = step % period;
  return m == 0 || m == 1;
}

}  // namespace

constexpr int NPROF = 8192;   // event pairs recorded before an intermediate collection

struct Prof {
  bool on = false;
  uint32_t mask = ~0u;   // kinds to time (bit per OV_KIND_*)
  int n = 0;
  cudaEvent_t a[NPROF] = {}, b[NPROF] = {};
  int kind[NPROF] = {};
  double ms[OV_NKIND] = {};
  int64_t cnt[OV_NKIND] = {};
};

struct ov_context {
  cudaStream_t st = nullptr;
  ov_options opt{};
  void* buf[NBUF] = {};
  size_t cap[NBUF] = {};
  bool host_buf[NBUF] = {};     // allocated as mapped pinned host memory (options.basis_memory)
  // coefficients of the last forward pass (for ov_tsl_coefficients)
  int last_k = 0, last_nsrc = 0;
  // shape of the last forward pass whose bases stay in B_BV / B_BW (for ov_tsl_ritz_triples)
  int last_block = 0, last_seg = 0, last_prec = -1;
  int32_t last_dims[4] = {0, 0, 0, 0};
  cudaEvent_t ev[8] = {};
  Prof* prof = nullptr;
  int64_t launches = 0;
  int tuned_apply[2] = {0, 0};  // per precision (OV_FP64, OV_MIXED)
  int tuned_pair[2] = {0, 0};
  bool owns_stream = false;     // worker contexts of ov_tsl_batch own theirs
  std::vector<ov_context*> workers;
  // captured sweeps (options.graphs): key of the captured call shape, executable graph,
  // kernels it launches; the capture stream and the events ordering it with `st`
  struct SweepGraph {
    std::vector<unsigned char> key;    // shape of the captured graph
    std::vector<unsigned char> seen;   // shape of the last call launched directly
    cudaGraphExec_t exec = nullptr;
    int64_t nlaunch = 0;
  } gfwd, grev, gnest;   // forward sweep, reverse sweep, nested k x k stage
  cudaStream_t cap_st = nullptr;
  cudaEvent_t cap_ev[2] = {nullptr, nullptr};
  // one-shot host-side fault injection (ov_debug_inject)
  int inj_kind = OV_INJECT_NONE, inj_step = 0;
  int inj_word[2] = {0, 0};     // host copy of the error word written by an injected breakdown
  double inj_nan[2] = {0.0, 0.0};
  void* blas = nullptr;         // cuBLAS handle of the tensor-core k x k products (options.gemm)
};

namespace {

// add the recorded event pairs to the per-kind totals (synchronises the stream)
void prof_collect(ov_context* c) {
  Prof* p = c->prof;
  if (!p || p->n == 0) return;
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < p->n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->a[i], p->b[i]));
    p->ms[p->kind[i]] += ms;
    p->cnt[p->kind[i]] += 1;
  }
  p->n = 0;
}

// run a launcher that enqueues `nl` kernels; time it when profiling is on
template <typename F>
void run(ov_context* c, int kind, int64_t nl, F&& f) {
  Prof* p = c->prof;
  const bool rec = p && p->on && ((p->mask >> kind) & 1u);
  if (rec && p->n == NPROF) prof_collect(c);
  if (rec) CK(cudaEventRecord(p->a[p->n], c->st));
  f();
  if (rec) {
    CK(cudaEventRecord(p->b[p->n], c->st));
    p->kind[p->n++] = kind;
  }
  c->launches += nl;
}

void* ws(ov_context* c, int id, size_t bytes, bool zero);

// C_p = op(A_p) op(B_p), k x k complex, for the problems p < nb with act[p] set (all
// when act is null; act_dev is the device copy): on the BF16 tensor cores by the exact
// digit splitting (options.gemm), else FP64 arithmetic
// whether the k x k products of this context run on the tensor cores (options.gemm)
bool kk_split(const ov_context* c, int k) {
  return k <= OZ_MAX_K && (c->opt.gemm == 2 || (c->opt.gemm == 0 && k >= 128));
}

void kk_gemm(ov_context* c, const zd* A, int64_t sA, int hA, const zd* B, int64_t sB, int hB, zd* C, int64_t sC,
             int k, int nb, const std::vector<int>* act, const int* act_dev) {
  const bool split = kk_split(c, k);
  if (!split) {
    run(c, OV_KIND_DENSE_GEMM, 1,
        [&] { dense_gemm_batch(A, sA, hA, B, sB, hB, C, sC, k, nb, act ? act_dev : nullptr, c->st); });
    return;
  }
  if (!c->blas) {
    c->blas = oz_create_handle();
    if (!c->blas) throw Status{OV_ERR_CUDA};
  }
  void* w = ws(c, B_OZ, oz_workspace_bytes(k), false);
  for (int p = 0; p < nb; ++p) {
    if (act && !(*act)[p]) continue;
    run(c, OV_KIND_DENSE_GEMM, 0, [&] {
      const int r = oz_zgemm(c->blas, A + p * sA, hA, B + p * sB, hB, C + p * sC, k, w, c->st);
      if (r < 0) throw Status{OV_ERR_CUDA};
      c->launches += r;
    });
  }
}

void free_buf(ov_context* c, int id) {
  if (!c->buf[id]) return;
  if (c->host_buf[id]) {
    CK(cudaStreamSynchronize(c->st));
    CK(cudaFreeHost(c->buf[id]));
  } else {
    CK(cudaFree(c->buf[id]));
  }
  c->buf[id] = nullptr;
  c->cap[id] = 0;
  c->host_buf[id] = false;
}

// Append the bytes of a plain value to a graph key.
template <typename T>
void key_add(std::vector<unsigned char>& key, const T& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
  key.insert(key.end(), p, p + sizeof(T));
}

// Run `enqueue` (kernel launches on c->st only, no allocation, no host copy, no
// synchronisation) directly, or through a CUDA graph: a key seen for the first time
// runs directly; when the next call repeats it, that call is captured (so a shape
// used once never pays for a capture), and later calls with the key replay the
// graph.  The capture runs on a private non-blocking stream (the legacy default
// stream cannot be captured), ordered with c->st by events; a replay costs one
// graph launch instead of one launch per kernel.
template <typename F>
void captured(ov_context* c, ov_context::SweepGraph& g, const std::vector<unsigned char>& key, F&& enqueue) {
  const bool can = c->opt.graphs && !(c->prof && c->prof->on) && c->inj_kind == OV_INJECT_NONE;
  if (!can || (!(g.exec && g.key == key) && g.seen != key)) {
    if (can) g.seen = key;
    enqueue();
    return;
  }
  if (!c->cap_st) {
    CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->cap_ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->cap_ev[1], cudaEventDisableTiming));
  }
  if (!(g.exec && g.key == key)) {
    if (g.exec) {
      CK(cudaGraphExecDestroy(g.exec));
      g.exec = nullptr;
    }
    cudaStream_t user = c->st;
    const int64_t l0 = c->launches;
    CK(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
    c->st = c->cap_st;
    cudaGraph_t graph = nullptr;
    try {
      enqueue();
    } catch (...) {
      c->st = user;
      cudaStreamEndCapture(c->cap_st, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    c->st = user;
    CK(cudaStreamEndCapture(c->cap_st, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    g.key = key;
    g.nlaunch = c->launches - l0;
    c->launches = l0;
  }
  CK(cudaEventRecord(c->cap_ev[0], c->st));
  CK(cudaStreamWaitEvent(c->cap_st, c->cap_ev[0], 0));
  CK(cudaGraphLaunch(g.exec, c->cap_st));
  CK(cudaEventRecord(c->cap_ev[1], c->cap_st));
  CK(cudaStreamWaitEvent(c->st, c->cap_ev[1], 0));
  c->launches += g.nlaunch;
}

void* ws(ov_context* c, int id, size_t bytes, bool zero = false) {
  if (bytes == 0) bytes = 16;
  const bool host = (id == B_BV || id == B_BW) && c->opt.basis_memory == 1;
  if (c->cap[id] < bytes || c->host_buf[id] != host) {
    if (c->inj_kind == OV_INJECT_OOM) {
      if (c->inj_step-- <= 0) {
        c->inj_kind = OV_INJECT_NONE;
        throw Status{OV_ERR_OOM};
      }
    }
    free_buf(c, id);
    size_t nb = (bytes + 255) & ~(size_t)255;
    if (host) {
      // pinned host memory mapped into the device's address space: the kernels reach it
      // through its device alias; it is cleared on the host before the device sees it
      void* hp = nullptr;
      void* dp = nullptr;
      if (cudaHostAlloc(&hp, nb, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        throw Status{OV_ERR_OOM};
      }
      std::memset(hp, 0, nb);
      if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess || dp != hp) {
        // the library relies on one address for host and device (unified addressing)
        cudaGetLastError();
        cudaFreeHost(hp);
        throw Status{OV_ERR_CUDA};
      }
      c->buf[id] = hp;
      c->cap[id] = nb;
      c->host_buf[id] = true;
      return hp;
    }
    cudaError_t e = cudaMalloc(&c->buf[id], nb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Status{OV_ERR_OOM};
    }
    c->cap[id] = nb;
    // The whole capacity starts at zero, not only the bytes asked for now: ticket
    // counters rely on it when a later call (more sources) uses more of the buffer
    // without reallocating it.
    CK(cudaMemsetAsync(c->buf[id], 0, nb, c->st));
    return c->buf[id];
  }
  if (zero) CK(cudaMemsetAsync(c->buf[id], 0, bytes, c->st));
  return c->buf[id];
}

template <typename T> T* wsT(ov_context* c, int id, int64_t n, bool zero = false) {
  return static_cast<T*>(ws(c, id, (size_t)n * sizeof(T), zero));
}

void check_ptr(const void* p) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) throw Status{OV_ERR_INVALID_ARG};
}

Geom make_geom(const int32_t dims[4]) {
  if (!dims) throw Status{OV_ERR_INVALID_ARG};
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 1 || dims[i] > 4096) throw Status{OV_ERR_INVALID_ARG};
  Geom g;
  g.nx = dims[0]; g.ny = dims[1]; g.nz = dims[2]; g.nt = dims[3];
  g.V = (int64_t)g.nx * g.ny * g.nz * g.nt;
  if (g.V > (int64_t)1 << 28) throw Status{OV_ERR_INVALID_ARG};
  return g;
}

// fm = 2 sets up block mode: fields of 2V sites (upper and lower halves)
template <typename R>
Lat<R> setup(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc, int k,
             bool basis, int fm = 1, int kcap = 0) {
  Lat<R> L{};
  L.g = make_geom(dims);
  L.gl = L.g;
  if (nsrc < 1 || nsrc > 4096) throw Status{OV_ERR_INVALID_ARG};
  if (!(std::isfinite(mu) && std::isfinite(m_w)) || 2.0 * m_w + 8.0 == 0.0) throw Status{OV_ERR_INVALID_ARG};
  check_ptr(U);
  const int64_t V = L.g.V;
  L.kappa = (R)(1.0 / (2.0 * m_w + 8.0));
  L.ef = (R)std::exp(mu);
  L.efinv = (R)std::exp(-mu);
  L.nsrc = nsrc;
  L.k = k;
  L.vs = ((24 * V + 63) / 64) * 64;
  R* u = wsT<R>(c, B_LINKS, link_reals<R>() * V);
  L.u = u;
  run(c, OV_KIND_LAYOUT, 1, [&] { pack_links<R>(static_cast<const double*>(U), u, V, c->st); });
  launch_check();
  if (fm == 2) {
    L.block = 1;
    L.g.V = 2 * V;
    L.vs = ((48 * V + 63) / 64) * 64;
  }
  const int64_t Vf = L.g.V;
  L.kcap = kcap > 0 ? kcap : k;
  L.jbase = 0;
  if (basis) {
    L.bv = wsT<R>(c, B_BV, (int64_t)nsrc * L.kcap * L.vs);
    L.bw = wsT<R>(c, B_BW, (int64_t)nsrc * L.kcap * L.vs);
  }
  L.p = wsT<R>(c, B_P, nsrc * L.vs);
  L.q = wsT<R>(c, B_Q, nsrc * L.vs);
  L.r = wsT<R>(c, B_R, nsrc * L.vs);
  L.s = wsT<R>(c, B_S, nsrc * L.vs);
  L.sc = wsT<SrcScal>(c, B_SC, nsrc);
  L.alpha = wsT<zd>(c, B_ALPHA, (int64_t)nsrc * k);
  L.beta = wsT<zd>(c, B_BETA, (int64_t)nsrc * k);
  L.delta = wsT<double>(c, B_DELTA, (int64_t)nsrc * k);
  // room for up to 8 partial values per block of the site kernels (blocks of 32
  // threads on small lattices)
  const int64_t nblk = (Vf + 31) / 32;
  L.part_stride = 8 * (nblk < 64 ? 64 : nblk);
  L.part = wsT<zd>(c, B_PART, nsrc * L.part_stride);
  L.cnt = wsT<unsigned>(c, B_CNT, (int64_t)nsrc * 16);
  return L;
}

std::vector<SrcScal> read_scalars(ov_context* c, const SrcScal* d, int nsrc) {
  std::vector<SrcScal> h(nsrc);
  CK(cudaMemcpyAsync(h.data(), d, sizeof(SrcScal) * nsrc, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return h;
}

int scalar_status(const std::vector<SrcScal>& h, int* k_reached, int k) {
  int st = OV_OK, kr = k;
  for (const auto& s : h) {
    if (s.err) {
      if (s.err_step >= 0 && s.err_step < kr) kr = s.err_step;
      if (s.err & ERRB_BREAKDOWN) st = OV_ERR_BREAKDOWN;
      else if (st == OV_OK) st = OV_ERR_NONFINITE;
    }
  }
  if (k_reached) *k_reached = kr;
  return st;
}

// Host-side fault injection (ov_debug_inject): after the stencil of step j, a NaN
// in alpha_j of source 0; after the update of step j, source 0 flagged as broken
// down exactly as the update kernel flags it.  Plain copies of ordinary values.
template <typename R>
void inject_after_stencil(ov_context* c, const Lat<R>& L, int j) {
  if (c->inj_kind != OV_INJECT_NONFINITE || c->inj_step != j) return;
  c->inj_kind = OV_INJECT_NONE;
  c->inj_nan[0] = c->inj_nan[1] = std::nan("");
  CK(cudaMemcpyAsync(L.alpha + j, c->inj_nan, sizeof(zd), cudaMemcpyHostToDevice, c->st));
}
template <typename R>
void inject_after_update(ov_context* c, const Lat<R>& L, int j) {
  if (c->inj_kind != OV_INJECT_BREAKDOWN || c->inj_step != j) return;
  c->inj_kind = OV_INJECT_NONE;
  c->inj_word[0] = ERRB_BREAKDOWN;
  c->inj_word[1] = j + 1;
  CK(cudaMemcpyAsync(&L.sc[0].err, c->inj_word, 2 * sizeof(int), cudaMemcpyHostToDevice, c->st));
}

// Forward Krylov recurrence for all sources; bases, coefficients stay on device.
template <typename R>
void forward_krylov(ov_context* c, Lat<R>& L) {
  const int k = L.k;
  const int64_t nsb = (L.g.V + 127) / 128;
  zd* coef = wsT<zd>(c, B_COEF, (int64_t)L.nsrc * 2 * k);
  zd* cpart = wsT<zd>(c, B_CPART, (int64_t)L.nsrc * 2 * k * nsb);
  std::vector<unsigned char> key;
  key_add(key, L);
  key_add(key, coef);
  key_add(key, cpart);
  key_add(key, c->opt);
  key_add(key, c->tuned_pair[c->opt.precision]);
  captured(c, c->gfwd, key, [&] {
    run(c, OV_KIND_UPDATE, 1, [&] { tsl_init(L, c->st); });
    for (int j = 0; j < k; ++j) {
      run(c, OV_KIND_STENCIL_PAIR, 1,
          [&] { tsl_stencil(L, j, j < k - 1, c->st, c->tuned_pair[c->opt.precision]); });
      inject_after_stencil(c, L, j);
      if (j == k - 1) break;
      const int reb = rebiorth_at(j + 1, c->opt.rebiorth);
      run(c, OV_KIND_UPDATE, 1, [&] { tsl_update(L, j, !reb, c->st); });
      if (reb) {
        for (int ps = 0; ps < c->opt.passes; ++ps) {
          run(c, OV_KIND_PROJ_DOTS, 2, [&] { proj_dots(L, j, 0, L.r, L.s, L.vs, coef, cpart, c->st); });
          run(c, OV_KIND_PROJ_UPDATE, 1,
              [&] { proj_update(L, j, 0, L.r, L.s, L.vs, coef, ps == c->opt.passes - 1, c->st, ps > 0); });
        }
      }
      inject_after_update(c, L, j);
    }
    launch_check();
  });
}

// Run diagnostics (options.diagnostics) after a forward recurrence whose
// coefficients are all valid: the sampled loss of biorthogonality of the stored
// bases (dots of the last basis pair with every basis vector; not with
// segments) and the Ritz values of each source's T_k on the host.  Returns
// OV_ERR_SIGN_ILLPOSED when a Ritz value lies within 1e-14 ||T_k||_inf of the
// imaginary axis (where sgn is undefined), OV_ERR_NOCONV when the eigenvalue
// iteration fails, else OV_OK.
template <typename R>
int run_diagnostics(ov_context* c, const Lat<R>& L, bool segments, ov_tsl_info* info) {
  const int k = L.k, nsrc = L.nsrc;
  double loss = -1.0;
  if (!segments) {
    const int64_t nsb = (L.g.V + 127) / 128;
    zd* coef = wsT<zd>(c, B_COEF, (int64_t)nsrc * 2 * k);
    zd* cpart = wsT<zd>(c, B_CPART, (int64_t)nsrc * 2 * k * nsb);
    run(c, OV_KIND_PROJ_DOTS, 2, [&] {
      proj_dots(L, k - 1, 0, L.basis_v(0, k - 1), L.basis_w(0, k - 1), (int64_t)L.kcap * L.vs, coef, cpart,
                c->st);
    });
    launch_check();
    std::vector<zd> h((size_t)nsrc * 2 * k);
    CK(cudaMemcpyAsync(h.data(), coef, sizeof(zd) * h.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    loss = 0.0;
    for (int src = 0; src < nsrc; ++src)
      for (int i = 0; i < k; ++i)
        for (int side = 0; side < 2; ++side) {
          zd z = h[(size_t)src * 2 * k + 2 * i + side];
          if (i == k - 1) z.re -= 1.0;
          const double a = std::sqrt(z.re * z.re + z.im * z.im);
          loss = std::isfinite(a) ? std::max(loss, a) : INFINITY;
        }
  }
  std::vector<double> a(2 * (size_t)nsrc * k), b(2 * (size_t)nsrc * k), d((size_t)nsrc * k), e(2 * (size_t)k);
  CK(cudaMemcpyAsync(a.data(), L.alpha, sizeof(double) * a.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(b.data(), L.beta, sizeof(double) * b.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(d.data(), L.delta, sizeof(double) * d.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double min_re = INFINITY, tnorm = 0.0;
  int st = OV_OK;
  for (int src = 0; src < nsrc; ++src) {
    const double* as = a.data() + (size_t)src * 2 * k;
    const double* bs = b.data() + (size_t)src * 2 * k;
    const double* ds = d.data() + (size_t)src * k;
    double nrm = 0.0;   // infinity norm: largest absolute row sum
    for (int j = 0; j < k; ++j) {
      double row = std::hypot(as[2 * j], as[2 * j + 1]);
      if (j > 0) row += ds[j];
      if (j + 1 < k) row += std::hypot(bs[2 * (j + 1)], bs[2 * (j + 1) + 1]);
      nrm = std::max(nrm, row);
    }
    const int es = ov_tridiag_eigenvalues(k, as, bs, ds, e.data());
    if (es != OV_OK) {
      st = es;
      continue;
    }
    double m = INFINITY;
    for (int j = 0; j < k; ++j) m = std::min(m, std::fabs(e[2 * j]));
    min_re = std::min(min_re, m);
    tnorm = std::max(tnorm, nrm);
    if (m <= 1e-14 * nrm && st == OV_OK) st = OV_ERR_SIGN_ILLPOSED;
  }
  if (info) {
    info->biorth_loss = loss;
    info->min_abs_re_ritz = min_re;
    info->t_norm = tnorm;
  }
  return st;
}

// ---------------------------------------------------------------------------
// Two-pass TSL with segment replay (options.segment = S > 0, no
// re-biorthogonalisation).  Segments are aligned to the top: [k - S, k),
// [k - 2S, k - S), ..., the lowest one possibly shorter.  The basis window holds
// v_{j0-1} .. v_{j1} of the current segment [j0, j1).  At every segment start
// the recurrence state (r, s, v_{j0-1}, w_{j0-1} and the per-source scalars) is
// checkpointed; replaying a segment from its checkpoint runs the same kernels
// on the same data, so it reproduces its vectors and coefficients bit for bit.
// ---------------------------------------------------------------------------
struct SegPlan {
  int S = 0;
  std::vector<int> lo, hi;   // ascending segments [lo[t], hi[t])
};
SegPlan seg_plan(int k, int S) {
  SegPlan p;
  p.S = S;
  std::vector<int> b;
  for (int x = k; x > 0; x -= S) b.push_back(x);
  b.push_back(0);
  for (int t = (int)b.size() - 1; t > 0; --t) {
    p.lo.push_back(b[t]);
    p.hi.push_back(b[t - 1]);
  }
  return p;
}

template <typename R>
struct SegStore {
  R *r, *s, *v, *w;   // [segment][src][vs]
  SrcScal* sc;        // [segment][src]
};
template <typename R>
SegStore<R> seg_store(ov_context* c, const Lat<R>& L, int nseg) {
  const int64_t n = (int64_t)nseg * L.nsrc * L.vs;
  return SegStore<R>{wsT<R>(c, B_CKR, n), wsT<R>(c, B_CKS, n), wsT<R>(c, B_CKV, n), wsT<R>(c, B_CKW, n),
                     wsT<SrcScal>(c, B_CKSC, (int64_t)nseg * L.nsrc)};
}
// copy the window's first vector (v_{jbase}, w_{jbase}) of every source to or from a checkpoint
template <typename R>
void window_slot(ov_context* c, const Lat<R>& L, int slot, R* v, R* w, bool to_window) {
  const size_t pitch = sizeof(R) * L.kcap * L.vs, width = sizeof(R) * L.vs;
  R* bv = L.bv + (int64_t)slot * L.vs;
  R* bw = L.bw + (int64_t)slot * L.vs;
  if (to_window) {
    CK(cudaMemcpy2DAsync(bv, pitch, v, width, width, L.nsrc, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpy2DAsync(bw, pitch, w, width, width, L.nsrc, cudaMemcpyDeviceToDevice, c->st));
  } else {
    CK(cudaMemcpy2DAsync(v, width, bv, pitch, width, L.nsrc, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpy2DAsync(w, width, bw, pitch, width, L.nsrc, cudaMemcpyDeviceToDevice, c->st));
  }
}
// steps j0 .. j1-1 without re-biorthogonalisation; with `next`, also the stencil of
// step j1, which writes v_{j1} and w_{j1} into the window
template <typename R>
void seg_steps(ov_context* c, Lat<R>& L, int j0, int j1, bool next) {
  const int k = L.k;
  const int jend = next ? j1 + 1 : j1;
  for (int j = j0; j < jend; ++j) {
    run(c, OV_KIND_STENCIL_PAIR, 1, [&] { tsl_stencil(L, j, j < k - 1, c->st, c->tuned_pair[c->opt.precision]); });
    inject_after_stencil(c, L, j);
    if (j == k - 1 || j == j1) break;
    run(c, OV_KIND_UPDATE, 1, [&] { tsl_update(L, j, true, c->st); });
    inject_after_update(c, L, j);
  }
}
// pass 1: the recurrence over all segments, checkpointing each segment start
template <typename R>
void seg_forward(ov_context* c, Lat<R>& L, const SegPlan& P, const SegStore<R>& K) {
  const int64_t fs = (int64_t)L.nsrc * L.vs;
  run(c, OV_KIND_UPDATE, 1, [&] { tsl_init(L, c->st); });
  for (size_t t = 0; t < P.lo.size(); ++t) {
    const int j0 = P.lo[t];
    if (t > 0) {
      // v_{j0-1} moves from the end of the previous window to its first slot
      window_slot(c, L, j0 - L.jbase - 1, K.v + (int64_t)t * fs, K.w + (int64_t)t * fs, false);
      L.jbase = j0 - 1;
      window_slot(c, L, 0, K.v + (int64_t)t * fs, K.w + (int64_t)t * fs, true);
    } else {
      L.jbase = j0 - 1;
    }
    CK(cudaMemcpyAsync(K.r + t * fs, L.r, sizeof(R) * fs, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(K.s + t * fs, L.s, sizeof(R) * fs, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(K.sc + t * L.nsrc, L.sc, sizeof(SrcScal) * L.nsrc, cudaMemcpyDeviceToDevice, c->st));
    seg_steps(c, L, j0, P.hi[t], false);
  }
  launch_check();
}
// replay segment t from its checkpoint (with `next`: also v_{j1}, w_{j1})
template <typename R>
void seg_replay(ov_context* c, Lat<R>& L, const SegPlan& P, const SegStore<R>& K, int t, bool next) {
  const int64_t fs = (int64_t)L.nsrc * L.vs;
  const int j0 = P.lo[t];
  L.jbase = j0 - 1;
  if (t > 0) window_slot(c, L, 0, K.v + (int64_t)t * fs, K.w + (int64_t)t * fs, true);
  CK(cudaMemcpyAsync(L.r, K.r + t * fs, sizeof(R) * fs, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(L.s, K.s + t * fs, sizeof(R) * fs, cudaMemcpyDeviceToDevice, c->st));
  // only the forward scalars: the reverse sweep keeps its own in the same structs
  CK(cudaMemcpy2DAsync(L.sc, sizeof(SrcScal), K.sc + t * L.nsrc, sizeof(SrcScal), offsetof(SrcScal, g_alpha),
                       L.nsrc, cudaMemcpyDeviceToDevice, c->st));
  seg_steps(c, L, j0, P.hi[t], next && P.hi[t] < L.k);
  launch_check();
}

// Scaled Newton iteration for sgn (mirrors the oracle's stopping rules).
// a[0] holds the start matrix; a[1] is scratch.  Block form: when e != nullptr
// the iteration runs on [[A, E], [0, A]] (e[0] holds E) and E converges to the
// upper-right block.  Returns the iteration count (or -1 on a non-finite step)
// and the index of the buffer holding the result in *which.
struct NewtonRecord {
  zd* inv = nullptr;        // NREC slots of k x k inverses
  double* logdet = nullptr; // NREC log|det| values
  std::vector<int> scaling; // scaling flag of each recorded iteration
  int cap = 0;
  bool ok = true;           // false when the iteration outgrew the record
};
constexpr int NREC = 48;

// status of the k x k stage from its device error word: a device-side wait that
// ran past its limit, an ill-posed sign (singular or non-finite), or success
int sign_status(ov_context* c, const int* derr) {
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return (herr & ERRB_TIMEOUT) ? OV_ERR_TIMEOUT : herr ? OV_ERR_SIGN_ILLPOSED : OV_OK;
}
int sign_failed(ov_context* c, const int* derr) {
  return sign_status(c, derr) == OV_ERR_TIMEOUT ? OV_ERR_TIMEOUT : OV_ERR_SIGN_ILLPOSED;
}

int newton(ov_context* c, zd* a[2], zd* e[2], int k, int* err_dev, int* which, NewtonRecord* rec = nullptr) {
  const int64_t n = (int64_t)k * k;
  zd* ai = wsT<zd>(c, B_XI, n);
  zd* t1 = e ? wsT<zd>(c, B_TMP1, n) : nullptr;
  zd* t2 = e ? wsT<zd>(c, B_TMP2, n) : nullptr;
  int* ipiv = wsT<int>(c, B_IPIV, k);
  int* used = wsT<int>(c, B_COL, k);
  unsigned long long* keys = wsT<unsigned long long>(c, B_PROW, (int64_t)(k + 1) * GJ_KEY_SLOTS);
  zd* w0 = wsT<zd>(c, B_W0, n);
  zd* w1 = wsT<zd>(c, B_W1, n);
  double* dstat = wsT<double>(c, B_DSTAT, 4);   // [0] diff^2, [1] norm^2, [2] log|det| (or its norm form)
  zd* dpart = wsT<zd>(c, B_DPART, (n + 255) / 256 + 64);
  unsigned* dcnt = wsT<unsigned>(c, B_DCNT, 4);
  zd* npart = wsT<zd>(c, B_NSPART, 64);
  unsigned* ncnt = wsT<unsigned>(c, B_NSCNT, 1);
  const bool norm_rules = c->opt.newton == 0;
  bool scaling = true, last = false;
  double prev = INFINITY;
  int cur = 0, it = 0;
  double hs[3];
  for (it = 1; it <= 100; ++it) {
    CK(cudaMemsetAsync(dstat, 0, 3 * sizeof(double), c->st));
    run(c, OV_KIND_DENSE, 0, [&] {
      // log|det| only where the determinant scaling uses it
      c->launches += dense_inverse(a[cur], ai, w0, w1, k, 1, nullptr, ipiv, used, keys,
                                   !norm_rules && scaling ? dstat + 2 : nullptr, 0, err_dev, c->opt.dense, c->st);
    });
    if (norm_rules && scaling)
      run(c, OV_KIND_DENSE, 1, [&] { dense_norm_scale(a[cur], ai, k, 1, nullptr, dstat + 2, 0, npart, ncnt, c->st); });
    if (rec) {
      const int slot = it - 1;
      if (slot < rec->cap) {
        run(c, OV_KIND_DENSE, 1, [&] { dense_copy(ai, rec->inv + (int64_t)slot * n, n, c->st); });
        CK(cudaMemcpyAsync(rec->logdet + slot, dstat + 2, sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        rec->scaling.push_back(scaling ? 1 : 0);
      } else {
        rec->ok = false;
      }
    }
    if (e) {
      kk_gemm(c, ai, 0, 0, e[cur], 0, 0, t1, 0, k, 1, nullptr, nullptr);
      kk_gemm(c, t1, 0, 0, ai, 0, 0, t2, 0, k, 1, nullptr, nullptr);
    }
    // the block determinant is det(A)^2: its 1/(2k)-th root is det(A)^(1/k)
    run(c, OV_KIND_DENSE, e ? 2 : 1, [&] {
      dense_newton_combine(a[cur], ai, a[1 - cur], k, dstat + 2, scaling ? 1 : 0, 1.0, e ? 2.0 : 1.0, dstat,
                           dpart, dcnt, c->st);
      if (e)
        dense_newton_combine(e[cur], t2, e[1 - cur], k, dstat + 2, scaling ? 1 : 0, -1.0, 1.0, dstat, dpart,
                             dcnt, c->st);
    });
    launch_check();
    CK(cudaMemcpyAsync(hs, dstat, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    cur = 1 - cur;
    const double step = std::sqrt(hs[0] / hs[1]);
    if (!std::isfinite(step)) return -1;
    if (last || step <= 1e-14) break;
    const bool was_unscaled = !scaling;
    if (step < 1e-2) scaling = false;
    if (norm_rules && was_unscaled && step * step * step / (prev * prev) <= 1e-12) last = true;
    if (it > 6 && !scaling && step >= 0.5 * prev) break;
    prev = step;
  }
  *which = cur;
  return it > 100 ? 100 : it;
}

// The same scaled Newton iteration for nb problems at once (matrices at stride
// k*k in a[0] and a[1]).  Each problem follows the stopping rules above on its
// own and is switched off when it stops; its result is then in a[which[p]].
// With rec_inv, the inverse and log|det| of every iteration of problem p are
// recorded in slot i of rec_inv + p*cap*k*k and rec_ld + p*cap (scalings and
// overflow in scaling / rec_ok).  Returns the largest iteration count, or -1.
int newton_batch(ov_context* c, zd* a[2], int k, int nb, int* err_dev, std::vector<int>& which,
                 std::vector<int>& iters, zd* rec_inv = nullptr, double* rec_ld = nullptr, int cap = 0,
                 std::vector<std::vector<int>>* scaling_rec = nullptr, std::vector<char>* rec_ok = nullptr) {
  const int64_t n = (int64_t)k * k;
  const int64_t pstride = (n + 255) / 256 + 64;
  zd* ai = wsT<zd>(c, B_XI, nb * n);
  zd* w0 = wsT<zd>(c, B_W0, nb * n);
  zd* w1 = wsT<zd>(c, B_W1, nb * n);
  int* ipiv = wsT<int>(c, B_IPIV, (int64_t)nb * k);
  int* used = wsT<int>(c, B_COL, (int64_t)nb * k);
  unsigned long long* keys = wsT<unsigned long long>(c, B_PROW, (int64_t)nb * (k + 1) * GJ_KEY_SLOTS);
  double* dstat = wsT<double>(c, B_DSTAT, 4 * (int64_t)nb);
  zd* dpart = wsT<zd>(c, B_DPART, nb * pstride);
  unsigned* dcnt = wsT<unsigned>(c, B_DCNT, 4 * (int64_t)nb);
  int* act_dev = wsT<int>(c, B_ACT, nb);
  int* scal_dev = wsT<int>(c, B_SCAL, nb);
  zd* npart = wsT<zd>(c, B_NSPART, 64 * (int64_t)nb);
  unsigned* ncnt = wsT<unsigned>(c, B_NSCNT, nb);
  const bool norm_rules = c->opt.newton == 0;
  std::vector<int> act(nb, 1), scaling(nb, 1), last(nb, 0);
  std::vector<double> prev(nb, INFINITY), hs(4 * (size_t)nb);
  which.assign(nb, 0);
  iters.assign(nb, 0);
  if (scaling_rec) scaling_rec->assign(nb, {});
  if (rec_ok) rec_ok->assign(nb, 1);
  int cur = 0, itmax = 0;
  for (int it = 1; it <= 100; ++it) {
    if (std::find(act.begin(), act.end(), 1) == act.end()) break;
    CK(cudaMemcpyAsync(act_dev, act.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(scal_dev, scaling.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(dstat, 0, sizeof(double) * 4 * nb, c->st));
    run(c, OV_KIND_DENSE, 0, [&] {
      // log|det| only where the determinant scaling uses it
      const bool want_ld = !norm_rules && std::find(scaling.begin(), scaling.end(), 1) != scaling.end();
      c->launches += dense_inverse(a[cur], ai, w0, w1, k, nb, act_dev, ipiv, used, keys,
                                   want_ld ? dstat + 2 : nullptr, 4, err_dev, c->opt.dense, c->st);
    });
    if (norm_rules && std::find(scaling.begin(), scaling.end(), 1) != scaling.end())
      run(c, OV_KIND_DENSE, 1, [&] { dense_norm_scale(a[cur], ai, k, nb, act_dev, dstat + 2, 4, npart, ncnt, c->st); });
    if (rec_inv) {
      const int slot = it - 1;
      for (int p = 0; p < nb; ++p) {
        if (!act[p]) continue;
        if (slot < cap) {
          (*scaling_rec)[p].push_back(scaling[p]);
          CK(cudaMemcpyAsync(rec_ld + (int64_t)p * cap + slot, dstat + 4 * p + 2, sizeof(double),
                             cudaMemcpyDeviceToDevice, c->st));
        } else {
          (*rec_ok)[p] = 0;
        }
      }
      if (slot < cap)
        run(c, OV_KIND_DENSE, 1,
            [&] { dense_copy_batch(ai, n, rec_inv + (int64_t)slot * n, (int64_t)cap * n, n, nb, act_dev, c->st); });
    }
    run(c, OV_KIND_DENSE, 1, [&] {
      dense_newton_combine_batch(a[cur], ai, a[1 - cur], k, nb, act_dev, dstat + 2, 4, scal_dev, 1, 1.0, 1.0, dstat,
                                 dpart, pstride, dcnt, c->st);
    });
    launch_check();
    CK(cudaMemcpyAsync(hs.data(), dstat, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    cur = 1 - cur;
    for (int p = 0; p < nb; ++p) {
      if (!act[p]) continue;
      const double step = std::sqrt(hs[4 * p] / hs[4 * p + 1]);
      iters[p] = it;
      which[p] = cur;
      itmax = std::max(itmax, it);
      if (!std::isfinite(step)) return -1;
      if (last[p] || step <= 1e-14) {
        act[p] = 0;
        continue;
      }
      const bool was_unscaled = !scaling[p];
      if (step < 1e-2) scaling[p] = 0;
      if (norm_rules && was_unscaled && step * step * step / (prev[p] * prev[p]) <= 1e-12) last[p] = 1;
      if (it > 6 && !scaling[p] && step >= 0.5 * prev[p]) {
        act[p] = 0;
        continue;
      }
      prev[p] = step;
    }
  }
  return itmax;
}

// y_p = beta0_p Q_p sgn(H_p) e_1 for nb tridiagonals T_p (alpha, beta, delta at
// stride k): the nested Krylov sign with inner size m_in (Sec. 4.1,
// one nesting level; nested.cu).  The Hessenberg matrices go through the same
// scaled Newton iteration as the full k x k sign, all problems in one batch when
// their inner spaces have the same size.
int nested_sign(ov_context* c, int m_in, const zd* alpha, const zd* beta, const double* delta, int k, int nb,
                const std::vector<double>& beta0, zd* y, int* iters) {
  const int m = std::min(m_in, k);
  const int64_t mm = (int64_t)m * m;
  NestWs W{wsT<zd>(c, B_NLU, (int64_t)nb * 4 * k), wsT<int>(c, B_NPIV, (int64_t)nb * k),
           wsT<zd>(c, B_NS, (int64_t)nb * k * k),  wsT<zd>(c, B_NQ, (int64_t)nb * m * k),
           wsT<zd>(c, B_NW, (int64_t)nb * k),      wsT<zd>(c, B_NH, nb * mm),
           wsT<int>(c, B_NMEFF, nb),               wsT<zd>(c, B_NHB, (int64_t)nb * m),
           wsT<double>(c, B_NWN, nb)};
  int* derr = wsT<int>(c, B_DERR, 1, true);
  // the set-up and the m Arnoldi steps (~6 m launches) replay as one graph when the shape repeats
  std::vector<unsigned char> key;
  key_add(key, k);
  key_add(key, nb);
  key_add(key, m);
  for (const void* ptr : {(const void*)alpha, (const void*)beta, (const void*)delta, (const void*)W.lu,
                          (const void*)W.piv, (const void*)W.s, (const void*)W.q, (const void*)W.w, (const void*)W.h,
                          (const void*)W.meff, (const void*)W.hb, (const void*)W.wn, (const void*)derr})
    key_add(key, ptr);
  captured(c, c->gnest, key, [&] {
    run(c, OV_KIND_DENSE, 0, [&] { c->launches += nested_prepare(alpha, beta, delta, k, nb, m, W, derr, c->st); });
    run(c, OV_KIND_DENSE, 0, [&] { c->launches += nested_arnoldi(k, nb, m, W, derr, c->st); });
  });
  launch_check();
  std::vector<int> meff(nb);
  CK(cudaMemcpyAsync(meff.data(), W.meff, sizeof(int) * nb, cudaMemcpyDeviceToHost, c->st));
  {
    const int ss = sign_status(c, derr);
    if (ss != OV_OK) return ss;
  }
  // The Hessenberg matrices' inversions in the step form (one launch per elimination
  // column, graph-replayed): at m = 60 .. 150 it is faster than the cooperative form,
  // whose per-step inter-block handshake dominates at these sizes (k = 800: 6.7 / 10.3 /
  // 14.9 ms per stage against 8.1 / 14.4 / 20.5 at m = 60 / 100 / 150); both forms give
  // the same bits.
  struct DenseForm {
    ov_context* c;
    int saved;
    ~DenseForm() { c->opt.dense = saved; }
  } form{c, c->opt.dense};
  c->opt.dense = GJ_STEPS;
  int itmax = 0;
  if (m >= 2 && std::all_of(meff.begin(), meff.end(), [&](int v) { return v == m; })) {
    zd* a[2] = {W.h, wsT<zd>(c, B_NHN, nb * mm)};
    std::vector<int> which, its;
    itmax = newton_batch(c, a, m, nb, derr, which, its);
    if (itmax < 0) return sign_failed(c, derr);
    for (int p = 0; p < nb; ++p)
      run(c, OV_KIND_DENSE, 1, [&] {
        nested_combine(W.q + (int64_t)p * m * k, a[which[p]] + p * mm, m, k, m, beta0[p], y + (int64_t)p * k, c->st);
      });
  } else {
    // a closed inner space: each problem on its own m_eff x m_eff leading block
    for (int p = 0; p < nb; ++p) {
      const int me = meff[p];
      zd* a[2] = {wsT<zd>(c, B_NHC, (int64_t)me * me), wsT<zd>(c, B_NHCN, (int64_t)me * me)};
      if (me == 1) {
        // a 1 x 1 Hessenberg matrix: sgn(h) = sgn(Re h), on the host
        zd h{};
        CK(cudaMemcpyAsync(&h, W.h + p * mm, sizeof(zd), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (!std::isfinite(h.re) || !std::isfinite(h.im) || h.re == 0.0) return OV_ERR_SIGN_ILLPOSED;
        const zd f{h.re > 0.0 ? 1.0 : -1.0, 0.0};
        CK(cudaMemcpyAsync(a[0], &f, sizeof(zd), cudaMemcpyHostToDevice, c->st));
        run(c, OV_KIND_DENSE, 1,
            [&] { nested_combine(W.q + (int64_t)p * m * k, a[0], 1, k, 1, beta0[p], y + (int64_t)p * k, c->st); });
        CK(cudaStreamSynchronize(c->st));   // f lives on this stack frame
        itmax = std::max(itmax, 1);
        continue;
      }
      CK(cudaMemcpy2DAsync(a[0], sizeof(zd) * me, W.h + p * mm, sizeof(zd) * m, sizeof(zd) * me, me,
                           cudaMemcpyDeviceToDevice, c->st));
      std::vector<int> which, its;
      const int it = newton_batch(c, a, me, 1, derr, which, its);
      if (it < 0) return sign_failed(c, derr);
      itmax = std::max(itmax, it);
      run(c, OV_KIND_DENSE, 1, [&] {
        nested_combine(W.q + (int64_t)p * m * k, a[which[0]], me, k, me, beta0[p], y + (int64_t)p * k, c->st);
      });
    }
  }
  launch_check();
  {
    const int ss = sign_status(c, derr);
    if (ss != OV_OK) return ss;
  }
  if (iters) *iters = itmax;
  return OV_OK;
}

// y_p = beta0_p sgn(T_p) e_1 for nb tridiagonals (alpha, beta, delta at stride k):
// the full k x k sign by the scaled Newton iteration, all problems in one batch
int full_sign(ov_context* c, const zd* alpha, const zd* beta, const double* delta, int k, int nb,
              const std::vector<double>& beta0, zd* y, int* iters) {
  const int64_t n = (int64_t)k * k;
  int* derr = wsT<int>(c, B_DERR, 1, true);
  zd* a[2] = {wsT<zd>(c, B_X, nb * n), wsT<zd>(c, B_XN, nb * n)};
  for (int p = 0; p < nb; ++p)
    run(c, OV_KIND_DENSE, 2, [&] {
      dense_build_t(alpha + (int64_t)p * k, beta + (int64_t)p * k, delta + (int64_t)p * k, k, a[0] + p * n, c->st);
    });
  std::vector<int> which, its;
  const int itmax = newton_batch(c, a, k, nb, derr, which, its);
  if (itmax < 0) return sign_failed(c, derr);
  for (int p = 0; p < nb; ++p)
    run(c, OV_KIND_DENSE, 1, [&] { dense_extract_y(a[which[p]] + p * n, beta0[p], k, y + (int64_t)p * k, c->st); });
  {
    const int ss = sign_status(c, derr);
    if (ss != OV_OK) return ss;
  }
  if (iters) *iters = itmax;
  return OV_OK;
}

// y_src = beta0 sgn(T_k) e_1 for every source (nested when options.nested > 0)
template <typename R>
int sign_all(ov_context* c, Lat<R>& L, const std::vector<SrcScal>& hsc, zd* y, int* iters) {
  std::vector<double> b0(L.nsrc);
  for (int src = 0; src < L.nsrc; ++src) b0[src] = hsc[src].beta0;
  if (c->opt.nested > 0) return nested_sign(c, c->opt.nested, L.alpha, L.beta, L.delta, L.k, L.nsrc, b0, y, iters);
  return full_sign(c, L.alpha, L.beta, L.delta, L.k, L.nsrc, b0, y, iters);
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

template <typename R>
int tsl_sign_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                  const void* b, int k, void* x, ov_tsl_info* info) {
  check_ptr(b);
  check_ptr(x);
  const int S = c->opt.segment > 0 && c->opt.segment < k ? c->opt.segment : 0;
  Lat<R> L = setup<R>(c, dims, U, mu, m_w, nsrc, k, true, 1, S > 0 ? S + 2 : 0);
  run(c, OV_KIND_LAYOUT, 2, [&] {
    pack_spinors<R>(static_cast<const double*>(b), L.r, nsrc, L.g.V, L.vs, c->st);
    pack_spinors<R>(static_cast<const double*>(b), L.s, nsrc, L.g.V, L.vs, c->st);
  });
  SegPlan P;
  SegStore<R> K{};
  CK(cudaEventRecord(c->ev[0], c->st));
  if (S > 0) {
    P = seg_plan(k, S);
    K = seg_store(c, L, (int)P.lo.size());
    seg_forward(c, L, P, K);
  } else {
    forward_krylov(c, L);
  }
  CK(cudaEventRecord(c->ev[1], c->st));
  auto hsc = read_scalars(c, L.sc, nsrc);
  int kr = k;
  int st = scalar_status(hsc, &kr, k);
  c->last_k = k;
  c->last_nsrc = nsrc;
  c->last_block = 0;
  c->last_seg = S > 0 ? 1 : 0;
  c->last_prec = c->opt.precision;
  std::copy(dims, dims + 4, c->last_dims);
  if (info) info->k_reached = kr;
  if (st != OV_OK) return st;
  if (c->opt.diagnostics) {
    st = run_diagnostics(c, L, S > 0, info);
    if (st != OV_OK) return st;
  }
  zd* y = wsT<zd>(c, B_Y, (int64_t)nsrc * k);
  int iters = 0;
  st = sign_all(c, L, hsc, y, &iters);
  if (st != OV_OK) return st;
  CK(cudaEventRecord(c->ev[2], c->st));
  if (S > 0) {
    // second pass: x = V_k y, one replayed segment at a time
    for (size_t t = 0; t < P.lo.size(); ++t) {
      seg_replay(c, L, P, K, (int)t, false);
      run(c, OV_KIND_COMBINE, 1, [&] {
        combine_range(L, P.lo[t], P.hi[t] - P.lo[t], y, static_cast<double*>(x), t > 0, c->st);
      });
    }
  } else {
    run(c, OV_KIND_COMBINE, 1, [&] { combine(L, k, y, static_cast<double*>(x), c->st); });
  }
  launch_check();
  CK(cudaEventRecord(c->ev[3], c->st));
  CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
  if (info) {
    info->newton_iters = iters;
    info->t_ms[0] = elapsed(c->ev[0], c->ev[1]);
    info->t_ms[1] = elapsed(c->ev[1], c->ev[2]);
    info->t_ms[2] = elapsed(c->ev[2], c->ev[3]);
  }
  return OV_OK;
}

// Theorem 1: TSL on B = [[H, dH], [0, H]] from (top, bottom) (top may be null:
// zero) with left start proportional to (top + bottom, bottom); writes the two
// halves of the result.
template <typename R>
int block_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
               const void* top, const void* bottom, int k, const void* E, double m_dir, void* out_top,
               void* out_bottom, ov_tsl_info* info) {
  check_ptr(bottom);
  check_ptr(out_top);
  check_ptr(out_bottom);
  if (top) check_ptr(top);
  if (E) check_ptr(E);
  if (!std::isfinite(m_dir) || c->opt.segment > 0) throw Status{OV_ERR_INVALID_ARG};
  Lat<R> L = setup<R>(c, dims, U, mu, m_w, nsrc, k, true, 2);
  const int64_t V = L.gl.V, Vf = L.g.V;
  if (E) {
    R* ue = wsT<R>(c, B_ELINKS, link_reals<R>() * V);
    run(c, OV_KIND_LAYOUT, 1, [&] { pack_links<R>(static_cast<const double*>(E), ue, V, c->st); });
    L.ue = ue;
  }
  L.mdir = (R)m_dir;
  run(c, OV_KIND_LAYOUT, 1, [&] {
    pack_block_start<R>(static_cast<const double*>(top), static_cast<const double*>(bottom), L.r, L.s, nsrc, V,
                        L.vs, c->st);
  });
  CK(cudaEventRecord(c->ev[0], c->st));
  forward_krylov(c, L);
  CK(cudaEventRecord(c->ev[1], c->st));
  auto hsc = read_scalars(c, L.sc, nsrc);
  int kr = k;
  int st = scalar_status(hsc, &kr, k);
  c->last_k = k;
  c->last_nsrc = nsrc;
  c->last_block = 1;
  c->last_seg = 0;
  c->last_prec = c->opt.precision;
  std::copy(dims, dims + 4, c->last_dims);
  if (info) info->k_reached = kr;
  if (st != OV_OK) return st;
  if (c->opt.diagnostics) {
    st = run_diagnostics(c, L, false, info);
    if (st != OV_OK) return st;
  }
  zd* y = wsT<zd>(c, B_Y, (int64_t)nsrc * k);
  int iters = 0;
  st = sign_all(c, L, hsc, y, &iters);
  if (st != OV_OK) return st;
  CK(cudaEventRecord(c->ev[2], c->st));
  double* out = wsT<double>(c, B_BLOCKOUT, (int64_t)nsrc * Vf * 24);
  run(c, OV_KIND_COMBINE, 1, [&] { combine(L, k, y, out, c->st); });
  launch_check();
  const size_t half = (size_t)V * 24 * sizeof(double);
  for (int src = 0; src < nsrc; ++src) {
    CK(cudaMemcpyAsync(static_cast<char*>(out_top) + src * half, out + (int64_t)src * Vf * 24, half,
                       cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(static_cast<char*>(out_bottom) + src * half, out + (int64_t)src * Vf * 24 + V * 24, half,
                       cudaMemcpyDeviceToDevice, c->st));
  }
  CK(cudaEventRecord(c->ev[3], c->st));
  CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
  if (info) {
    info->newton_iters = iters;
    info->t_ms[0] = elapsed(c->ev[0], c->ev[1]);
    info->t_ms[1] = elapsed(c->ev[1], c->ev[2]);
    info->t_ms[2] = elapsed(c->ev[2], c->ev[3]);
  }
  return OV_OK;
}

// A-posteriori estimates of Sec. 4.1: the sign applied twice, each time by its
// own k-step TSL, then ||sgn^2 b - b|| / (2 ||b||) per source (Eq. error_est),
// or for the block matrix from (0, b) (Eq. bA_error_est) when block is set.
void merge_info(ov_tsl_info* acc, const ov_tsl_info& one) {
  if (!acc) return;
  if (one.k_reached < acc->k_reached) acc->k_reached = one.k_reached;
  if (one.newton_iters > acc->newton_iters) acc->newton_iters = one.newton_iters;
  for (int i = 0; i < 8; ++i) acc->t_ms[i] += one.t_ms[i];
}

// Ritz triples of the last forward pass (eigen-triples for deflation, Sec. 3):
// eigenvalues theta of T_k on the host, the candidates smallest in |theta|, their
// right and left eigenvectors y, z of T_k (inverse iteration, z^dag y = 1), the Ritz
// vectors R = V_k y and L = W_k z on the device, and the true residual
// ||H R - theta R|| / ||R||; candidates at or below tol are returned in |theta| order.
template <typename R>
int ritz_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int src, int k, int lmax,
              double tol, int32_t* l_out, double* lam, void* Rv, void* Lv, double* resid) {
  check_ptr(Rv);
  check_ptr(Lv);
  Lat<R> L = setup<R>(c, dims, U, mu, m_w, c->last_nsrc, k, true);
  const int64_t V = L.g.V, n = 12 * V, fd = 24 * V;
  std::vector<double> al(2 * k), be(2 * k), de(k), th(2 * k);
  CK(cudaMemcpyAsync(al.data(), L.alpha + (int64_t)src * k, sizeof(zd) * k, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(be.data(), L.beta + (int64_t)src * k, sizeof(zd) * k, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(de.data(), L.delta + (int64_t)src * k, sizeof(double) * k, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  int st = ov_tridiag_eigenvalues(k, al.data(), be.data(), de.data(), th.data());
  if (st != OV_OK) return st;
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return std::hypot(th[2 * a], th[2 * a + 1]) < std::hypot(th[2 * b], th[2 * b + 1]);
  });
  // a Ritz pair is checked with H only when the bottom entry of its unit eigenvector,
  // times the largest subdiagonal of T_k, is at most 10 tol (the Lanczos residual of
  // (theta, V_k y) is delta_{k+1} |y_k| ||v_{k+1}||); at most 2 lmax + 8 such checks
  const int nchecks = 2 * lmax + 8;
  double dmax = 0.0;
  for (int j = 1; j < k; ++j) dmax = std::max(dmax, std::abs(de[j]));
  zd* yd = wsT<zd>(c, B_RZY, 2 * (int64_t)k);
  double* hf = wsT<double>(c, B_RZH, fd);      // H R
  zd* dd = wsT<zd>(c, B_RZD, 160);             // dots and their partials
  Lat<R> L1 = L;
  L1.nsrc = 1;
  std::vector<double> y(2 * k), z(2 * k);
  double* rout = static_cast<double*>(Rv);
  double* lout = static_cast<double*>(Lv);
  int got = 0, checks = 0;
  for (int ci = 0; ci < k && got < lmax && checks < nchecks; ++ci) {
    const int i = order[ci];
    const double t2[2] = {th[2 * i], th[2 * i + 1]};
    if (ov_tridiag_eigenvector(k, al.data(), be.data(), de.data(), t2, 0, y.data()) != OV_OK) continue;
    if (std::hypot(y[2 * (k - 1)], y[2 * (k - 1) + 1]) * dmax > 10.0 * tol) continue;
    ++checks;
    if (ov_tridiag_eigenvector(k, al.data(), be.data(), de.data(), t2, 1, z.data()) != OV_OK) continue;
    // z <- z / conj(z^dag y), so that z^dag y = 1
    double sr = 0.0, si = 0.0;
    for (int j = 0; j < k; ++j) {
      sr += z[2 * j] * y[2 * j] + z[2 * j + 1] * y[2 * j + 1];
      si += z[2 * j] * y[2 * j + 1] - z[2 * j + 1] * y[2 * j];
    }
    const double s2 = sr * sr + si * si;
    if (!(s2 > 1e-16)) continue;   // a nearly defective Ritz value: left and right nearly orthogonal
    for (int j = 0; j < k; ++j) {  // z / conj(s) = z s / |s|^2
      const double a = z[2 * j], b = z[2 * j + 1];
      z[2 * j] = (a * sr - b * si) / s2;
      z[2 * j + 1] = (a * si + b * sr) / s2;
    }
    double* ro = rout + (int64_t)got * fd;
    double* lo = lout + (int64_t)got * fd;
    CK(cudaMemcpyAsync(yd, y.data(), sizeof(zd) * k, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(yd + k, z.data(), sizeof(zd) * k, cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 2, [&] {
      ritz_combine(L, src, 0, k, yd, ro, c->st);
      ritz_combine(L, src, 1, k, yd + k, lo, c->st);
    });
    // residual: H R - theta R
    run(c, OV_KIND_LAYOUT, 1, [&] { pack_spinors<R>(ro, L.r, 1, V, L.vs, c->st); });
    run(c, OV_KIND_APPLY_H, 1, [&] { apply_h(L1, L.r, L.p, 0, c->st, 0, nullptr); });
    run(c, OV_KIND_LAYOUT, 1, [&] { unpack_spinors<R>(L.p, hf, 1, V, L.vs, c->st); });
    const zd mth = mk(-t2[0], -t2[1]);
    CK(cudaMemcpyAsync(dd, &mth, sizeof(zd), cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 3, [&] {
      vec_update(hf, ro, fd, 1, dd, 1.0, n, c->st);
      vec_dots(hf, fd, 1, hf, n, dd + 1, dd + 4, c->st);
      vec_dots(ro, fd, 1, ro, n, dd + 2, dd + 4, c->st);
    });
    launch_check();
    zd nrm[2];
    CK(cudaMemcpyAsync(nrm, dd + 1, 2 * sizeof(zd), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const double res = std::sqrt(nrm[0].re / nrm[1].re);
    if (!(res <= tol)) continue;
    lam[2 * got] = t2[0];
    lam[2 * got + 1] = t2[1];
    if (resid) resid[got] = res;
    ++got;
  }
  *l_out = got;
  return OV_OK;
}

// Deflation (Sec. 3): the projected start vector(s) from the caller's eigen-triples,
// the (block) TSL on them, and the exact part added back; every vector operation
// is a kernel on the user-layout fields (complex128).
template <typename R>
int deflated_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                  const void* b, int k, const void* E, double m_dir, bool block, int l, const double* lam,
                  const void* Rf, const void* Lf, const void* dRf, const void* dLf, void* dx, void* x,
                  ov_tsl_info* info) {
  check_ptr(b);
  check_ptr(x);
  if (block) check_ptr(dx);
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || dims[3] < 1 || nsrc < 1) throw Status{OV_ERR_INVALID_ARG};
  if (l > 0) {
    if (!lam) throw Status{OV_ERR_INVALID_ARG};
    check_ptr(Rf);
    check_ptr(Lf);
    if (block) {
      check_ptr(dRf);
      check_ptr(dLf);
    }
  }
  const int64_t V = (int64_t)dims[0] * dims[1] * dims[2] * dims[3];
  const int64_t n = 12 * V;          // complex entries per field
  const int64_t fd = 2 * n;          // doubles per field
  std::vector<double> sg(std::max(l, 1), 0.0);
  for (int i = 0; i < l; ++i) {
    if (!std::isfinite(lam[2 * i]) || !std::isfinite(lam[2 * i + 1])) throw Status{OV_ERR_INVALID_ARG};
    if (lam[2 * i] == 0.0) throw Status{OV_ERR_SIGN_ILLPOSED};
    sg[i] = lam[2 * i] > 0.0 ? 1.0 : -1.0;
  }
  const int lm = std::max(l, 1);
  zd* a = wsT<zd>(c, B_DFA, (int64_t)nsrc * lm);
  zd* cc = wsT<zd>(c, B_DFC, (int64_t)nsrc * lm);
  zd* sa = wsT<zd>(c, B_DFSA, (int64_t)nsrc * lm);
  zd* sc = wsT<zd>(c, B_DFSC, (int64_t)nsrc * lm);
  zd* part = wsT<zd>(c, B_DFPART, 152 * (int64_t)lm);
  double* sgd = wsT<double>(c, B_DFSG, lm);
  double* bot = wsT<double>(c, B_DFBOT, nsrc * fd);
  double* top = block ? wsT<double>(c, B_DFTOP, nsrc * fd) : nullptr;
  const double* bd = static_cast<const double*>(b);
  const double* rd = static_cast<const double*>(Rf);
  const double* ld = static_cast<const double*>(Lf);
  const double* drd = static_cast<const double*>(dRf);
  const double* dld = static_cast<const double*>(dLf);
  CK(cudaMemcpyAsync(sgd, sg.data(), sizeof(double) * lm, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(bot, bd, sizeof(double) * nsrc * fd, cudaMemcpyDeviceToDevice, c->st));
  if (block) CK(cudaMemsetAsync(top, 0, sizeof(double) * nsrc * fd, c->st));
  if (l > 0) {
    for (int p = 0; p < nsrc; ++p) {
      run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(ld, fd, l, bd + p * fd, n, a + (int64_t)p * l, part, c->st); });
      if (block)
        run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(dld, fd, l, bd + p * fd, n, cc + (int64_t)p * l, part, c->st); });
      // Pbar: bottom' = b - sum R_i a_i;  top' = -sum (R_i c_i + dR_i a_i)
      run(c, OV_KIND_COMBINE, 1, [&] { vec_update(bot + p * fd, rd, fd, l, a + (int64_t)p * l, -1.0, n, c->st); });
      if (block)
        run(c, OV_KIND_COMBINE, 2, [&] {
          vec_update(top + p * fd, rd, fd, l, cc + (int64_t)p * l, -1.0, n, c->st);
          vec_update(top + p * fd, drd, fd, l, a + (int64_t)p * l, -1.0, n, c->st);
        });
    }
    run(c, OV_KIND_COMBINE, 2, [&] {
      coef_sign(a, sgd, sa, l, nsrc, c->st);
      if (block) coef_sign(cc, sgd, sc, l, nsrc, c->st);
    });
  }
  launch_check();
  const int st = block ? block_impl<R>(c, dims, U, mu, m_w, nsrc, top, bot, k, E, m_dir, dx, x, info)
                       : tsl_sign_impl<R>(c, dims, U, mu, m_w, nsrc, bot, k, x, info);
  if (st != OV_OK) return st;
  if (l > 0) {
    double* xd = static_cast<double*>(x);
    double* dxd = static_cast<double*>(dx);
    for (int p = 0; p < nsrc; ++p) {
      // the exact part: sum_i sgn(lambda_i) (R_i c_i + dR_i a_i, R_i a_i)
      run(c, OV_KIND_COMBINE, 1, [&] { vec_update(xd + p * fd, rd, fd, l, sa + (int64_t)p * l, 1.0, n, c->st); });
      if (block)
        run(c, OV_KIND_COMBINE, 2, [&] {
          vec_update(dxd + p * fd, rd, fd, l, sc + (int64_t)p * l, 1.0, n, c->st);
          vec_update(dxd + p * fd, drd, fd, l, sa + (int64_t)p * l, 1.0, n, c->st);
        });
    }
  }
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  return OV_OK;
}

template <typename R>
int eps_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc, const void* b,
             int k, bool block, const void* E, double m_dir, double* eps, ov_tsl_info* info) {
  check_ptr(b);
  if (!eps) throw Status{OV_ERR_INVALID_ARG};
  const Geom g = make_geom(dims);
  if (nsrc < 1 || nsrc > 4096) throw Status{OV_ERR_INVALID_ARG};
  const int64_t n = g.V * 24;   // doubles per source
  double* t1 = block ? wsT<double>(c, B_EPS1T, nsrc * n) : nullptr;
  double* b1 = wsT<double>(c, B_EPS1B, nsrc * n);
  double* t2 = block ? wsT<double>(c, B_EPS2T, nsrc * n) : nullptr;
  double* b2 = wsT<double>(c, B_EPS2B, nsrc * n);
  double* nrm = wsT<double>(c, B_EPSN, 3 * (int64_t)nsrc);
  if (info) info->k_reached = k;
  ov_tsl_info one{};
  int st;
  if (block) {
    st = block_impl<R>(c, dims, U, mu, m_w, nsrc, nullptr, b, k, E, m_dir, t1, b1, &one);
    merge_info(info, one);
    if (st != OV_OK) return st;
    one = ov_tsl_info{};
    st = block_impl<R>(c, dims, U, mu, m_w, nsrc, t1, b1, k, E, m_dir, t2, b2, &one);
  } else {
    st = tsl_sign_impl<R>(c, dims, U, mu, m_w, nsrc, b, k, b1, &one);
    merge_info(info, one);
    if (st != OV_OK) return st;
    one = ov_tsl_info{};
    st = tsl_sign_impl<R>(c, dims, U, mu, m_w, nsrc, b1, k, b2, &one);
  }
  merge_info(info, one);
  if (st != OV_OK) return st;
  run(c, OV_KIND_COMBINE, 1, [&] { eps_norms(t2, b2, static_cast<const double*>(b), nsrc, n, nrm, c->st); });
  launch_check();
  std::vector<double> h(3 * (size_t)nsrc);
  CK(cudaMemcpyAsync(h.data(), nrm, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int src = 0; src < nsrc; ++src)
    eps[src] = std::sqrt(h[3 * src] + h[3 * src + 1]) / (2.0 * std::sqrt(h[3 * src + 2]));
  return OV_OK;
}

// What the reverse mode needs from the forward pass: the lattice state (bases or
// segment checkpoints, coefficients), the host scalars, y, and per source the
// recorded inverses of the Newton sign iteration, its scalings and its result.
template <typename R>
struct FwdState {
  Lat<R> L{};
  std::vector<SrcScal> hsc;
  int k = 0, nsrc = 0, S = 0;
  SegPlan P;
  SegStore<R> K{};
  zd* y = nullptr;        // [src][k]
  zd* rec_inv = nullptr;  // [src][NREC][k*k]
  double* rec_ld = nullptr;  // [src][NREC]
  zd* fsign = nullptr;    // [src][k*k]
  std::vector<std::vector<int>> scaling;
  std::vector<int> iters;
  std::vector<char> rec_ok;
  int iters_max = 0;
};

// forward recurrence and, per source, y = beta0 sgn(T_k) e1 by Newton with every
// inverse recorded (for the Frechet adjoint of the reverse mode)
template <typename R>
int vjp_forward(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                const void* b, int k, FwdState<R>& F, ov_tsl_info* info) {
  check_ptr(b);
  // the reverse mode differentiates the full k x k sign (Theorem 1 by Newton), not the nested one
  if (c->opt.nested > 0) throw Status{OV_ERR_INVALID_ARG};
  const int S = c->opt.segment > 0 && c->opt.segment < k ? c->opt.segment : 0;
  F.S = S;
  F.k = k;
  F.nsrc = nsrc;
  F.L = setup<R>(c, dims, U, mu, m_w, nsrc, k, true, 1, S > 0 ? S + 2 : 0);
  Lat<R>& L = F.L;
  const int64_t V = L.g.V, vs = L.vs;
  run(c, OV_KIND_LAYOUT, 2, [&] {
    pack_spinors<R>(static_cast<const double*>(b), L.r, nsrc, V, vs, c->st);
    pack_spinors<R>(static_cast<const double*>(b), L.s, nsrc, V, vs, c->st);
  });
  CK(cudaEventRecord(c->ev[0], c->st));
  if (S > 0) {
    F.P = seg_plan(k, S);
    F.K = seg_store(c, L, (int)F.P.lo.size());
    seg_forward(c, L, F.P, F.K);
  } else {
    forward_krylov(c, L);
  }
  CK(cudaEventRecord(c->ev[1], c->st));
  F.hsc = read_scalars(c, L.sc, nsrc);
  int kr = k;
  int st = scalar_status(F.hsc, &kr, k);
  c->last_k = k;
  c->last_nsrc = nsrc;
  c->last_block = 0;
  c->last_seg = S > 0 ? 1 : 0;
  c->last_prec = c->opt.precision;
  std::copy(dims, dims + 4, c->last_dims);
  if (info) info->k_reached = kr;
  if (st != OV_OK) return st;
  if (c->opt.diagnostics) {
    st = run_diagnostics(c, L, S > 0, info);
    if (st != OV_OK) return st;
  }
  const int64_t n = (int64_t)k * k;
  F.y = wsT<zd>(c, B_Y, (int64_t)nsrc * k);
  F.rec_inv = wsT<zd>(c, B_REC, (int64_t)nsrc * NREC * n);
  F.rec_ld = wsT<double>(c, B_RECLD, (int64_t)nsrc * NREC);
  F.fsign = wsT<zd>(c, B_FSIGN, (int64_t)nsrc * n);
  int* derr = wsT<int>(c, B_DERR, 1, true);
  zd* a[2] = {wsT<zd>(c, B_X, nsrc * n), wsT<zd>(c, B_XN, nsrc * n)};
  for (int src = 0; src < nsrc; ++src)
    run(c, OV_KIND_DENSE, 2, [&] {
      dense_build_t(L.alpha + (int64_t)src * k, L.beta + (int64_t)src * k, L.delta + (int64_t)src * k, k,
                    a[0] + src * n, c->st);
    });
  std::vector<int> which;
  F.iters_max = newton_batch(c, a, k, nsrc, derr, which, F.iters, F.rec_inv, F.rec_ld, NREC, &F.scaling, &F.rec_ok);
  if (F.iters_max < 0) return sign_failed(c, derr);
  for (int src = 0; src < nsrc; ++src)
    run(c, OV_KIND_DENSE, 2, [&] {
      dense_copy(a[which[src]] + src * n, F.fsign + (int64_t)src * n, n, c->st);
      dense_extract_y(a[which[src]] + src * n, F.hsc[src].beta0, k, F.y + (int64_t)src * k, c->st);
    });
  {
    const int ss = sign_status(c, derr);
    if (ss != OV_OK) return ss;
  }
  CK(cudaEventRecord(c->ev[2], c->st));
  if (info) {
    info->newton_iters = F.iters_max;
    info->t_ms[0] = elapsed(c->ev[0], c->ev[1]);
    info->t_ms[1] = elapsed(c->ev[1], c->ev[2]);
  }
  return OV_OK;
}

// reverse mode from a forward state: g_y = V^dag xbar, G_T by the Frechet adjoint,
// x = V y (if x is given), the reverse sweep and the force
template <typename R>
int vjp_reverse(ov_context* c, FwdState<R>& F, const void* xbar, void* x, void* dU, double* dmu,
                ov_tsl_info* info) {
  check_ptr(xbar);
  check_ptr(dU);
  if (!dmu) throw Status{OV_ERR_INVALID_ARG};
  if (x) check_ptr(x);
  Lat<R>& L = F.L;
  const int k = F.k, nsrc = F.nsrc, S = F.S;
  const SegPlan& P = F.P;
  const SegStore<R>& K = F.K;
  const auto& hsc = F.hsc;
  zd* y = F.y;
  const int64_t V = L.g.V, vs = L.vs;
  CK(cudaEventRecord(c->ev[2], c->st));
  // g_y = V^dag xbar
  R* xb = wsT<R>(c, B_XBAR, nsrc * vs);
  run(c, OV_KIND_LAYOUT, 1, [&] { pack_spinors<R>(static_cast<const double*>(xbar), xb, nsrc, V, vs, c->st); });
  const int64_t nsb = (V + 127) / 128;
  zd* gy = wsT<zd>(c, B_GY, (int64_t)nsrc * 2 * k);
  zd* cpart = wsT<zd>(c, B_CPART, (int64_t)nsrc * 2 * k * nsb);
  if (S > 0) {
    // second pass: g_y one replayed segment at a time
    for (size_t t = 0; t < P.lo.size(); ++t) {
      seg_replay(c, L, P, K, (int)t, false);
      run(c, OV_KIND_COMBINE, 2, [&] {
        basis_dots_range(L, P.lo[t], P.hi[t] - P.lo[t], xb, vs, gy + 2 * P.lo[t], cpart, c->st);
      });
    }
  } else {
    run(c, OV_KIND_COMBINE, 2, [&] { basis_dots(L, k, xb, vs, gy, cpart, c->st); });
  }
  launch_check();
  // G_T = L_sgn(T^dag, beta0 g_y e1^T).  The Theorem-1 block iteration on
  // [[T^dag, G], [0, T^dag]] has diagonal iterates X_i^dag (X_i: the iterates on
  // T, same scalings), so its upper-right block follows from the recorded X_i^{-1}:
  //   E <- (g_i E - X_i^{-dag} E X_i^{-dag} / g_i) / 2,
  // continued with X^{-1} = sgn(T) once the diagonal has converged.
  zd* gaT = wsT<zd>(c, B_GA, (int64_t)nsrc * k);
  zd* gbT = wsT<zd>(c, B_GB, (int64_t)nsrc * k);
  double* gdT = wsT<double>(c, B_GD, (int64_t)nsrc * k);
  int* derr = wsT<int>(c, B_DERR, 1, true);
  int iters_adj = 0;
  {
    // all sources together: source p runs its own recorded iterations (switched
    // off after F.iters[p]), then up to four steps with sgn(T) until its own
    // stopping rule holds
    const int64_t n = (int64_t)k * k;
    const int64_t pstride = (n + 255) / 256 + 64;
    zd* e[2] = {wsT<zd>(c, B_E, nsrc * n), wsT<zd>(c, B_EN, nsrc * n)};
    zd* t1 = wsT<zd>(c, B_TMP1, nsrc * n);
    zd* t2 = wsT<zd>(c, B_TMP2, nsrc * n);
    double* dstat = wsT<double>(c, B_DSTAT, 4 * (int64_t)nsrc);
    zd* dpart = wsT<zd>(c, B_DPART, nsrc * pstride);
    unsigned* dcnt = wsT<unsigned>(c, B_DCNT, 4 * (int64_t)nsrc);
    int* act_dev = wsT<int>(c, B_ACT, nsrc);
    int* rscal = wsT<int>(c, B_RSCAL, (int64_t)nsrc * NREC);
    std::vector<int> hscal((size_t)nsrc * NREC, 0), act(nsrc, 0), cur(nsrc, 0), extra(nsrc, 0);
    std::vector<double> prev(nsrc, INFINITY), hs(4 * (size_t)nsrc);
    int rec_max = 0;
    std::vector<double> hb0(nsrc, 0.0);
    std::vector<int> okm(nsrc, 0);
    for (int src = 0; src < nsrc; ++src) {
      hb0[src] = hsc[src].beta0;
      if (!F.rec_ok[src]) continue;
      okm[src] = 1;
      for (size_t i = 0; i < F.scaling[src].size(); ++i) hscal[(size_t)src * NREC + i] = F.scaling[src][i];
      rec_max = std::max(rec_max, F.iters[src]);
    }
    CK(cudaMemcpyAsync(rscal, hscal.data(), sizeof(int) * hscal.size(), cudaMemcpyHostToDevice, c->st));
    // Low-rank start: E_0 = beta0 g_y e_1^T has rank one and each iteration at most
    // doubles the rank, so while it is small E = A B^H is kept as k x r factors:
    //   A <- [g A / 2 | -Y A / (2 g)],  B <- [B | Y^H B]   (Y = X_i^{-H}),
    // two k x k x r products instead of two k^3 ones; E is formed once the rank
    // would pass rmax.  (Factors beyond a source's own rank stay zero.)
    // (with the tensor-core products a full k x k product costs about what two FP64
    // k x k x 16 ones do, so the factored form stops at rank 8 there)
    int rmax = 0;
    const int rcap = kk_split(c, k) ? 8 : 256;
    for (int r = 2; r <= rcap && r <= k / 2; r *= 2) rmax = r;
    if (rmax < 2) rmax = 1;
    zd* fa = wsT<zd>(c, B_LRA, (int64_t)nsrc * k * rmax);
    zd* fb = wsT<zd>(c, B_LRB, (int64_t)nsrc * k * rmax);
    double* b0dev = wsT<double>(c, B_BETA0, nsrc);
    CK(cudaMemcpyAsync(b0dev, hb0.data(), sizeof(double) * nsrc, cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_DENSE, 1, [&] { dense_lr_init(fa, fb, k, rmax, gy, 2 * (int64_t)k, 2, b0dev, nsrc, c->st); });
    int i0 = 0, rank = 1;
    const int64_t fs = (int64_t)k * rmax;
    while (2 * rank <= rmax && i0 < rec_max) {
      for (int src = 0; src < nsrc; ++src) act[src] = F.rec_ok[src] && i0 < F.iters[src];
      CK(cudaMemcpyAsync(act_dev, act.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, c->st));
      const zd* yi = F.rec_inv + (int64_t)i0 * n;
      run(c, OV_KIND_DENSE_GEMM, 2, [&] {
        dense_gemm_rect_batch(yi, (int64_t)NREC * n, k, 1, fa, fs, rmax, 0, fa + rank, fs, rmax, k, rank, k, nsrc,
                              act_dev, c->st);
        dense_gemm_rect_batch(yi, (int64_t)NREC * n, k, 0, fb, fs, rmax, 0, fb + rank, fs, rmax, k, rank, k, nsrc,
                              act_dev, c->st);
      });
      run(c, OV_KIND_DENSE, 1, [&] {
        dense_lr_scale(fa, k, rmax, rank, F.rec_ld + i0, NREC, rscal + i0, NREC, nsrc, act_dev, c->st);
      });
      rank *= 2;
      ++i0;
    }
    CK(cudaMemcpyAsync(act_dev, okm.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_DENSE_GEMM, 1, [&] {
      dense_gemm_rect_batch(fa, fs, rmax, 0, fb, fs, rmax, 1, e[0], n, k, k, k, rank, nsrc, act_dev, c->st);
    });
    for (int i = i0; i < rec_max; ++i) {
      const int ce = (i - i0) & 1;
      for (int src = 0; src < nsrc; ++src) act[src] = F.rec_ok[src] && i < F.iters[src];
      CK(cudaMemcpyAsync(act_dev, act.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, c->st));
      const zd* yi = F.rec_inv + (int64_t)i * n;
      kk_gemm(c, yi, (int64_t)NREC * n, 1, e[ce], n, 0, t1, n, k, nsrc, &act, act_dev);
      kk_gemm(c, t1, n, 0, yi, (int64_t)NREC * n, 1, t2, n, k, nsrc, &act, act_dev);
      run(c, OV_KIND_DENSE, 1, [&] {
        dense_newton_combine_batch(e[ce], t2, e[1 - ce], k, nsrc, act_dev, F.rec_ld + i, NREC, rscal + i, NREC, -1.0,
                                   1.0, dstat, dpart, pstride, dcnt, c->st);
      });
    }
    // bring every source's iterate to e[0] (its parity is its own count of dense iterations)
    for (int src = 0; src < nsrc; ++src) {
      if (!F.rec_ok[src]) continue;
      if (std::max(F.iters[src] - i0, 0) & 1)
        run(c, OV_KIND_DENSE, 1, [&] { dense_copy(e[1] + src * n, e[0] + src * n, n, c->st); });
      act[src] = 1;
    }
    for (int x = 1; x <= 4; ++x) {
      if (std::find(act.begin(), act.end(), 1) == act.end()) break;
      const int ce = (x - 1) & 1;
      CK(cudaMemcpyAsync(act_dev, act.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, c->st));
      CK(cudaMemsetAsync(dstat, 0, sizeof(double) * 4 * nsrc, c->st));
      kk_gemm(c, F.fsign, n, 1, e[ce], n, 0, t1, n, k, nsrc, &act, act_dev);
      kk_gemm(c, t1, n, 0, F.fsign, n, 1, t2, n, k, nsrc, &act, act_dev);
      run(c, OV_KIND_DENSE, 1, [&] {
        dense_newton_combine_batch(e[ce], t2, e[1 - ce], k, nsrc, act_dev, dstat + 2, 4, nullptr, 0, -1.0, 1.0,
                                   dstat, dpart, pstride, dcnt, c->st);
      });
      CK(cudaMemcpyAsync(hs.data(), dstat, sizeof(double) * 4 * nsrc, cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      for (int src = 0; src < nsrc; ++src) {
        if (!act[src]) continue;
        const double step = std::sqrt(hs[4 * src] / hs[4 * src + 1]);
        if (!std::isfinite(step)) return sign_failed(c, derr);
        extra[src] = x;
        cur[src] = 1 - ce;
        if (step <= 1e-14 || step >= 0.5 * prev[src]) act[src] = 0;
        prev[src] = step;
      }
    }
    for (int src = 0; src < nsrc; ++src) {
      if (!F.rec_ok[src]) continue;
      iters_adj = std::max(iters_adj, F.iters[src] + extra[src]);
      run(c, OV_KIND_DENSE, 1, [&] {
        dense_extract_tri(e[cur[src]] + src * n, k, gaT + (int64_t)src * k, gbT + (int64_t)src * k,
                          gdT + (int64_t)src * k, c->st);
      });
    }
    // a sign that needed more iterations than the record holds: the block iteration itself
    for (int src = 0; src < nsrc; ++src) {
      if (F.rec_ok[src]) continue;
      zd* a[2] = {wsT<zd>(c, B_X, nsrc * n), wsT<zd>(c, B_XN, nsrc * n)};
      zd* t = wsT<zd>(c, B_T, n);
      zd* eb[2] = {e[0] + src * n, e[1] + src * n};
      run(c, OV_KIND_DENSE, 5, [&] {
        dense_build_t(L.alpha + (int64_t)src * k, L.beta + (int64_t)src * k, L.delta + (int64_t)src * k, k, t,
                      c->st);
        dense_adjoint(t, a[0], k, c->st);
        dense_set_column0(eb[0], gy + (int64_t)src * 2 * k, 2, hsc[src].beta0, k, c->st);
      });
      int wb = 0;
      const int itb = newton(c, a, eb, k, derr, &wb);
      if (itb < 0) return sign_failed(c, derr);
      if (itb > iters_adj) iters_adj = itb;
      run(c, OV_KIND_DENSE, 1, [&] {
        dense_extract_tri(eb[wb], k, gaT + (int64_t)src * k, gbT + (int64_t)src * k, gdT + (int64_t)src * k,
                          c->st);
      });
    }
  }
  {
    const int ss = sign_status(c, derr);
    if (ss != OV_OK) return ss;
  }
  CK(cudaEventRecord(c->ev[3], c->st));
  // (with segments, x is accumulated while the reverse sweep replays each segment)
  int tcur = S > 0 ? (int)P.lo.size() - 1 : 0;   // the window holds the top segment after the second pass
  auto seg_combine = [&](int t) {
    if (x)
      run(c, OV_KIND_COMBINE, 1, [&] {
        combine_range(L, P.lo[t], P.hi[t] - P.lo[t], y, static_cast<double*>(x), t != (int)P.lo.size() - 1,
                      c->st);
      });
  };
  if (S > 0) {
    seg_combine(tcur);
  } else if (x) {
    run(c, OV_KIND_COMBINE, 1, [&] { combine(L, k, y, static_cast<double*>(x), c->st); });
  }
  CK(cudaEventRecord(c->ev[4], c->st));
  // reverse sweep
  std::vector<int> reb;
  for (int j = k - 2; j >= 0; --j)
    if (rebiorth_at(j + 1, c->opt.rebiorth)) reb.push_back(j);
  const int nreb_max = reb.empty() ? 1 : (int)reb.size();
  // force ring length; with segments a divisor of S, so that every flush ends at a segment boundary
  int m = k < 32 ? k : 32;
  if (S > 0)
    for (m = std::min(32, S); S % m; --m) {
    }
  Rev<R> B{};
  B.nsrc = nsrc;
  B.vs = vs;
  B.m = m;
  B.gv = wsT<R>(c, B_GV, nsrc * vs);
  B.gw = wsT<R>(c, B_GW, nsrc * vs);
  B.gv_new = wsT<R>(c, B_GV2, nsrc * vs);
  B.gw_new = wsT<R>(c, B_GW2, nsrc * vs);
  B.gr_ring = wsT<R>(c, B_GR, (int64_t)m * nsrc * vs);
  B.gs_ring = wsT<R>(c, B_GS, (int64_t)m * nsrc * vs);
  B.gp_ring = wsT<R>(c, B_GP, (int64_t)m * nsrc * vs);
  B.hin = wsT<R>(c, B_HIN, (int64_t)nsrc * vs);
  B.xbar = xb;
  B.y = y;
  B.gaT = gaT;
  B.gbT = gbT;
  B.gdT = gdT;
  B.nreb_max = nreb_max;
  B.ev = wsT<zd>(c, B_EV, (int64_t)nsrc * nreb_max * k, true);
  B.ew = wsT<zd>(c, B_EW, (int64_t)nsrc * nreb_max * k, true);
  B.reb_steps = wsT<int>(c, B_REB, nreb_max);
  if (!reb.empty())
    CK(cudaMemcpyAsync(B.reb_steps, reb.data(), sizeof(int) * reb.size(), cudaMemcpyHostToDevice, c->st));
  B.force = wsT<double>(c, B_FORCE, 72 * V, true);
  {
    const int ns = force_splits(V);
    B.force_parts = ns > 1 ? wsT<double>(c, B_FPARTS, (int64_t)ns * 72 * V) : nullptr;
  }
  B.dmu = wsT<double>(c, B_DMU, 1, true);
  B.dmu_part = wsT<zd>(c, B_DMUPART, kForceSplitMax * ((V + 127) / 128) + 64);
  B.dmu_cnt = wsT<unsigned>(c, B_DMUCNT, 4);
  zd* coef = wsT<zd>(c, B_COEF, (int64_t)nsrc * 2 * k);
  auto sweep = [&] {
  run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_init(L, B, c->st); });
  run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_combine(L, B, k - 1, 0, c->st); });
  run(c, OV_KIND_REV_STENCIL, 1, [&] { rev_stencil(L, B, k - 1, 0, -1, 0, c->st); });
  std::swap(B.gv, B.gv_new);
  std::swap(B.gw, B.gw_new);
  int slot = 1, j0 = k - 1, nrec = 0;
  for (int j = k - 2; j >= 0; --j) {
    if (slot == m) {
      run(c, OV_KIND_FORCE, 4, [&] { force_flush(L, B, nullptr, m, j0, c->st); });
      slot = 0;
      j0 = j;
    }
    if (S > 0 && j < P.lo[tcur]) {
      // entering the segment below: its vectors (and v_{j+1}, w_{j+1}) from its checkpoint
      --tcur;
      seg_replay(c, L, P, K, tcur, true);
      seg_combine(tcur);
    }
    const int prev = slot == 0 ? m - 1 : slot - 1;
    run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_dots(L, B, j, c->st); });
    const int rb = rebiorth_at(j + 1, c->opt.rebiorth);
    run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_form(L, B, j, slot, !rb, c->st); });
    if (rb) {
      R* grs = B.gr_ring + (int64_t)slot * nsrc * vs;
      R* gss = B.gs_ring + (int64_t)slot * nsrc * vs;
      for (int ps = 0; ps < c->opt.passes; ++ps) {
        run(c, OV_KIND_PROJ_DOTS, 2, [&] { proj_dots(L, j, 1, grs, gss, vs, coef, cpart, c->st); });
        run(c, OV_KIND_PROJ_UPDATE, 1, [&] { proj_update(L, j, 1, grs, gss, vs, coef, false, c->st, ps > 0); });
        run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_proj_record(L, B, j, nrec, coef, c->st); });
      }
      run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_alpha_dots(L, B, j, slot, c->st); });
      ++nrec;
    }
    run(c, OV_KIND_REV_SCALAR, 1, [&] { rev_combine(L, B, j, slot, c->st); });
    run(c, OV_KIND_REV_STENCIL, 1, [&] { rev_stencil(L, B, j, slot, prev, nrec, c->st); });
    std::swap(B.gv, B.gv_new);
    std::swap(B.gw, B.gw_new);
    ++slot;
  }
  run(c, OV_KIND_FORCE, 4, [&] { force_flush(L, B, nullptr, slot, j0, c->st); });
  };
  if (S > 0) {
    sweep();   // segment replays copy checkpoints between the steps: launched directly
  } else {
    std::vector<unsigned char> key;
    const Rev<R> B0 = B;   // the sweep swaps B's gradient buffers: key on its state at entry
    key_add(key, L);
    key_add(key, B0);
    key_add(key, coef);
    key_add(key, cpart);
    key_add(key, c->opt);
    key_add(key, xb);
    captured(c, c->grev, key, sweep);
  }
  CK(cudaEventRecord(c->ev[5], c->st));
  run(c, OV_KIND_LAYOUT, 1, [&] { unpack_force(B.force, static_cast<double*>(dU), V, c->st); });
  launch_check();
  CK(cudaMemcpyAsync(dmu, B.dmu, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  auto hsc2 = read_scalars(c, L.sc, nsrc);
  prof_collect(c);
  const int st = scalar_status(hsc2, nullptr, k);
  if (st != OV_OK) return st;
  if (info) {
    info->newton_iters = F.iters_max;
    info->newton_iters_adj = iters_adj;
    info->t_ms[2] = elapsed(c->ev[2], c->ev[3]);
    info->t_ms[3] = elapsed(c->ev[3], c->ev[4]);
    info->t_ms[4] = elapsed(c->ev[4], c->ev[5]);
  }
  return OV_OK;
}

template <typename R>
int tsl_vjp_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                 const void* b, int k, const void* xbar, void* x, void* dU, double* dmu, ov_tsl_info* info) {
  check_ptr(xbar);
  check_ptr(dU);
  if (!dmu) throw Status{OV_ERR_INVALID_ARG};
  if (x) check_ptr(x);
  FwdState<R> F;
  const int st = vjp_forward<R>(c, dims, U, mu, m_w, nsrc, b, k, F, info);
  if (st != OV_OK) return st;
  return vjp_reverse<R>(c, F, xbar, x, dU, dmu, info);
}

// ---------------------------------------------------------------------------
// Overlap operator D_ov = 1 + gamma5 sgn(H(mu)) (Sec. 1, Eq. overlap, a = 1) on
// the user layout: D_ov b = b + gamma5 x with x the TSL approximation of
// sgn(H(mu)) b; D_ov^dag b = b + sgn(H(-mu)) gamma5 b (H(mu)^dag = H(-mu) by
// gamma5-hermiticity, and sgn(H)^dag = sgn(H^dag) since sgn(lambda) is real).
// ---------------------------------------------------------------------------
template <typename R>
int overlap_apply_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                       const void* b, int k, int dagger, void* out, ov_tsl_info* info) {
  check_ptr(b);
  check_ptr(out);
  const Geom g = make_geom(dims);
  if (nsrc < 1 || nsrc > 4096) throw Status{OV_ERR_INVALID_ARG};
  const int64_t n = (int64_t)nsrc * 12 * g.V;   // complex elements
  const double* bd = static_cast<const double*>(b);
  double* od = static_cast<double*>(out);
  double* xs = wsT<double>(c, B_OVX, 2 * n);
  int st;
  if (!dagger) {
    st = tsl_sign_impl<R>(c, dims, U, mu, m_w, nsrc, b, k, xs, info);
    if (st != OV_OK) return st;
    run(c, OV_KIND_COMBINE, 1, [&] { ov_combine(bd, xs, od, n, 1, c->st); });
  } else {
    double* g5b = wsT<double>(c, B_OVB, 2 * n);
    run(c, OV_KIND_COMBINE, 1, [&] { gamma5_scale(bd, g5b, n, 1.0, 0.0, c->st); });
    st = tsl_sign_impl<R>(c, dims, U, -mu, m_w, nsrc, g5b, k, xs, info);
    if (st != OV_OK) return st;
    run(c, OV_KIND_COMBINE, 1, [&] { ov_combine(bd, xs, od, n, 0, c->st); });
  }
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  return OV_OK;
}

// Restarted GMRES(m) (Saad and Schultz 1986) for D_ov x = rhs (or D_ov^dag x = rhs),
// one right-hand side, x_0 = 0: Arnoldi with classical Gram-Schmidt applied
// twice (dots and updates on the device), complex Givens rotations and the
// triangular solve on the host, the true residual recomputed at every restart.
// The operator applies the k-step TSL, which is linear in its vector only to
// its approximation error, so the attainable residual is of that order.
// Returns OV_ERR_NOCONV when the relative residual is still above tol after
// maxit operator applications (*iters, *resid report where it stopped).
constexpr int GMRES_M = 30;
// Restarted GMRES(m) on vectors of n complex entries (user layout) for the operator
// `apply(in, out)`; the same algorithm serves the overlap solve and the shifted
// solves of the eigenvector derivatives.
template <typename Apply>
int gmres_solve(ov_context* c, int64_t n, const double* rhs, double* x, double tol, int maxit, Apply&& apply,
                int* iters, double* resid) {
  const int64_t n2 = 2 * n;
  const int m = std::max(1, std::min(maxit, GMRES_M));
  double* Vb = wsT<double>(c, B_GMV, (int64_t)(m + 1) * n2);
  double* r = wsT<double>(c, B_GMR, n2);
  double* ax = wsT<double>(c, B_GMW, n2);
  zd* hd = wsT<zd>(c, B_GMH, 2 * (int64_t)(m + 1));
  zd* part = wsT<zd>(c, B_GMP, 152 * (int64_t)(m + 1));
  auto dots = [&](const double* basis, int nvec, const double* w, std::vector<zd>& out) {
    run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(basis, n2, nvec, w, n, hd, part, c->st); });
    out.resize(nvec);
    CK(cudaMemcpyAsync(out.data(), hd, sizeof(zd) * nvec, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  };
  std::vector<zd> tmp;
  dots(rhs, 1, rhs, tmp);
  const double bnorm = std::sqrt(tmp[0].re);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n2, c->st));
  *iters = 0;
  *resid = 0.0;
  if (!(bnorm > 0.0)) return std::isfinite(bnorm) ? OV_OK : OV_ERR_NONFINITE;
  CK(cudaMemcpyAsync(r, rhs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->st));
  double rn = bnorm;
  int it = 0;
  while (rn > tol * bnorm && it < maxit) {
    run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(r, Vb, 1.0 / rn, 0.0, n, c->st); });
    std::vector<std::complex<double>> H((size_t)(m + 1) * m, 0.0), gv(m + 1, 0.0), sn(m, 0.0);
    std::vector<double> cs(m, 0.0);
    gv[0] = rn;
    int j = 0;
    while (j < m && it < maxit) {
      double* w = Vb + (int64_t)(j + 1) * n2;
      apply(Vb + (int64_t)j * n2, w);
      std::vector<std::complex<double>> hc(j + 2, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        run(c, OV_KIND_COMBINE, 3, [&] {
          vec_dots(Vb, n2, j + 1, w, n, hd, part, c->st);
          vec_update(w, Vb, n2, j + 1, hd, -1.0, n, c->st);
        });
        std::vector<zd> hh(j + 1);
        CK(cudaMemcpyAsync(hh.data(), hd, sizeof(zd) * (j + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int i = 0; i <= j; ++i) hc[i] += std::complex<double>(hh[i].re, hh[i].im);
      }
      dots(w, 1, w, tmp);
      const double hn = std::sqrt(tmp[0].re);
      if (!std::isfinite(hn)) return OV_ERR_NONFINITE;
      hc[j + 1] = hn;
      if (hn > 0.0) run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(w, w, 1.0 / hn, 0.0, n, c->st); });
      // previous rotations, then the one that zeroes H[j+1][j]
      for (int i = 0; i < j; ++i) {
        const std::complex<double> a = hc[i], b2 = hc[i + 1];
        hc[i] = cs[i] * a + sn[i] * b2;
        hc[i + 1] = -std::conj(sn[i]) * a + cs[i] * b2;
      }
      const std::complex<double> a = hc[j], b2 = hc[j + 1];
      const double rho = std::hypot(std::abs(a), std::abs(b2));
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = std::abs(a) / rho;
        sn[j] = (a / std::abs(a)) * std::conj(b2) / rho;
      }
      hc[j] = cs[j] * a + sn[j] * b2;
      hc[j + 1] = 0.0;
      gv[j + 1] = -std::conj(sn[j]) * gv[j];
      gv[j] = cs[j] * gv[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
      ++j;
      ++it;
      if (std::abs(gv[j]) <= tol * bnorm) break;
    }
    // y = R^{-1} g by back substitution, x += V y
    std::vector<std::complex<double>> y(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      std::complex<double> t = gv[i];
      for (int q = i + 1; q < j; ++q) t -= H[(size_t)i * m + q] * y[q];
      y[i] = t / H[(size_t)i * m + i];
    }
    std::vector<zd> yd(j);
    for (int i = 0; i < j; ++i) yd[i] = mk(y[i].real(), y[i].imag());
    CK(cudaMemcpyAsync(hd, yd.data(), sizeof(zd) * j, cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 1, [&] { vec_update(x, Vb, n2, j, hd, 1.0, n, c->st); });
    // true residual
    apply(x, ax);
    run(c, OV_KIND_COMBINE, 1, [&] { vec_sub(rhs, ax, r, n, c->st); });
    dots(r, 1, r, tmp);
    rn = std::sqrt(tmp[0].re);
    if (!std::isfinite(rn)) return OV_ERR_NONFINITE;
  }
  *iters = it;
  *resid = rn / bnorm;
  return rn <= tol * bnorm ? OV_OK : OV_ERR_NOCONV;
}

template <typename R>
int overlap_solve_one(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, const double* rhs,
                      int k, int dagger, double tol, int maxit, double* x, int* iters, double* resid) {
  const Geom g = make_geom(dims);
  return gmres_solve(
      c, 12 * g.V, rhs, x, tol, maxit,
      [&](const double* in, double* out) {
        const int st = overlap_apply_impl<R>(c, dims, U, mu, m_w, 1, in, k, dagger, out, nullptr);
        if (st != OV_OK) throw Status{st};
      },
      iters, resid);
}

// A x = rhs by conjugate gradients on the normal equations A A^dag y = rhs, x = A^dag y
// (the minimum-norm solution for a consistent singular A), on vectors of n complex
// entries; the residual ||rhs - A x|| is the CG residual.  maxit counts CG steps.
template <typename ApplyA, typename ApplyAdag>
int cg_normal_solve(ov_context* c, int64_t n, const double* rhs, double* x, double tol, int maxit, ApplyA&& apply_a,
                    ApplyAdag&& apply_adag, int* iters, double* resid) {
  const int64_t n2 = 2 * n;
  double* y = wsT<double>(c, B_CGY, n2);
  double* r = wsT<double>(c, B_CGR, n2);
  double* p = wsT<double>(c, B_CGP, n2);
  double* q = wsT<double>(c, B_CGQ, n2);
  double* t = wsT<double>(c, B_CGT, n2);
  zd* cd = wsT<zd>(c, B_CGC, 160);
  auto dot = [&](const double* a, const double* b) {
    run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(a, n2, 1, b, n, cd + 1, cd + 4, c->st); });
    zd h;
    CK(cudaMemcpyAsync(&h, cd + 1, sizeof(zd), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return h.re;
  };
  auto axpy = [&](double* w, const double* v, double a) {   // w += a v (a real)
    const zd ca = mk(a, 0.0);
    CK(cudaMemcpyAsync(cd, &ca, sizeof(zd), cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 1, [&] { vec_update(w, v, n2, 1, cd, 1.0, n, c->st); });
  };
  CK(cudaMemsetAsync(y, 0, sizeof(double) * n2, c->st));
  CK(cudaMemcpyAsync(r, rhs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(p, rhs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->st));
  const double bn = std::sqrt(dot(rhs, rhs));
  double rr = bn * bn;
  int it = 0;
  *iters = 0;
  *resid = 0.0;
  if (!std::isfinite(bn)) return OV_ERR_NONFINITE;
  if (bn > 0.0) {
    while (std::sqrt(rr) > tol * bn && it < maxit) {
      apply_adag(p, t);
      apply_a(t, q);
      const double pq = dot(p, q);
      if (!(pq > 0.0) || !std::isfinite(pq)) break;
      const double al = rr / pq;
      axpy(y, p, al);
      axpy(r, q, -al);
      const double rn = dot(r, r);
      if (!std::isfinite(rn)) return OV_ERR_NONFINITE;
      const double be = rn / rr;
      rr = rn;
      run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(p, p, be, 0.0, n, c->st); });
      axpy(p, r, 1.0);
      ++it;
    }
  }
  apply_adag(y, x);
  *iters = it;
  *resid = bn > 0.0 ? std::sqrt(rr) / bn : 0.0;
  return std::sqrt(rr) <= tol * bn ? OV_OK : OV_ERR_NOCONV;
}

// Eigenvalue and eigenvector derivatives along (E, m_dir) (App. B, computed as App. E
// does, by shifted inversions with CG on the normal equations), FP64, for the
// eigen-triples (lambda_i, R_i, L_i):
//   dlambda_i = <L_i| dH R_i>,
//   (lambda_i - H) dR_i = Q_i (dH - dlambda_i) R_i,           Q_i = 1 - R_i <L_i|,
//   (conj lambda_i - H^dag) dL_i = Q_i^dag (dH^dag - conj dlambda_i) L_i,
// each by cg_normal_solve (restarted GMRES stagnates on these indefinite shifted
// operators), then <L_i|dR_i> = 0 and <dL_i|R_i> = 0 imposed (the singular shifted
// operators fix dR_i, dL_i only up to R_i, L_i).
int eigderiv_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, const void* E,
                  double m_dir, int l, const double* lam, const void* Rf, const void* Lf, double tol, int maxit,
                  double* dlam, void* dRf, void* dLf, double* resid) {
  check_ptr(Rf);
  check_ptr(Lf);
  check_ptr(dRf);
  check_ptr(dLf);
  if (E) check_ptr(E);
  if (!(tol > 0.0) || maxit < 1 || !std::isfinite(m_dir)) throw Status{OV_ERR_INVALID_ARG};
  Lat<double> L1 = setup<double>(c, dims, U, mu, m_w, 1, 2, false);
  const int64_t V = L1.g.V, n = 12 * V, fd = 24 * V;
  if (E) {
    double* ue = wsT<double>(c, B_ELINKS, link_reals<double>() * V);
    run(c, OV_KIND_LAYOUT, 1, [&] { pack_links<double>(static_cast<const double*>(E), ue, V, c->st); });
    L1.ue = ue;
  }
  L1.mdir = m_dir;
  double* t1 = wsT<double>(c, B_EDT1, fd);
  double* t2 = wsT<double>(c, B_EDT2, fd);
  zd* cd = wsT<zd>(c, B_EDC, 160);    // [0..3] coefficients, [4..] dot partials
  auto op = [&](const double* in, double* out, int which, int dagger) {   // which: 0 H, 1 dH
    run(c, OV_KIND_LAYOUT, 1, [&] { pack_spinors<double>(in, L1.r, 1, V, L1.vs, c->st); });
    run(c, OV_KIND_APPLY_H, 1, [&] {
      if (which) apply_dh(L1, L1.r, L1.p, dagger, c->st);
      else apply_h(L1, L1.r, L1.p, dagger, c->st, 0, nullptr);
    });
    run(c, OV_KIND_LAYOUT, 1, [&] { unpack_spinors<double>(L1.p, out, 1, V, L1.vs, c->st); });
  };
  auto dot = [&](const double* a, const double* b) {   // a^dag b
    run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(a, fd, 1, b, n, cd + 1, cd + 4, c->st); });
    zd h;
    CK(cudaMemcpyAsync(&h, cd + 1, sizeof(zd), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return h;
  };
  auto axpy = [&](double* w, const double* v, zd a) {   // w += a v
    CK(cudaMemcpyAsync(cd, &a, sizeof(zd), cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 1, [&] { vec_update(w, v, fd, 1, cd, 1.0, n, c->st); });
  };
  const double* Rb = static_cast<const double*>(Rf);
  const double* Lb = static_cast<const double*>(Lf);
  double* dRb = static_cast<double*>(dRf);
  double* dLb = static_cast<double*>(dLf);
  int worst = OV_OK;
  for (int i = 0; i < l; ++i) {
    const double* Ri = Rb + (int64_t)i * fd;
    const double* Li = Lb + (int64_t)i * fd;
    const zd li = mk(lam[2 * i], lam[2 * i + 1]);
    // dlambda_i and the right-hand side of the right derivative
    op(Ri, t1, 1, 0);
    const zd dl = dot(Li, t1);
    dlam[2 * i] = dl.re;
    dlam[2 * i + 1] = dl.im;
    axpy(t1, Ri, mk(-dl.re, -dl.im));
    const zd pr = dot(Li, t1);
    axpy(t1, Ri, mk(-pr.re, -pr.im));
    double* x = dRb + (int64_t)i * fd;
    int it = 0;
    double rr = 0.0;
    const zd lic = mk(li.re, -li.im);
    auto a_r = [&](const double* in, double* out) {   // out = lambda_i in - H in
      op(in, out, 0, 0);
      run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(out, out, -1.0, 0.0, n, c->st); });
      axpy(out, in, li);
    };
    auto a_rdag = [&](const double* in, double* out) {   // out = conj(lambda_i) in - H^dag in
      op(in, out, 0, 1);
      run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(out, out, -1.0, 0.0, n, c->st); });
      axpy(out, in, lic);
    };
    int st = cg_normal_solve(c, n, t1, x, tol, maxit, a_r, a_rdag, &it, &rr);
    if (st != OV_OK && st != OV_ERR_NOCONV) return st;
    if (st == OV_ERR_NOCONV) worst = st;
    const zd cr = dot(Li, x);
    axpy(x, Ri, mk(-cr.re, -cr.im));
    if (resid) resid[2 * i] = rr;
    // the left derivative
    op(Li, t2, 1, 1);
    axpy(t2, Li, mk(-dl.re, dl.im));       // - conj(dlambda) L_i
    const zd pl = dot(Ri, t2);
    axpy(t2, Li, mk(-pl.re, -pl.im));
    double* y = dLb + (int64_t)i * fd;
    st = cg_normal_solve(c, n, t2, y, tol, maxit, a_rdag, a_r, &it, &rr);
    if (st != OV_OK && st != OV_ERR_NOCONV) return st;
    if (st == OV_ERR_NOCONV) worst = st;
    const zd cl = dot(Ri, y);
    axpy(y, Li, mk(-cl.re, -cl.im));
    if (resid) resid[2 * i + 1] = rr;
  }
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  return worst;
}

// Eigen-triples of H(U, mu) smallest in |lambda| by shift-and-invert Arnoldi (the
// role ARPACK plays in the paper, Sec. 3, 4.1): m Arnoldi steps on H^{-1} (right) and
// on H^{-dag} (left) from the caller's start vector, each inversion by
// cg_normal_solve, classical Gram-Schmidt twice; the m x m Hessenberg matrices'
// eigenpairs (ov_hessenberg_eigen) with the largest |mu| give lambda = 1/mu and the
// Ritz vectors; left and right are paired by eigenvalue, scaled to L^dag R = 1, and
// the residual ||H R - lambda R|| / ||R|| is reported.  FP64.
int eigsmall_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int l, int m,
                  const void* start, double tol, int maxit, int32_t* l_out, double* lam, void* Rf, void* Lf,
                  double* resid) {
  check_ptr(start);
  check_ptr(Rf);
  check_ptr(Lf);
  if (!(tol > 0.0) || maxit < 1 || m < l || m > 1024) throw Status{OV_ERR_INVALID_ARG};
  Lat<double> L1 = setup<double>(c, dims, U, mu, m_w, 1, 2, false);
  const int64_t V = L1.g.V, n = 12 * V, fd = 24 * V;
  double* Q = wsT<double>(c, B_SIQ, (int64_t)(m + 1) * fd);
  double* lt = wsT<double>(c, B_SILT, (int64_t)l * fd);
  double* t1 = wsT<double>(c, B_SIT1, fd);
  zd* cd = wsT<zd>(c, B_SIC, (int64_t)m + 8);          // [0, m) coefficients, [m] a dot
  zd* dots = cd + m;
  zd* part = wsT<zd>(c, B_SIP, 152 * (int64_t)(m + 1)); // partial sums of vec_dots (152 per vector)
  auto opH = [&](const double* in, double* out, int dagger) {
    run(c, OV_KIND_LAYOUT, 1, [&] { pack_spinors<double>(in, L1.r, 1, V, L1.vs, c->st); });
    run(c, OV_KIND_APPLY_H, 1, [&] { apply_h(L1, L1.r, L1.p, dagger, c->st, 0, nullptr); });
    run(c, OV_KIND_LAYOUT, 1, [&] { unpack_spinors<double>(L1.p, out, 1, V, L1.vs, c->st); });
  };
  auto dot = [&](const double* a, const double* b) {
    run(c, OV_KIND_COMBINE, 2, [&] { vec_dots(a, fd, 1, b, n, dots, part, c->st); });
    zd h;
    CK(cudaMemcpyAsync(&h, dots, sizeof(zd), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return std::complex<double>(h.re, h.im);
  };
  std::vector<std::complex<double>> lamr, laml;
  std::vector<int> keep_r;
  double* Rb = static_cast<double*>(Rf);
  double* Lb = static_cast<double*>(Lf);
  int worst = OV_OK;
  for (int side = 0; side < 2; ++side) {
    const int dg = side;   // A = H (right) or H^dag (left)
    const double s0 = std::sqrt(dot(static_cast<const double*>(start), static_cast<const double*>(start)).real());
    if (!(s0 > 0.0) || !std::isfinite(s0)) throw Status{OV_ERR_INVALID_ARG};
    run(c, OV_KIND_COMBINE, 1,
        [&] { vec_scale(static_cast<const double*>(start), Q, 1.0 / s0, 0.0, n, c->st); });
    std::vector<std::complex<double>> hm((size_t)(m + 1) * m, 0.0);
    int mm = m;
    for (int j = 0; j < m; ++j) {
      double* w = Q + (int64_t)(j + 1) * fd;
      int it = 0;
      double rr = 0.0;
      const int st = cg_normal_solve(
          c, n, Q + (int64_t)j * fd, w, tol, maxit, [&](const double* in, double* out) { opH(in, out, dg); },
          [&](const double* in, double* out) { opH(in, out, 1 - dg); }, &it, &rr);
      if (st != OV_OK && st != OV_ERR_NOCONV) return st;
      if (st == OV_ERR_NOCONV) worst = st;
      for (int pass = 0; pass < 2; ++pass) {
        run(c, OV_KIND_COMBINE, 3, [&] {
          vec_dots(Q, fd, j + 1, w, n, cd, part, c->st);
          vec_update(w, Q, fd, j + 1, cd, -1.0, n, c->st);
        });
        std::vector<zd> hh(j + 1);
        CK(cudaMemcpyAsync(hh.data(), cd, sizeof(zd) * (j + 1), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        for (int i = 0; i <= j; ++i) hm[(size_t)i * m + j] += std::complex<double>(hh[i].re, hh[i].im);
      }
      const double hn = std::sqrt(dot(w, w).real());
      if (!std::isfinite(hn)) return OV_ERR_NONFINITE;
      hm[(size_t)(j + 1) * m + j] = hn;
      if (!(hn > 1e-14 * std::abs(hm[(size_t)j * m + j]))) {   // an invariant subspace: stop here
        mm = j + 1;
        break;
      }
      run(c, OV_KIND_COMBINE, 1, [&] { vec_scale(w, w, 1.0 / hn, 0.0, n, c->st); });
    }
    // eigenpairs of the leading mm x mm Hessenberg block
    std::vector<double> hv(2 * (size_t)mm * mm), ev(2 * (size_t)mm), vv(2 * (size_t)mm * mm);
    for (int i = 0; i < mm; ++i)
      for (int jj = 0; jj < mm; ++jj) {
        hv[2 * ((size_t)i * mm + jj)] = hm[(size_t)i * m + jj].real();
        hv[2 * ((size_t)i * mm + jj) + 1] = hm[(size_t)i * m + jj].imag();
      }
    const int st = ov_hessenberg_eigen(mm, hv.data(), ev.data(), vv.data());
    if (st != OV_OK) return st;
    std::vector<int> order(mm);
    for (int i = 0; i < mm; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return std::hypot(ev[2 * a], ev[2 * a + 1]) > std::hypot(ev[2 * b], ev[2 * b + 1]);
    });
    const int take = std::min(l, mm);
    std::vector<std::complex<double>>& lamv = side ? laml : lamr;
    for (int q = 0; q < take; ++q) {
      const int i = order[q];
      const std::complex<double> muv(ev[2 * i], ev[2 * i + 1]);
      if (std::abs(muv) == 0.0) break;
      lamv.push_back(side ? std::conj(1.0 / muv) : 1.0 / muv);   // an eigenvalue of H either way
      std::vector<zd> y(mm);
      for (int jj = 0; jj < mm; ++jj) y[jj] = mk(vv[2 * ((size_t)jj * mm + i)], vv[2 * ((size_t)jj * mm + i) + 1]);
      CK(cudaMemcpyAsync(cd, y.data(), sizeof(zd) * mm, cudaMemcpyHostToDevice, c->st));
      double* out = (side ? lt : Rb) + (int64_t)q * fd;
      CK(cudaMemsetAsync(out, 0, sizeof(double) * fd, c->st));
      run(c, OV_KIND_COMBINE, 1, [&] { vec_update(out, Q, fd, mm, cd, 1.0, n, c->st); });
    }
  }
  // pair every right eigenvalue with the nearest left one; scale L to L^dag R = 1
  int got = 0;
  std::vector<char> used(laml.size(), 0);
  for (size_t i = 0; i < lamr.size(); ++i) {
    int best = -1;
    double bd = INFINITY;
    for (size_t j = 0; j < laml.size(); ++j) {
      if (used[j]) continue;
      const double d = std::abs(laml[j] - lamr[i]);
      if (d < bd) {
        bd = d;
        best = (int)j;
      }
    }
    if (best < 0 || !(bd <= 1e-6 * std::abs(lamr[i]) + 1e-12)) continue;
    used[best] = 1;
    double* ro = Rb + (int64_t)got * fd;
    double* lo = Lb + (int64_t)got * fd;
    if ((int64_t)got != (int64_t)i)
      CK(cudaMemcpyAsync(ro, Rb + (int64_t)i * fd, sizeof(double) * fd, cudaMemcpyDeviceToDevice, c->st));
    const std::complex<double> sdot = dot(lt + (int64_t)best * fd, ro);   // L^dag R
    if (std::abs(sdot) < 1e-12) continue;
    const std::complex<double> f = 1.0 / std::conj(sdot);
    run(c, OV_KIND_COMBINE, 1,
        [&] { vec_scale(lt + (int64_t)best * fd, lo, f.real(), f.imag(), n, c->st); });
    // residual ||H R - lambda R|| / ||R||
    opH(ro, t1, 0);
    const zd ml = mk(-lamr[i].real(), -lamr[i].imag());
    CK(cudaMemcpyAsync(cd, &ml, sizeof(zd), cudaMemcpyHostToDevice, c->st));
    run(c, OV_KIND_COMBINE, 1, [&] { vec_update(t1, ro, fd, 1, cd, 1.0, n, c->st); });
    const double rn = std::sqrt(dot(t1, t1).real() / dot(ro, ro).real());
    lam[2 * got] = lamr[i].real();
    lam[2 * got + 1] = lamr[i].imag();
    if (resid) resid[got] = rn;
    ++got;
  }
  *l_out = got;
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  return worst;
}

template <typename R>
int overlap_solve_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                       const void* rhs, int k, int dagger, double tol, int maxit, void* x, int32_t* iters,
                       double* resid) {
  check_ptr(rhs);
  check_ptr(x);
  if (nsrc < 1 || nsrc > 4096 || !(tol > 0.0) || maxit < 1) throw Status{OV_ERR_INVALID_ARG};
  const Geom g = make_geom(dims);
  const int64_t n2 = 24 * g.V;
  int worst = OV_OK, itmax = 0;
  double rmax = 0.0;
  for (int s = 0; s < nsrc; ++s) {
    int it = 0;
    double rr = 0.0;
    const int st = overlap_solve_one<R>(c, dims, U, mu, m_w, static_cast<const double*>(rhs) + s * n2, k, dagger,
                                        tol, maxit, static_cast<double*>(x) + s * n2, &it, &rr);
    if (st != OV_OK && st != OV_ERR_NOCONV) return st;
    if (st == OV_ERR_NOCONV) worst = st;
    itmax = std::max(itmax, it);
    rmax = std::max(rmax, rr);
  }
  if (iters) *iters = itmax;
  if (resid) *resid = rmax;
  return worst;
}

// U(1) current estimator (Sec. 4.3, Eq. lat_vec_cur) over nnoise noise vectors:
//   j_{x,nu} = (1/N) sum_eta < gamma5 chi, d(sgn(H) eta)/dTheta_{x,nu} >,  chi = D_ov^{-dag} eta,
// from one forward TSL on eta and two reverse sweeps (cotangents gamma5 chi and
// i gamma5 chi: the real and imaginary parts), each link gradient turned into a
// Theta derivative with dU = i U dTheta.  trace_mu (may be null) receives the
// same estimator of Tr(D_ov^{-1} dD_ov/dmu) from the two sweeps' mu derivatives.
template <typename R>
int u1_current_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nnoise,
                    const void* eta, int k, double tol, int maxit, void* j, double* trace_mu, ov_tsl_info* info) {
  check_ptr(eta);
  check_ptr(j);
  check_ptr(U);
  if (nnoise < 1 || nnoise > 4096) throw Status{OV_ERR_INVALID_ARG};
  const Geom g = make_geom(dims);
  const int64_t n = 12 * g.V, n2 = 2 * n;
  double* chi = wsT<double>(c, B_CHI, n2);
  double* xb1 = wsT<double>(c, B_CURX1, n2);
  double* xb2 = wsT<double>(c, B_CURX2, n2);
  double* g1 = wsT<double>(c, B_CURG1, 72 * g.V);
  double* g2 = wsT<double>(c, B_CURG2, 72 * g.V);
  double tr_re = 0.0, tr_im = 0.0;
  for (int s = 0; s < nnoise; ++s) {
    const double* es = static_cast<const double*>(eta) + s * n2;
    int it = 0;
    double rr = 0.0;
    int st = overlap_solve_one<R>(c, dims, U, mu, m_w, es, k, 1, tol, maxit, chi, &it, &rr);
    if (st != OV_OK) return st;
    run(c, OV_KIND_COMBINE, 2, [&] {
      gamma5_scale(chi, xb1, n, 1.0, 0.0, c->st);
      gamma5_scale(chi, xb2, n, 0.0, 1.0, c->st);
    });
    FwdState<R> F;
    st = vjp_forward<R>(c, dims, U, mu, m_w, 1, es, k, F, info);
    if (st != OV_OK) return st;
    double d1 = 0.0, d2 = 0.0;
    st = vjp_reverse<R>(c, F, xb1, nullptr, g1, &d1, nullptr);
    if (st != OV_OK) return st;
    st = vjp_reverse<R>(c, F, xb2, nullptr, g2, &d2, nullptr);
    if (st != OV_OK) return st;
    run(c, OV_KIND_COMBINE, 1, [&] {
      theta_current(static_cast<const double*>(U), g1, g2, static_cast<double*>(j), 4 * g.V, 1.0 / nnoise, s > 0,
                    c->st);
    });
    tr_re += d1 / nnoise;
    tr_im += d2 / nnoise;
  }
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  if (trace_mu) {
    trace_mu[0] = tr_re;
    trace_mu[1] = tr_im;
  }
  return OV_OK;
}

template <typename R>
int apply_h_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                 const void* in, void* out, int dagger) {
  check_ptr(in);
  check_ptr(out);
  Lat<R> L = setup<R>(c, dims, U, mu, m_w, nsrc, 1, false);
  int* aerr = wsT<int>(c, B_AERR, 1, true);
  const int var = c->tuned_apply[c->opt.precision];
  if constexpr (std::is_same<R, float>::value) {
    if (var == APPLY_IL) {   // the sources-interleaved form has its own field layout
      run(c, OV_KIND_LAYOUT, 1,
          [&] { pack_spinors_il(static_cast<const double*>(in), L.r, nsrc, L.g.V, c->st); });
      run(c, OV_KIND_APPLY_H, 1, [&] { apply_h_il(L, L.r, L.p, dagger, c->st); });
      run(c, OV_KIND_LAYOUT, 1,
          [&] { unpack_spinors_il(L.p, static_cast<double*>(out), nsrc, L.g.V, c->st); });
    }
  }
  if (!std::is_same<R, float>::value || var != APPLY_IL) {
    run(c, OV_KIND_LAYOUT, 1,
        [&] { pack_spinors<R>(static_cast<const double*>(in), L.r, nsrc, L.g.V, L.vs, c->st); });
    run(c, OV_KIND_APPLY_H, 1, [&] { apply_h(L, L.r, L.p, dagger, c->st, var, aerr); });
    run(c, OV_KIND_LAYOUT, 1,
        [&] { unpack_spinors<R>(L.p, static_cast<double*>(out), nsrc, L.g.V, L.vs, c->st); });
  }
  launch_check();
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, aerr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
  return (herr & ERRB_TIMEOUT) ? OV_ERR_TIMEOUT : OV_OK;
}

template <typename R>
int autotune_impl(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int nsrc,
                  ov_tune_report* rep) {
  Lat<R> L = setup<R>(c, dims, U, mu, m_w, nsrc, 2, true);
  CK(cudaMemsetAsync(L.r, 0, sizeof(R) * nsrc * L.vs, c->st));
  CK(cudaMemsetAsync(L.s, 0, sizeof(R) * nsrc * L.vs, c->st));
  CK(cudaMemsetAsync(L.sc, 0, sizeof(SrcScal) * nsrc, c->st));
  cudaEvent_t e0 = c->ev[6], e1 = c->ev[7];
  auto time_us = [&](auto&& launch) {
    launch();
    CK(cudaEventRecord(e0, c->st));
    for (int r = 0; r < 5; ++r) launch();
    CK(cudaEventRecord(e1, c->st));
    CK(cudaEventSynchronize(e1));
    launch_check();
    return 1e3f * elapsed(e0, e1) / 5.f;
  };
  ov_tune_report r{};
  r.n_apply = apply_h_variants();
  r.n_pair = tsl_stencil_variants();
  int* aerr = wsT<int>(c, B_AERR, 1, true);
  for (int v = 0; v < r.n_apply && v < 16; ++v)
    r.apply_us[v] = time_us([&] {
      if constexpr (std::is_same<R, float>::value) {
        if (v == APPLY_IL) return apply_h_il(L, L.r, L.p, 0, c->st);   // same buffers, its own layout
      }
      apply_h(L, L.r, L.p, 0, c->st, v, aerr);
    });
  for (int v = 0; v < r.n_pair && v < 16; ++v)
    r.pair_us[v] = time_us([&] { tsl_stencil(L, 0, true, c->st, v); });
  // a variant replaces the current choice only when it is more than 2% faster: the
  // variants differ in their reduction blocks, so a choice made on timing noise
  // would change the results from run to run at rounding level
  for (int v = 1; v < r.n_apply && v < 16; ++v)
    if (r.apply_us[v] < 0.98f * r.apply_us[r.apply_variant]) r.apply_variant = v;
  for (int v = 1; v < r.n_pair && v < 16; ++v)
    if (r.pair_us[v] < 0.98f * r.pair_us[r.pair_variant]) r.pair_variant = v;
  int herr = 0;
  CK(cudaMemcpyAsync(&herr, aerr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (herr & ERRB_TIMEOUT) return OV_ERR_TIMEOUT;
  c->tuned_apply[c->opt.precision] = r.apply_variant;
  c->tuned_pair[c->opt.precision] = r.pair_variant;
  c->launches += 6 * (r.n_apply + r.n_pair);
  if (rep) *rep = r;
  return OV_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const Status& s) {
    return s.code;
  } catch (...) {
    return OV_ERR_CUDA;
  }
}

bool valid_options(const ov_options* o) {
  return o->precision >= 0 && o->precision <= 1 && o->rebiorth >= 0 && o->passes >= 1 && o->passes <= 4 &&
         o->segment >= 0 && (o->segment == 0 || o->rebiorth == 0) && (o->dense == 0 || o->dense == 1) &&
         (o->diagnostics == 0 || o->diagnostics == 1) && (o->newton == 0 || o->newton == 1) &&
         (o->basis_memory == 0 || o->basis_memory == 1) && (o->graphs == 0 || o->graphs == 1) &&
         o->gemm >= 0 && o->gemm <= 2 && o->nested >= 0 && o->nested <= OV_NESTED_MAX;
}

// x = V_k y from a forward state (a second pass over the segments if there are any)
template <typename R>
void fwd_combine(ov_context* c, FwdState<R>& F, void* x) {
  Lat<R>& L = F.L;
  if (F.S > 0) {
    for (size_t t = 0; t < F.P.lo.size(); ++t) {
      seg_replay(c, L, F.P, F.K, (int)t, false);
      run(c, OV_KIND_COMBINE, 1, [&] {
        combine_range(L, F.P.lo[t], F.P.hi[t] - F.P.lo[t], F.y, static_cast<double*>(x), t > 0, c->st);
      });
    }
  } else {
    run(c, OV_KIND_COMBINE, 1, [&] { combine(L, F.k, F.y, static_cast<double*>(x), c->st); });
  }
  launch_check();
  CK(cudaStreamSynchronize(c->st));
  prof_collect(c);
}

}  // namespace

// A forward pass kept for reverse mode: a private context whose workspace holds
// the bases (or segment checkpoints), the coefficients and the Newton record.
struct ov_tape {
  ov_context* parent = nullptr;
  ov_context* ctx = nullptr;
  FwdState<double>* f64 = nullptr;
  FwdState<float>* f32 = nullptr;
};

extern "C" {

int ov_context_create(ov_context** ctx, const ov_options* opt, void* stream) {
  if (!ctx) return OV_ERR_INVALID_ARG;
  *ctx = nullptr;
  ov_options o{};
  o.precision = OV_FP64;
  o.rebiorth = 1;
  o.passes = 2;
  o.graphs = 1;
  if (opt) {
    if (!valid_options(opt)) return OV_ERR_INVALID_ARG;
    o = *opt;
  }
  ov_context* c = new (std::nothrow) ov_context();
  if (!c) return OV_ERR_OOM;
  c->st = static_cast<cudaStream_t>(stream);
  c->opt = o;
  for (auto& e : c->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return OV_ERR_CUDA;
    }
  }
  *ctx = c;
  return OV_OK;
}

int ov_context_destroy(ov_context* c) {
  if (!c) return OV_ERR_INVALID_ARG;
  for (ov_context* w : c->workers) ov_context_destroy(w);
  c->workers.clear();
  cudaStreamSynchronize(c->st);
  if (c->cap_st) cudaStreamSynchronize(c->cap_st);
  if (c->gfwd.exec) cudaGraphExecDestroy(c->gfwd.exec);
  if (c->grev.exec) cudaGraphExecDestroy(c->grev.exec);
  if (c->gnest.exec) cudaGraphExecDestroy(c->gnest.exec);
  for (auto& e : c->cap_ev)
    if (e) cudaEventDestroy(e);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  oz_destroy_handle(c->blas);
  for (int i = 0; i < NBUF; ++i) {
    if (!c->buf[i]) continue;
    if (c->host_buf[i])
      cudaFreeHost(c->buf[i]);
    else
      cudaFree(c->buf[i]);
  }
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->prof) {
    for (int i = 0; i < NPROF; ++i) {
      if (c->prof->a[i]) cudaEventDestroy(c->prof->a[i]);
      if (c->prof->b[i]) cudaEventDestroy(c->prof->b[i]);
    }
    delete c->prof;
  }
  if (c->owns_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
  return OV_OK;
}

static int prof_create(ov_context* c) {
  if (c->prof) return OV_OK;
  c->prof = new (std::nothrow) Prof();
  if (!c->prof) return OV_ERR_OOM;
  for (int i = 0; i < NPROF; ++i) {
    if (cudaEventCreate(&c->prof->a[i]) != cudaSuccess || cudaEventCreate(&c->prof->b[i]) != cudaSuccess) {
      cudaGetLastError();
      return OV_ERR_CUDA;
    }
  }
  return OV_OK;
}

int ov_profile_enable(ov_context* c, int32_t enable) {
  if (!c) return OV_ERR_INVALID_ARG;
  if (!c->prof && !enable) return OV_OK;
  const int st = prof_create(c);
  if (st != OV_OK) return st;
  c->prof->on = enable != 0;
  return OV_OK;
}

int ov_profile_select(ov_context* c, uint32_t kind_mask) {
  if (!c) return OV_ERR_INVALID_ARG;
  int st = prof_create(c);
  if (st != OV_OK) return st;
  // pairs already recorded keep their kinds; collect them under the old mask
  st = guarded([&] { prof_collect(c); return OV_OK; });
  if (st != OV_OK) return st;
  c->prof->mask = kind_mask;
  return OV_OK;
}

int ov_profile_read(ov_context* c, int32_t kind, int64_t* launches, double* ms, int32_t reset) {
  if (!c || kind < 0 || kind >= OV_NKIND || !launches || !ms) return OV_ERR_INVALID_ARG;
  if (!c->prof) {
    *launches = 0;
    *ms = 0.0;
    return OV_OK;
  }
  const int st = guarded([&] { prof_collect(c); return OV_OK; });
  if (st != OV_OK) return st;
  *launches = c->prof->cnt[kind];
  *ms = c->prof->ms[kind];
  if (reset) {
    for (int i = 0; i < OV_NKIND; ++i) { c->prof->cnt[i] = 0; c->prof->ms[i] = 0.0; }
  }
  return OV_OK;
}

int64_t ov_launch_count(ov_context* c) { return c ? c->launches : -1; }

int ov_selftest_wait(ov_context* c, uint64_t limit_ns, double* elapsed_ms) {
  if (!c || !elapsed_ms || limit_ns == 0 || limit_ns > 100000000ull) return OV_ERR_INVALID_ARG;
  return guarded([&] {
    // [0, 1]: the key word nothing writes, [2]: error word, [3], [4]: how each block left
    int* w = wsT<int>(c, B_DERR, 8);
    CK(cudaMemsetAsync(w, 0, 8 * sizeof(int), c->st));
    CK(cudaEventRecord(c->ev[0], c->st));
    dense_wait_probe(reinterpret_cast<unsigned long long*>(w), w + 2, w + 3, limit_ns, c->st);
    launch_check();
    c->launches += 1;
    CK(cudaEventRecord(c->ev[1], c->st));
    int h[8] = {};
    CK(cudaMemcpyAsync(h, w, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    *elapsed_ms = elapsed(c->ev[0], c->ev[1]);
    // both blocks must have given up, the second through the first one's flag
    if (h[0] != 0 || h[1] != 0 || !(h[2] & ERRB_TIMEOUT) || h[3] != 1 || h[4] != 1) return OV_ERR_CUDA;
    return OV_ERR_TIMEOUT;
  });
}

int ov_context_set_options(ov_context* c, const ov_options* opt) {
  if (!c || !opt || !valid_options(opt)) return OV_ERR_INVALID_ARG;
  c->opt = *opt;
  return OV_OK;
}

int ov_apply_H(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
               const void* in, void* out, int32_t dagger) {
  if (!c) return OV_ERR_INVALID_ARG;
  return guarded([&] {
    return c->opt.precision == OV_MIXED ? apply_h_impl<float>(c, dims, U, mu, m_w, nsrc, in, out, dagger)
                                        : apply_h_impl<double>(c, dims, U, mu, m_w, nsrc, in, out, dagger);
  });
}

int ov_tsl_sign(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                const void* b, int32_t k, void* x, ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED ? tsl_sign_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, x, info)
                                        : tsl_sign_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, x, info);
  });
}

int ov_tsl_sign_vjp(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                    const void* b, int32_t k, const void* xbar, void* x, void* dU, double* dmu,
                    ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? tsl_vjp_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, xbar, x, dU, dmu, info)
               : tsl_vjp_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, xbar, x, dU, dmu, info);
  });
}

int ov_autotune(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                ov_tune_report* rep) {
  if (!c) return OV_ERR_INVALID_ARG;
  return guarded([&] {
    return c->opt.precision == OV_MIXED ? autotune_impl<float>(c, dims, U, mu, m_w, nsrc, rep)
                                        : autotune_impl<double>(c, dims, U, mu, m_w, nsrc, rep);
  });
}

int ov_set_stencil_variants(ov_context* c, int32_t apply_variant, int32_t pair_variant) {
  if (!c || apply_variant < 0 || apply_variant >= apply_h_variants() || pair_variant < 0 ||
      pair_variant >= tsl_stencil_variants())
    return OV_ERR_INVALID_ARG;
  c->tuned_apply[c->opt.precision] = apply_variant;
  c->tuned_pair[c->opt.precision] = pair_variant;
  return OV_OK;
}

int ov_block_tsl_sign(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                      const void* top, const void* bottom, int32_t k, const void* E, double m_dir, void* out_top,
                      void* out_bottom, ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? block_impl<float>(c, dims, U, mu, m_w, nsrc, top, bottom, k, E, m_dir, out_top, out_bottom, info)
               : block_impl<double>(c, dims, U, mu, m_w, nsrc, top, bottom, k, E, m_dir, out_top, out_bottom, info);
  });
}

int ov_tsl_sign_jvp(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                    const void* b, int32_t k, const void* E, double m_dir, void* dx, void* x, ov_tsl_info* info) {
  return ov_block_tsl_sign(c, dims, U, mu, m_w, nsrc, nullptr, b, k, E, m_dir, dx, x, info);
}

int ov_tsl_ritz_triples(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t src,
                        int32_t k, int32_t lmax, double tol, int32_t* l_out, double* lam, void* R, void* L,
                        double* resid) {
  if (!c || !dims || !l_out || !lam || lmax < 1 || lmax > 4096 || !(tol > 0.0) || k < 2 || k != c->last_k ||
      src < 0 || src >= c->last_nsrc || c->last_block || c->last_seg || c->last_prec != c->opt.precision ||
      !std::equal(dims, dims + 4, c->last_dims))
    return OV_ERR_INVALID_ARG;
  *l_out = 0;
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? ritz_impl<float>(c, dims, U, mu, m_w, src, k, lmax, tol, l_out, lam, R, L, resid)
               : ritz_impl<double>(c, dims, U, mu, m_w, src, k, lmax, tol, l_out, lam, R, L, resid);
  });
}

int ov_eigen_derivatives(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, const void* E,
                         double m_dir, int32_t l, const double* lam, const void* R, const void* L, double tol,
                         int32_t maxit, double* dlam, void* dR, void* dL, double* resid) {
  if (!c || !dims || l < 1 || l > 4096 || !lam || !dlam) return OV_ERR_INVALID_ARG;
  return guarded([&] {
    return eigderiv_impl(c, dims, U, mu, m_w, E, m_dir, l, lam, R, L, tol, maxit, dlam, dR, dL, resid);
  });
}

int ov_eigen_smallest(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t l,
                      int32_t m, const void* start, double tol, int32_t maxit, int32_t* l_out, double* lam, void* R,
                      void* L, double* resid) {
  if (!c || !dims || !l_out || !lam || l < 1 || l > 1024 || m < l || m > 1024) return OV_ERR_INVALID_ARG;
  *l_out = 0;
  return guarded([&] {
    return eigsmall_impl(c, dims, U, mu, m_w, l, m, start, tol, maxit, l_out, lam, R, L, resid);
  });
}

int ov_tsl_sign_deflated(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                         const void* b, int32_t k, int32_t l, const double* lam, const void* R, const void* L,
                         void* x, ov_tsl_info* info) {
  if (!c || !dims || k < 2 || k > 4096 || l < 0 || l > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? deflated_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, nullptr, 0.0, false, l, lam, R, L, nullptr,
                                      nullptr, nullptr, x, info)
               : deflated_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, nullptr, 0.0, false, l, lam, R, L, nullptr,
                                       nullptr, nullptr, x, info);
  });
}

int ov_tsl_sign_jvp_deflated(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w,
                             int32_t nsrc, const void* b, int32_t k, const void* E, double m_dir, int32_t l,
                             const double* lam, const void* R, const void* L, const void* dR, const void* dL,
                             void* dx, void* x, ov_tsl_info* info) {
  if (!c || !dims || k < 2 || k > 4096 || l < 0 || l > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? deflated_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, E, m_dir, true, l, lam, R, L, dR, dL, dx, x,
                                      info)
               : deflated_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, E, m_dir, true, l, lam, R, L, dR, dL, dx,
                                       x, info);
  });
}

int ov_tsl_eps(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
               const void* b, int32_t k, double* eps, ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? eps_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, false, nullptr, 0.0, eps, info)
               : eps_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, false, nullptr, 0.0, eps, info);
  });
}

int ov_block_tsl_eps(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                     const void* b, int32_t k, const void* E, double m_dir, double* eps, ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? eps_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, true, E, m_dir, eps, info)
               : eps_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, true, E, m_dir, eps, info);
  });
}

int ov_tsl_batch(ov_context* c, int32_t nprob, ov_problem* probs, int32_t nworkers) {
  if (!c || nprob < 0 || (nprob > 0 && !probs) || nworkers < 1 || nworkers > 16) return OV_ERR_INVALID_ARG;
  for (int32_t i = 0; i < nprob; ++i) probs[i].status = OV_OK;
  if (nprob == 0) return OV_OK;
  const int nw = std::min<int>(nworkers, nprob);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OV_ERR_CUDA;
  }
  while ((int)c->workers.size() < nw) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return OV_ERR_CUDA;
    }
    ov_context* w = nullptr;
    const int st = ov_context_create(&w, &c->opt, s);
    if (st != OV_OK) {
      cudaStreamDestroy(s);
      return st;
    }
    w->owns_stream = true;
    c->workers.push_back(w);
  }
  // most work first (V k^2 per source; the VJP about twice the forward)
  std::vector<int> order(nprob);
  std::vector<double> cost(nprob);
  for (int i = 0; i < nprob; ++i) {
    const ov_problem& p = probs[i];
    const double V = (double)p.dims[0] * p.dims[1] * p.dims[2] * p.dims[3];
    cost[i] = V * (double)p.k * p.k * std::max(1, p.nsrc) * (p.xbar ? 2.0 : 1.0);
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  // the caller's stream orders the inputs before the workers and the workers before later work
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> done(nw, nullptr);
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(start, c->st) != cudaSuccess) {
    cudaGetLastError();
    if (start) cudaEventDestroy(start);
    return OV_ERR_CUDA;
  }
  std::vector<int64_t> l0(nw);
  for (int w = 0; w < nw; ++w) {
    ov_context* wc = c->workers[w];
    wc->opt = c->opt;
    std::copy(c->tuned_apply, c->tuned_apply + 2, wc->tuned_apply);
    std::copy(c->tuned_pair, c->tuned_pair + 2, wc->tuned_pair);
    cudaStreamWaitEvent(wc->st, start, 0);
    l0[w] = wc->launches;
  }
  std::atomic<int> next{0};
  auto work = [&](ov_context* wc) {
    cudaSetDevice(dev);
    for (;;) {
      const int n = next.fetch_add(1);
      if (n >= nprob) break;
      ov_problem& p = probs[order[n]];
      p.status = p.xbar ? ov_tsl_sign_vjp(wc, p.dims, p.U, p.mu, p.m_w, p.nsrc, p.b, p.k, p.xbar, p.x, p.dU,
                                          p.dmu, &p.info)
                        : ov_tsl_sign(wc, p.dims, p.U, p.mu, p.m_w, p.nsrc, p.b, p.k, p.x, &p.info);
    }
  };
  std::vector<std::thread> threads;
  for (int w = 1; w < nw; ++w) threads.emplace_back(work, c->workers[w]);
  work(c->workers[0]);
  for (auto& t : threads) t.join();
  int status = OV_OK;
  for (int w = 0; w < nw; ++w) {
    ov_context* wc = c->workers[w];
    c->launches += wc->launches - l0[w];
    if (cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(done[w], wc->st) == cudaSuccess)
      cudaStreamWaitEvent(c->st, done[w], 0);
    else if (status == OV_OK)
      status = OV_ERR_CUDA;
  }
  cudaEventDestroy(start);
  for (auto e : done)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  for (int32_t i = 0; i < nprob && status == OV_OK; ++i) status = probs[i].status;
  return status;
}

int ov_tape_destroy(ov_tape* t) {
  if (!t) return OV_ERR_INVALID_ARG;
  delete t->f64;
  delete t->f32;
  if (t->ctx) ov_context_destroy(t->ctx);
  delete t;
  return OV_OK;
}

int ov_tsl_sign_fwd(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                    const void* b, int32_t k, void* x, ov_tsl_info* info, ov_tape** tape) {
  if (!c || !tape || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  *tape = nullptr;
  if (info) std::memset(info, 0, sizeof(*info));
  ov_tape* t = new (std::nothrow) ov_tape();
  if (!t) return OV_ERR_OOM;
  t->parent = c;
  int st = ov_context_create(&t->ctx, &c->opt, c->st);
  if (st != OV_OK) {
    delete t;
    return st;
  }
  std::copy(c->tuned_apply, c->tuned_apply + 2, t->ctx->tuned_apply);
  std::copy(c->tuned_pair, c->tuned_pair + 2, t->ctx->tuned_pair);
  st = guarded([&] {
    check_ptr(x);
    int s;
    if (c->opt.precision == OV_MIXED) {
      t->f32 = new FwdState<float>();
      s = vjp_forward<float>(t->ctx, dims, U, mu, m_w, nsrc, b, k, *t->f32, info);
      if (s == OV_OK) fwd_combine(t->ctx, *t->f32, x);
    } else {
      t->f64 = new FwdState<double>();
      s = vjp_forward<double>(t->ctx, dims, U, mu, m_w, nsrc, b, k, *t->f64, info);
      if (s == OV_OK) fwd_combine(t->ctx, *t->f64, x);
    }
    return s;
  });
  c->launches += t->ctx->launches;
  t->ctx->launches = 0;
  if (st != OV_OK) {
    ov_tape_destroy(t);
    return st;
  }
  *tape = t;
  return OV_OK;
}

int ov_tsl_sign_vjp_tape(ov_tape* t, const void* xbar, void* dU, double* dmu, ov_tsl_info* info) {
  if (!t || !t->ctx || (!t->f64 && !t->f32)) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  const int st = guarded([&] {
    if (t->f32) {
      if (info) info->k_reached = t->f32->k;
      return vjp_reverse<float>(t->ctx, *t->f32, xbar, nullptr, dU, dmu, info);
    }
    if (info) info->k_reached = t->f64->k;
    return vjp_reverse<double>(t->ctx, *t->f64, xbar, nullptr, dU, dmu, info);
  });
  t->parent->launches += t->ctx->launches;
  t->ctx->launches = 0;
  return st;
}

int ov_tsl_coefficients(ov_context* c, int32_t src, int32_t k, double* alpha, double* beta, double* delta) {
  if (!c || src < 0 || src >= c->last_nsrc || k != c->last_k || !alpha || !beta || !delta)
    return OV_ERR_INVALID_ARG;
  return guarded([&] {
    CK(cudaMemcpyAsync(alpha, static_cast<zd*>(c->buf[B_ALPHA]) + (int64_t)src * k, sizeof(zd) * k,
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(beta, static_cast<zd*>(c->buf[B_BETA]) + (int64_t)src * k, sizeof(zd) * k,
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(delta, static_cast<double*>(c->buf[B_DELTA]) + (int64_t)src * k, sizeof(double) * k,
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return OV_OK;
  });
}

int ov_tridiag_sign_nested(ov_context* c, int32_t k, const double* alpha, const double* beta, const double* delta,
                           int32_t m, double beta0, double* y, int32_t* newton_iters) {
  if (!c || k < 2 || k > 4096 || m < 0 || m > OV_NESTED_MAX || !alpha || !beta || !delta || !y ||
      !std::isfinite(beta0))
    return OV_ERR_INVALID_ARG;
  return guarded([&] {
    zd* da = wsT<zd>(c, B_NTA, k);
    zd* db = wsT<zd>(c, B_NTB, k);
    double* dd = wsT<double>(c, B_NTD, k);
    zd* dy = wsT<zd>(c, B_NTY, k);
    CK(cudaMemcpyAsync(da, alpha, sizeof(zd) * k, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(db, beta, sizeof(zd) * k, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dd, delta, sizeof(double) * k, cudaMemcpyHostToDevice, c->st));
    const std::vector<double> b0{beta0};
    int it = 0;
    const int st = m > 0 ? nested_sign(c, m, da, db, dd, k, 1, b0, dy, &it) : full_sign(c, da, db, dd, k, 1, b0, dy, &it);
    if (st != OV_OK) return st;
    CK(cudaMemcpyAsync(y, dy, sizeof(zd) * k, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (newton_iters) *newton_iters = it;
    return OV_OK;
  });
}

int ov_kk_gemm(ov_context* c, const void* A, int32_t hA, const void* B, int32_t hB, void* C, int32_t k,
               int32_t mode) {
  if (!c || k < 1 || (mode != 1 && mode != 2) || (mode == 2 && k > OZ_MAX_K) || (hA != 0 && hA != 1) ||
      (hB != 0 && hB != 1))
    return OV_ERR_INVALID_ARG;
  return guarded([&] {
    check_ptr(A);
    check_ptr(B);
    check_ptr(C);
    const int saved = c->opt.gemm;
    c->opt.gemm = mode;
    try {
      kk_gemm(c, static_cast<const zd*>(A), 0, hA, static_cast<const zd*>(B), 0, hB, static_cast<zd*>(C), 0, k, 1,
              nullptr, nullptr);
    } catch (...) {
      c->opt.gemm = saved;
      throw;
    }
    c->opt.gemm = saved;
    launch_check();
    CK(cudaStreamSynchronize(c->st));
    return OV_OK;
  });
}

int ov_overlap_apply(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                     const void* b, int32_t k, int32_t dagger, void* out, ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? overlap_apply_impl<float>(c, dims, U, mu, m_w, nsrc, b, k, dagger, out, info)
               : overlap_apply_impl<double>(c, dims, U, mu, m_w, nsrc, b, k, dagger, out, info);
  });
}

int ov_overlap_solve(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nsrc,
                     const void* rhs, int32_t k, int32_t dagger, double tol, int32_t maxit, void* x, int32_t* iters,
                     double* resid) {
  if (!c || k < 2 || k > 4096) return OV_ERR_INVALID_ARG;
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? overlap_solve_impl<float>(c, dims, U, mu, m_w, nsrc, rhs, k, dagger, tol, maxit, x, iters, resid)
               : overlap_solve_impl<double>(c, dims, U, mu, m_w, nsrc, rhs, k, dagger, tol, maxit, x, iters, resid);
  });
}

int ov_u1_current(ov_context* c, const int32_t dims[4], const void* U, double mu, double m_w, int32_t nnoise,
                  const void* eta, int32_t k, double tol, int32_t maxit, void* j, double* trace_mu,
                  ov_tsl_info* info) {
  if (!c || k < 2 || k > 4096 || !(tol > 0.0) || maxit < 1) return OV_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  return guarded([&] {
    return c->opt.precision == OV_MIXED
               ? u1_current_impl<float>(c, dims, U, mu, m_w, nnoise, eta, k, tol, maxit, j, trace_mu, info)
               : u1_current_impl<double>(c, dims, U, mu, m_w, nnoise, eta, k, tol, maxit, j, trace_mu, info);
  });
}

int ov_debug_inject(ov_context* c, int32_t kind, int32_t step) {
  if (!c || kind < OV_INJECT_NONE || kind > OV_INJECT_OOM || step < 0) return OV_ERR_INVALID_ARG;
  c->inj_kind = kind;
  c->inj_step = step;
  return OV_OK;
}

const char* ov_strerror(int s) {
  switch (s) {
    case OV_OK: return "success";
    case OV_ERR_INVALID_ARG: return "invalid argument";
    case OV_ERR_OOM: return "device workspace allocation failed";
    case OV_ERR_BREAKDOWN: return "Lanczos breakdown (|omega| <= 1e-14 ||r|| ||s||)";
    case OV_ERR_SIGN_ILLPOSED:
      return "k x k sign ill-posed (singular or non-convergent Newton iterate, or a Ritz value on the "
             "imaginary axis)";
    case OV_ERR_NOCONV:
      return "an iteration did not converge (the Ritz values of the diagnostics, or the overlap solver)";
    case OV_ERR_CUDA: return "CUDA runtime error";
    case OV_ERR_NONFINITE: return "non-finite recurrence coefficient";
    case OV_ERR_SCRATCH_LIMIT: return "problem too large for the fixed 32 MiB scratch of ov_apply_H_noalloc";
    case OV_ERR_TIMEOUT: return "a device-side wait ran past its time limit";
    default: return "unknown status";
  }
}

}  // extern "C"
