// C ABI of the phaseless-AFQMC hot path (declared in include/afqmc.h).
//
// The context carves one caller-provided device workspace into the buffers of
// the walker batch and the Hamiltonian store, runs the set-up, and enqueues
// the kernels of each step on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <complex>
#include <map>
#include <mutex>
#include <random>
#include <thread>
#include <type_traits>
#include <string>
#include <vector>

#include <cuda.h>

#include "afqmc.h"
#include "kernels_simt.cuh"
#include "cv_kernels.cuh"
#include "tc_gemm.cuh"
#include "setup_kernels.cuh"

using namespace afq;

namespace {

thread_local char g_err[1024] = "";

afqmc_status fail(afqmc_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CU(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(AFQMC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CHECK_LAUNCH(ctx)                                                                      \
  do {                                                                                         \
    (ctx)->launches++;                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess) return fail(AFQMC_ECUDA, "kernel launch failed (%s:%d): %s", __FILE__, __LINE__, \
                                       cudaGetErrorString(e_));                                \
  } while (0)

constexpr int kHistory = 4096;    // energy measurements buffered on the device by afqmc_run
constexpr int kMaxOcc = 64;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Dims {
  int N, X, na, nb, W, ncol, nblk, c0[2], nbk[2];
  bool restricted;
  int prec;
  int gchunk, nchunk;
  bool cplx = false;   // complex Hamiltonian: X = 2 x the complex Cholesky vectors (Hermitian fields)
  size_t rsz() const { return prec == AFQMC_PREC_FP64 ? 8 : 4; }
  size_t cm() const { return cplx ? 2 : 1; }   // trial, htilde, Ltilde, L, E_h and set-up arrays: complex
  bool tensor() const { return prec == AFQMC_PREC_BF16 || prec == AFQMC_PREC_BF16X3; }
};

// Offsets of every device buffer inside the workspace.
struct Layout {
  size_t psi, thetaT, tA, tB, tC, psi_tmp, th_tmp, logO, logO_tmp, w, w_tmp, wph;
  size_t phi, phi_r, hrot, hrot_r, lbar, slbar, lrot, chol, eh;
  size_t msum, lsum, pden, e1, e2;   // set-up: sum L L, sum lbar L, trial density, two N x N temporaries
  size_t vbias, x, xbar, coef, cmf, xxbar, vhs;
  size_t exch_part, eloc, hist, status, step, src, cum, neww, slot, sflag;
  size_t etr;         // {E_T, sum ENumer, sum EDenom} when E_T follows the running estimate
  size_t tc;          // tensor-core operand buffers (BF16 forms)
  size_t stage;       // set-up staging of Cholesky chunks (aliases vhs, which the set-up does not use)
  size_t stage_bytes, stage_bytes_avail, vhs_bytes, tc_bytes;
  size_t total;
};

Layout plan(const Dims& d) {
  Layout L{};
  size_t cur = 0;
  auto take = [&](size_t bytes) { size_t o = align_up(cur, 256); cur = o + bytes; return o; };
  const size_t R = d.rsz(), C = 2 * R;
  const size_t W = d.W, N = d.N, X = d.X, nc = d.ncol;
  L.psi = take(W * N * nc * C);
  L.thetaT = take(W * nc * N * C);
  L.tA = take(W * N * nc * C);
  L.tB = take(W * N * nc * C);
  L.tC = take(W * N * nc * C);
  L.psi_tmp = take(W * N * nc * C);
  L.th_tmp = take(W * nc * N * C);
  L.logO = take(W * 16);
  L.logO_tmp = take(W * 16);
  L.w = take(W * 8);
  L.w_tmp = take(W * 8);
  L.wph = take(W * 8);
  const size_t cm = d.cm();
  L.phi = take(N * nc * 8 * cm);
  L.phi_r = take(N * nc * R * cm);
  L.hrot = take(nc * N * 8 * cm);
  L.hrot_r = take(nc * N * R * cm);
  L.lbar = take(X * 8);
  L.slbar = take(X * 8);
  L.lrot = take(X * nc * N * R * cm);
  // L in the working precision feeds the CUDA-core VHS GEMM; the tensor-core forms read only their
  // bf16 copy of L^T
  L.chol = take(d.tensor() ? 0 : X * N * N * R * cm);
  L.eh = take(N * N * R * cm);
  L.msum = take(N * N * 8 * cm);
  L.lsum = take(N * N * 8 * cm);
  L.pden = take(N * N * 8 * cm);
  L.e1 = take(N * N * 8 * cm);
  L.e2 = take(N * N * 8 * cm);
  L.vbias = take(W * X * C);
  L.x = take(W * X * 8);
  L.xbar = take(W * X * 16);
  L.coef = take(W * X * C);
  L.cmf = take(W * 16);
  L.xxbar = take(W * 16);
  L.exch_part = take(W * (size_t)d.nchunk * 16);
  L.eloc = take(W * 3 * 16);
  L.hist = take((size_t)kHistory * 4 * 8);
  L.status = take(256);
  L.step = take(256);
  L.src = take(W * 4);
  L.cum = take(W * 8);
  L.neww = take(256);
  L.slot = take(256);
  L.sflag = take(256);   // set-up: input check flags, the 1-norm of the exponent
  L.etr = take(256);
  {
    tc::TcState tmp;
    L.tc_bytes = tc::plan(&tmp, d.prec, d.W, d.N, d.X, d.ncol, d.c0, d.nbk, d.nblk, d.cplx);
  }
  L.tc = take(L.tc_bytes);
  L.vhs_bytes = W * N * N * C;
  // staging of at least one gamma: a host chunk's copy (binary64), its cast for the set-up GEMMs and
  // the chunk's Ltilde (binary64)
  // (complex: the chunk's copy, its two Hermitian fields and their Ltilde, all complex binary64)
  L.stage_bytes = d.cplx ? align_up(N * N * 16, 256) + align_up(2 * N * N * 16, 256) + align_up(2 * nc * N * 16, 256) + 1024
                         : align_up(N * N * 8, 256) * 2 + align_up(nc * N * 8, 256) + 1024;
  L.stage_bytes_avail = std::max(L.vhs_bytes, L.stage_bytes);
  L.vhs = take(L.stage_bytes_avail);
  L.stage = L.vhs;
  L.total = align_up(cur, 256);
  return L;
}

afqmc_status make_dims(int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta, const double* psiT,
                       const afqmc_params* p, Dims* d, bool cplx = false) {
  if (!p) return fail(AFQMC_EINVAL, "params is NULL");
  if (norb < 1 || naux < 1) return fail(AFQMC_EINVAL, "norb and naux must be >= 1 (got %d, %d)", norb, naux);
  if (nalpha < 1 || nbeta < 0 || nalpha > norb || nbeta > norb || nalpha > kMaxOcc || nbeta > kMaxOcc)
    return fail(AFQMC_EINVAL, "need 1 <= nalpha <= min(norb, %d), 0 <= nbeta <= min(norb, %d) (got %d, %d)",
                kMaxOcc, kMaxOcc, nalpha, nbeta);
  if (p->nwalkers < 1 || p->nwalkers > 65535) return fail(AFQMC_EINVAL, "nwalkers must be in [1, 65535]");
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(AFQMC_EINVAL, "dt must be positive and finite");
  if (p->taylor_order < 1 || p->taylor_order > 12) return fail(AFQMC_EINVAL, "taylor_order must be in [1, 12]");
  if (p->prec < AFQMC_PREC_FP64 || p->prec > AFQMC_PREC_BF16X3) return fail(AFQMC_EINVAL, "unknown prec %d", p->prec);
  if (p->reserved != 0) return fail(AFQMC_EINVAL, "params.reserved must be 0");
  if (!psiT) return fail(AFQMC_EINVAL, "psiT is NULL");
  if ((long long)norb * norb > (1ll << 31) / 2) return fail(AFQMC_EINVAL, "norb too large");
  if (cplx && (long long)naux * 2 > (1ll << 30)) return fail(AFQMC_EINVAL, "naux too large");
  d->N = norb; d->X = cplx ? 2 * naux : naux; d->na = nalpha; d->nb = nbeta; d->W = p->nwalkers; d->prec = p->prec;
  d->cplx = cplx;
  bool same = nalpha == nbeta;
  const int nt = nalpha + nbeta;
  const int e = cplx ? 2 : 1;   // doubles per trial entry
  for (int r = 0; same && r < norb; ++r)
    for (int c = 0; c < nalpha * e; ++c)
      if (psiT[((size_t)r * nt) * e + c] != psiT[((size_t)r * nt + nalpha) * e + c]) { same = false; break; }
  d->restricted = same;
  d->ncol = same ? nalpha : nt;
  d->nblk = (same || nbeta == 0) ? 1 : 2;
  d->c0[0] = 0; d->nbk[0] = nalpha;
  d->c0[1] = nalpha; d->nbk[1] = same ? 0 : nbeta;
  d->gchunk = 8;
  d->nchunk = (d->X + d->gchunk - 1) / d->gchunk;
  if (d->tensor()) {   // exchange partials come per (spin block, M tile) of the tensor-core kernel
    tc::TcState tmp;
    tc::plan(&tmp, d->prec, d->W, d->N, d->X, d->ncol, d->c0, d->nbk, d->nblk, cplx);
    d->nchunk = tmp.nchunk;
  }
  return AFQMC_OK;
}

// Host binary64 helpers for the set-up ------------------------------------------------
template <typename S>
bool invert_small(std::vector<S>& a, int n) {   // Gauss-Jordan with partial pivoting, in place
  std::vector<S> inv((size_t)n * n, S(0.0));
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = S(1.0);
  for (int k = 0; k < n; ++k) {
    int pv = k;
    for (int i = k + 1; i < n; ++i) if (std::abs(a[(size_t)i * n + k]) > std::abs(a[(size_t)pv * n + k])) pv = i;
    if (std::abs(a[(size_t)pv * n + k]) == 0.0) return false;
    for (int j = 0; j < n; ++j) { std::swap(a[(size_t)k * n + j], a[(size_t)pv * n + j]); std::swap(inv[(size_t)k * n + j], inv[(size_t)pv * n + j]); }
    const S d = a[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) { a[(size_t)k * n + j] /= d; inv[(size_t)k * n + j] /= d; }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const S f = a[(size_t)i * n + k];
      if (f == S(0.0)) continue;
      for (int j = 0; j < n; ++j) { a[(size_t)i * n + j] -= f * a[(size_t)k * n + j]; inv[(size_t)i * n + j] -= f * inv[(size_t)k * n + j]; }
    }
  }
  a = inv;
  return true;
}

inline double conj_s(double x) { return x; }
inline std::complex<double> conj_s(std::complex<double> x) { return std::conj(x); }

}  // namespace

struct afqmc_ctx {
  Dims d;
  Layout L;
  char* base;
  cudaStream_t stream;
  double dt, sdt, cap, ecore, e_c, e_var, e_trial, smul;
  int taylor;
  unsigned long long seed, host_step, launches;
  bool theta_fresh, vbias_fresh;
  int hist_used;
  // chunked set-up (afqmc_create_begin / afqmc_add_cholesky / afqmc_create_end)
  bool building = false;     // true until afqmc_create_end succeeds
  double e_trial_param = 0.0;   // params.e_trial (NaN: E_var once it is measured)
  int chol_next = 0;         // first gamma not passed yet
  bool setup_f32 = false;    // set-up GEMMs (sum L L, Ltilde) in binary32 (large problems, reduced forms)
  std::vector<double> h1e_host;
  // free projection (Section "Free projection AFQMC"): no force-bias shift, complex weights
  // w e^{i phi} (phases in L.wph), no phaseless projection and no comb
  bool free_proj = false;
  // E_T replaced at each comb by the running mixed estimate (device words L.etr)
  bool et_update = false;
  tc::TcState tcs;
  CvState cv;
  int tile_cap = 4;          // largest CUDA-core GEMM register tile (4: 64-wide block tiles, 2: 32, 1: 16)
  int prop_path = 0;         // 0: tensor cores (BF16 forms) else fused CUDA-core kernel where they fit,
                             // 1: batched GEMMs, 2: fused CUDA-core kernel
  int prop_tile = 0;         // fused propagation register tile: 0: 4 rows x 2 columns, 1: 8 x 2, 2: 4 x 4
  // CUDA graphs of the driver loop's step patterns (captured lazily on a private stream)
  bool graphs_on = true;
  cudaStream_t cap_stream = nullptr;
  // the energy estimator kernel runs on `side` beside the following step's fields, VHS and
  // propagation (it reads Theta, vbias, the exchange partials and the weights, which only the
  // step's overlap rewrites); the overlap joins it first
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool join_pending = false;
  // afqmc_run_async's per-measurement copies to the caller's host array run on `copy_stream`
  // (after each step graph, off the main stream; the main stream waits for them only before the
  // device history is reused and at the end of the call)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copy = nullptr, ev_copied = nullptr;
  // the tensor-core exchange draws the current step's normals into L.x with a spare warp (its
  // binary64 work overlaps the contraction); the next fields kernel uses them instead of drawing
  bool normals_pending = false;
  bool thb_valid = false;    // the bf16 Theta^T exchange operand (tensor forms) matches Theta^T
  cudaGraphExec_t g_step[8] = {};       // bit 0: energy measured, bit 1: Theta refreshed first,
  unsigned long long g_step_k[8] = {};  // bit 2: the energy reuses the bf16 Theta operand
  cudaGraphExec_t g_qr = nullptr, g_comb[2] = {};
  unsigned long long g_qr_k = 0, g_comb_k[2] = {};
  unsigned long long graph_gen = 0;   // bumped whenever captured launch parameters go stale
  void drop_graphs() {
    ++graph_gen;
    for (auto& g : g_step) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (auto& g : g_comb) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (g_qr) { cudaGraphExecDestroy(g_qr); g_qr = nullptr; }
  }
  // tracing
  bool prof = false;
  std::vector<cudaEvent_t> free_events;
  struct Pending { int stage; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  double stage_ms[AFQMC_NSTAGES] = {};
  long long stage_n[AFQMC_NSTAGES] = {};
  ~afqmc_ctx() {
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    if (ev_copy) cudaEventDestroy(ev_copy);
    if (ev_copied) cudaEventDestroy(ev_copied);
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : free_events) cudaEventDestroy(e);
  }
  cudaEvent_t take_event() {
    if (!free_events.empty()) { cudaEvent_t e = free_events.back(); free_events.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  void drain() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        stage_ms[p.stage] += ms;
        stage_n[p.stage] += 1;
      }
      free_events.push_back(p.a);
      free_events.push_back(p.b);
    }
    pending.clear();
  }
  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

namespace {

// Records a CUDA event pair around a stage when tracing is on.
struct StageTimer {
  afqmc_ctx* c;
  int id;
  cudaEvent_t a = nullptr;
  StageTimer(afqmc_ctx* ctx, int stage) : c(ctx), id(stage) {
    if (!c->prof) return;
    if (c->pending.size() > 4096) c->drain();
    a = c->take_event();
    if (a) cudaEventRecord(a, c->stream);
  }
  ~StageTimer() {
    if (!a) return;
    cudaEvent_t b = c->take_event();
    if (!b) { c->free_events.push_back(a); return; }
    cudaEventRecord(b, c->stream);
    c->pending.push_back({id, a, b});
  }
};

// --------------------------------------------------------------------------------------
template <typename R, bool CA, bool CB, int TM, int TN>
afqmc_status gemm_tiled(afqmc_ctx* c, const GemmDesc& g) {
  dim3 grid((g.Nc + 16 * TN - 1) / (16 * TN), (g.M + 16 * TM - 1) / (16 * TM), g.batch);
  if (grid.y > 65535 || grid.z > 65535) return fail(AFQMC_EINVAL, "GEMM grid too large");
  k_gemm<R, CA, CB, TM, TN><<<grid, 256, 0, c->stream>>>(g);
  CHECK_LAUNCH(c);
  return AFQMC_OK;
}

// Block tile picked from the output shape: 64-wide tiles for large dimensions, 32 or 16 for small
// ones, so that tiny or skinny batched products do not run mostly on padding.
template <typename R, bool CA, bool CB>
afqmc_status gemm(afqmc_ctx* c, const GemmDesc& g) {
  if (g.M <= 0 || g.Nc <= 0 || g.batch <= 0) return AFQMC_OK;
  int tm = std::min(c->tile_cap, g.M >= 48 ? 4 : (g.M > 16 ? 2 : 1));
  int tn = std::min(c->tile_cap, g.Nc >= 48 ? 4 : (g.Nc > 16 ? 2 : 1));
  auto ctas = [&](int a, int b) {
    return (long long)((g.M + 16 * a - 1) / (16 * a)) * ((g.Nc + 16 * b - 1) / (16 * b)) * g.batch;
  };
  while (ctas(tm, tn) < 148 && (tm > 1 || tn > 1)) {   // fill the SMs before using larger tiles
    if (tm >= tn) tm /= 2; else tn /= 2;
  }
  if (tm == 4 && tn == 1) tn = 2;
  if (tm == 4 && tn == 4) return gemm_tiled<R, CA, CB, 4, 4>(c, g);
  if (tm == 4) return gemm_tiled<R, CA, CB, 4, 2>(c, g);
  if (tm == 2 && tn == 4) return gemm_tiled<R, CA, CB, 2, 4>(c, g);
  if (tm == 2) return gemm_tiled<R, CA, CB, 2, 2>(c, g);
  if (tn >= 2) return gemm_tiled<R, CA, CB, 1, 4>(c, g);
  return gemm_tiled<R, CA, CB, 1, 1>(c, g);
}

GemmDesc gdesc(int M, int Nc, int K, int batch) {
  GemmDesc g{};
  g.M = M; g.Nc = Nc; g.K = K; g.batch = batch;
  g.alpha_re = 1.0;
  return g;
}

template <typename R>
OverlapArgs<R> overlap_args(afqmc_ctx* c, int mode) {
  OverlapArgs<R> a{};
  a.N = c->d.N; a.ncol = c->d.ncol; a.nblk = c->d.nblk;
  a.c0[0] = c->d.c0[0]; a.c0[1] = c->d.c0[1]; a.nb[0] = c->d.nbk[0]; a.nb[1] = c->d.nbk[1];
  a.smul = c->smul;
  a.psi = c->at<cplx_t<R>>(c->L.psi);
  a.phi = c->at<double>(c->L.phi);
  a.phi_r = c->at<R>(c->L.phi_r);
  a.phi_c = c->d.cplx ? c->at<cplx_t<R>>(c->L.phi_r) : nullptr;
  a.thetaT = c->at<cplx_t<R>>(c->L.thetaT);
  a.logO = c->at<double2>(c->L.logO);
  a.w = c->at<double>(c->L.w);
  a.status = c->at<int>(c->L.status);
  a.mode = mode;
  a.cmf = c->at<double2>(c->L.cmf);
  a.xxbar = c->at<double2>(c->L.xxbar);
  a.dt = c->dt; a.e_trial = c->e_trial; a.e_c = c->e_c;
  a.eshift = std::exp(c->dt * (c->e_trial - c->e_c));
  a.etr = (mode == 1 && c->et_update && !c->free_proj) ? c->at<double>(c->L.etr) : nullptr;
  a.step = mode == 1 ? c->at<unsigned long long>(c->L.step) : nullptr;
  a.wph = (mode == 1 && c->free_proj) ? c->at<double>(c->L.wph) : nullptr;
  for (int s = 0; s < 2; ++s)
    a.thb[s] = (c->d.tensor() && s < c->d.nblk && c->tcs.blk[s].n > 0)
                   ? reinterpret_cast<__nv_bfloat16*>(c->at<char>(c->L.tc) + c->tcs.blk[s].off_th)
                   : nullptr;
  a.kst = c->tcs.kst;
  a.nseg = c->tcs.nseg;
  a.kst0 = (c->d.cplx && c->d.tensor()) ? c->tcs.kst0 : 0;
  return a;
}

bool overlap_stage(const Dims& d) {
  const int nmax = std::max(d.nbk[0], d.nblk > 1 ? d.nbk[1] : 0);
  const size_t sm = d.prec == AFQMC_PREC_FP64 ? overlap_lu_smem<double>(d.N, nmax, true, d.cplx)
                                              : overlap_lu_smem<float>(d.N, nmax, true, d.cplx);
  return sm <= 100 * 1024;   // leaves room for two CTAs per SM
}
size_t overlap_smem(const Dims& d) {
  const int nmax = std::max(d.nbk[0], d.nblk > 1 ? d.nbk[1] : 0);
  const bool st = overlap_stage(d);
  return d.prec == AFQMC_PREC_FP64 ? overlap_lu_smem<double>(d.N, nmax, st, d.cplx)
                                   : overlap_lu_smem<float>(d.N, nmax, st, d.cplx);
}

bool qr_stage_psi(const Dims& d) {
  const int nmax = std::max(d.nbk[0], d.nblk > 1 ? d.nbk[1] : 0);
  return (d.prec == AFQMC_PREC_FP64 ? qr_smem_bytes<double>(d.N, nmax, true) : qr_smem_bytes<float>(d.N, nmax, true)) <=
         227 * 1024;
}
size_t qr_smem(const Dims& d) {
  const int nmax = std::max(d.nbk[0], d.nblk > 1 ? d.nbk[1] : 0);
  const bool st = qr_stage_psi(d);
  return d.prec == AFQMC_PREC_FP64 ? qr_smem_bytes<double>(d.N, nmax, st) : qr_smem_bytes<float>(d.N, nmax, st);
}

size_t prop_smem(const Dims& d) { return prop_smem_floats(d.N, d.ncol, nullptr, nullptr) * sizeof(float); }

bool use_fused_propagation(const Dims& d) {
  return d.prec != AFQMC_PREC_FP64 && !d.cplx && prop_smem(d) <= 227 * 1024;   // real E_h only
}

bool use_tc_propagation(const afqmc_ctx* c) { return c->d.tensor() && c->tcs.pg.ok && c->prop_path == 0; }

// The stream waits for an energy estimator launched beside it (no-op when none is pending).
afqmc_status join_energy(afqmc_ctx* c) {
  if (!c->join_pending) return AFQMC_OK;
  c->join_pending = false;
  CU(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  return AFQMC_OK;
}

template <typename R>
afqmc_status launch_overlap(afqmc_ctx* c, int mode) {
  afqmc_status js = join_energy(c);   // the overlap rewrites Theta and the weights the estimator reads
  if (js != AFQMC_OK) return js;
  StageTimer timer(c, AFQMC_STAGE_OVERLAP);
  const size_t sm = overlap_smem(c->d);
  const bool stg = overlap_stage(c->d);
  // psi and Phi that do not fit shared memory (large N) are read in place by a wide CTA per walker
  if (c->d.cplx) {
    if (stg) k_overlap_lu<R, true, true><<<c->d.W, 128, sm, c->stream>>>(overlap_args<R>(c, mode));
    else k_overlap_lu_wide<R, true><<<c->d.W, 512, sm, c->stream>>>(overlap_args<R>(c, mode));
  } else if (stg) {
    k_overlap_lu<R, true><<<c->d.W, 128, sm, c->stream>>>(overlap_args<R>(c, mode));
  } else {
    k_overlap_lu_wide<R><<<c->d.W, 512, sm, c->stream>>>(overlap_args<R>(c, mode));
  }
  c->thb_valid = c->d.tensor();
  CHECK_LAUNCH(c);
  return AFQMC_OK;
}

size_t exchange_smem(const Dims& d) {
  const size_t R = d.rsz();
  const int nmax = std::max(d.nbk[0], d.nblk > 1 ? d.nbk[1] : 0);
  const size_t cn = (size_t)d.ncol * d.N;
  return cn * 2 * R + (d.cplx ? 2 * cn : cn + (cn & 1)) * R + (size_t)nmax * nmax * 2 * R;
}

template <typename R>
afqmc_status launch_exchange(afqmc_ctx* c, int with_exchange, const int* widx = nullptr, int rows = -1) {
  ExchangeArgs<R> a{};
  a.N = c->d.N; a.X = c->d.X; a.ncol = c->d.ncol; a.nblk = c->d.nblk;
  a.c0[0] = c->d.c0[0]; a.c0[1] = c->d.c0[1]; a.nb[0] = c->d.nbk[0]; a.nb[1] = c->d.nbk[1];
  a.smul = c->smul; a.gchunk = c->d.gchunk; a.nchunk = c->d.nchunk;
  a.thetaT = c->at<cplx_t<R>>(c->L.thetaT);
  a.lrot = c->at<R>(c->L.lrot);
  a.lrot_c = c->d.cplx ? c->at<cplx_t<R>>(c->L.lrot) : nullptr;
  a.vbias = c->at<cplx_t<R>>(c->L.vbias);
  a.exch_part = c->at<double2>(c->L.exch_part);
  a.with_exchange = with_exchange;
  a.widx = widx;
  a.with_vbias = widx ? 0 : 1;
  dim3 grid(c->d.nchunk, rows < 0 ? c->d.W : rows);
  if (c->d.cplx) k_exchange<R, true><<<grid, 256, exchange_smem(c->d), c->stream>>>(a);
  else k_exchange<R><<<grid, 256, exchange_smem(c->d), c->stream>>>(a);
  CHECK_LAUNCH(c);
  return AFQMC_OK;
}

afqmc_status allow_max_dynamic_smem(const void* fn) {
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  CU(cudaFuncGetAttributes(&fa, fn));
  CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
  return AFQMC_OK;
}

template <typename R>
afqmc_status set_smem_limits(const Dims& d) {
  afqmc_status st_;
  const size_t ov = overlap_smem(d), ex = d.tensor() ? 0 : exchange_smem(d), qr = qr_smem(d);
  const size_t lim = 227 * 1024;
  if (ov > lim || ex > lim || qr > lim)
    return fail(AFQMC_EINVAL, "problem too large for the CUDA-core kernels' shared-memory staging "
                              "(overlap %zu, exchange %zu, qr %zu bytes > %zu)", ov, ex, qr, lim);
  // The attribute is per kernel, shared by every context in the process: allow the largest
  // dynamic size the device permits next to the kernel's static shared memory (each launch still
  // requests only its own size).
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu<R, true>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu<R, false>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_exchange<R>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_exchange<R, true>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu<R, true, true>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu<R, false, true>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_qr_chol<R>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_qr_chol_wide<R>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu_wide<R>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_lu_wide<R, true>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_propagate_smem<4, 2>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_propagate_smem<8, 2>))) != AFQMC_OK) return st_;
  if ((st_ = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_propagate_smem<4, 4>))) != AFQMC_OK) return st_;
  return AFQMC_OK;
}

// Local energy at the current walkers into eloc and the weighted sums into sums_dev.
template <typename R>
afqmc_status energy_cv_impl(afqmc_ctx* c, double* sums_dev, int* slot, bool run);

// run: a measurement of the run loop, which also feeds the running sums of E_T when it follows them.
template <typename R>
EnergyArgs<R> energy_args(afqmc_ctx* c, double* sums_dev, int* slot, bool run = false) {
  EnergyArgs<R> a{};
  a.N = c->d.N; a.X = c->d.X; a.ncol = c->d.ncol;
  a.smul = c->smul; a.ecore = c->ecore; a.nchunk = c->d.nchunk;
  a.thetaT = c->at<cplx_t<R>>(c->L.thetaT);
  a.hrot = c->at<void>(c->L.hrot_r);
  a.vbias = c->at<cplx_t<R>>(c->L.vbias);
  a.exch_part = c->at<double2>(c->L.exch_part);
  a.exch_part_f = c->d.tensor() ? c->at<float2>(c->L.exch_part) : nullptr;   // the tensor-core exchange's format
  a.eloc = c->at<double2>(c->L.eloc);
  a.W = c->d.W;
  a.wgt = c->at<double>(c->L.w);
  a.wph = c->free_proj ? c->at<double>(c->L.wph) : nullptr;
  a.out = sums_dev;
  a.slot = slot;
  a.done = reinterpret_cast<unsigned int*>(c->base + c->L.slot + 64);
  a.etacc = (run && c->et_update && !c->free_proj) ? c->at<double>(c->L.etr) : nullptr;
  return a;
}

// beside: a step follows at once, so the estimator kernel may run on the side stream until that
// step's overlap (not while stage timing is on, which times it on the main stream).
template <typename R>
afqmc_status energy_impl(afqmc_ctx* c, double* sums_dev, int* slot = nullptr, bool beside = false,
                         double* sums_host = nullptr, bool run = false) {
  if (c->cv.enabled) {
    afqmc_status sc = energy_cv_impl<R>(c, sums_dev, slot, run);
    if (sc == AFQMC_OK && sums_host)
      CU(cudaMemcpyAsync(sums_host, sums_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sc;
  }
  afqmc_status st;
  if (!c->theta_fresh) {
    if ((st = launch_overlap<R>(c, 2)) != AFQMC_OK) return st;
    c->theta_fresh = true;
  }
  StageTimer* tx = new StageTimer(c, AFQMC_STAGE_EXCHANGE);
  if (c->d.prec == AFQMC_PREC_BF16 || c->d.prec == AFQMC_PREC_BF16X3) {
    tc::NormalsJob nj{c->at<double>(c->L.x), c->seed, c->at<unsigned long long>(c->L.step), c->d.W, c->d.X};
    if ((st = tc::exchange(&c->tcs, c->stream, c->at<char>(c->L.tc), c->smul, c->at<float2>(c->L.thetaT),
                           c->at<float2>(c->L.vbias), c->at<float2>(c->L.exch_part), c->at<int>(c->L.status),
                           nullptr, c->d.W, &c->launches, g_err, sizeof(g_err), &nj, c->thb_valid)) != AFQMC_OK)
      return st;
    c->normals_pending = true;   // valid for the next step_impl while the step counter is unchanged
  } else {
    if ((st = launch_exchange<R>(c, 1)) != AFQMC_OK) return st;
  }
  delete tx;
  const bool fork = beside && !c->prof && c->side != nullptr;
  cudaStream_t es = c->stream;
  if (fork) {
    CU(cudaEventRecord(c->ev_fork, c->stream));
    CU(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    es = c->side;
  }
  StageTimer te(c, AFQMC_STAGE_ENERGY);
  auto kern = c->d.cplx ? k_energy<R, true> : k_energy<R, false>;
  kern<<<c->d.W, 256, 0, es>>>(energy_args<R>(c, sums_dev, slot, run));
  CHECK_LAUNCH(c);
  if (sums_host) CU(cudaMemcpyAsync(sums_host, sums_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, es));
  if (fork) {
    CU(cudaEventRecord(c->ev_join, c->side));
    c->join_pending = true;
  }
  c->vbias_fresh = true;
  return AFQMC_OK;
}

template <typename R>
FieldArgs<R> field_args(afqmc_ctx* c) {
  using R2 = cplx_t<R>;
  const Dims& d = c->d;
  FieldArgs<R> fa{};
  fa.X = d.X; fa.sdt = c->sdt; fa.cap = c->cap; fa.seed = c->seed;
  fa.step = c->at<unsigned long long>(c->L.step);
  fa.vbias = c->at<R2>(c->L.vbias); fa.lbar = c->at<double>(c->L.lbar); fa.slbar = c->at<double>(c->L.slbar);
  fa.x = c->at<double>(c->L.x); fa.xbar = c->at<double2>(c->L.xbar); fa.coef = c->at<R2>(c->L.coef);
  fa.cmf = c->at<double2>(c->L.cmf); fa.xxbar = c->at<double2>(c->L.xxbar);
  fa.free_proj = c->free_proj ? 1 : 0;
  if (d.tensor()) {
    fa.coefb = reinterpret_cast<__nv_bfloat16*>(c->at<char>(c->L.tc) + c->tcs.off_coef);
    fa.kx = c->tcs.kx;
    fa.nseg = c->tcs.nseg;
    fa.kx0 = d.cplx ? c->tcs.kx0 : 0;
  }
  return fa;
}

// Draws the current step's normals into L.x (unless the energy's tensor-core exchange already has).
afqmc_status draw_normals(afqmc_ctx* c) {
  const long long pairs = (long long)c->d.W * ((c->d.X + 1) / 2);
  const int grid = (int)std::max(1LL, std::min<long long>(1LL << 20, (pairs + 127) / 128));
  k_normals<<<grid, 128, 0, c->stream>>>(c->seed, c->at<unsigned long long>(c->L.step), c->d.W, c->d.X,
                                         c->at<double>(c->L.x));
  CHECK_LAUNCH(c);
  return AFQMC_OK;
}

template <typename R>
afqmc_status step_impl(afqmc_ctx* c) {
  afqmc_status st;
  const Dims& d = c->d;
  using R2 = cplx_t<R>;
  if (!c->theta_fresh) {
    if ((st = launch_overlap<R>(c, 2)) != AFQMC_OK) return st;
    c->theta_fresh = true;
  }
  if (!c->vbias_fresh && !c->free_proj) {   // free projection draws unshifted fields
    StageTimer timer(c, AFQMC_STAGE_FORCE_BIAS);
    {
      // vbias[w][g] = smul * sum_k thetaT[w][k] * lrot[g][k],  k = (c, p)
      GemmDesc g = gdesc(d.W, d.X, d.ncol * d.N, 1);
      g.A = c->at<R2>(c->L.thetaT); g.sAm = (long long)d.ncol * d.N; g.sAk = 1;
      g.B = c->at<R>(c->L.lrot); g.sBk = 1; g.sBn = (long long)d.ncol * d.N;
      g.C = c->at<R2>(c->L.vbias); g.sCm = d.X; g.sCn = 1;
      g.alpha_re = c->smul;
      if ((st = d.cplx ? gemm<R, true, true>(c, g) : gemm<R, true, false>(c, g)) != AFQMC_OK) return st;
    }
  }
  StageTimer* tf = new StageTimer(c, AFQMC_STAGE_FIELDS);
  if (!c->normals_pending && (st = draw_normals(c)) != AFQMC_OK) return st;
  c->normals_pending = false;
  k_fields<R><<<d.W, 256, 0, c->stream>>>(field_args<R>(c));
  delete tf;
  CHECK_LAUNCH(c);
  const long long NN = (long long)d.N * d.N, Nc = (long long)d.N * d.ncol;
  // VHS[w][pq] = sum_g coef[w][g] L[g][pq]
  StageTimer* tv = new StageTimer(c, AFQMC_STAGE_VHS);
  const bool tc_prop = use_tc_propagation(c);
  if (tc_prop) {   // bf16 hi/lo planes for the tensor-core propagation
    if ((st = tc::vhs_planes(&c->tcs, c->stream, c->at<char>(c->L.tc), c->at<float2>(c->L.coef),
                             c->at<int>(c->L.status), &c->launches, g_err, sizeof(g_err), true)) != AFQMC_OK)
      return st;
  } else if (d.tensor()) {   // planar fp32 output: VHS_w = vhs[w][0][:] + i vhs[w][1][:]
    if ((st = tc::vhs(&c->tcs, c->stream, c->at<char>(c->L.tc), c->at<float2>(c->L.coef), c->at<float>(c->L.vhs),
                      c->at<int>(c->L.status), &c->launches, g_err, sizeof(g_err))) != AFQMC_OK)
      return st;
  } else {
    GemmDesc g = gdesc(d.W, (int)NN, d.X, 1);
    g.A = c->at<R2>(c->L.coef); g.sAm = d.X; g.sAk = 1;
    g.B = c->at<R>(c->L.chol); g.sBk = NN; g.sBn = 1;
    g.C = c->at<R2>(c->L.vhs); g.sCm = NN; g.sCn = 1;
    if ((st = d.cplx ? gemm<R, true, true>(c, g) : gemm<R, true, false>(c, g)) != AFQMC_OK) return st;
  }
  delete tv;
  // psi <- E_h Taylor(VHS) E_h psi   (tA = accumulator, tB/tC = Taylor terms)
  const double* skip = c->at<double>(c->L.w);
  StageTimer* tp = new StageTimer(c, AFQMC_STAGE_PROPAGATE);
  if (tc_prop) {
    if ((st = tc::propagate(&c->tcs, c->stream, c->at<char>(c->L.tc), c->taylor, c->at<float2>(c->L.psi), skip,
                            c->at<int>(c->L.status), &c->launches, g_err, sizeof(g_err))) != AFQMC_OK)
      return st;
    delete tp;
    if ((st = launch_overlap<R>(c, 1)) != AFQMC_OK) return st;
    c->theta_fresh = true;
    c->vbias_fresh = false;
    c->host_step++;
    return AFQMC_OK;
  }
  if (use_fused_propagation(d) && c->prop_path != 1) {
    PropArgs pa{};
    pa.N = d.N; pa.ncol = d.ncol; pa.order = c->taylor;
    prop_smem_floats(d.N, d.ncol, &pa.ldv, &pa.ldc);
    pa.eh = c->at<float>(c->L.eh);
    pa.vhs = c->base + c->L.vhs;
    pa.planar = d.tensor() ? 1 : 0;
    pa.psi = c->at<float2>(c->L.psi);
    pa.w = skip;
    pa.W = d.W;
    pa.status = c->at<int>(c->L.status);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tm = c->prop_tile == 1 ? 8 : 4, tcw = c->prop_tile == 2 ? 4 : 2;
    const int tiles = ((d.N + tm - 1) / tm) * (pa.ldc / tcw);
    const int threads = std::min(512, std::max(64, (tiles + 31) / 32 * 32));
    const int grid = std::min(d.W, sms);
    if (c->prop_tile == 1) k_propagate_smem<8, 2><<<grid, threads, prop_smem(d), c->stream>>>(pa);
    else if (c->prop_tile == 2) k_propagate_smem<4, 4><<<grid, threads, prop_smem(d), c->stream>>>(pa);
    else k_propagate_smem<4, 2><<<grid, threads, prop_smem(d), c->stream>>>(pa);
    delete tp;
    CHECK_LAUNCH(c);
    if ((st = launch_overlap<R>(c, 1)) != AFQMC_OK) return st;
    c->theta_fresh = true;
    c->vbias_fresh = false;
    c->host_step++;
    return AFQMC_OK;
  }
  {
    GemmDesc g = gdesc(d.N, d.ncol, d.N, d.W);
    g.A = c->at<R>(c->L.eh); g.sAb = 0; g.sAm = d.N; g.sAk = 1;
    g.B = c->at<R2>(c->L.psi); g.sBb = Nc; g.sBk = d.ncol; g.sBn = 1;
    g.C = c->at<R2>(c->L.tB); g.sCb = Nc; g.sCm = d.ncol; g.sCn = 1;
    g.D = c->at<R2>(c->L.tA); g.sDb = Nc; g.sDm = d.ncol; g.sDn = 1; g.d_add = 0;
    g.skip = skip;
    if ((st = d.cplx ? gemm<R, true, true>(c, g) : gemm<R, false, true>(c, g)) != AFQMC_OK) return st;
  }
  size_t tin = c->L.tB, tout = c->L.tC;
  for (int k = 1; k <= c->taylor; ++k) {
    GemmDesc g = gdesc(d.N, d.ncol, d.N, d.W);
    g.A = c->at<R2>(c->L.vhs); g.sAb = NN; g.sAm = d.N; g.sAk = 1;
    if (d.tensor()) { g.a_planar = 1; g.a_im_off = NN; g.sAb = 2 * NN; }
    g.B = c->at<R2>(tin); g.sBb = Nc; g.sBk = d.ncol; g.sBn = 1;
    g.C = k < c->taylor ? c->at<R2>(tout) : nullptr; g.sCb = Nc; g.sCm = d.ncol; g.sCn = 1;
    g.D = c->at<R2>(c->L.tA); g.sDb = Nc; g.sDm = d.ncol; g.sDn = 1; g.d_add = 1;
    g.alpha_re = 1.0 / k;
    g.skip = skip;
    if ((st = gemm<R, true, true>(c, g)) != AFQMC_OK) return st;
    std::swap(tin, tout);
  }
  {
    GemmDesc g = gdesc(d.N, d.ncol, d.N, d.W);
    g.A = c->at<R>(c->L.eh); g.sAb = 0; g.sAm = d.N; g.sAk = 1;
    g.B = c->at<R2>(c->L.tA); g.sBb = Nc; g.sBk = d.ncol; g.sBn = 1;
    g.C = c->at<R2>(c->L.psi); g.sCb = Nc; g.sCm = d.ncol; g.sCn = 1;
    g.skip = skip;
    if ((st = d.cplx ? gemm<R, true, true>(c, g) : gemm<R, false, true>(c, g)) != AFQMC_OK) return st;
  }
  delete tp;
  if ((st = launch_overlap<R>(c, 1)) != AFQMC_OK) return st;
  c->theta_fresh = true;
  c->vbias_fresh = false;
  c->host_step++;
  return AFQMC_OK;
}

template <typename R>
QrArgs<R> qr_args(afqmc_ctx* c) {
  const Dims& d = c->d;
  return QrArgs<R>{d.N, d.ncol, d.nblk, d.c0[0], d.nbk[0], d.c0[1], d.nbk[1], c->smul,
                   c->at<cplx_t<R>>(c->L.psi), c->at<double2>(c->L.logO), c->at<double>(c->L.w),
                   c->at<int>(c->L.status), qr_stage_psi(d) ? 1 : 0};
}

template <typename R>
afqmc_status qr_impl(afqmc_ctx* c) {
  const Dims& d = c->d;
  StageTimer timer(c, AFQMC_STAGE_QR);
  if (qr_stage_psi(d)) k_qr_chol<R><<<d.W, 256, qr_smem(d), c->stream>>>(qr_args<R>(c));
  else k_qr_chol_wide<R><<<d.W, 1024, qr_smem(d), c->stream>>>(qr_args<R>(c));   // psi read in place (large N)
  CHECK_LAUNCH(c);
  // Theta = psi (Phi^T psi)^-1 is unchanged by psi -> psi R^-1 (Phi^T psi picks up the same R^-1),
  // so Theta, its bf16 copy and the force bias stay valid; log O was updated by -sum log R_ii.
  return AFQMC_OK;
}

template <typename R>
afqmc_status comb_impl(afqmc_ctx* c) {
  const Dims& d = c->d;
  using R2 = cplx_t<R>;
  if (c->free_proj) return fail(AFQMC_EINVAL, "population control is not part of free projection");
  StageTimer timer(c, AFQMC_STAGE_COMB);
  k_comb_plan<<<1, 256, 0, c->stream>>>(d.W, c->seed, c->at<unsigned long long>(c->L.step), c->at<double>(c->L.w),
                                        c->at<double>(c->L.cum), c->at<int>(c->L.src), c->at<double>(c->L.neww),
                                        c->at<int>(c->L.status), c->et_update ? c->at<double>(c->L.etr) : nullptr);
  CHECK_LAUNCH(c);
  const int pe = d.N * d.ncol;
  if (!c->theta_fresh) {
    afqmc_status st = launch_overlap<R>(c, 2);
    if (st != AFQMC_OK) return st;
    c->theta_fresh = true;
  }
  k_comb_gather<R><<<d.W, 256, 0, c->stream>>>(d.W, pe, pe, c->at<int>(c->L.src), c->at<double>(c->L.neww),
                                               c->at<R2>(c->L.psi), c->at<R2>(c->L.psi_tmp), c->at<R2>(c->L.thetaT),
                                               c->at<R2>(c->L.th_tmp), c->at<double2>(c->L.logO),
                                               c->at<double2>(c->L.logO_tmp), c->at<double>(c->L.w),
                                               c->at<double>(c->L.w_tmp));
  CHECK_LAUNCH(c);
  const size_t pb = (size_t)d.W * pe * sizeof(R2);
  CU(cudaMemcpyAsync(c->base + c->L.psi, c->base + c->L.psi_tmp, pb, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->base + c->L.thetaT, c->base + c->L.th_tmp, pb, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->base + c->L.logO, c->base + c->L.logO_tmp, d.W * 16, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->base + c->L.w, c->base + c->L.w_tmp, d.W * 8, cudaMemcpyDeviceToDevice, c->stream));
  c->vbias_fresh = false;
  c->thb_valid = false;   // the gather reordered Theta^T, not its bf16 copy
  return AFQMC_OK;
}

afqmc_status read_status(afqmc_ctx* c) {
  int st = 0;
  CU(cudaMemcpyAsync(&st, c->base + c->L.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (st == 0) return AFQMC_OK;
  CU(cudaMemsetAsync(c->base + c->L.status, 0, sizeof(int), c->stream));
  if (st & kStatusTimeout) return fail(AFQMC_ETIMEOUT, "a kernel gave up waiting for an asynchronous copy or tensor-core operation (bounded wait)");
  if (st & kStatusNoWalkers) return fail(AFQMC_ENOWALKERS, "all walker weights are zero");
  if (st & kStatusNonFinite) return fail(AFQMC_ENONFINITE, "a walker weight became non-finite (set to 0)");
  return fail(AFQMC_ESINGULAR, "a walker overlap matrix was singular (weight set to 0)");
}

#define DISPATCH(ctx, fn, ...)                                                      \
  ((ctx)->d.prec == AFQMC_PREC_FP64 ? fn<double>(ctx, ##__VA_ARGS__) : fn<float>(ctx, ##__VA_ARGS__))

// ---- chunked set-up ----------------------------------------------------------------------
// begin: trial quantities (host, O(N^2 n)), zeroed accumulators on the device.  S is the host scalar
// of the Hamiltonian (double, or std::complex<double> for a complex one, whose arrays are
// interleaved (re, im) pairs).
template <typename R, typename S>
afqmc_status setup_begin_s(afqmc_ctx* c, const double* h1e_d, const double* psiT_d) {
  const Dims& d = c->d;
  const int N = d.N, nc = d.ncol, nt = d.na + d.nb;
  const S* h1e = reinterpret_cast<const S*>(h1e_d);
  const S* psiT = reinterpret_cast<const S*>(psiT_d);
  afqmc_status st;
  if ((st = set_smem_limits<R>(d)) != AFQMC_OK) return st;
  c->h1e_host.assign(h1e_d, h1e_d + (size_t)N * N * d.cm());
  // trial columns that are stored (restricted: alpha only)
  std::vector<S> phi((size_t)N * nc);
  for (int p = 0; p < N; ++p)
    for (int col = 0; col < nc; ++col) phi[(size_t)p * nc + col] = psiT[(size_t)p * nt + col];
  // P = sum_s Phi_s (Phi_s^+ Phi_s)^-1 Phi_s^+ over both spins
  std::vector<S> P((size_t)N * N, S(0.0));
  for (int s = 0; s < 2; ++s) {
    const int off = s == 0 ? 0 : d.na, n = s == 0 ? d.na : d.nb;
    if (n == 0) continue;
    std::vector<S> Sm((size_t)n * n, S(0.0));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        S acc(0.0);
        for (int p = 0; p < N; ++p) acc += conj_s(psiT[(size_t)p * nt + off + i]) * psiT[(size_t)p * nt + off + j];
        Sm[(size_t)i * n + j] = acc;
      }
    if (!invert_small(Sm, n)) return fail(AFQMC_EINVAL, "trial orbitals of spin %d are linearly dependent", s);
    std::vector<S> tmp((size_t)N * n, S(0.0));   // Phi S^-1
    for (int p = 0; p < N; ++p)
      for (int j = 0; j < n; ++j) {
        S acc(0.0);
        for (int i = 0; i < n; ++i) acc += psiT[(size_t)p * nt + off + i] * Sm[(size_t)i * n + j];
        tmp[(size_t)p * n + j] = acc;
      }
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < N; ++q) {
        S acc(0.0);
        for (int j = 0; j < n; ++j) acc += tmp[(size_t)p * n + j] * conj_s(psiT[(size_t)q * nt + off + j]);
        P[(size_t)p * N + q] += acc;
      }
  }
  // htilde = Phi^+ h  [nc][N]
  std::vector<S> hrot((size_t)nc * N, S(0.0));
  for (int col = 0; col < nc; ++col)
    for (int p = 0; p < N; ++p) {
      const S f = conj_s(phi[(size_t)p * nc + col]);
      if (f == S(0.0)) continue;
      for (int q = 0; q < N; ++q) hrot[(size_t)col * N + q] += f * h1e[(size_t)p * N + q];
    }
  CU(cudaMemcpyAsync(c->base + c->L.phi, phi.data(), phi.size() * sizeof(S), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->base + c->L.hrot, hrot.data(), hrot.size() * sizeof(S), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->base + c->L.pden, P.data(), P.size() * sizeof(S), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemsetAsync(c->base + c->L.msum, 0, (size_t)N * N * sizeof(S), c->stream));
  CU(cudaMemsetAsync(c->base + c->L.lsum, 0, (size_t)N * N * sizeof(S), c->stream));
  CU(cudaMemsetAsync(c->base + c->L.sflag, 0, 256, c->stream));
  const size_t cm = d.cm();
  k_convert<R><<<64, 256, 0, c->stream>>>((size_t)N * nc * cm, c->at<double>(c->L.phi), c->at<R>(c->L.phi_r));
  CHECK_LAUNCH(c);
  k_convert<R><<<64, 256, 0, c->stream>>>((size_t)N * nc * cm, c->at<double>(c->L.hrot), c->at<R>(c->L.hrot_r));
  CHECK_LAUNCH(c);
  // binary32 set-up GEMMs where binary64 would take seconds (reduced forms only): their rounding,
  // ~1e-7 relative per sum, stays far below the forms' own
  const double flops = 2.0 * d.X * (double)N * N * N * cm * cm + 2.0 * d.X * (double)nc * N * N * cm * cm;
  c->setup_f32 = d.prec != AFQMC_PREC_FP64 && flops > 4e11;
  if (d.tensor()) {
    tc::plan(&c->tcs, d.prec, d.W, N, d.X, nc, d.c0, d.nbk, d.nblk, d.cplx);
    if ((st = tc::begin(&c->tcs, c->stream, c->at<char>(c->L.tc), g_err, sizeof(g_err))) != AFQMC_OK) return st;
  }
  // the synchronisation keeps the host vectors alive until their copies are done
  CU(cudaStreamSynchronize(c->stream));
  return AFQMC_OK;
}

template <typename R>
afqmc_status setup_begin(afqmc_ctx* c, const double* h1e, const double* psiT) {
  return c->d.cplx ? setup_begin_s<R, std::complex<double>>(c, h1e, psiT) : setup_begin_s<R, double>(c, h1e, psiT);
}

// One sub-chunk of gammas [g0, g0 + ng) already on the device (src, type T): checks, lbar, the
// accumulators, Ltilde, and the working-precision / tensor-core copies of L.
template <typename R, typename T, typename G>
afqmc_status setup_chunk(afqmc_ctx* c, int g0, int ng, const T* src, char* scratch) {
  const Dims& d = c->d;
  const int N = d.N, nc = d.ncol;
  const size_t NN = (size_t)N * N;
  afqmc_status st;
  k_chol_check<T><<<592, 256, 0, c->stream>>>(ng, N, src, c->at<int>(c->L.sflag));
  CHECK_LAUNCH(c);
  double* lbar = c->at<double>(c->L.lbar) + g0;
  k_chunk_lbar<T><<<ng, 256, 0, c->stream>>>(N, src, c->at<double>(c->L.pden), lbar);
  CHECK_LAUNCH(c);
  k_chunk_lsum<T><<<(unsigned)std::min<size_t>(4 * 148, (NN + 255) / 256), 256, 0, c->stream>>>(
      ng, NN, src, lbar, c->at<double>(c->L.lsum));
  CHECK_LAUNCH(c);
  // the chunk in the GEMM type
  const G* sg;
  char* cur = scratch;
  if (std::is_same<T, G>::value) {
    sg = reinterpret_cast<const G*>(src);
  } else {
    G* cast = reinterpret_cast<G*>(cur);
    cur += align_up((size_t)ng * NN * sizeof(G), 256);
    k_cast<T, G><<<592, 256, 0, c->stream>>>((size_t)ng * NN, src, cast);
    CHECK_LAUNCH(c);
    sg = cast;
  }
  {   // msum += sum_g L^g L^g = B^T B with B the chunk viewed as [ng N][N] (L^g symmetric)
    GemmDesc g = gdesc(N, N, ng * N, 1);
    g.A = sg; g.sAm = 1; g.sAk = N;
    g.B = sg; g.sBk = N; g.sBn = 1;
    if (std::is_same<G, double>::value) {
      g.D = c->at<double>(c->L.msum); g.sDm = N; g.sDn = 1; g.d_add = 1;
      if ((st = gemm<G, false, false>(c, g)) != AFQMC_OK) return st;
    } else {   // binary32 partial sum of the chunk, added into the binary64 total
      g.C = c->at<G>(c->L.e1); g.sCm = N; g.sCn = 1;
      if ((st = gemm<G, false, false>(c, g)) != AFQMC_OK) return st;
      k_add_f32_to_f64<<<592, 256, 0, c->stream>>>(NN, c->at<float>(c->L.e1), c->at<double>(c->L.msum));
      CHECK_LAUNCH(c);
    }
  }
  G* lrot = reinterpret_cast<G*>(cur);
  {   // Ltilde[g] = Phi^T L^g  ([nc][N] per gamma)
    GemmDesc g = gdesc(nc, N, N, ng);
    g.A = std::is_same<G, double>::value ? c->at<void>(c->L.phi) : c->at<void>(c->L.phi_r);
    g.sAb = 0; g.sAm = 1; g.sAk = nc;
    g.B = sg; g.sBb = (long long)NN; g.sBk = N; g.sBn = 1;
    g.C = lrot; g.sCb = (long long)nc * N; g.sCm = N; g.sCn = 1;
    if ((st = gemm<G, false, false>(c, g)) != AFQMC_OK) return st;
  }
  k_cast<G, R><<<592, 256, 0, c->stream>>>((size_t)ng * nc * N, lrot, c->at<R>(c->L.lrot) + (size_t)g0 * nc * N);
  CHECK_LAUNCH(c);
  if (d.tensor()) {
    if ((st = tc::load_chunk<T, G>(&c->tcs, c->stream, c->at<char>(c->L.tc), g0, ng, src, lrot, &c->launches, g_err,
                                   sizeof(g_err))) != AFQMC_OK)
      return st;
  } else {
    k_cast<T, R><<<592, 256, 0, c->stream>>>((size_t)ng * NN, src, c->at<R>(c->L.chol) + (size_t)g0 * NN);
    CHECK_LAUNCH(c);
  }
  return AFQMC_OK;
}

// Complex Hamiltonian: one sub-chunk of complex Cholesky vectors [g0, g0 + ng) (src, interleaved
// (re, im) of type T) becomes the Hermitian fields 2 g0 .. 2 (g0 + ng) - 1; their lbar, sums, Ltilde
// and working-precision copies as in setup_chunk, with complex GEMMs (M^g Hermitian, so
// sum M M = sum M^+ M, and Ltilde = Phi^+ M).
template <typename R, typename T, typename G>
afqmc_status setup_chunk_c(afqmc_ctx* c, int g0, int ng, const T* src, char* scratch) {
  using G2 = cplx_t<G>;
  const Dims& d = c->d;
  const int N = d.N, nc = d.ncol, nf = 2 * ng, f0 = 2 * g0;
  const size_t NN = (size_t)N * N;
  afqmc_status st;
  k_chol_check_c<T><<<592, 256, 0, c->stream>>>(ng, N, src, c->at<int>(c->L.sflag));
  CHECK_LAUNCH(c);
  G* fields = reinterpret_cast<G*>(scratch);
  char* cur = scratch + align_up((size_t)nf * NN * 2 * sizeof(G), 256);
  k_hermitian_fields<T, G><<<592, 256, 0, c->stream>>>(ng, N, src, fields);
  CHECK_LAUNCH(c);
  double* lbar = c->at<double>(c->L.lbar) + f0;
  k_chunk_lbar_c<G><<<nf, 256, 0, c->stream>>>(N, fields, c->at<double>(c->L.pden), lbar);
  CHECK_LAUNCH(c);
  // lsum += sum_f lbar_f M^f: lbar is real, so the interleaved arrays are summed as real ones
  k_chunk_lsum<G><<<(unsigned)std::min<size_t>(4 * 148, (2 * NN + 255) / 256), 256, 0, c->stream>>>(
      nf, 2 * NN, fields, lbar, c->at<double>(c->L.lsum));
  CHECK_LAUNCH(c);
  {   // msum += sum_f M^f+ M^f = B^+ B with B the fields viewed as [nf N][N]
    GemmDesc g = gdesc(N, N, nf * N, 1);
    g.A = fields; g.sAm = 1; g.sAk = N; g.conj_a = 1;
    g.B = fields; g.sBk = N; g.sBn = 1;
    if (std::is_same<G, double>::value) {
      g.D = c->at<double2>(c->L.msum); g.sDm = N; g.sDn = 1; g.d_add = 1;
      if ((st = gemm<G, true, true>(c, g)) != AFQMC_OK) return st;
    } else {
      g.C = c->at<G2>(c->L.e1); g.sCm = N; g.sCn = 1;
      if ((st = gemm<G, true, true>(c, g)) != AFQMC_OK) return st;
      k_add_f32_to_f64<<<592, 256, 0, c->stream>>>(2 * NN, c->at<float>(c->L.e1), c->at<double>(c->L.msum));
      CHECK_LAUNCH(c);
    }
  }
  G2* lrot = reinterpret_cast<G2*>(cur);
  {   // Ltilde[f] = Phi^+ M^f  ([nc][N] per field)
    GemmDesc g = gdesc(nc, N, N, nf);
    g.A = std::is_same<G, double>::value ? c->at<void>(c->L.phi) : c->at<void>(c->L.phi_r);
    g.sAb = 0; g.sAm = 1; g.sAk = nc; g.conj_a = 1;
    g.B = fields; g.sBb = (long long)NN; g.sBk = N; g.sBn = 1;
    g.C = lrot; g.sCb = (long long)nc * N; g.sCm = N; g.sCn = 1;
    if ((st = gemm<G, true, true>(c, g)) != AFQMC_OK) return st;
  }
  k_cast<G, R><<<592, 256, 0, c->stream>>>((size_t)nf * nc * N * 2, reinterpret_cast<const G*>(lrot),
                                            c->at<R>(c->L.lrot) + (size_t)f0 * nc * N * 2);
  CHECK_LAUNCH(c);
  if (d.tensor())   // the realified bf16 operands of the exchange and the VHS build
    return tc::load_chunk_c<G>(&c->tcs, c->stream, c->at<char>(c->L.tc), f0, nf, fields,
                               reinterpret_cast<const G*>(lrot), &c->launches, g_err, sizeof(g_err));
  k_cast<G, R><<<592, 256, 0, c->stream>>>((size_t)nf * NN * 2, fields, c->at<R>(c->L.chol) + (size_t)f0 * NN * 2);
  CHECK_LAUNCH(c);
  return AFQMC_OK;
}

// Host-side check of a host chunk (before it is copied): finite entries, symmetric L^g.  One pass
// over the upper triangle of each L^g, the vectors split over host threads; the first bad vector
// (in gamma order) is reported.
template <typename T>
afqmc_status check_host_chunk(int g0, int ng, int N, const T* chol) {
  const size_t NN = (size_t)N * N;
  auto bad_in = [&](int g, int* kind, int* bp, int* bq) {
    const T* Lg = chol + (size_t)g * NN;
    for (int p = 0; p < N; ++p) {
      if (!std::isfinite((double)Lg[(size_t)p * N + p])) { *kind = 1; *bp = p; *bq = p; return true; }
      for (int q = p + 1; q < N; ++q) {
        const double v = Lg[(size_t)p * N + q], u = Lg[(size_t)q * N + p];
        if (!std::isfinite(v) || !std::isfinite(u)) { *kind = 1; *bp = p; *bq = q; return true; }
        if (std::fabs(v - u) > 1e-12 * std::max(1.0, std::max(std::fabs(v), std::fabs(u)))) {
          *kind = 2; *bp = p; *bq = q; return true;
        }
      }
    }
    return false;
  };
  const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  const int per = (ng + nth - 1) / nth;
  std::vector<int> first(nth, -1), kinds(nth, 0), ps(nth, 0), qs(nth, 0);
  auto work = [&](int t) {
    for (int g = t * per; g < std::min(ng, (t + 1) * per); ++g)
      if (bad_in(g, &kinds[t], &ps[t], &qs[t])) { first[t] = g; return; }
  };
  if ((size_t)ng * NN < ((size_t)1 << 20) || nth == 1) {
    work(0);
    for (int t = 1; t < nth; ++t) work(t);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  for (int t = 0; t < nth; ++t) {
    if (first[t] < 0) continue;
    const int g = g0 + first[t];
    if (kinds[t] == 1) return fail(AFQMC_EINVAL, "chol has a non-finite entry (vector %d, %d, %d)", g, ps[t], qs[t]);
    return fail(AFQMC_EINVAL, "chol[%d] is not symmetric at (%d, %d)", g, ps[t], qs[t]);
  }
  return AFQMC_OK;
}

// Gammas [g0, g0 + ng) from host or device memory, in sub-chunks that fit the staging region.
template <typename R, typename T>
afqmc_status setup_add(afqmc_ctx* c, int g0, int ng, const T* chol, bool on_device, bool host_checked) {
  const Dims& d = c->d;
  const size_t NN = (size_t)d.N * d.N * d.cm();   // T elements per vector (complex: interleaved)
  const size_t per = d.cplx ? (on_device ? 0 : align_up(NN * sizeof(T), 256)) + align_up(2 * NN * 8, 256) +
                                  align_up((size_t)2 * d.ncol * d.N * 16, 256)
                            : (on_device ? 0 : align_up(NN * sizeof(T), 256)) + align_up(NN * 8, 256) +
                                  align_up((size_t)d.ncol * d.N * 8, 256);
  // 1024 bytes of slack cover the 256-byte alignment of the three staged arrays
  const size_t cap = std::max<size_t>(1, (c->L.stage_bytes_avail - 1024) / per);
  for (int a = 0; a < ng; a += (int)cap) {
    const int n = (int)std::min<size_t>(cap, (size_t)(ng - a));
    const T* part = chol + (size_t)a * NN;
    char* scratch = c->base + c->L.stage;
    const T* src = part;
    if (!on_device) {
      afqmc_status st;
      if (!d.cplx && !host_checked && (st = check_host_chunk<T>(g0 + a, n, d.N, part)) != AFQMC_OK) return st;
      T* dst = reinterpret_cast<T*>(scratch);
      CU(cudaMemcpyAsync(dst, part, (size_t)n * NN * sizeof(T), cudaMemcpyHostToDevice, c->stream));
      scratch += align_up((size_t)n * NN * sizeof(T), 256);
      src = dst;
    }
    afqmc_status st = d.cplx ? (c->setup_f32 ? setup_chunk_c<R, T, float>(c, g0 + a, n, src, scratch)
                                             : setup_chunk_c<R, T, double>(c, g0 + a, n, src, scratch))
                             : (c->setup_f32 ? setup_chunk<R, T, float>(c, g0 + a, n, src, scratch)
                                             : setup_chunk<R, T, double>(c, g0 + a, n, src, scratch));
    if (st != AFQMC_OK) return st;
    // the staging region is reused by the next sub-chunk (stream order), and a host chunk's
    // pageable source must stay readable until its copy is done
    if (!on_device) CU(cudaStreamSynchronize(c->stream));
  }
  // the caller may free or reuse a device chunk once the call returns
  if (on_device) CU(cudaStreamSynchronize(c->stream));
  return AFQMC_OK;
}

// end: h_eff, exp(-dt/2 h_eff), the mean-field constants, operand descriptors, walkers, E_var.
template <typename R>
afqmc_status setup_end(afqmc_ctx* c) {
  const Dims& d = c->d;
  const int N = d.N, X = d.X, nc = d.ncol;
  const size_t NN = (size_t)N * N;
  afqmc_status st;
  int flags = 0;
  CU(cudaMemcpyAsync(&flags, c->base + c->L.sflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> lbar(X);
  CU(cudaMemcpyAsync(lbar.data(), c->base + c->L.lbar, (size_t)X * 8, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (flags & kSetupNonFinite) return fail(AFQMC_EINVAL, "chol has a non-finite entry");
  if (flags & kSetupAsymmetric) return fail(AFQMC_EINVAL, "chol is not symmetric");
  double l2 = 0.0;
  for (int g = 0; g < X; ++g) l2 += lbar[g] * lbar[g];
  c->e_c = c->ecore - 0.5 * l2;
  std::vector<double> slbar(X);   // sqrt(dt) lbar for the fields kernel
  for (int g = 0; g < X; ++g) slbar[g] = c->sdt * lbar[g];
  CU(cudaMemcpyAsync(c->base + c->L.slbar, slbar.data(), slbar.size() * 8, cudaMemcpyHostToDevice, c->stream));
  // A = -dt/2 h_eff (e1), from h (e2)
  double* A = c->at<double>(c->L.e1);
  double* H = c->at<double>(c->L.e2);
  const bool cx = d.cplx;
  CU(cudaMemcpyAsync(H, c->h1e_host.data(), NN * 8 * d.cm(), cudaMemcpyHostToDevice, c->stream));
  const unsigned eg = (unsigned)std::min<size_t>(4 * 148, (NN + 255) / 256);
  if (cx) k_heff_c<<<eg, 256, 0, c->stream>>>(N, -0.5 * c->dt, H, c->at<double>(c->L.msum), c->at<double>(c->L.lsum), A);
  else k_heff<<<eg, 256, 0, c->stream>>>(N, -0.5 * c->dt, H, c->at<double>(c->L.msum), c->at<double>(c->L.lsum), A);
  CHECK_LAUNCH(c);
  double* dnorm = c->at<double>(c->L.sflag) + 8;
  if (cx) k_norm1_c<<<1, 1024, 0, c->stream>>>(N, A, dnorm);
  else k_norm1<<<1, 1024, 0, c->stream>>>(N, A, dnorm);
  CHECK_LAUNCH(c);
  double norm = 0.0;
  CU(cudaMemcpyAsync(&norm, dnorm, 8, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));   // also ends the uses of slbar and h1e_host
  if (!std::isfinite(norm)) return fail(AFQMC_EINVAL, "h_eff is not finite");
  // exp(A) = (exp(A / 2^s))^(2^s), ||A|| / 2^s <= 1/4, Taylor to degree m in Horner form
  int sq = 0;
  while (norm / std::ldexp(1.0, sq) > 0.25) ++sq;
  const double sc = std::ldexp(1.0, -sq), theta = norm * sc;
  int m = 2;
  {
    double term = theta * theta / 2.0;   // theta^(m+1) / (m+1)! for the first omitted term
    term = term * theta / 3.0;
    while (term > 5e-18 && m < 30) { ++m; term = term * theta / (m + 1); }
  }
  double* T = c->at<double>(c->L.msum);   // sum L L and lsum are no longer needed
  double* Tn = c->at<double>(c->L.lsum);
  auto idplus = [&](double alpha, double diag, const double* B, double* out) -> afqmc_status {
    if (cx) k_identity_plus_c<<<eg, 256, 0, c->stream>>>(N, alpha, diag, B, out);
    else k_identity_plus<<<eg, 256, 0, c->stream>>>(N, alpha, diag, B, out);
    CHECK_LAUNCH(c);
    return AFQMC_OK;
  };
  auto mm = [&](const double* X1, const double* X2, double* out, double alpha) -> afqmc_status {
    GemmDesc g = gdesc(N, N, N, 1);
    g.A = X1; g.sAm = N; g.sAk = 1;
    g.B = X2; g.sBk = N; g.sBn = 1;
    g.C = out; g.sCm = N; g.sCn = 1;
    g.alpha_re = alpha;
    return cx ? gemm<double, true, true>(c, g) : gemm<double, false, false>(c, g);
  };
  if ((st = idplus(sc / m, 1.0, A, T)) != AFQMC_OK) return st;
  for (int k = m - 1; k >= 1; --k) {   // T <- I + (sc / k) A T
    if ((st = mm(A, T, Tn, sc / k)) != AFQMC_OK) return st;
    if ((st = idplus(1.0, 1.0, Tn, Tn)) != AFQMC_OK) return st;
    std::swap(T, Tn);
  }
  for (int s = 0; s < sq; ++s) {
    if ((st = mm(T, T, Tn, 1.0)) != AFQMC_OK) return st;
    std::swap(T, Tn);
  }
  k_convert<R><<<64, 256, 0, c->stream>>>(NN * d.cm(), T, c->at<R>(c->L.eh));
  CHECK_LAUNCH(c);
  if (d.tensor()) {
    if ((st = tc::finish(&c->tcs, c->at<char>(c->L.tc), g_err, sizeof(g_err))) != AFQMC_OK) return st;
    if (c->tcs.pg.ok) {   // F = E_h - I in binary64 for the tensor-core propagation
      if ((st = idplus(1.0, -1.0, T, Tn)) != AFQMC_OK) return st;
      if ((st = tc::prepare_prop(&c->tcs, c->stream, c->at<char>(c->L.tc), Tn, &c->launches, g_err,
                                 sizeof(g_err))) != AFQMC_OK)
        return st;
    }
  }
  CU(cudaMemsetAsync(c->base + c->L.status, 0, 256, c->stream));
  CU(cudaMemsetAsync(c->base + c->L.step, 0, 256, c->stream));
  CU(cudaMemsetAsync(c->base + c->L.slot, 0, 256, c->stream));   // history slot, energy completion counter
  CU(cudaMemsetAsync(c->base + c->L.etr, 0, 256, c->stream));
  CU(cudaMemsetAsync(c->base + c->L.wph, 0, (size_t)d.W * 8, c->stream));
  k_init_walkers<R><<<296, 256, 0, c->stream>>>(d.W, N, nc, c->at<double>(c->L.phi), c->at<cplx_t<R>>(c->L.psi),
                                                c->at<double>(c->L.w), cx ? 1 : 0);
  CHECK_LAUNCH(c);
  if ((st = launch_overlap<R>(c, 0)) != AFQMC_OK) return st;
  c->theta_fresh = true;
  c->vbias_fresh = false;
  // E_var = E_L(psiT) (every walker is the trial)
  if ((st = energy_impl<R>(c, c->at<double>(c->L.hist))) != AFQMC_OK) return st;
  double2 e0;
  CU(cudaMemcpyAsync(&e0, c->base + c->L.eloc, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->e_var = e0.x;
  c->h1e_host.clear();
  c->h1e_host.shrink_to_fit();
  return read_status(c);
}

// Every entry point but afqmc_propagate first orders the stream after an energy estimator still
// running beside it (afqmc_local_energy_async); afqmc_propagate leaves that to the step's overlap.
afqmc_status check_ctx(afqmc_ctx* c) {
  if (!c) return fail(AFQMC_EINVAL, "context is NULL");
  if (c->building) return fail(AFQMC_EINVAL, "the context's set-up is not complete (afqmc_create_end)");
  return join_energy(c);
}

#include "cv_host.inc"

// Captures `body` (which enqueues on c->stream) into a graph.  Host-side state is restored
// afterwards; the caller applies the state change of one replay itself.
template <typename F>
afqmc_status capture_graph(afqmc_ctx* c, F body, cudaGraph_t* out, unsigned long long* nkernels) {
  if (!c->cap_stream) CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const bool tf = c->theta_fresh, vf = c->vbias_fresh, tb = c->thb_valid;
  const unsigned long long hs = c->host_step, l0 = c->launches;
  cudaStream_t user = c->stream;
  // a captured step draws its normals unless the same capture's energy does (never from a flag
  // left by earlier direct calls); after a replay no drawn normals are pending
  c->normals_pending = false;
  CU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap_stream;
  afqmc_status st = body();
  c->stream = user;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  *nkernels = c->launches - l0;
  c->theta_fresh = tf; c->vbias_fresh = vf; c->host_step = hs; c->launches = l0; c->normals_pending = false;
  c->thb_valid = tb;
  c->join_pending = false;   // every captured body ends after the overlap that joins the estimator
  if (st != AFQMC_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
  *out = graph;
  return AFQMC_OK;
}

// Captures `body` (which enqueues on c->stream) into an executable graph.  Host-side state is
// restored afterwards; the caller applies the state change of one replay itself.
template <typename F>
afqmc_status capture(afqmc_ctx* c, F body, cudaGraphExec_t* out, unsigned long long* nkernels) {
  cudaGraph_t graph = nullptr;
  afqmc_status st = capture_graph(c, body, &graph, nkernels);
  if (st != AFQMC_OK) return st;
  const cudaError_t e2 = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return fail(AFQMC_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
  return AFQMC_OK;
}

// One driver-loop step (optional energy into the history slot, then propagation) via a graph.
afqmc_status graph_step(afqmc_ctx* c, bool energy) {
  const int v = (energy ? 1 : 0) | (c->theta_fresh ? 0 : 2) | (energy && c->theta_fresh && c->thb_valid ? 4 : 0);
  if (!c->g_step[v]) {
    afqmc_status st = capture(c, [&]() -> afqmc_status {
      afqmc_status s2;
      if (energy &&
          (s2 = DISPATCH(c, energy_impl, c->at<double>(c->L.hist), c->at<int>(c->L.slot), true, nullptr, true)) !=
              AFQMC_OK)
        return s2;
      return DISPATCH(c, step_impl);
    }, &c->g_step[v], &c->g_step_k[v]);
    if (st != AFQMC_OK) return st;
  }
  CU(cudaGraphLaunch(c->g_step[v], c->stream));
  c->normals_pending = false;
  c->thb_valid = c->d.tensor();   // the step ends with the overlap
  c->launches += c->g_step_k[v];
  c->theta_fresh = true;
  c->vbias_fresh = false;
  c->host_step++;
  return AFQMC_OK;
}

afqmc_status graph_qr(afqmc_ctx* c) {
  if (!c->g_qr) {
    afqmc_status st = capture(c, [&]() { return DISPATCH(c, qr_impl); }, &c->g_qr, &c->g_qr_k);
    if (st != AFQMC_OK) return st;
  }
  CU(cudaGraphLaunch(c->g_qr, c->stream));
  c->normals_pending = false;
  c->launches += c->g_qr_k;
  return AFQMC_OK;   // Theta and its copies stay valid (see qr_impl)
}

afqmc_status graph_comb(afqmc_ctx* c) {
  const int v = c->theta_fresh ? 0 : 1;
  if (!c->g_comb[v]) {
    afqmc_status st = capture(c, [&]() { return DISPATCH(c, comb_impl); }, &c->g_comb[v], &c->g_comb_k[v]);
    if (st != AFQMC_OK) return st;
  }
  CU(cudaGraphLaunch(c->g_comb[v], c->stream));
  c->normals_pending = false;
  c->thb_valid = false;
  c->launches += c->g_comb_k[v];
  c->theta_fresh = true;
  c->vbias_fresh = false;
  return AFQMC_OK;
}

}  // namespace

// ======================================================================================
extern "C" {

const char* afqmc_last_error(void) { return g_err; }

afqmc_status afqmc_workspace_size(int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta, const double* psiT,
                                  const afqmc_params* params, size_t* bytes) {
  if (!bytes) return fail(AFQMC_EINVAL, "bytes is NULL");
  Dims d{};
  afqmc_status st = make_dims(norb, naux, nalpha, nbeta, psiT, params, &d);
  if (st != AFQMC_OK) return st;
  *bytes = plan(d).total;
  return AFQMC_OK;
}

}  // extern "C"

namespace {
afqmc_status create_begin_impl(const double* h1e, double ecore, int32_t norb, int32_t naux, int32_t nalpha,
                               int32_t nbeta, const double* psiT, const afqmc_params* params, void* workspace,
                               size_t workspace_bytes, afqmc_ctx** out, bool cplx) {
  if (!out) return fail(AFQMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h1e) return fail(AFQMC_EINVAL, "h1e is NULL");
  Dims d{};
  afqmc_status st = make_dims(norb, naux, nalpha, nbeta, psiT, params, &d, cplx);
  if (st != AFQMC_OK) return st;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(AFQMC_EINVAL, "workspace must be a non-NULL 256-byte aligned device pointer");
  Layout L = plan(d);
  if (workspace_bytes < L.total)
    return fail(AFQMC_ENOMEM, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
  if (!std::isfinite(ecore)) return fail(AFQMC_EINVAL, "ecore is not finite");
  const size_t N = norb, nt = nalpha + nbeta, e = cplx ? 2 : 1;
  double hmax = 0.0;
  for (size_t i = 0; i < N * N * e; ++i) {
    if (!std::isfinite(h1e[i])) return fail(AFQMC_EINVAL, "h1e has a non-finite entry");
    hmax = std::max(hmax, std::fabs(h1e[i]));
  }
  for (size_t i = 0; i < N * nt * e; ++i)
    if (!std::isfinite(psiT[i])) return fail(AFQMC_EINVAL, "psiT has a non-finite entry");
  for (size_t p = 0; p < N; ++p)
    for (size_t q = (cplx ? p : p + 1); q < N; ++q) {   // symmetric, or Hermitian (h_qp = conj h_pq)
      const double dr = h1e[(p * N + q) * e] - h1e[(q * N + p) * e];
      const double di = cplx ? h1e[(p * N + q) * e + 1] + h1e[(q * N + p) * e + 1] : 0.0;
      if (std::fabs(dr) + std::fabs(di) > 1e-12 * std::max(1.0, hmax))
        return fail(AFQMC_EINVAL, "h1e is not %s at (%zu, %zu)", cplx ? "Hermitian" : "symmetric", p, q);
    }
  afqmc_ctx* c = new afqmc_ctx();
  c->d = d;
  c->L = L;
  c->base = static_cast<char*>(workspace);
  c->stream = static_cast<cudaStream_t>(params->stream);
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    c->side = nullptr;   // the estimator then stays on the main stream
  }
  c->dt = params->dt;
  c->sdt = std::sqrt(params->dt);
  c->cap = params->fb_cap;
  c->ecore = ecore;
  c->taylor = params->taylor_order;
  c->seed = params->seed;
  c->smul = d.restricted ? 2.0 : 1.0;
  c->host_step = 0;
  c->launches = 0;
  c->hist_used = 0;
  c->e_trial = std::isnan(params->e_trial) ? 0.0 : params->e_trial;
  c->e_trial_param = params->e_trial;
  c->building = true;
  c->chol_next = 0;
  st = DISPATCH(c, setup_begin, h1e, psiT);
  if (st != AFQMC_OK) {
    delete c;
    return st;
  }
  *out = c;
  return AFQMC_OK;
}

}  // namespace

extern "C" {

afqmc_status afqmc_create_begin(const double* h1e, double ecore, int32_t norb, int32_t naux, int32_t nalpha,
                                int32_t nbeta, const double* psiT, const afqmc_params* params, void* workspace,
                                size_t workspace_bytes, afqmc_ctx** out) {
  return create_begin_impl(h1e, ecore, norb, naux, nalpha, nbeta, psiT, params, workspace, workspace_bytes, out,
                           false);
}

afqmc_status afqmc_create_begin_complex(const double* h1e, double ecore, int32_t norb, int32_t naux, int32_t nalpha,
                                        int32_t nbeta, const double* psiT, const afqmc_params* params,
                                        void* workspace, size_t workspace_bytes, afqmc_ctx** out) {
  return create_begin_impl(h1e, ecore, norb, naux, nalpha, nbeta, psiT, params, workspace, workspace_bytes, out,
                           true);
}

afqmc_status afqmc_workspace_size_complex(int32_t norb, int32_t naux, int32_t nalpha, int32_t nbeta,
                                          const double* psiT, const afqmc_params* params, size_t* bytes) {
  if (!bytes) return fail(AFQMC_EINVAL, "bytes is NULL");
  Dims d{};
  afqmc_status st = make_dims(norb, naux, nalpha, nbeta, psiT, params, &d, true);
  if (st != AFQMC_OK) return st;
  *bytes = plan(d).total;
  return AFQMC_OK;
}

afqmc_status afqmc_add_cholesky(afqmc_ctx* ctx, int32_t gamma0, int32_t ngamma, const void* chol, int32_t dtype,
                                int32_t location) {
  if (!ctx) return fail(AFQMC_EINVAL, "context is NULL");
  if (!ctx->building) return fail(AFQMC_EINVAL, "afqmc_add_cholesky: the context's set-up is already complete");
  if (!chol) return fail(AFQMC_EINVAL, "afqmc_add_cholesky: chol is NULL");
  const bool cdt = dtype == AFQMC_DTYPE_C128 || dtype == AFQMC_DTYPE_C64;
  if (dtype != AFQMC_DTYPE_F64 && dtype != AFQMC_DTYPE_F32 && !cdt)
    return fail(AFQMC_EINVAL, "afqmc_add_cholesky: dtype %d", dtype);
  if (cdt != ctx->d.cplx)
    return fail(AFQMC_EINVAL, "afqmc_add_cholesky: %s vectors for a %s context", cdt ? "complex" : "real",
                ctx->d.cplx ? "complex" : "real");
  if (location != AFQMC_HOST && location != AFQMC_DEVICE)
    return fail(AFQMC_EINVAL, "afqmc_add_cholesky: location %d", location);
  if (gamma0 != ctx->chol_next)
    return fail(AFQMC_EINVAL, "afqmc_add_cholesky: expected gamma0 = %d (vectors are passed in order, once)",
                ctx->chol_next);
  const int nvec = ctx->d.cplx ? ctx->d.X / 2 : ctx->d.X;
  if (ngamma < 1 || gamma0 + (long long)ngamma > nvec)
    return fail(AFQMC_EINVAL, "afqmc_add_cholesky: gammas [%d, %lld) outside [0, %d)", gamma0,
                gamma0 + (long long)ngamma, nvec);
  const bool dev = location == AFQMC_DEVICE;
  afqmc_status st;
  if (dtype == AFQMC_DTYPE_F64 || dtype == AFQMC_DTYPE_C128)
    st = DISPATCH(ctx, setup_add, gamma0, ngamma, static_cast<const double*>(chol), dev, false);
  else
    st = DISPATCH(ctx, setup_add, gamma0, ngamma, static_cast<const float*>(chol), dev, false);
  if (st != AFQMC_OK) return st;
  ctx->chol_next = gamma0 + ngamma;
  return AFQMC_OK;
}

afqmc_status afqmc_create_end(afqmc_ctx* ctx) {
  if (!ctx) return fail(AFQMC_EINVAL, "context is NULL");
  if (!ctx->building) return fail(AFQMC_EINVAL, "afqmc_create_end: the context's set-up is already complete");
  const int nvec = ctx->d.cplx ? ctx->d.X / 2 : ctx->d.X;
  if (ctx->chol_next != nvec)
    return fail(AFQMC_EINVAL, "afqmc_create_end: %d of %d Cholesky vectors passed", ctx->chol_next, nvec);
  afqmc_status st = DISPATCH(ctx, setup_end);
  if (st != AFQMC_OK) return st;
  ctx->building = false;
  ctx->e_trial = std::isnan(ctx->e_trial_param) ? ctx->e_var : ctx->e_trial_param;
  return AFQMC_OK;
}

afqmc_status afqmc_create(const double* h1e, const double* chol, double ecore, int32_t norb, int32_t naux,
                          int32_t nalpha, int32_t nbeta, const double* psiT, const afqmc_params* params,
                          void* workspace, size_t workspace_bytes, afqmc_ctx** out) {
  if (!out) return fail(AFQMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h1e || !chol) return fail(AFQMC_EINVAL, "h1e or chol is NULL");
  Dims d{};
  afqmc_status st = make_dims(norb, naux, nalpha, nbeta, psiT, params, &d);
  if (st != AFQMC_OK) return st;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(AFQMC_EINVAL, "workspace must be a non-NULL 256-byte aligned device pointer");
  Layout L = plan(d);
  if (workspace_bytes < L.total)
    return fail(AFQMC_ENOMEM, "workspace has %zu bytes, %zu needed", workspace_bytes, L.total);
  // every host input is checked before the device is touched
  if ((st = check_host_chunk<double>(0, naux, norb, chol)) != AFQMC_OK) return st;
  afqmc_ctx* c = nullptr;
  if ((st = afqmc_create_begin(h1e, ecore, norb, naux, nalpha, nbeta, psiT, params, workspace, workspace_bytes,
                               &c)) != AFQMC_OK)
    return st;
  st = DISPATCH(c, setup_add, 0, naux, chol, false, true);
  if (st == AFQMC_OK) {
    c->chol_next = naux;
    st = afqmc_create_end(c);
  }
  if (st != AFQMC_OK) {
    afqmc_destroy(c);
    return st;
  }
  *out = c;
  return AFQMC_OK;
}

void afqmc_destroy(afqmc_ctx* ctx) {
  if (ctx && ctx->side) cudaStreamSynchronize(ctx->side);   // a copy into the caller's memory may be pending
  delete ctx;
}

uint64_t afqmc_launch_count(afqmc_ctx* ctx) { return ctx ? ctx->launches : 0; }

afqmc_status afqmc_profile(afqmc_ctx* ctx, int32_t enable) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (enable) {
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->drain();
    for (int i = 0; i < AFQMC_NSTAGES; ++i) { ctx->stage_ms[i] = 0.0; ctx->stage_n[i] = 0; }
  }
  ctx->prof = enable != 0;
  return AFQMC_OK;
}

afqmc_status afqmc_stage_times(afqmc_ctx* ctx, double* ms, int64_t* count) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->drain();
  for (int i = 0; i < AFQMC_NSTAGES; ++i) {
    if (ms) ms[i] = ctx->stage_ms[i];
    if (count) count[i] = ctx->stage_n[i];
  }
  return AFQMC_OK;
}

afqmc_status afqmc_propagate(afqmc_ctx* ctx, int32_t nsteps) {
  if (!ctx) return fail(AFQMC_EINVAL, "context is NULL");   // an estimator beside it is joined by the overlap
  if (ctx->building) return fail(AFQMC_EINVAL, "the context's set-up is not complete (afqmc_create_end)");
  afqmc_status st;
  if (nsteps < 0) return fail(AFQMC_EINVAL, "nsteps < 0");
  if (nsteps == 0 && (st = join_energy(ctx)) != AFQMC_OK) return st;
  for (int s = 0; s < nsteps; ++s)
    if ((st = DISPATCH(ctx, step_impl)) != AFQMC_OK) return st;
  return AFQMC_OK;
}

afqmc_status afqmc_local_energy(afqmc_ctx* ctx, double* sums, double* eloc) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (eloc && ctx->cv.enabled)
    return fail(AFQMC_EINVAL, "per-walker energies are not formed in the control-variate form (exchange is subsampled)");
  double* dsums = ctx->at<double>(ctx->L.hist) + 4 * (kHistory - 1);
  if ((st = DISPATCH(ctx, energy_impl, dsums)) != AFQMC_OK) return st;
  if (sums) CU(cudaMemcpyAsync(sums, dsums, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (eloc)
    CU(cudaMemcpyAsync(eloc, ctx->base + ctx->L.eloc, (size_t)ctx->d.W * 3 * sizeof(double2), cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (sums || eloc) return read_status(ctx);
  return AFQMC_OK;
}

afqmc_status afqmc_local_energy_async(afqmc_ctx* ctx, double* sums_host) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!sums_host) return fail(AFQMC_EINVAL, "afqmc_local_energy_async: sums_host is NULL");
  // the estimator (and the copy) may run beside a following afqmc_propagate; any other entry
  // point orders the stream after it first
  double* dsums = ctx->at<double>(ctx->L.hist) + 4 * (kHistory - 1);
  return DISPATCH(ctx, energy_impl, dsums, nullptr, true, sums_host);
}

afqmc_status afqmc_reortho(afqmc_ctx* ctx) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  return DISPATCH(ctx, qr_impl);
}

afqmc_status afqmc_popcontrol(afqmc_ctx* ctx) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  return DISPATCH(ctx, comb_impl);
}

afqmc_status afqmc_run(afqmc_ctx* ctx, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                       int32_t comb_every, double* energies, int32_t* nmeas) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (nsteps < 0) return fail(AFQMC_EINVAL, "nsteps < 0");
  if (ctx->free_proj && comb_every > 0) return fail(AFQMC_EINVAL, "free projection: comb_every must be <= 0");
  int used = 0, total = 0;
  double* hist = ctx->at<double>(ctx->L.hist);
  const bool graphs = ctx->graphs_on && !ctx->prof;
  auto flush = [&]() -> afqmc_status {
    if (used > 0 && energies)
      CU(cudaMemcpyAsync(energies + 4 * (size_t)(total - used), hist, (size_t)used * 4 * sizeof(double),
                         cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    used = 0;
    if (graphs) CU(cudaMemsetAsync(ctx->base + ctx->L.slot, 0, sizeof(int), ctx->stream));
    return AFQMC_OK;
  };
  if (graphs) CU(cudaMemsetAsync(ctx->base + ctx->L.slot, 0, sizeof(int), ctx->stream));
  for (int s = 0; s < nsteps; ++s) {
    const bool energy = energy_every > 0 && ctx->host_step % (unsigned long long)energy_every == 0;
    if (energy && used == kHistory - 1 && (st = flush()) != AFQMC_OK) return st;
    if (graphs) {
      if ((st = graph_step(ctx, energy)) != AFQMC_OK) return st;
    } else {
      if (energy && (st = DISPATCH(ctx, energy_impl, hist + 4 * used, nullptr, true, nullptr, true)) != AFQMC_OK)
        return st;
      if ((st = DISPATCH(ctx, step_impl)) != AFQMC_OK) return st;
    }
    if (energy) { ++used; ++total; }
    if (reortho_every > 0 && ctx->host_step % (unsigned long long)reortho_every == 0)
      if ((st = graphs ? graph_qr(ctx) : DISPATCH(ctx, qr_impl)) != AFQMC_OK) return st;
    if (comb_every > 0 && ctx->host_step % (unsigned long long)comb_every == 0)
      if ((st = graphs ? graph_comb(ctx) : DISPATCH(ctx, comb_impl)) != AFQMC_OK) return st;
  }
  if ((st = flush()) != AFQMC_OK) return st;
  if (nmeas) *nmeas = total;
  return read_status(ctx);
}

afqmc_status afqmc_run_async(afqmc_ctx* ctx, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                             int32_t comb_every, double* energies_host, int32_t* nmeas) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (nsteps < 0) return fail(AFQMC_EINVAL, "nsteps < 0");
  if (ctx->free_proj && comb_every > 0) return fail(AFQMC_EINVAL, "free projection: comb_every must be <= 0");
  if (energy_every > 0 && !energies_host) return fail(AFQMC_EINVAL, "afqmc_run_async: energies_host is NULL");
  int used = 0, total = 0;
  double* hist = ctx->at<double>(ctx->L.hist);
  const bool graphs = ctx->graphs_on && !ctx->prof;
  if (graphs && energy_every > 0 && !ctx->copy_stream) {
    CU(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&ctx->ev_copy, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming));
  }
  bool copies = false;   // copies enqueued on copy_stream that the main stream has not waited for
  auto wait_copies = [&]() -> afqmc_status {
    if (!copies) return AFQMC_OK;
    CU(cudaEventRecord(ctx->ev_copied, ctx->copy_stream));
    CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_copied, 0));
    copies = false;
    return AFQMC_OK;
  };
  if (graphs) CU(cudaMemsetAsync(ctx->base + ctx->L.slot, 0, sizeof(int), ctx->stream));
  for (int s = 0; s < nsteps; ++s) {
    const bool energy = energy_every > 0 && ctx->host_step % (unsigned long long)energy_every == 0;
    if (energy && used == kHistory - 1) {   // the device history wraps: its copies come first
      used = 0;
      if ((st = wait_copies()) != AFQMC_OK) return st;
      if (graphs) CU(cudaMemsetAsync(ctx->base + ctx->L.slot, 0, sizeof(int), ctx->stream));
    }
    if (graphs) {
      if ((st = graph_step(ctx, energy)) != AFQMC_OK) return st;
      if (energy) {   // after the step graph, which joins the estimator's branch; off the main stream
        CU(cudaEventRecord(ctx->ev_copy, ctx->stream));
        CU(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_copy, 0));
        CU(cudaMemcpyAsync(energies_host + 4 * (size_t)total, hist + 4 * used, 4 * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->copy_stream));
        copies = true;
      }
    } else {
      if (energy &&
          (st = DISPATCH(ctx, energy_impl, hist + 4 * used, nullptr, true, energies_host + 4 * (size_t)total, true)) !=
              AFQMC_OK)
        return st;
      if ((st = DISPATCH(ctx, step_impl)) != AFQMC_OK) return st;
    }
    if (energy) { ++used; ++total; }
    if (reortho_every > 0 && ctx->host_step % (unsigned long long)reortho_every == 0)
      if ((st = graphs ? graph_qr(ctx) : DISPATCH(ctx, qr_impl)) != AFQMC_OK) return st;
    if (comb_every > 0 && ctx->host_step % (unsigned long long)comb_every == 0)
      if ((st = graphs ? graph_comb(ctx) : DISPATCH(ctx, comb_impl)) != AFQMC_OK) return st;
  }
  if ((st = wait_copies()) != AFQMC_OK) return st;   // the main stream's work after this call sees them
  if (nmeas) *nmeas = total;
  return AFQMC_OK;
}

afqmc_status afqmc_get_walkers(afqmc_ctx* ctx, double* psi, double* logO, double* w, uint64_t* step) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  const Dims& d = ctx->d;
  if (psi) {
    const size_t n = (size_t)d.W * d.N * d.ncol;
    std::vector<double> buf(2 * n);
    if (d.prec == AFQMC_PREC_FP64) {
      CU(cudaMemcpyAsync(buf.data(), ctx->base + ctx->L.psi, n * 16, cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
    } else {
      std::vector<float> f(2 * n);
      CU(cudaMemcpyAsync(f.data(), ctx->base + ctx->L.psi, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      for (size_t i = 0; i < 2 * n; ++i) buf[i] = f[i];
    }
    const int nt = d.na + d.nb;
    for (int wk = 0; wk < d.W; ++wk)
      for (int p = 0; p < d.N; ++p)
        for (int col = 0; col < nt; ++col) {
          const int sc = (d.restricted && col >= d.na) ? col - d.na : col;
          const size_t si = ((size_t)wk * d.N + p) * d.ncol + sc, di = ((size_t)wk * d.N + p) * nt + col;
          psi[2 * di] = buf[2 * si];
          psi[2 * di + 1] = buf[2 * si + 1];
        }
  }
  if (logO) CU(cudaMemcpyAsync(logO, ctx->base + ctx->L.logO, (size_t)d.W * 16, cudaMemcpyDeviceToHost, ctx->stream));
  if (w) CU(cudaMemcpyAsync(w, ctx->base + ctx->L.w, (size_t)d.W * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (step) *step = ctx->host_step;
  return AFQMC_OK;
}

afqmc_status afqmc_set_walkers(afqmc_ctx* ctx, const double* psi, const double* w, uint64_t step) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  const Dims& d = ctx->d;
  if (!psi || !w) return fail(AFQMC_EINVAL, "psi and w are required");
  const int nt = d.na + d.nb;
  const size_t n = (size_t)d.W * d.N * d.ncol;
  std::vector<double> buf(2 * n);
  for (int wk = 0; wk < d.W; ++wk) {
    if (!(w[wk] >= 0.0) || !std::isfinite(w[wk])) return fail(AFQMC_EINVAL, "weight %d is negative or non-finite", wk);
    for (int p = 0; p < d.N; ++p)
      for (int col = 0; col < nt; ++col) {
        const size_t si = ((size_t)wk * d.N + p) * nt + col;
        if (!std::isfinite(psi[2 * si]) || !std::isfinite(psi[2 * si + 1]))
          return fail(AFQMC_EINVAL, "psi has a non-finite entry");
        if (d.restricted && col >= d.na) {
          const size_t ai = ((size_t)wk * d.N + p) * nt + (col - d.na);
          if (psi[2 * si] != psi[2 * ai] || psi[2 * si + 1] != psi[2 * ai + 1])
            return fail(AFQMC_EINVAL, "restricted context: alpha and beta blocks of walker %d differ", wk);
          continue;
        }
        const size_t di = ((size_t)wk * d.N + p) * d.ncol + col;
        buf[2 * di] = psi[2 * si];
        buf[2 * di + 1] = psi[2 * si + 1];
      }
  }
  if (d.prec == AFQMC_PREC_FP64) {
    CU(cudaMemcpyAsync(ctx->base + ctx->L.psi, buf.data(), n * 16, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    std::vector<float> f(buf.begin(), buf.end());
    CU(cudaMemcpyAsync(ctx->base + ctx->L.psi, f.data(), n * 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  CU(cudaMemcpyAsync(ctx->base + ctx->L.w, w, (size_t)d.W * 8, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(ctx->base + ctx->L.wph, 0, (size_t)d.W * 8, ctx->stream));
  unsigned long long s64 = step;
  CU(cudaMemcpyAsync(ctx->base + ctx->L.step, &s64, 8, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->host_step = step;
  ctx->theta_fresh = false;
  ctx->normals_pending = false;
  ctx->vbias_fresh = false;
  st = DISPATCH(ctx, launch_overlap, 0);
  if (st != AFQMC_OK) return st;
  ctx->theta_fresh = true;
  return read_status(ctx);
}

afqmc_status afqmc_get_fields(afqmc_ctx* ctx, double* x, double* xbar) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  const size_t n = (size_t)ctx->d.W * ctx->d.X;
  if (x) CU(cudaMemcpyAsync(x, ctx->base + ctx->L.x, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (xbar) CU(cudaMemcpyAsync(xbar, ctx->base + ctx->L.xbar, n * 16, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return AFQMC_OK;
}

afqmc_status afqmc_draw_normals(uint64_t seed, uint64_t step, uint32_t stream_id, int32_t nwalkers, int32_t naux,
                                double* out, void* stream) {
  if (nwalkers < 0 || naux < 0 || nwalkers > 65535) return fail(AFQMC_EINVAL, "bad sizes");
  if (stream_id > 0xffff) return fail(AFQMC_EINVAL, "stream_id must fit 16 bits");
  if (nwalkers == 0 || naux == 0) return AFQMC_OK;
  if (!out) return fail(AFQMC_EINVAL, "out is NULL");
  k_draw_normals<<<nwalkers, 256, 0, static_cast<cudaStream_t>(stream)>>>(seed, step, stream_id, nwalkers, naux, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "draw_normals launch: %s", cudaGetErrorString(e));
  return AFQMC_OK;
}

afqmc_status afqmc_get_info(afqmc_ctx* ctx, afqmc_info* info) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!info) return fail(AFQMC_EINVAL, "info is NULL");
  info->norb = ctx->d.N; info->naux = ctx->d.X; info->nalpha = ctx->d.na; info->nbeta = ctx->d.nb;
  info->nwalkers = ctx->d.W; info->restricted = ctx->d.restricted ? 1 : 0; info->prec = ctx->d.prec;
  info->reserved = 0;
  info->step = ctx->host_step;
  if (ctx->et_update) {   // E_T lives on the device, where each comb updates it
    double et;
    CU(cudaMemcpyAsync(&et, ctx->base + ctx->L.etr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->e_trial = et;
  }
  info->e_var = ctx->e_var; info->e_trial = ctx->e_trial; info->e_core_mf = ctx->e_c;
  info->workspace_bytes = ctx->L.total;
  return AFQMC_OK;
}

afqmc_status afqmc_set_etrial(afqmc_ctx* ctx, double e_trial) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!std::isfinite(e_trial)) return fail(AFQMC_EINVAL, "e_trial must be finite");
  if (ctx->et_update) {   // the device copy is the one in use (the running sums stay)
    CU(cudaMemcpyAsync(ctx->base + ctx->L.etr, &e_trial, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  } else if (e_trial != ctx->e_trial) {
    CU(cudaStreamSynchronize(ctx->stream));   // captured graphs hold the old value: rebuild them
    ctx->drop_graphs();
  }
  ctx->e_trial = e_trial;
  return AFQMC_OK;
}

afqmc_status afqmc_set_etrial_update(afqmc_ctx* ctx, int32_t enable) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!enable && !ctx->et_update) return AFQMC_OK;
  CU(cudaStreamSynchronize(ctx->stream));   // captured graphs hold the other form's arguments
  if (ctx->et_update) {                     // keep the value reached so far
    double et;
    CU(cudaMemcpyAsync(&et, ctx->base + ctx->L.etr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->e_trial = et;
  }
  ctx->drop_graphs();
  if (enable) {   // E_T from its current value, the running sums from zero
    const double words[3] = {ctx->e_trial, 0.0, 0.0};
    CU(cudaMemcpyAsync(ctx->base + ctx->L.etr, words, sizeof(words), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  ctx->et_update = enable != 0;
  return AFQMC_OK;
}

afqmc_status afqmc_set_free_projection(afqmc_ctx* ctx, int32_t enable) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (enable && ctx->cv.enabled) return fail(AFQMC_EINVAL, "free projection: disable the control variate first");
  if ((enable != 0) == ctx->free_proj) return AFQMC_OK;
  CU(cudaStreamSynchronize(ctx->stream));   // captured graphs hold the other form's arguments
  ctx->drop_graphs();
  CU(cudaMemsetAsync(ctx->base + ctx->L.wph, 0, (size_t)ctx->d.W * 8, ctx->stream));
  ctx->free_proj = enable != 0;
  ctx->vbias_fresh = false;   // free projection may leave it stale: re-formed before a phaseless step
  return AFQMC_OK;
}

afqmc_status afqmc_get_weight_phases(afqmc_ctx* ctx, double* phase) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!phase) return fail(AFQMC_EINVAL, "phase is NULL");
  CU(cudaMemcpyAsync(phase, ctx->base + ctx->L.wph, (size_t)ctx->d.W * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return AFQMC_OK;
}

// ---------------------------------------------------------------- learned control variate
afqmc_status afqmc_cv_workspace_size(afqmc_ctx* ctx, int32_t capacity, int32_t batch, size_t* bytes) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!bytes || capacity < 1 || batch < 1) return fail(AFQMC_EINVAL, "cv: capacity and batch must be >= 1");
  CvState tmp;
  *bytes = cv_plan(&tmp, 2 * ctx->d.N + 8, ctx->d.W, capacity, batch, nullptr);
  return AFQMC_OK;
}

afqmc_status afqmc_cv_attach(afqmc_ctx* ctx, int32_t capacity, int32_t batch, double sample_frac, uint64_t init_seed,
                             void* dev, size_t bytes) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (capacity < 1 || batch < 1) return fail(AFQMC_EINVAL, "cv: capacity and batch must be >= 1");
  if (ctx->d.cplx) return fail(AFQMC_EINVAL, "cv: the control variate takes real Hamiltonians");
  if (!(sample_frac > 0.0 && sample_frac <= 1.0)) return fail(AFQMC_EINVAL, "cv: sample_frac must be in (0, 1]");
  if (ctx->d.W > 8192) return fail(AFQMC_EINVAL, "cv: at most 8192 walkers (subsample drawn in one block)");
  if (!dev || (reinterpret_cast<uintptr_t>(dev) & 255)) return fail(AFQMC_EINVAL, "cv: device block must be 256-byte aligned");
  CvState v;
  const size_t need = cv_plan(&v, 2 * ctx->d.N + 8, ctx->d.W, capacity, batch, nullptr);
  if (bytes < need) return fail(AFQMC_ENOMEM, "cv: device block has %zu bytes, %zu needed", bytes, need);
  cv_plan(&v, 2 * ctx->d.N + 8, ctx->d.W, capacity, batch, static_cast<char*>(dev));
  v.attached = true;
  v.cap = capacity;
  v.B = batch;
  v.frac = sample_frac;
  v.m = std::max(1, std::min(ctx->d.W, (int)std::lround(sample_frac * ctx->d.W)));
  v.seed = init_seed;
  v.bytes = need;
  // Glorot-uniform weights, zero biases
  std::vector<float> p(v.nparams, 0.f);
  std::mt19937_64 rng(init_seed);
  auto glorot = [&](size_t off, int a, int b) {
    std::uniform_real_distribution<double> u(-std::sqrt(6.0 / (a + b)), std::sqrt(6.0 / (a + b)));
    for (size_t i = 0; i < (size_t)a * b; ++i) p[off + i] = (float)u(rng);
  };
  glorot(v.oW1, v.D, v.H);
  glorot(v.oW2, v.H, v.H);
  glorot(v.oW3, v.H, v.H);
  glorot(v.oW4, v.H, 1);
  CU(cudaMemcpyAsync(v.P, p.data(), v.nparams * 4, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaMemsetAsync(v.Mo, 0, v.nparams * 4, ctx->stream));
  CU(cudaMemsetAsync(v.Vo, 0, v.nparams * 4, ctx->stream));
  const float ident[2] = {0.f, 1.f};
  CU(cudaMemcpyAsync(v.ystat, ident, 8, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if ((st = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_cv_select))) != AFQMC_OK) return st;
  if ((st = tc::gemm_f32_prepare(g_err, sizeof(g_err))) != AFQMC_OK) return fail(st, "cv: %s", g_err);
  ctx->drop_graphs();
  ctx->cv = v;
  return AFQMC_OK;
}

afqmc_status afqmc_cv_collect(afqmc_ctx* ctx, int32_t nsteps, int32_t reortho_every, int32_t comb_every,
                              int32_t* npairs) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!ctx->cv.attached) return fail(AFQMC_EINVAL, "cv: not attached");
  if (ctx->cv.scaled) return fail(AFQMC_EINVAL, "cv: training data are already standardised (collect before training)");
  if ((st = DISPATCH(ctx, cv_collect_impl, nsteps, reortho_every, comb_every)) != AFQMC_OK) return st;
  if (npairs) *npairs = ctx->cv.ndata;
  return read_status(ctx);
}

afqmc_status afqmc_cv_train(afqmc_ctx* ctx, int32_t epochs, double lr, double* losses) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!ctx->cv.attached) return fail(AFQMC_EINVAL, "cv: not attached");
  if (epochs < 0 || !(lr > 0.0)) return fail(AFQMC_EINVAL, "cv: epochs >= 0 and lr > 0 required");
  return cv_train_impl(ctx, epochs, lr, losses);
}

afqmc_status afqmc_cv_enable(afqmc_ctx* ctx, int32_t enable) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (enable && !ctx->cv.attached) return fail(AFQMC_EINVAL, "cv: not attached");
  if (enable && ctx->free_proj) return fail(AFQMC_EINVAL, "cv: not available in free projection");
  if ((enable != 0) != ctx->cv.enabled) {
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->drop_graphs();
  }
  ctx->cv.enabled = enable != 0;
  ctx->vbias_fresh = false;
  return AFQMC_OK;
}

afqmc_status afqmc_cv_params(afqmc_ctx* ctx, int32_t set, float* host) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!ctx->cv.attached || !host) return fail(AFQMC_EINVAL, "cv: not attached or NULL buffer");
  const size_t b = ctx->cv.nparams * 4;
  if (set) CU(cudaMemcpyAsync(ctx->cv.P, host, b, cudaMemcpyHostToDevice, ctx->stream));
  else CU(cudaMemcpyAsync(host, ctx->cv.P, b, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return AFQMC_OK;
}

afqmc_status afqmc_cv_eval(afqmc_ctx* ctx, const float* x, const float* y, int32_t rows, float* out, float* loss,
                           float* grads) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  CvState& v = ctx->cv;
  if (!v.attached || !x) return fail(AFQMC_EINVAL, "cv: not attached or NULL input");
  if (rows < 1 || rows > v.B) return fail(AFQMC_EINVAL, "cv: rows must be in [1, batch = %d]", v.B);
  CU(cudaMemcpyAsync(v.X, x, (size_t)rows * v.D * 4, cudaMemcpyHostToDevice, ctx->stream));
  if ((st = cv_forward(ctx, rows, v.X, v.A1, v.A2, v.A3, v.out)) != AFQMC_OK) return st;
  if (y) {
    CU(cudaMemcpyAsync(v.yb, y, (size_t)rows * 4, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(v.loss, 0, 4, ctx->stream));
    if ((st = cv_backward(ctx, rows)) != AFQMC_OK) return st;
    if (loss) CU(cudaMemcpyAsync(loss, v.loss, 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (grads) CU(cudaMemcpyAsync(grads, v.G, v.nparams * 4, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (out) CU(cudaMemcpyAsync(out, v.out, (size_t)rows * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return AFQMC_OK;
}

afqmc_status afqmc_cv_info(afqmc_ctx* ctx, int32_t* dim, uint64_t* nparams, int32_t* npairs, int32_t* nsample) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  const CvState& v = ctx->cv;
  if (dim) *dim = 2 * ctx->d.N + 8;
  if (nparams) { CvState tmp; cv_plan(&tmp, 2 * ctx->d.N + 8, 1, 1, 1, nullptr); *nparams = tmp.nparams; }
  if (npairs) *npairs = v.ndata;
  if (nsample) *nsample = v.m;
  return AFQMC_OK;
}

// ---------------------------------------------------------------- autotuner
afqmc_status afqmc_set_tuning(afqmc_ctx* ctx, const afqmc_tuning* t) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (!t || (t->tile_cap != 1 && t->tile_cap != 2 && t->tile_cap != 4)) return fail(AFQMC_EINVAL, "tuning: tile_cap 1, 2 or 4");
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->drop_graphs();
  if (ctx->d.tensor() && ctx->tcs.packed && t->prop_path != 0)
    return fail(AFQMC_EINVAL, "tuning: with packed L^T (norb > 128) only the tensor-core propagation (prop_path 0) runs");
  ctx->tile_cap = t->tile_cap;
  ctx->prop_path = (t->prop_path >= 0 && t->prop_path <= 2) ? t->prop_path : 0;
  ctx->prop_tile = (t->prop_tile >= 0 && t->prop_tile <= 2) ? t->prop_tile : 0;
  if (ctx->d.tensor())
    tc::set_exchange_groups(&ctx->tcs, ctx->at<char>(ctx->L.tc), t->exch_groups, t->exch_form == 1 ? 1 : 0);
  return AFQMC_OK;
}

afqmc_status afqmc_autotune(afqmc_ctx* ctx, int32_t steps, afqmc_tuning* chosen) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  if (steps < 1) return fail(AFQMC_EINVAL, "autotune: steps >= 1");
  const Dims& d = ctx->d;
  // snapshot of the walkers (host copies), restored after every trial
  const size_t pb = (size_t)d.W * d.N * d.ncol * 2 * d.rsz();
  std::vector<char> psi(pb), logo((size_t)d.W * 16), w((size_t)d.W * 8), wph((size_t)d.W * 8);
  CU(cudaMemcpyAsync(psi.data(), ctx->base + ctx->L.psi, pb, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(logo.data(), ctx->base + ctx->L.logO, logo.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(w.data(), ctx->base + ctx->L.w, w.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaMemcpyAsync(wph.data(), ctx->base + ctx->L.wph, wph.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  const unsigned long long step0 = ctx->host_step;
  auto restore = [&]() -> afqmc_status {
    CU(cudaMemcpyAsync(ctx->base + ctx->L.psi, psi.data(), pb, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->base + ctx->L.logO, logo.data(), logo.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->base + ctx->L.w, w.data(), w.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->base + ctx->L.wph, wph.data(), wph.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->base + ctx->L.step, &step0, 8, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->host_step = step0;
    ctx->theta_fresh = false;
    ctx->vbias_fresh = false;
    return AFQMC_OK;
  };
  std::vector<afqmc_tuning> cands;
  const bool fused_ok = use_fused_propagation(d), tc_ok = d.tensor() && ctx->tcs.pg.ok;
  std::vector<int> groups = {0};
  if (d.tensor()) groups = {1, 2, 3, 4};
  for (int tc_cap : {4, 2})
    for (int g : groups) {
      if (tc_ok)
        for (int form : {0, 1})
          if (form == 0 || (tc_cap == 4 && d.prec == AFQMC_PREC_BF16X3)) cands.push_back(afqmc_tuning{tc_cap, 0, g, 0, form, 0.f});
      if (d.tensor() && ctx->tcs.packed) continue;   // packed L^T: the tensor-core propagation only
      if (fused_ok)
        for (int pt : {0, 1, 2}) cands.push_back(afqmc_tuning{tc_cap, 2, g, pt, 0, 0.f});
      cands.push_back(afqmc_tuning{tc_cap, 1, g, 0, 0, 0.f});
    }
  const bool graphs_was = ctx->graphs_on, prof_was = ctx->prof;
  ctx->graphs_on = false;
  ctx->prof = false;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  afqmc_tuning best{4, 0, 0, 0, 0, 1e30f};
  double* scratch = ctx->at<double>(ctx->L.hist) + 4 * (kHistory - 1);
  for (auto& cnd : cands) {
    if ((st = afqmc_set_tuning(ctx, &cnd)) != AFQMC_OK) break;
    if ((st = restore()) != AFQMC_OK) break;
    if ((st = DISPATCH(ctx, energy_impl, scratch)) != AFQMC_OK) break;   // warm-up step
    if ((st = DISPATCH(ctx, step_impl)) != AFQMC_OK) break;
    CU(cudaEventRecord(e0, ctx->stream));
    for (int k = 0; k < steps && st == AFQMC_OK; ++k) {
      st = DISPATCH(ctx, energy_impl, scratch);
      if (st == AFQMC_OK) st = DISPATCH(ctx, step_impl);
    }
    if (st != AFQMC_OK) break;
    CU(cudaEventRecord(e1, ctx->stream));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    cnd.ms_per_step = ms / steps;
    if (cnd.ms_per_step < best.ms_per_step) best = cnd;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->graphs_on = graphs_was;
  ctx->prof = prof_was;
  if (st != AFQMC_OK) return st;
  if ((st = afqmc_set_tuning(ctx, &best)) != AFQMC_OK) return st;
  if ((st = restore()) != AFQMC_OK) return st;
  if (chosen) *chosen = best;
  return read_status(ctx);
}

afqmc_status afqmc_set_graphs(afqmc_ctx* ctx, int32_t enable) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  ctx->graphs_on = enable != 0;
  return AFQMC_OK;
}

afqmc_status afqmc_synchronize(afqmc_ctx* ctx, double timeout_s) {
  afqmc_status st = check_ctx(ctx);
  if (st != AFQMC_OK) return st;
  cudaEvent_t ev;
  CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, ctx->stream);
  if (e != cudaSuccess) { cudaEventDestroy(ev); return fail(AFQMC_ECUDA, "event record: %s", cudaGetErrorString(e)); }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return fail(AFQMC_ECUDA, "event query: %s", cudaGetErrorString(e)); }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) { cudaEventDestroy(ev); return fail(AFQMC_ETIMEOUT, "stream still busy after %.3f s", el); }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  return read_status(ctx);
}

}  // extern "C"

// ======================================================================================
// Comb plan without allocation (afqmc_comb_plan_noalloc).  The prefix-sum scratch of
// k_comb_plan lives in this file-scope device array instead of a workspace: words
// [0, AFQMC_NOALLOC_MAX_WALKERS) hold the prefix sums, the tail holds the step counter
// and the kernel's status word (internal: the caller's signal is neww).  Host code never
// dereferences the symbol: it looks up the array's device address once per device and
// context and passes that pointer to the kernels.
namespace {

static __device__ __align__(256) unsigned long long g_comb_scratch[AFQMC_NOALLOC_MAX_WALKERS + 64];

constexpr int kMaxDevices = 256;
struct ScratchAddr {
  unsigned long long ctx_id = 0;   // unique id of the CUDA context the address belongs to (0: none)
  void* ptr = nullptr;
};
std::mutex g_comb_scratch_mu;
ScratchAddr g_comb_scratch_addr[kMaxDevices];

typedef CUresult (*PFN_ctx_current)(CUcontext*);
typedef CUresult (*PFN_ctx_id)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current CUDA context (0 when there is none).  A context
// that is destroyed and created again (cudaDeviceReset) gets a new id, so a cached symbol
// address is looked up again instead of being reused.  The driver functions come through the
// runtime's entry-point query, so the library does not link the driver library itself.
cudaError_t current_context_id(unsigned long long* id) {
  static PFN_ctx_current get_current = nullptr;
  static PFN_ctx_id get_id = nullptr;
  *id = 0;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess) return e;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<PFN_ctx_current>(f1);
    get_id = reinterpret_cast<PFN_ctx_id>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  if (!ctx) return cudaSuccess;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
  return cudaSuccess;
}

__global__ void k_store_step(unsigned long long* dst, unsigned long long v) { *dst = v; }

}  // namespace

extern "C" afqmc_status afqmc_comb_plan_noalloc(const double* w, int32_t nwalkers, uint64_t seed, uint64_t step,
                                                int32_t* src, double* neww, void* stream) {
  if (nwalkers < 1 || nwalkers > AFQMC_NOALLOC_MAX_WALKERS)
    return fail(AFQMC_EINVAL, "afqmc_comb_plan_noalloc: nwalkers = %d outside [1, %d] (the static scratch holds "
                              "%d prefix sums)", nwalkers, AFQMC_NOALLOC_MAX_WALKERS, AFQMC_NOALLOC_MAX_WALKERS);
  if (!w || !src || !neww) return fail(AFQMC_EINVAL, "afqmc_comb_plan_noalloc: w, src and neww are required");
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(AFQMC_EINVAL, "afqmc_comb_plan_noalloc: device %d unsupported", dev);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_comb_scratch_mu);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess)
      return fail(AFQMC_ECUDA, "afqmc_comb_plan_noalloc: current context: %s", cudaGetErrorString(e));
    ScratchAddr& slot = g_comb_scratch_addr[dev];
    if (id == 0 || slot.ptr == nullptr || slot.ctx_id != id) {
      // set-up for this device and context: the array's device address (the first lookup in a
      // process may create the context and load the module)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_comb_scratch);
      if (e != cudaSuccess || !p)
        return fail(AFQMC_ECUDA, "afqmc_comb_plan_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      if (id == 0 && (e = current_context_id(&id)) != cudaSuccess)
        return fail(AFQMC_ECUDA, "afqmc_comb_plan_noalloc: current context: %s", cudaGetErrorString(e));
      slot.ctx_id = id;
      slot.ptr = p;
    }
    base = slot.ptr;
  }
  unsigned long long* words = static_cast<unsigned long long*>(base);
  double* cum = reinterpret_cast<double*>(words);
  unsigned long long* step_word = words + AFQMC_NOALLOC_MAX_WALKERS;
  int* status = reinterpret_cast<int*>(words + AFQMC_NOALLOC_MAX_WALKERS + 1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CU(cudaMemsetAsync(status, 0, sizeof(int), s));
  k_store_step<<<1, 1, 0, s>>>(step_word, (unsigned long long)step);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "afqmc_comb_plan_noalloc launch: %s", cudaGetErrorString(e));
  k_comb_plan<<<1, 256, 0, s>>>(nwalkers, seed, step_word, w, cum, src, neww, status, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "afqmc_comb_plan_noalloc launch: %s", cudaGetErrorString(e));
  return AFQMC_OK;
}

// ======================================================================================
// Batched independent systems: one graph launch per step with one branch per system.
struct afqmc_batch {
  std::vector<afqmc_ctx*> sys;
  struct Exec {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned long long> nk;
    std::vector<char> end_theta, end_vbias, end_thb;
  };
  std::map<int, Exec> cache;   // child-graph form: one child graph per system and step kind
  // Grouped form (every system in a tensor-core form, real, phaseless): one launch per stage over
  // the work of every system, the step captured as one graph per step kind.
  int mode = AFQMC_BATCH_AUTO;
  int exch_groups = 0;          // epilogue warpgroups of the grouped exchange (0: the most that fit)
  int nbranch_req = 0;          // branches of the grouped step (0: two where there are two systems)
  bool g_ready = false;
  struct Branch {               // the systems of one branch and their grouped launches
    std::vector<int> sys;       // indices into the batch's contexts
    afq::tc::GroupGemm exch, vhs;
    afq::tc::GroupProp prop;
    void *a_first = nullptr, *a_energy = nullptr, *a_fields = nullptr, *a_overlap = nullptr, *a_stage = nullptr,
         *a_qr = nullptr, *a_comb = nullptr, *a_zero = nullptr;
    int total_w = 0;
    size_t max_vbias = 0;
    // the overlap and QR launches: walker ranges [w0, w1) of systems with similar shared memory
    struct SmemClass { int w0, w1; size_t smem; };
    std::vector<SmemClass> ovl, qr;
  };
  std::vector<Branch> br;
  std::vector<void*> g_dev;     // device argument arrays of the grouped per-walker kernels
  static constexpr int kMaxBranches = 4;
  cudaStream_t bs[kMaxBranches - 1] = {};   // further streams of the grouped step's forks
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxBranches - 1] = {};
  struct GExec {
    cudaGraphExec_t exec = nullptr;
    unsigned long long nk = 0;
  };
  std::map<int, GExec> gcache;
  std::vector<unsigned long long> gens;   // the contexts' graph generations the caches were built at
  // stage tracing of the grouped form (direct launches with CUDA events around each stage)
  bool prof = false;
  struct Pending { int stage; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  double stage_ms[AFQMC_NSTAGES] = {};
  long long stage_n[AFQMC_NSTAGES] = {};
  cudaEvent_t event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drop_grouped() {
    for (auto& kv : gcache)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    gcache.clear();
    for (auto& x : br) {
      afq::tc::group_free(&x.exch);
      afq::tc::group_free(&x.vhs);
      afq::tc::group_prop_free(&x.prop);
    }
    br.clear();
    for (void* d : g_dev) cudaFree(d);
    g_dev.clear();
    g_ready = false;
  }
  void drop_all() {
    for (auto& kv : cache)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    cache.clear();
    drop_grouped();
  }
  ~afqmc_batch() {
    drop_all();
    for (auto x : bs)
      if (x) cudaStreamDestroy(x);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto e : ev_join)
      if (e) cudaEventDestroy(e);
    for (auto& q : pending) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
    for (auto e : free_events) cudaEventDestroy(e);
  }
};

namespace {

// ---------------------------------------------------------------------------------------------
// Grouped batch: every stage of the step is one launch over the work of all systems.

// Whether every context admits the grouped form (else *why says what does not).
bool grouped_ok(const afqmc_batch* b, const char** why) {
  const afqmc_ctx* c0 = b->sys[0];
  for (const afqmc_ctx* c : b->sys) {
    if (!c->d.tensor()) { *why = "a context is not in a tensor-core form"; return false; }
    if (c->d.prec != c0->d.prec) { *why = "the contexts use different precision forms"; return false; }
    if (c->d.cplx) { *why = "a context has a complex Hamiltonian"; return false; }
    if (c->free_proj) { *why = "a context runs free projection"; return false; }
    if (!use_tc_propagation(c)) { *why = "a context does not use the tensor-core propagation"; return false; }
    if (c->taylor != c0->taylor) { *why = "the contexts use different Taylor orders"; return false; }
    if (c->prof) { *why = "a context is being traced"; return false; }
  }
  return true;
}

template <typename T>
afqmc_status upload(afqmc_batch* b, const std::vector<T>& v, void** dev) {
  *dev = nullptr;
  if (v.empty()) return AFQMC_OK;
  void* p = nullptr;
  CU(cudaMalloc(&p, v.size() * sizeof(T)));
  b->g_dev.push_back(p);
  CU(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dev = p;
  return AFQMC_OK;
}

// The grouped launches of one branch: the tcgen05 problems (exchange, VHS, propagation) and the
// argument arrays of the per-walker kernels, in device memory.
afqmc_status branch_plan(afqmc_batch* b, afqmc_batch::Branch& x) {
  using R = float;
  const int nsys = (int)x.sys.size();
  std::vector<tc::GroupSystem> gs(nsys);
  std::vector<tc::GroupPropSystem> ps(nsys);
  std::vector<EnergyArgs<R>> ea(nsys);
  std::vector<FieldArgs<R>> fa(nsys);
  std::vector<OverlapArgs<R>> oa(nsys);
  std::vector<QrArgs<R>> qa(nsys);
  std::vector<CombArgs<R>> ca(nsys);
  std::vector<ZeroArgs> za(nsys);
  std::vector<int> stage(nsys), first(nsys + 1, 0);
  // systems in order of their overlap kernel's shared memory, so that the overlap and QR launches can
  // take runs of systems with similar needs (a launch reserves its largest system's shared memory)
  std::stable_sort(x.sys.begin(), x.sys.end(),
                   [&](int p, int q) { return overlap_smem(b->sys[p]->d) < overlap_smem(b->sys[q]->d); });
  std::vector<size_t> osm(nsys), qsm(nsys);
  for (int i = 0; i < nsys; ++i) {
    afqmc_ctx* c = b->sys[x.sys[i]];
    const Dims& d = c->d;
    char* tcbuf = c->at<char>(c->L.tc);
    int* status = c->at<int>(c->L.status);
    gs[i] = tc::GroupSystem{&c->tcs, tcbuf, c->smul, c->at<float2>(c->L.thetaT), c->at<float2>(c->L.vbias),
                            c->at<float2>(c->L.exch_part), status,
                            tc::NormalsJob{c->at<double>(c->L.x), c->seed, c->at<unsigned long long>(c->L.step), d.W,
                                           d.X}};
    ps[i] = tc::GroupPropSystem{&c->tcs, tcbuf, c->at<float2>(c->L.psi), c->at<double>(c->L.w), status};
    ea[i] = energy_args<R>(c, c->at<double>(c->L.hist), c->at<int>(c->L.slot), true);
    fa[i] = field_args<R>(c);
    oa[i] = overlap_args<R>(c, 1);
    stage[i] = overlap_stage(d) ? 1 : 0;
    osm[i] = overlap_smem(d);
    qa[i] = qr_args<R>(c);
    qsm[i] = qr_smem(d);
    ca[i] = CombArgs<R>{d.W, d.N * d.ncol, c->seed, c->at<unsigned long long>(c->L.step), c->at<double>(c->L.cum),
                        c->at<int>(c->L.src), c->at<double>(c->L.neww), status, c->at<float2>(c->L.psi),
                        c->at<float2>(c->L.psi_tmp), c->at<float2>(c->L.thetaT), c->at<float2>(c->L.th_tmp),
                        c->at<double2>(c->L.logO), c->at<double2>(c->L.logO_tmp), c->at<double>(c->L.w),
                        c->at<double>(c->L.w_tmp), c->et_update ? c->at<double>(c->L.etr) : nullptr};
    za[i] = ZeroArgs{c->at<float2>(c->L.vbias), (size_t)d.W * d.X};
    x.max_vbias = std::max(x.max_vbias, (size_t)d.W * d.X);
    first[i + 1] = first[i] + d.W;
  }
  x.total_w = first[nsys];
  // runs of systems whose shared memory is within a factor of two of the run's first (at most 4 runs)
  auto classes = [&](const std::vector<size_t>& sm, std::vector<afqmc_batch::Branch::SmemClass>& out) {
    out.clear();
    int i0 = 0;
    for (int i = 1; i <= nsys; ++i)
      if (i == nsys || (sm[i] > 2 * std::max<size_t>(sm[i0], 16384) && out.size() < 3)) {
        size_t m = 0;
        for (int k = i0; k < i; ++k) m = std::max(m, sm[k]);
        out.push_back({first[i0], first[i], m});
        i0 = i;
      }
  };
  classes(osm, x.ovl);
  classes(qsm, x.qr);
  afqmc_status st;
  if ((st = tc::group_exchange_plan(gs.data(), nsys, b->exch_groups, &x.exch, g_err, sizeof(g_err))) != AFQMC_OK ||
      (st = tc::group_vhs_plan(gs.data(), nsys, &x.vhs, g_err, sizeof(g_err))) != AFQMC_OK ||
      (st = tc::group_prop_plan(ps.data(), nsys, b->sys[0]->taylor, &x.prop, g_err, sizeof(g_err))) != AFQMC_OK)
    return st;
  if ((st = upload(b, first, &x.a_first)) != AFQMC_OK || (st = upload(b, ea, &x.a_energy)) != AFQMC_OK ||
      (st = upload(b, fa, &x.a_fields)) != AFQMC_OK || (st = upload(b, oa, &x.a_overlap)) != AFQMC_OK ||
      (st = upload(b, stage, &x.a_stage)) != AFQMC_OK || (st = upload(b, qa, &x.a_qr)) != AFQMC_OK ||
      (st = upload(b, ca, &x.a_comb)) != AFQMC_OK || (st = upload(b, za, &x.a_zero)) != AFQMC_OK)
    return st;
  return AFQMC_OK;
}

// The systems split into branches of about equal work (the exchange, VHS and propagation flops; the
// largest first, each to the lightest branch), each branch planned on its own.
afqmc_status batch_grouped_plan(afqmc_batch* b) {
  using R = float;
  b->drop_grouped();
  const int nsys = (int)b->sys.size();
  const int nb = std::max(1, std::min(nsys, b->nbranch_req > 0 ? b->nbranch_req : 2));
  std::vector<double> cost(nsys);
  for (int i = 0; i < nsys; ++i) {
    const afqmc_ctx* c = b->sys[i];
    const Dims& d = c->d;
    double n2 = 0.0;
    for (int k = 0; k < d.nblk; ++k) n2 += (double)d.nbk[k] * d.nbk[k];
    cost[i] = 4.0 * n2 * d.N * d.X * d.W + 4.0 * d.X * (double)d.N * d.N * d.W +
              8.0 * (c->taylor + 2) * (double)d.N * d.N * d.ncol * d.W;
  }
  std::vector<int> order(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->br.assign(nb, afqmc_batch::Branch{});
  std::vector<double> load(nb, 0.0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->br[k].sys.push_back(i);
    load[k] += cost[i];
  }
  for (auto& x : b->br) std::sort(x.sys.begin(), x.sys.end());
  afqmc_status st;
  for (auto& x : b->br)
    if ((st = branch_plan(b, x)) != AFQMC_OK) {
      b->drop_grouped();
      return st;
    }
  if ((st = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_overlap_group<R>))) != AFQMC_OK ||
      (st = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_qr_group<R>))) != AFQMC_OK) {
    b->drop_grouped();
    return st;
  }
  for (int k = 0; k < afqmc_batch::kMaxBranches - 1; ++k) {
    if (!b->bs[k]) CU(cudaStreamCreateWithFlags(&b->bs[k], cudaStreamNonBlocking));
    if (!b->ev_join[k]) CU(cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming));
  }
  if (!b->ev_fork) CU(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
  b->g_ready = true;
  return AFQMC_OK;
}

// Streams bs[0 .. n) wait for s (fork) / s waits for them (join): independent grouped launches (the
// branches; within a lone branch the exchange classes and the small- and large-form propagation)
// run side by side.
afqmc_status batch_fork(afqmc_batch* b, cudaStream_t s, int n = 1) {
  CU(cudaEventRecord(b->ev_fork, s));
  for (int k = 0; k < n; ++k) CU(cudaStreamWaitEvent(b->bs[k], b->ev_fork, 0));
  return AFQMC_OK;
}
afqmc_status batch_join(afqmc_batch* b, cudaStream_t s, int n = 1) {
  for (int k = 0; k < n; ++k) {
    CU(cudaEventRecord(b->ev_join[k], b->bs[k]));
    CU(cudaStreamWaitEvent(s, b->ev_join[k], 0));
  }
  return AFQMC_OK;
}

// Events around one stage of a directly launched grouped step (tracing on).
struct BatchStage {
  afqmc_batch* b;
  cudaStream_t s;
  int stage;
  cudaEvent_t e0 = nullptr;
  BatchStage(afqmc_batch* b_, cudaStream_t s_, int st) : b(b_), s(s_), stage(st) {
    if (b->prof) {
      e0 = b->event();
      cudaEventRecord(e0, s);
    }
  }
  ~BatchStage() {
    if (!e0) return;
    cudaEvent_t e1 = b->event();
    cudaEventRecord(e1, s);
    b->pending.push_back({stage, e0, e1});
  }
};

// One grouped step on stream s: the exchange (force bias, exchange partials, the step's normals;
// the Theta operands rebuilt first unless thb), the energy estimator (energy), fields, the VHS
// planes, the propagation and the new overlaps of every system, then QR and the comb.
afqmc_status branch_step(afqmc_batch* b, afqmc_batch::Branch& x, cudaStream_t s, bool energy, bool qr, bool comb,
                         bool thb, bool forks, unsigned long long* nk) {
  using R = float;
  const int nsys = (int)x.sys.size();
  const int* first = static_cast<const int*>(x.a_first);
  afqmc_status st;
  {
    BatchStage t(b, s, AFQMC_STAGE_FORCE_BIAS);   // the cleared vbias and the bf16 Theta operands
    const unsigned zb = (unsigned)std::min<size_t>(1184, (x.max_vbias + 255) / 256);
    k_zero_group<<<dim3(zb, nsys), 256, 0, s>>>(static_cast<const ZeroArgs*>(x.a_zero));
    ++*nk;
    if (!thb && (st = tc::group_theta(x.exch, s, nk, g_err, sizeof(g_err))) != AFQMC_OK) return st;
  }
  {
    BatchStage t(b, s, AFQMC_STAGE_EXCHANGE);
    const bool two = forks && x.exch.nparts > 1;
    if (two && (st = batch_fork(b, s)) != AFQMC_OK) return st;
    if ((st = tc::group_gemm(x.exch, s, true, nk, g_err, sizeof(g_err), two ? b->bs[0] : nullptr)) != AFQMC_OK)
      return st;
    if (two && (st = batch_join(b, s)) != AFQMC_OK) return st;
  }
  if (energy) {
    BatchStage t(b, s, AFQMC_STAGE_ENERGY);
    k_energy_group<R><<<x.total_w, 256, 0, s>>>(static_cast<const EnergyArgs<R>*>(x.a_energy), first, nsys);
    ++*nk;
  }
  {
    BatchStage t(b, s, AFQMC_STAGE_FIELDS);
    k_fields_group<R><<<x.total_w, 256, 0, s>>>(static_cast<const FieldArgs<R>*>(x.a_fields), first, nsys);
    ++*nk;
  }
  {
    BatchStage t(b, s, AFQMC_STAGE_VHS);
    if ((st = tc::group_gemm(x.vhs, s, false, nk, g_err, sizeof(g_err))) != AFQMC_OK) return st;
  }
  {
    BatchStage t(b, s, AFQMC_STAGE_PROPAGATE);
    const bool two = forks && x.prop.nsmall > 0 && x.prop.nlarge > 0;
    if (two && (st = batch_fork(b, s)) != AFQMC_OK) return st;
    if ((st = tc::group_propagate(x.prop, s, nk, g_err, sizeof(g_err), two ? b->bs[0] : nullptr)) != AFQMC_OK)
      return st;
    if (two && (st = batch_join(b, s)) != AFQMC_OK) return st;
  }
  {
    BatchStage t(b, s, AFQMC_STAGE_OVERLAP);
    for (const auto& k : x.ovl) {
      k_overlap_group<R><<<k.w1 - k.w0, 128, k.smem, s>>>(static_cast<const OverlapArgs<R>*>(x.a_overlap), first,
                                                          static_cast<const int*>(x.a_stage), nsys, k.w0);
      ++*nk;
    }
  }
  if (qr) {
    BatchStage t(b, s, AFQMC_STAGE_QR);
    for (const auto& k : x.qr) {
      k_qr_group<R><<<k.w1 - k.w0, 256, k.smem, s>>>(static_cast<const QrArgs<R>*>(x.a_qr), first, nsys, k.w0);
      ++*nk;
    }
  }
  if (comb) {
    BatchStage t(b, s, AFQMC_STAGE_COMB);
    const CombArgs<R>* ca = static_cast<const CombArgs<R>*>(x.a_comb);
    k_comb_plan_group<R><<<nsys, 256, 0, s>>>(ca);
    k_comb_gather_group<R><<<x.total_w, 256, 0, s>>>(ca, first, nsys);
    k_comb_back_group<R><<<x.total_w, 256, 0, s>>>(ca, first, nsys);
    *nk += 3;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "grouped batch step: %s", cudaGetErrorString(e));
  return AFQMC_OK;
}

// One grouped step of every branch: side by side on s and the further streams, or in turn on s (one
// branch, or tracing, where the stages' events must not overlap); a lone branch forks its
// independent launches instead.
afqmc_status batch_grouped_step(afqmc_batch* b, cudaStream_t s, bool energy, bool qr, bool comb, bool thb,
                                unsigned long long* nk) {
  afqmc_status st;
  if (b->br.size() == 1 || b->prof) {   // tracing: every launch alone, so each stage times its kernels
    for (auto& x : b->br)
      if ((st = branch_step(b, x, s, energy, qr, comb, thb, !b->prof, nk)) != AFQMC_OK) return st;
    return AFQMC_OK;
  }
  const int n = (int)b->br.size() - 1;
  if ((st = batch_fork(b, s, n)) != AFQMC_OK) return st;
  for (int k = 0; k <= n; ++k)
    if ((st = branch_step(b, b->br[k], k ? b->bs[k - 1] : s, energy, qr, comb, thb, false, nk)) != AFQMC_OK)
      return st;
  return batch_join(b, s, n);
}

// The executable graph of one grouped step kind (key: energy | qr << 1 | comb << 2 | thb << 3).
afqmc_status batch_grouped_exec(afqmc_batch* b, int key, afqmc_batch::GExec** out) {
  auto it = b->gcache.find(key);
  if (it != b->gcache.end()) { *out = &it->second; return AFQMC_OK; }
  afqmc_ctx* c0 = b->sys[0];
  if (!c0->cap_stream) CU(cudaStreamCreateWithFlags(&c0->cap_stream, cudaStreamNonBlocking));
  afqmc_batch::GExec ex;
  CU(cudaStreamBeginCapture(c0->cap_stream, cudaStreamCaptureModeThreadLocal));
  afqmc_status st = batch_grouped_step(b, c0->cap_stream, key & 1, key & 2, key & 4, key & 8, &ex.nk);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c0->cap_stream, &g);
  if (st != AFQMC_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "grouped batch capture: %s", cudaGetErrorString(e));
  const cudaError_t ie = cudaGraphInstantiate(&ex.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return fail(AFQMC_ECUDA, "grouped batch graph instantiation: %s", cudaGetErrorString(ie));
  auto res = b->gcache.emplace(key, ex);
  *out = &res.first->second;
  return AFQMC_OK;
}

afqmc_status batch_exec(afqmc_batch* b, int key, bool energy, bool qr, bool comb, afqmc_batch::Exec** out) {
  auto it = b->cache.find(key);
  if (it != b->cache.end()) { *out = &it->second; return AFQMC_OK; }
  afqmc_batch::Exec ex;
  cudaGraph_t bg = nullptr;
  CU(cudaGraphCreate(&bg, 0));
  for (afqmc_ctx* c : b->sys) {
    cudaGraph_t g = nullptr;
    unsigned long long nk = 0;
    bool end_tf = false, end_vf = false, end_tb = false;
    afqmc_status st = capture_graph(c, [&]() -> afqmc_status {
      afqmc_status s2;
      if (energy &&
          (s2 = DISPATCH(c, energy_impl, c->at<double>(c->L.hist), c->at<int>(c->L.slot), true, nullptr, true)) !=
              AFQMC_OK)
        return s2;
      if ((s2 = DISPATCH(c, step_impl)) != AFQMC_OK) return s2;
      if (qr && (s2 = DISPATCH(c, qr_impl)) != AFQMC_OK) return s2;
      if (comb && (s2 = DISPATCH(c, comb_impl)) != AFQMC_OK) return s2;
      end_tf = c->theta_fresh;
      end_tb = c->thb_valid;
      end_vf = c->vbias_fresh;
      return AFQMC_OK;
    }, &g, &nk);
    if (st != AFQMC_OK) { cudaGraphDestroy(bg); return st; }
    cudaGraphNode_t node;
    const cudaError_t e = cudaGraphAddChildGraphNode(&node, bg, nullptr, 0, g);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { cudaGraphDestroy(bg); return fail(AFQMC_ECUDA, "batch graph: %s", cudaGetErrorString(e)); }
    ex.nk.push_back(nk);
    ex.end_theta.push_back(end_tf);
    ex.end_thb.push_back(end_tb);
    ex.end_vbias.push_back(end_vf);
  }
  const cudaError_t e = cudaGraphInstantiate(&ex.exec, bg, 0);
  cudaGraphDestroy(bg);
  if (e != cudaSuccess) return fail(AFQMC_ECUDA, "batch graph instantiation: %s", cudaGetErrorString(e));
  auto res = b->cache.emplace(key, std::move(ex));
  *out = &res.first->second;
  return AFQMC_OK;
}

}  // namespace

extern "C" {

afqmc_status afqmc_batch_create(int32_t nsys, afqmc_ctx* const* ctxs, afqmc_batch** out) {
  if (!out || !ctxs || nsys < 1) return fail(AFQMC_EINVAL, "batch: need nsys >= 1 contexts");
  *out = nullptr;
  for (int i = 0; i < nsys; ++i) {
    if (!ctxs[i]) return fail(AFQMC_EINVAL, "batch: context %d is NULL", i);
    if (ctxs[i]->building) return fail(AFQMC_EINVAL, "batch: context %d has not finished its set-up", i);
    if (ctxs[i]->host_step != ctxs[0]->host_step) return fail(AFQMC_EINVAL, "batch: contexts must be at the same step");
    if (ctxs[i]->cv.enabled) return fail(AFQMC_EINVAL, "batch: the control-variate form is not batched");
  }
  afqmc_batch* b = new afqmc_batch();
  b->sys.assign(ctxs, ctxs + nsys);
  *out = b;
  return AFQMC_OK;
}

void afqmc_batch_destroy(afqmc_batch* b) { delete b; }

afqmc_status afqmc_batch_set_mode(afqmc_batch* b, int32_t mode, int32_t exch_groups, int32_t branches) {
  if (!b) return fail(AFQMC_EINVAL, "batch is NULL");
  if (mode < AFQMC_BATCH_AUTO || mode > AFQMC_BATCH_GRAPHS) return fail(AFQMC_EINVAL, "batch: unknown mode %d", mode);
  if (exch_groups < 0 || exch_groups > 4) return fail(AFQMC_EINVAL, "batch: exch_groups must be in [0, 4]");
  if (branches < 0 || branches > afqmc_batch::kMaxBranches)
    return fail(AFQMC_EINVAL, "batch: branches must be in [0, %d]", afqmc_batch::kMaxBranches);
  for (afqmc_ctx* c : b->sys) CU(cudaStreamSynchronize(c->stream));
  if (mode != b->mode || exch_groups != b->exch_groups || branches != b->nbranch_req) b->drop_grouped();
  b->mode = mode;
  b->exch_groups = exch_groups;
  b->nbranch_req = branches;
  return AFQMC_OK;
}

afqmc_status afqmc_batch_profile(afqmc_batch* b, int32_t enable) {
  if (!b) return fail(AFQMC_EINVAL, "batch is NULL");
  b->prof = enable != 0;
  if (b->prof) {
    std::fill(b->stage_ms, b->stage_ms + AFQMC_NSTAGES, 0.0);
    std::fill(b->stage_n, b->stage_n + AFQMC_NSTAGES, 0LL);
  }
  return AFQMC_OK;
}

afqmc_status afqmc_batch_stage_times(afqmc_batch* b, double* ms, int64_t* count) {
  if (!b) return fail(AFQMC_EINVAL, "batch is NULL");
  CU(cudaStreamSynchronize(b->sys[0]->stream));
  for (auto& q : b->pending) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, q.a, q.b));
    b->stage_ms[q.stage] += t;
    b->stage_n[q.stage] += 1;
    b->free_events.push_back(q.a);
    b->free_events.push_back(q.b);
  }
  b->pending.clear();
  for (int i = 0; i < AFQMC_NSTAGES; ++i) {
    if (ms) ms[i] = b->stage_ms[i];
    if (count) count[i] = b->stage_n[i];
  }
  return AFQMC_OK;
}

afqmc_status afqmc_batch_describe(afqmc_batch* b, char* buf, size_t len) {
  if (!b || !buf || len == 0) return fail(AFQMC_EINVAL, "batch or buffer is NULL");
  std::string out;
  char line[256];
  if (!b->g_ready) {
    out = "grouped launches not planned (runs in the graphs form, or before the first grouped run)\n";
  } else {
    auto part = [&](const char* what, const tc::GroupLaunch& gl) {
      snprintf(line, sizeof(line),
               "%s: %d problems, %d tiles, grid %d, %d stages of %d B, %d epilogue groups x %d B (width %d), "
               "%d TMEM cols, %zu B smem\n",
               what, gl.nprob, gl.tiles, gl.grid, gl.stages, gl.stage_stride, gl.epi_groups, gl.epi_bytes, gl.nb,
               gl.tmem_cols, gl.smem);
      out += line;
    };
    for (size_t k = 0; k < b->br.size(); ++k) {
      const afqmc_batch::Branch& x = b->br[k];
      snprintf(line, sizeof(line), "branch %zu of %zu: %zu systems, %d walkers\n", k + 1, b->br.size(), x.sys.size(),
               x.total_w);
      out += line;
      for (int j = 0; j < x.exch.nparts; ++j) part("  exchange", x.exch.part[j]);
      for (int j = 0; j < x.vhs.nparts; ++j) part("  vhs", x.vhs.part[j]);
      snprintf(line, sizeof(line), "  propagate: %d small-form systems (grid %d, %zu B smem), %d large-form systems "
               "(%d tiles, grid %d, %d stages)\n", x.prop.nsmall, x.prop.small_grid, x.prop.small_smem,
               x.prop.nlarge, x.prop.large_tiles, x.prop.large_grid, x.prop.large_stages);
      out += line;
    }
  }
  snprintf(buf, len, "%s", out.c_str());
  return AFQMC_OK;
}

afqmc_status afqmc_batch_get_mode(afqmc_batch* b, int32_t* mode) {
  if (!b || !mode) return fail(AFQMC_EINVAL, "batch or mode is NULL");
  const char* why = "";
  *mode = (b->mode != AFQMC_BATCH_GRAPHS && grouped_ok(b, &why)) ? AFQMC_BATCH_GROUPED : AFQMC_BATCH_GRAPHS;
  return AFQMC_OK;
}

afqmc_status afqmc_batch_run(afqmc_batch* b, int32_t nsteps, int32_t energy_every, int32_t reortho_every,
                             int32_t comb_every, double* energies, int32_t* nmeas) {
  if (!b) return fail(AFQMC_EINVAL, "batch is NULL");
  if (nsteps < 0) return fail(AFQMC_EINVAL, "nsteps < 0");
  afqmc_ctx* c0 = b->sys[0];
  cudaStream_t s = c0->stream;
  const int nsys = (int)b->sys.size();
  for (afqmc_ctx* c : b->sys)
    if (c->free_proj && comb_every > 0) return fail(AFQMC_EINVAL, "batch: free projection with comb_every > 0");
  int total = 0;
  for (int k = 0; k < nsteps; ++k)
    if (energy_every > 0 && (c0->host_step + k) % (unsigned long long)energy_every == 0) ++total;
  int used = 0, done = 0;
  auto flush = [&]() -> afqmc_status {
    for (int i = 0; i < nsys && energies && used > 0; ++i)
      CU(cudaMemcpyAsync(energies + ((size_t)i * total + done) * 4, b->sys[i]->at<double>(b->sys[i]->L.hist),
                         (size_t)used * 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    done += used;
    used = 0;
    for (afqmc_ctx* c : b->sys) CU(cudaMemsetAsync(c->base + c->L.slot, 0, sizeof(int), s));
    return AFQMC_OK;
  };
  for (afqmc_ctx* c : b->sys) {
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaMemsetAsync(c->base + c->L.slot, 0, sizeof(int), s));
  }
  afqmc_status st;
  // cached launches hold parameters (E_T, tuning) that a context may have changed since
  std::vector<unsigned long long> gens;
  for (afqmc_ctx* c : b->sys) gens.push_back(c->graph_gen);
  if (gens != b->gens) {
    b->drop_all();
    b->gens = gens;
  }
  const char* why = "";
  const bool grouped = b->mode != AFQMC_BATCH_GRAPHS && grouped_ok(b, &why);
  if (b->mode == AFQMC_BATCH_GROUPED && !grouped) return fail(AFQMC_EINVAL, "batch: grouped form: %s", why);
  if (grouped) {
    if (!b->g_ready && (st = batch_grouped_plan(b)) != AFQMC_OK) return st;
    bool thb = true;
    for (afqmc_ctx* c : b->sys) {   // every system starts from its own Theta (and the same step kind)
      if (!c->theta_fresh) {
        if ((st = DISPATCH(c, launch_overlap, 2)) != AFQMC_OK) return st;
        c->theta_fresh = true;
      }
      thb = thb && c->thb_valid;
      CU(cudaStreamSynchronize(c->stream));
    }
    for (int k = 0; k < nsteps; ++k) {
      const unsigned long long hs = c0->host_step;
      const bool energy = energy_every > 0 && hs % (unsigned long long)energy_every == 0;
      const bool qr = reortho_every > 0 && (hs + 1) % (unsigned long long)reortho_every == 0;
      const bool comb = comb_every > 0 && (hs + 1) % (unsigned long long)comb_every == 0;
      const int key = (energy ? 1 : 0) | (qr ? 2 : 0) | (comb ? 4 : 0) | (thb ? 8 : 0);
      if (energy && used == kHistory - 1 && (st = flush()) != AFQMC_OK) return st;
      if (b->prof) {   // direct launches, timed per stage
        unsigned long long nk = 0;
        if ((st = batch_grouped_step(b, s, energy, qr, comb, thb, &nk)) != AFQMC_OK) return st;
        c0->launches += nk;
      } else {
        afqmc_batch::GExec* ex = nullptr;
        if ((st = batch_grouped_exec(b, key, &ex)) != AFQMC_OK) return st;
        CU(cudaGraphLaunch(ex->exec, s));
        c0->launches += ex->nk;
      }
      for (afqmc_ctx* c : b->sys) {
        c->theta_fresh = true;
        c->thb_valid = !comb;   // the overlap writes the bf16 Theta operand; the comb reorders Theta only
        c->vbias_fresh = false;
        c->normals_pending = false;
        c->host_step++;
      }
      thb = !comb;
      if (energy) ++used;
    }
    if ((st = flush()) != AFQMC_OK) return st;
    if (nmeas) *nmeas = total;
    for (afqmc_ctx* c : b->sys)
      if ((st = read_status(c)) != AFQMC_OK) return st;
    return AFQMC_OK;
  }
  for (int k = 0; k < nsteps; ++k) {
    const unsigned long long hs = c0->host_step;
    const bool energy = energy_every > 0 && hs % (unsigned long long)energy_every == 0;
    const bool qr = reortho_every > 0 && (hs + 1) % (unsigned long long)reortho_every == 0;
    const bool comb = comb_every > 0 && (hs + 1) % (unsigned long long)comb_every == 0;
    const bool refresh = !c0->theta_fresh;
    const int key = (energy ? 1 : 0) | (refresh ? 2 : 0) | (qr ? 4 : 0) | (comb ? 8 : 0) |
                    (energy && !refresh && c0->thb_valid ? 16 : 0);
    if (energy && used == kHistory - 1 && (st = flush()) != AFQMC_OK) return st;
    afqmc_batch::Exec* ex = nullptr;
    if ((st = batch_exec(b, key, energy, qr, comb, &ex)) != AFQMC_OK) return st;
    CU(cudaGraphLaunch(ex->exec, s));
    for (int i = 0; i < nsys; ++i) {
      afqmc_ctx* c = b->sys[i];
      c->launches += ex->nk[i];
      c->theta_fresh = ex->end_theta[i];
      c->thb_valid = ex->end_thb[i];
      c->vbias_fresh = ex->end_vbias[i];
      c->normals_pending = false;
      c->host_step++;
    }
    if (energy) ++used;
  }
  if ((st = flush()) != AFQMC_OK) return st;
  if (nmeas) *nmeas = total;
  for (afqmc_ctx* c : b->sys)
    if ((st = read_status(c)) != AFQMC_OK) return st;
  return AFQMC_OK;
}

}  // extern "C"
