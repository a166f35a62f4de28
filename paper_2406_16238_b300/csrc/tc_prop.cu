// Tensor-core propagation for the BF16 forms (Eq. 8 with the mean-field form of h_eff):
//   t = E_h psi,  acc = t,  t <- V t / k and acc += t for k = 1..order,  psi <- E_h acc,
// with E_h = exp(-dt/2 h_eff) applied as psi + F psi, F = E_h - I (F is O(dt), so its split-bf16
// product error is far below that of E_h itself).
//
// Per walker and chunk of cw columns every product is a set of tcgen05 contractions D = A B^T with
// M = 128 rows p (orbitals) and K = q.  B holds the current term of the chunk once, as split bf16:
// rows 0 .. 2 cwp - 1 its hi parts (real parts of the columns, then imaginary parts, grouped by the
// epilogue's column slices), rows 2 cwp .. 4 cwp - 1 its lo parts.  Per 16-wide k-step two MMAs
// form A hi [B hi; B lo] (N = 4 cwp) and A lo B hi (N = 2 cwp, into the first half), so each
// accumulator holds the three split-bf16 partial products (hi*hi + lo*hi, hi*lo side by side; fp32
// in tensor memory).  An F product uses one accumulator D1 = F t; a V product two, D1 = Re V t and
// D2 = Im V t, and the epilogue forms Re (V t) = Re D1 - Im D2, Im (V t) = Im D1 + Re D2.
//
// Roles: warp 16 (one thread) loads F once and each walker's V planes by TMA and issues the MMAs;
// warps 0-15 read the accumulator, warp w covering lanes 32 (w % 4) .. + 31 (rows p) and a
// quarter of the chunk's columns: it keeps its part of row p of acc in registers and writes the
// matching entries of column k = p of the next B operand (hi and lo) into shared memory; the
// propagated chunk leaves through the B buffer, staged so that consecutive threads write
// consecutive addresses of psi.  V of the next walker is fetched as soon as the last Taylor
// product of the current one has completed.
// Rows p >= N of D (padding, and rows npad .. 127 which the MMA reads from the following buffer)
// are never used: those threads write zeros into B.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace afq {
namespace tc {

namespace {

struct PropTcParams {
  int N, npad, nk, ncol, cw, nch, order, W;
  int off_vlo, off_fhi, off_flo, off_b, off_bar;
  int tmem_cols;
  float2* psi;
  const double* w;
  int* status;
};

// Byte offset of element (row n, k) in a K-major, 128-byte-swizzled operand of `rows` rows
// stored as consecutive 64-wide K atoms of rows * 128 bytes each.
__device__ __forceinline__ uint32_t sw_off(int n, int k, int atom_bytes) {
  const int kk = k & 63;
  return (uint32_t)((k >> 6) * atom_bytes + (n >> 3) * 1024 + (n & 7) * 128 + (((kk >> 3) ^ (n & 7)) << 4) +
                    ((kk & 7) << 1));
}

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, __nv_bfloat16 v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = v;
}

// Column k = p of the next B operand for this thread's slice (columns j0 .. j0 + SW - 1) of the
// term (ur, ui).  B is K-major with 128-byte swizzling, two 64-wide K atoms of 4 CWP rows; the
// slice owns hi rows 2 j0 + jj (real parts) and 2 j0 + SW + jj (imaginary parts), and the lo rows
// 2 CWP further on, so its accumulator columns are consecutive.
// The byte offsets depend only on the thread.  Where 2 j0 is a multiple of 8 (SW = 4, 8) the rows
// of the slice have compile-time swizzle phases (n & 7) and each offset is two operations from a
// per-thread base; otherwise (SW = 2, 6) the 2 SW offsets are formed once and kept.
template <int CWP, int SW>
struct BOffsets {
  static constexpr bool kPhase = (2 * SW) % 8 == 0;
  static constexpr int ab = 4 * CWP * 128;
  uint32_t o[kPhase ? 2 : 2 * SW];
  __device__ __forceinline__ BOffsets(int p, int j0) {
    if constexpr (kPhase) {
      o[0] = (uint32_t)((p >> 6) * ab + ((2 * j0) >> 3) * 1024 + ((p & 7) << 1));
      o[1] = (uint32_t)((p & 63) >> 3);
    } else {
#pragma unroll
      for (int jj = 0; jj < SW; ++jj) {
        o[jj] = sw_off(2 * j0 + jj, p, ab);
        o[SW + jj] = sw_off(2 * j0 + SW + jj, p, ab);
      }
    }
  }
  // row 2 j0 + c of the slice (c = jj for real parts, SW + jj for imaginary parts)
  __device__ __forceinline__ uint32_t at(int c) const {
    if constexpr (kPhase) return o[0] + (uint32_t)((c >> 3) * 1024 + (c & 7) * 128) + ((o[1] ^ (uint32_t)(c & 7)) << 4);
    else return o[c];
  }
};

template <int CWP, int SW>
__device__ __forceinline__ void write_b(uint8_t* b, const BOffsets<CWP, SW>& bo, const float* ur, const float* ui) {
  constexpr uint32_t lo = 256u * CWP;   // 2 CWP rows further (2 CWP is a multiple of 8)
#pragma unroll
  for (int jj = 0; jj < SW; ++jj) {   // (real, imaginary) rounded as one pair
    const __nv_bfloat162 h = __floats2bfloat162_rn(ur[jj], ui[jj]);
    const __nv_bfloat162 l = __floats2bfloat162_rn(ur[jj] - __low2float(h), ui[jj] - __high2float(h));
    const uint32_t o_r = bo.at(jj), o_i = bo.at(SW + jj);
    st_bf16(b, o_r, __low2bfloat16(h));
    st_bf16(b, o_r + lo, __low2bfloat16(l));
    st_bf16(b, o_i, __high2bfloat16(h));
    st_bf16(b, o_i + lo, __high2bfloat16(l));
  }
}

// Generic-proxy writes of B become visible to the tensor core; one arrival per warp.
__device__ __forceinline__ void signal_b(uint64_t* bar_b, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar_b);
}

// Lane 0 waits, the warp follows its outcome (tcgen05.ld needs the whole warp).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) tc_fence_after();
  return ok != 0;
}

// NC consecutive accumulator columns of this thread's lane (no wait).
template <int NC>
__device__ __forceinline__ void ld_cols(uint32_t taddr, uint32_t* r) {
  if constexpr (NC == 4) {
    tmem_ld4_nowait(taddr, r);
  } else if constexpr (NC == 8) {
    tmem_ld8_nowait(taddr, r);
  } else if constexpr (NC == 12) {
    tmem_ld8_nowait(taddr, r);
    tmem_ld4_nowait(taddr + 8, r + 8);
  } else {
    static_assert(NC == 16, "slice width");
    tmem_ld16_nowait(taddr, r);
  }
}

// This thread's slice of row p of the product: dr[jj] + i di[jj] = (A t)[p][j0 + jj].  The hi and
// lo halves of each accumulator are added; a V product combines D1 = Re V t (columns 0 .. 4 CWP - 1)
// and D2 = Im V t (columns 4 CWP .. 8 CWP - 1).
template <int CWP, int SW, bool V>
__device__ __forceinline__ void load_d(uint32_t trow, int j0, float* dr, float* di) {
  constexpr int NC = 2 * SW;
  uint32_t h1[NC], l1[NC], h2[V ? NC : 1], l2[V ? NC : 1];
  ld_cols<NC>(trow + (uint32_t)(2 * j0), h1);
  ld_cols<NC>(trow + (uint32_t)(2 * CWP + 2 * j0), l1);
  if constexpr (V) {
    ld_cols<NC>(trow + (uint32_t)(4 * CWP + 2 * j0), h2);
    ld_cols<NC>(trow + (uint32_t)(6 * CWP + 2 * j0), l2);
  }
  tmem_wait();
#pragma unroll
  for (int jj = 0; jj < SW; ++jj) {
    const float ar = __uint_as_float(h1[jj]) + __uint_as_float(l1[jj]);
    const float ai = __uint_as_float(h1[SW + jj]) + __uint_as_float(l1[SW + jj]);
    if constexpr (V) {
      const float br = __uint_as_float(h2[jj]) + __uint_as_float(l2[jj]);
      const float bi = __uint_as_float(h2[SW + jj]) + __uint_as_float(l2[SW + jj]);
      dr[jj] = ar - bi;
      di[jj] = ai + br;
    } else {
      dr[jj] = ar;
      di[jj] = ai;
    }
  }
}

constexpr int kEpiWarps = 16;                 // 4 lane quadrants x 4 column slices
constexpr int kPropThreads = 32 * kEpiWarps + 32;

// The walkers one CTA propagates for one system: wk = first, first + stride, ... below end, the
// walkers of weight zero skipped.
struct WalkerRun {
  int first, stride, end;
};

__device__ __forceinline__ int run_next_live(const double* w, const WalkerRun& r, int from) {
  for (int k = from; k < r.end; k += r.stride)
    if (w[k] != 0.0) return k;
  return r.end;
}

// The 16 epilogue warps meet (bounded wait); shared-memory writes made before are visible after.
__device__ __forceinline__ bool epi_sync(uint64_t* bar_e, uint32_t& ph, volatile int* abort_flag, int lane) {
  __threadfence_block();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar_e);
  const bool ok = warp_wait(bar_e, ph, abort_flag, lane);
  ph ^= 1u;
  return ok;
}

// TMA and MMA issue (lane 0 of warp 16) for a run of walkers of one system: per walker and column
// chunk F psi, the Taylor terms V t / k, F acc.  F is loaded at the start of the run and each
// walker's V one walker ahead (into L2 as soon as the current walker's first V product may start,
// into shared memory once its last V product has completed).  idle: no product has been issued in
// this CTA yet, so F and the first V are requested at once; otherwise only after the first
// walker's B operand is ready (the epilogue writes it after reading the previous walker's last
// product, so no copy into this system's layout can meet a product still reading another's).
template <int CWP>
__device__ __forceinline__ bool prop_mma_run(uint8_t* sm, uint32_t tmem, const CUtensorMap* mapV,
                                             const CUtensorMap* mapF, const PropTcParams a, const WalkerRun r,
                                             bool& idle, uint64_t* bar_v, uint64_t* bar_f, uint64_t* bar_mma,
                                             uint64_t* bar_b, volatile int* abort_flag, uint32_t& ph_b,
                                             uint32_t& ph_v, uint32_t& ph_f, int lane) {
  if (lane != 0) return true;
  const uint32_t s0 = smem_u32(sm);
  const uint32_t vatom = (uint32_t)a.npad * 128u, batom = 4u * CWP * 128u;
  // descriptors are linear in the address: desc(base + off) = desc(base) + off / 16
  const uint64_t dvhi = sw128_desc(s0), dvlo = sw128_desc(s0 + (uint32_t)a.off_vlo);
  const uint64_t dfhi = sw128_desc(s0 + (uint32_t)a.off_fhi), dflo = sw128_desc(s0 + (uint32_t)a.off_flo);
  const uint64_t db = sw128_desc(s0 + (uint32_t)a.off_b);
  auto issue_v = [&](int w) {
    mbar_expect_tx(bar_v, 8u * vatom);
    for (int pl = 0; pl < 4; ++pl)
      for (int at = 0; at < 2; ++at) {
        const uint32_t dst = (pl < 2 ? 0u : (uint32_t)a.off_vlo) + (uint32_t)((pl & 1) * 2 + at) * vatom;
        tma_load_2d(sm + dst, mapV, bar_v, 64 * at, (w * 4 + pl) * a.npad);
      }
  };
  auto issue_f = [&]() {
    mbar_expect_tx(bar_f, 4u * vatom);
    for (int pl = 0; pl < 2; ++pl)
      for (int at = 0; at < 2; ++at)
        tma_load_2d(sm + (pl ? a.off_flo : a.off_fhi) + at * vatom, mapF, bar_f, 64 * at, pl * a.npad);
  };
  const uint32_t idesc_w = idesc_bf16(4 * CWP), idesc_n = idesc_bf16(2 * CWP);
  // F: D1 = F t.  V: D1 = Re V t (A atoms 0, 1), D2 = Im V t (A atoms 2, 3).  Per 16-wide k-step
  // A hi [B hi; B lo] (N = 4 CWP) and A lo B hi (N = 2 CWP).  Returns false once another role has
  // given up (recorded in the status word), so no further product is issued.
  auto product = [&](bool isv) {
    const uint64_t ah = isv ? dvhi : dfhi, al = isv ? dvlo : dflo;
    for (int h = 0; h < (isv ? 2 : 1); ++h) {
      const uint32_t d = tmem + (uint32_t)(h * 4 * CWP);
      for (int ks = 0; ks < a.nk; ++ks) {
        const uint32_t ko = (uint32_t)(ks & 3) * 32u;
        const uint64_t ao = ((uint32_t)(2 * h + (ks >> 2)) * vatom + ko) >> 4;
        const uint64_t bo = ((uint32_t)(ks >> 2) * batom + ko) >> 4;
        umma_bf16(d, ah + ao, db + bo, idesc_w, ks > 0 ? 1u : 0u);   // A hi [B hi; B lo]
        umma_bf16(d, al + ao, db + bo, idesc_n, 1u);                 // A lo B hi
      }
    }
    umma_commit(bar_mma);
    // An empty asm consuming blockIdx.x: with this nvcc the issue loop compiled with it runs the
    // propagation in 0.084 ms instead of 0.096 ms at N = 108, W = 640 (measured; the code generation
    // differs, why is not known).  It has no effect on the results.
    asm volatile("" ::"r"(blockIdx.x));
    if (*abort_flag) {   // another role gave up: record it and issue nothing more
      atomicOr(a.status, kStatusTimeout);
      return false;
    }
    return true;
  };
  int wk = run_next_live(a.w, r, r.first);
  if (wk >= r.end) return true;
  const bool early = idle;
  if (early) {
    issue_f();
    issue_v(wk);
  }
  idle = false;
  bool first = true;
  while (wk < r.end) {
    const int nxt = run_next_live(a.w, r, wk + r.stride);
    for (int ch = 0; ch < a.nch; ++ch) {
      if (!mbar_wait(bar_b, ph_b, abort_flag)) return false;
      ph_b ^= 1u;
      if (first) {
        if (!early) {
          issue_f();
          issue_v(wk);
        }
        if (!mbar_wait(bar_f, ph_f, abort_flag)) return false;
        ph_f ^= 1u;
        first = false;
      }
      tc_fence_after();
      if (!product(false)) return false;   // F psi
      for (int k = 1; k <= a.order; ++k) {
        if (!mbar_wait(bar_b, ph_b, abort_flag)) return false;
        ph_b ^= 1u;
        if (ch == 0 && k == 1) {
          if (!mbar_wait(bar_v, ph_v, abort_flag)) return false;
          ph_v ^= 1u;
          if (nxt < r.end)   // the next walker's V into L2 now, into shared memory later
            for (int pl = 0; pl < 4; ++pl)
              for (int at = 0; at < 2; ++at) tma_prefetch_l2_2d(mapV, 64 * at, (nxt * 4 + pl) * a.npad);
        }
        tc_fence_after();
        if (!product(true)) return false;   // V t_{k-1} / k
      }
      if (!mbar_wait(bar_b, ph_b, abort_flag)) return false;
      ph_b ^= 1u;
      if (ch == a.nch - 1 && nxt < r.end) issue_v(nxt);   // every V product of this walker has completed
      tc_fence_after();
      if (!product(false)) return false;   // F acc
    }
    wk = nxt;
  }
  return true;
}

// Epilogue (warps 0-15) for a run of walkers of one system: warp w covers lanes 32 (w % 4) .. + 31
// (rows p) and columns j0 .. j0 + SW - 1 of the chunk.  The next item's psi slice is loaded while
// the current item's products run: into registers (PF), or into L2 and read at the item's start
// (fewer live registers, for the grouped kernel).  The propagated chunk is staged in the B buffer
// (free once the last product has completed: N cwn complex entries fit in its 1024 CWP bytes for
// N <= 128) and written to psi by consecutive threads on consecutive addresses.
template <int CWP, bool PF>
__device__ __forceinline__ bool prop_epi_run(uint8_t* sm, uint32_t tmem, const PropTcParams& a, const WalkerRun r,
                                             int warp, int lane, uint64_t* bar_mma, uint64_t* bar_b, uint64_t* bar_e,
                                             volatile int* abort_flag, uint32_t& ph_m, uint32_t& ph_e) {
  constexpr int SW = CWP / 4;
  const int quad = warp & 3, j0 = (warp >> 2) * SW;
  const int p = 32 * quad + lane;
  const bool row = p < a.N;
  const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16);
  uint8_t* bsm = sm + a.off_b;
  float2* stage = reinterpret_cast<float2*>(bsm);
  const int tid = threadIdx.x;   // 0 .. 511 over the epilogue warps
  const BOffsets<CWP, SW> bo(p, j0);
  float accr[SW], acci[SW], dr[SW], di[SW];
  float2 nxv[PF ? SW : 1];
  auto slice_src = [&](int w_, int c_) { return a.psi + ((size_t)w_ * a.N + (row ? p : 0)) * a.ncol + c_ * a.cw; };
  auto load_slice = [&](int w_, int c_) {
    const int cwn = min(a.cw, a.ncol - c_ * a.cw);
    const float2* src = slice_src(w_, c_);
#pragma unroll
    for (int jj = 0; jj < SW; ++jj) nxv[PF ? jj : 0] = (row && j0 + jj < cwn) ? src[j0 + jj] : make_float2(0.f, 0.f);
  };
  // (wk, ch) the current item, (nwk, nch) the next one: found during the previous item, so the
  // weight read that finds it is hidden behind a product
  auto next_item = [&](int w_, int c_, int& w2, int& c2) {
    w2 = w_;
    c2 = c_ + 1;
    if (c2 == a.nch) {
      c2 = 0;
      w2 = run_next_live(a.w, r, w_ + r.stride);
    }
  };
  int wk = run_next_live(a.w, r, r.first), ch = 0, nwk, nch;
  if (wk < r.end) next_item(wk, ch, nwk, nch);
  if (PF && wk < r.end) load_slice(wk, 0);
  while (wk < r.end) {
    const int c0 = ch * a.cw, cwn = min(a.cw, a.ncol - c0);
    int nnwk = r.end, nnch = 0;
    if constexpr (PF) {
#pragma unroll
      for (int jj = 0; jj < SW; ++jj) {
        accr[jj] = dr[jj] = nxv[jj].x;
        acci[jj] = di[jj] = nxv[jj].y;
      }
    } else {
      const float2* src = slice_src(wk, ch);
#pragma unroll
      for (int jj = 0; jj < SW; ++jj) {
        const float2 v = (row && j0 + jj < cwn) ? src[j0 + jj] : make_float2(0.f, 0.f);
        accr[jj] = dr[jj] = v.x;
        acci[jj] = di[jj] = v.y;
      }
    }
    write_b<CWP, SW>(bsm, bo, dr, di);
    signal_b(bar_b, lane);
    if (nwk < r.end) {   // lands while this item's products run
      if constexpr (PF) {
        load_slice(nwk, nch);
      } else if (row && j0 == 0) {   // one thread per row: the first and last lines of its segment
        const float2* src = slice_src(nwk, nch);
        const int cwn2 = min(a.cw, a.ncol - nch * a.cw);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(src) : "memory");
        asm volatile("prefetch.global.L2 [%0];" ::"l"(src + cwn2 - 1) : "memory");
      }
    }
    if (!warp_wait(bar_mma, ph_m, abort_flag, lane)) return false;
    ph_m ^= 1u;
    load_d<CWP, SW, false>(trow, j0, dr, di);   // F psi
#pragma unroll
    for (int jj = 0; jj < SW; ++jj) {   // t_0 = psi + F psi
      accr[jj] = row ? accr[jj] + dr[jj] : 0.f;
      acci[jj] = row ? acci[jj] + di[jj] : 0.f;
    }
    write_b<CWP, SW>(bsm, bo, accr, acci);
    signal_b(bar_b, lane);
    next_item(nwk, nch, nnwk, nnch);   // while the first V product runs
    for (int k = 1; k <= a.order; ++k) {
      if (!warp_wait(bar_mma, ph_m, abort_flag, lane)) return false;
      ph_m ^= 1u;
      load_d<CWP, SW, true>(trow, j0, dr, di);   // t_k
      const float s = 1.f / (float)(k + 1);
#pragma unroll
      for (int jj = 0; jj < SW; ++jj) {
        const float tr = row ? dr[jj] : 0.f, ti = row ? di[jj] : 0.f;
        accr[jj] += tr;
        acci[jj] += ti;
        dr[jj] = tr * s;   // next operand t_k / (k + 1)
        di[jj] = ti * s;
      }
      if (k < a.order) write_b<CWP, SW>(bsm, bo, dr, di);
      else write_b<CWP, SW>(bsm, bo, accr, acci);
      signal_b(bar_b, lane);
    }
    if (!warp_wait(bar_mma, ph_m, abort_flag, lane)) return false;
    ph_m ^= 1u;
    load_d<CWP, SW, false>(trow, j0, dr, di);   // F acc
#pragma unroll
    for (int jj = 0; jj < SW; ++jj)
      if (row && j0 + jj < cwn) stage[p * cwn + j0 + jj] = make_float2(accr[jj] + dr[jj], acci[jj] + di[jj]);
    if (!epi_sync(bar_e, ph_e, abort_flag, lane)) return false;
    float2* dst = a.psi + (size_t)wk * a.N * a.ncol + c0;
    const int n = a.N * cwn;
    if (cwn == a.ncol) {   // the walker's rows are one contiguous block
      for (int e = tid; e < n; e += 32 * kEpiWarps) dst[e] = stage[e];
    } else {
      for (int e = tid; e < n; e += 32 * kEpiWarps) {
        const int pp = e / cwn;
        dst[(size_t)pp * a.ncol + (e - pp * cwn)] = stage[e];
      }
    }
    if (!epi_sync(bar_e, ph_e, abort_flag, lane)) return false;   // the B buffer is free again
    wk = nwk;
    ch = nch;
    nwk = nnwk;
    nch = nnch;
  }
  return true;
}

// Shared set-up of both small-form kernels: mbarriers, tensor memory.
struct PropBars {
  uint64_t *v, *f, *mma, *b, *e;
  volatile int* abort_flag;
  uint32_t tmem;
};

__device__ __forceinline__ PropBars prop_begin(uint8_t* sm, int off_bar, int tmem_cols, int warp) {
  PropBars pb;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + off_bar);
  pb.v = bars;
  pb.f = bars + 1;
  pb.mma = bars + 2;
  pb.b = bars + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  pb.abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  pb.e = bars + 5;
  if (threadIdx.x == 0) {
    mbar_init(pb.v, 1);
    mbar_init(pb.f, 1);
    mbar_init(pb.mma, 1);
    mbar_init(pb.b, kEpiWarps);
    mbar_init(pb.e, kEpiWarps);
    *pb.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pb.tmem = *tmem_slot;
  return pb;
}

// After an abort, in-flight copies and MMAs drain before tensor memory is freed.
__device__ __forceinline__ void prop_end(const PropBars& pb, int tmem_cols, int warp) {
  if (threadIdx.x == 0 && *pb.abort_flag) {
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < 2000000ull) {
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kEpiWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(pb.tmem), "r"(tmem_cols) : "memory");
}

template <int CWP>
__global__ void __launch_bounds__(kPropThreads, 1) k_prop_tc(const __grid_constant__ CUtensorMap mapV,
                                                             const __grid_constant__ CUtensorMap mapF,
                                                             const __grid_constant__ PropTcParams a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PropBars pb = prop_begin(sm, a.off_bar, a.tmem_cols, warp);
  const WalkerRun r{(int)blockIdx.x, (int)gridDim.x, a.W};
  bool go = true;
  if (warp == kEpiWarps) {
    uint32_t ph_b = 0, ph_v = 0, ph_f = 0;
    bool idle = true;
    go = prop_mma_run<CWP>(sm, pb.tmem, &mapV, &mapF, a, r, idle, pb.v, pb.f, pb.mma, pb.b, pb.abort_flag, ph_b,
                           ph_v, ph_f, lane);
  } else {
    uint32_t ph_m = 0, ph_e = 0;
    go = prop_epi_run<CWP, true>(sm, pb.tmem, a, r, warp, lane, pb.mma, pb.b, pb.e, pb.abort_flag, ph_m, ph_e);
  }
  if (!go && lane == 0) {
    atomicOr(a.status, kStatusTimeout);
    *pb.abort_flag = 1;
  }
  prop_end(pb, a.tmem_cols, warp);
}

// ---------------------------------------------------------------------------------------------
// Grouped small form: one launch over the walkers of several systems (N <= 128).  CTA b takes the
// walkers [cta_first[b], cta_first[b + 1]) of the launch's list (the systems in turn; contiguous
// ranges balanced by cost on the host, so a CTA rarely changes system), as one run of walkers per
// system.  Each system keeps its own shared-memory layout and operand width (CWP, dispatched per
// run); the mbarriers sit past the largest layout.  The next walker's V is prefetched only within
// a system.
struct PropTcProblem {   // aligned as its tensor maps
  CUtensorMap mapV, mapF;
  PropTcParams p;
  int cwp;
  int item0;   // the system's walker 0 in the launch's list
};

__global__ void __launch_bounds__(kPropThreads, 1) k_prop_tc_group(const PropTcProblem* __restrict__ probs, int nprob,
                                                                   const int* __restrict__ cta_first, int off_bar,
                                                                   int tmem_cols) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PropBars pb = prop_begin(sm, off_bar, tmem_cols, warp);
  const int i0 = cta_first[blockIdx.x], i1 = cta_first[blockIdx.x + 1];
  const bool mma = warp == kEpiWarps;
  bool go = true;
  {
    uint32_t ph_b = 0, ph_v = 0, ph_f = 0, ph_m = 0, ph_e = 0;
    bool idle = true;
    int cur = 0;
    for (int i = i0; i < i1 && go;) {
      while (cur + 1 < nprob && i >= probs[cur + 1].item0) ++cur;
      const PropTcProblem& pr = probs[cur];
      const int end = min(i1, pr.item0 + pr.p.W);
      const WalkerRun r{i - pr.item0, 1, end - pr.item0};
      if (mma) {
        const PropTcParams a = pr.p;   // a register copy: the MMAs' asm would force reloads of a reference
        switch (pr.cwp) {
          case 8: go = prop_mma_run<8>(sm, pb.tmem, &pr.mapV, &pr.mapF, a, r, idle, pb.v, pb.f, pb.mma, pb.b, pb.abort_flag, ph_b, ph_v, ph_f, lane); break;
          case 16: go = prop_mma_run<16>(sm, pb.tmem, &pr.mapV, &pr.mapF, a, r, idle, pb.v, pb.f, pb.mma, pb.b, pb.abort_flag, ph_b, ph_v, ph_f, lane); break;
          case 24: go = prop_mma_run<24>(sm, pb.tmem, &pr.mapV, &pr.mapF, a, r, idle, pb.v, pb.f, pb.mma, pb.b, pb.abort_flag, ph_b, ph_v, ph_f, lane); break;
          default: go = prop_mma_run<32>(sm, pb.tmem, &pr.mapV, &pr.mapF, a, r, idle, pb.v, pb.f, pb.mma, pb.b, pb.abort_flag, ph_b, ph_v, ph_f, lane); break;
        }
      } else {
        switch (pr.cwp) {
          case 8: go = prop_epi_run<8, false>(sm, pb.tmem, pr.p, r, warp, lane, pb.mma, pb.b, pb.e, pb.abort_flag, ph_m, ph_e); break;
          case 16: go = prop_epi_run<16, false>(sm, pb.tmem, pr.p, r, warp, lane, pb.mma, pb.b, pb.e, pb.abort_flag, ph_m, ph_e); break;
          case 24: go = prop_epi_run<24, false>(sm, pb.tmem, pr.p, r, warp, lane, pb.mma, pb.b, pb.e, pb.abort_flag, ph_m, ph_e); break;
          default: go = prop_epi_run<32, false>(sm, pb.tmem, pr.p, r, warp, lane, pb.mma, pb.b, pb.e, pb.abort_flag, ph_m, ph_e); break;
        }
      }
      i = end;
    }
  }
  if (!go && lane == 0) {
    for (int c = 0; c < nprob; ++c) atomicOr(probs[c].p.status, kStatusTimeout);
    *pb.abort_flag = 1;
  }
  prop_end(pb, tmem_cols, warp);
}

// ---------------------------------------------------------------------------------------------
// Large form (N > 128): one launch per product over all (walker, 128-row tile) pairs.  A is the
// walker's V (K = Re V | Im V) or F, streamed through a ring of TMA stages; B is the current term
// as split bf16 [hi, lo][2 ncolp rows][2 kq] (rows: real parts, then imaginary parts; K halves as
// in the fused kernel).  The epilogue (4 warps, thread = row p) adds the product to the Taylor
// sum acc [W][npad][ncolp] (complex64), writes the next term operand (column k = p of its rows,
// consecutive lanes on consecutive addresses), and the last product writes psi.
// mode 0: D = F psi, t_0 = psi + D;  mode k = 1..order: D = V t_{k-1} / k = t_k;
// mode order + 1: D = F acc, psi = acc + D.
struct PropGemmParams {
  int N, npad, kq, nq, ncol, ncolp, bn, mtiles, W, order, mode, stages;
  int cplx_f;   // complex F: four planes like V, F products over both K halves
  float2* psi;
  const double* w;
  float2* acc;
  __nv_bfloat16* bnext;   // next term operand, [W][2][bn][2 kq]
  int* status;
};

__device__ __forceinline__ int prop_kblocks(const PropGemmParams& a) {
  const bool freal = (a.mode == 0 || a.mode == a.order + 1) && !a.cplx_f;
  return 3 * (freal ? 1 : 2) * a.nq;
}

// TMA coordinates and k-steps of k-block j of tile (wk, mt): segments (A hi, B hi), (A lo, B hi),
// (A hi, B lo); V products run over two K halves (Re V against the first half of B, Im V against
// the second).
__device__ __forceinline__ void prop_kblock(const PropGemmParams& a, int wk, int mt, int j, int* ax, int* ay, int* bx,
                                            int* by, int* ksteps) {
  const bool fmode = a.mode == 0 || a.mode == a.order + 1;
  const bool freal = fmode && !a.cplx_f;
  const int halves = freal ? 1 : 2;
  const int seg = j / (halves * a.nq), h = (j / a.nq) % halves, qb = j % a.nq;
  const int alo = seg == 1 ? 1 : 0, blo = seg == 2 ? 1 : 0;
  *ax = qb * 64;
  *ay = freal ? alo * a.npad + mt * 128 : ((fmode ? 0 : wk) * 4 + 2 * alo + h) * a.npad + mt * 128;
  *bx = h * a.kq + qb * 64;
  *by = (wk * 2 + blo) * a.bn;
  *ksteps = min(4, (a.N - qb * 64 + 15) / 16);
}

// GROUP: one launch per product over the (walker, 128-row tile) pairs of several systems.  System i
// owns tiles [tile0, tile0 + tiles) of the launch; its maps (V, F and both term operands) and
// parameters are read from device memory, the product index comes from the launch, and the ring
// of stages and the accumulators are laid out for the widest system.
struct PropGemmProblem {   // aligned as its tensor maps
  CUtensorMap mapV, mapF, mapB[2];
  PropGemmParams p;            // p.mode is the launch's
  __nv_bfloat16* b[2];         // term operands: product m reads b[m % 2], writes b[(m + 1) % 2]
  int tile0, tiles;
};
struct PropGroupArgs {
  const PropGemmProblem* probs;
  int nprob, tiles, mode, stages, stride, tmem_cols, acc_stride;
};

template <bool GROUP>
__global__ void __launch_bounds__(192, 1) k_prop_gemm_t(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapB,
                                                        const __grid_constant__ PropGemmParams a0,
                                                        const __grid_constant__ PropGroupArgs ga) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int stages = GROUP ? ga.stages : a0.stages;
  const int stride = GROUP ? ga.stride : 16384 + a0.bn * 128;
  const uint32_t acc_stride = (uint32_t)(GROUP ? ga.acc_stride : a0.bn);
  const int tiles = GROUP ? ga.tiles : a0.W * a0.mtiles;
  const int tmem_cols = GROUP ? ga.tmem_cols
                              : (2 * a0.bn <= 32 ? 32 : (2 * a0.bn <= 64 ? 64 : (2 * a0.bn <= 128 ? 128 : (2 * a0.bn <= 256 ? 256 : 512))));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stride);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* tfull = bars + 2 * stages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // tile t: its system's parameters (with the launch's product) and maps, walker and row tile
  struct Item {
    PropGemmParams a;
    const CUtensorMap* ma;
    const CUtensorMap* mb;
    int wk, mt;
  };
  auto resolve = [&](int t, int& cur) -> Item {
    Item it;
    if constexpr (GROUP) {
      while (cur + 1 < ga.nprob && t >= ga.probs[cur + 1].tile0) ++cur;
      const PropGemmProblem& pr = ga.probs[cur];
      it.a = pr.p;
      it.a.mode = ga.mode;
      it.a.bnext = pr.b[(ga.mode + 1) % 2];
      const bool fmode = ga.mode == 0 || ga.mode == it.a.order + 1;
      it.ma = fmode ? &pr.mapF : &pr.mapV;
      it.mb = &pr.mapB[ga.mode % 2];
      t -= pr.tile0;
    } else {
      (void)cur;
      it.a = a0;
      it.ma = &mapA;
      it.mb = &mapB;
    }
    it.wk = t / it.a.mtiles;
    it.mt = t - it.wk * it.a.mtiles;
    return it;
  };
  auto give_up = [&](int* status) {
    if constexpr (GROUP) {
      (void)status;
      for (int i = 0; i < ga.nprob; ++i) atomicOr(ga.probs[i].p.status, kStatusTimeout);
    } else {
      atomicOr(status, kStatusTimeout);
    }
    *abort_flag = 1;
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      int stage = 0, cur = 0;
      uint32_t ph = 0;
      bool go = true;
      int* status = a0.status;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x) {
        const Item it = resolve(t, cur);
        const PropGemmParams& a = it.a;
        status = a.status;
        if (a.w[it.wk] == 0.0) continue;
        const int nkb = prop_kblocks(a), bytes = 16384 + a.bn * 128;
        for (int j = 0; j < nkb; ++j) {
          int ax, ay, bx, by, ks;
          prop_kblock(a, it.wk, it.mt, j, &ax, &ay, &bx, &by, &ks);
          if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag)) { go = false; break; }
          uint8_t* sa = smem + (size_t)stage * stride;
          mbar_expect_tx(&full[stage], (uint32_t)bytes);
          tma_load_2d(sa, it.ma, &full[stage], ax, ay);
          tma_load_2d(sa + 16384, it.mb, &full[stage], bx, by);
          if (++stage == stages) { stage = 0; ph ^= 1u; }
        }
      }
      if (!go) give_up(status);
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      int stage = 0, n_it = 0, cur = 0;
      uint32_t ph = 0;
      bool go = true;
      int* status = a0.status;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x) {
        const Item it = resolve(t, cur);
        const PropGemmParams& a = it.a;
        status = a.status;
        if (a.w[it.wk] == 0.0) continue;
        const uint32_t idesc = idesc_bf16(a.bn);
        const int nkb = prop_kblocks(a);
        const int acc = n_it & 1;
        const uint32_t aph = (uint32_t)(n_it >> 1) & 1u;
        ++n_it;
        if (!mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) { go = false; break; }
        tc_fence_after();
        const uint32_t dtm = tmem + (uint32_t)acc * acc_stride;
        bool first = true;
        for (int j = 0; j < nkb; ++j) {
          int ax, ay, bx, by, ks;
          prop_kblock(a, it.wk, it.mt, j, &ax, &ay, &bx, &by, &ks);
          if (!mbar_wait(&full[stage], ph, abort_flag)) { go = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)stage * stride), sb = sa + 16384;
          for (int k = 0; k < ks; ++k) {
            umma_bf16(dtm, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc, first ? 0u : 1u);
            first = false;
          }
          umma_commit(&empty[stage]);
          if (++stage == stages) { stage = 0; ph ^= 1u; }
        }
        if (!go) break;
        umma_commit(&tfull[acc]);
      }
      if (!go) give_up(status);
    }
  } else {   // epilogue: warps 2-5, lane quadrant warp % 4
    const int q = warp & 3;
    int n_it = 0, cur = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const Item it = resolve(t, cur);
      const PropGemmParams& a = it.a;
      const int wk = it.wk, mt = it.mt;
      if (a.w[wk] == 0.0) continue;
      const float s = (a.mode >= 1 && a.mode < a.order) ? 1.f / (float)(a.mode + 1) : 1.f;
      const size_t kk2 = (size_t)2 * a.kq;
      const int acc = n_it & 1;
      const uint32_t aph = (uint32_t)(n_it >> 1) & 1u;
      ++n_it;
      int ok = 0;
      if (lane == 0) ok = mbar_wait(&tfull[acc], aph, abort_flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) give_up(a.status);
        break;
      }
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_stride;
      const int p = mt * 128 + 32 * q + lane;
      const bool row = p < a.N, kpad = p < a.kq;
      float2* accrow = a.acc + ((size_t)wk * a.npad + (row ? p : 0)) * a.ncolp;
      float2* prow = a.psi + ((size_t)wk * a.N + (row ? p : 0)) * a.ncol;
      __nv_bfloat16* bw = a.bnext + (size_t)wk * 2 * a.bn * kk2;
      for (int c0 = 0; c0 < a.ncolp; c0 += 8) {
        uint32_t ur[8], ui[8];
        tmem_ld8_nowait(trow + (uint32_t)c0, ur);
        tmem_ld8_nowait(trow + (uint32_t)(a.ncolp + c0), ui);
        tmem_wait();
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int c = c0 + jj;
          float2 d = make_float2(__uint_as_float(ur[jj]), __uint_as_float(ui[jj]));
          float2 u = make_float2(0.f, 0.f);   // next operand entry
          bool both = true;
          if (row) {
            if (a.mode == 0) {
              const float2 ps = c < a.ncol ? prow[c] : make_float2(0.f, 0.f);
              u = make_float2(ps.x + d.x, ps.y + d.y);
              accrow[c] = u;
            } else if (a.mode <= a.order) {
              float2 sum = accrow[c];
              sum.x += d.x;
              sum.y += d.y;
              accrow[c] = sum;
              if (a.mode < a.order) {
                u = make_float2(d.x * s, d.y * s);
              } else {
                u = sum;
                both = a.cplx_f != 0;   // a real F product reads the first K half only
              }
            } else {
              const float2 sum = accrow[c];
              if (c < a.ncol) prow[c] = make_float2(sum.x + d.x, sum.y + d.y);
            }
          }
          if (a.mode <= a.order && kpad) {
            const __nv_bfloat16 rh = __float2bfloat16_rn(u.x), ih = __float2bfloat16_rn(u.y);
            const __nv_bfloat16 rl = __float2bfloat16_rn(u.x - __bfloat162float(rh));
            const __nv_bfloat16 il = __float2bfloat16_rn(u.y - __bfloat162float(ih));
            __nv_bfloat16* hre = bw + (size_t)c * kk2;                 // row c (real parts)
            __nv_bfloat16* him = bw + (size_t)(a.ncolp + c) * kk2;     // row ncolp + c (imaginary parts)
            const size_t lo = (size_t)a.bn * kk2;                      // the lo plane
            hre[p] = rh; hre[lo + p] = rl;
            him[p] = ih; him[lo + p] = il;
            if (both) {
              hre[a.kq + p] = __hneg(ih); hre[lo + a.kq + p] = __hneg(il);
              him[a.kq + p] = rh;         him[lo + a.kq + p] = rl;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  if (threadIdx.x == 0 && *abort_flag) {   // let in-flight copies and MMAs drain before freeing tensor memory
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 < 2000000ull) {
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}


// First operand of the large form: psi of every walker as split bf16 rows (real parts, then
// imaginary parts) over the first K half; K positions N .. kq - 1 and padding columns are zero.
struct PsiToB {
  int W, N, ncol, ncolp, kq, both;
  const float2* psi;
  __nv_bfloat16* b;
};
__device__ __forceinline__ void psi_to_b(const PsiToB& a, size_t first, size_t step) {
  const size_t kk2 = (size_t)2 * a.kq;
  const int bn = 2 * a.ncolp;
  const size_t total = (size_t)a.W * a.ncolp * a.kq;
  for (size_t idx = first; idx < total; idx += step) {
    const int p = (int)(idx % a.kq);
    const size_t r = idx / a.kq;
    const int c = (int)(r % a.ncolp);
    const int wk = (int)(r / a.ncolp);
    float2 v = make_float2(0.f, 0.f);
    if (p < a.N && c < a.ncol) v = a.psi[((size_t)wk * a.N + p) * a.ncol + c];
    const __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
    const __nv_bfloat16 rl = __float2bfloat16_rn(v.x - __bfloat162float(rh));
    const __nv_bfloat16 il = __float2bfloat16_rn(v.y - __bfloat162float(ih));
    __nv_bfloat16* bw = a.b + (size_t)wk * 2 * bn * kk2;
    const size_t lo = (size_t)bn * kk2;
    bw[(size_t)c * kk2 + p] = rh;
    bw[lo + (size_t)c * kk2 + p] = rl;
    bw[(size_t)(a.ncolp + c) * kk2 + p] = ih;
    bw[lo + (size_t)(a.ncolp + c) * kk2 + p] = il;
    if (a.both) {   // the second K half for a complex first product: rows [Re | -Im] and [Im | Re]
      bw[(size_t)c * kk2 + a.kq + p] = __hneg(ih);
      bw[lo + (size_t)c * kk2 + a.kq + p] = __hneg(il);
      bw[(size_t)(a.ncolp + c) * kk2 + a.kq + p] = rh;
      bw[lo + (size_t)(a.ncolp + c) * kk2 + a.kq + p] = rl;
    }
  }
}
__global__ void k_psi_to_b(PsiToB a) {
  psi_to_b(a, blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}
// Several systems at once: blockIdx.y is the system.
__global__ void k_psi_to_b_group(const PsiToB* __restrict__ jobs) {
  psi_to_b(jobs[blockIdx.y], blockIdx.x * (size_t)blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
}

// F = E_h - I (binary64 [N][N]) -> planes [hi, lo][npad][kq], zero outside N x N.  Complex F
// (interleaved binary64): planes [Re hi, Im hi, Re lo, Im lo], the order of the V planes.
__global__ void k_f_planes(int N, int npad, int kq, const double* f64, __nv_bfloat16* out, int cplx) {
  const int per = npad * kq, np = cplx ? 4 : 2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np * per; idx += gridDim.x * blockDim.x) {
    const int pl = idx / per, rem = idx % per, p = rem / kq, q = rem % kq;
    const int part = cplx ? (pl & 1) : 0, lo = cplx ? pl >> 1 : pl;
    const size_t e = (size_t)p * N + q;
    const double v = (p < N && q < N) ? (cplx ? f64[2 * e + part] : f64[e]) : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(v);
    out[idx] = lo ? __double2bfloat16(v - (double)__bfloat162float(hi)) : hi;
  }
}

template <int CWP>
afqmc_status launch_prop(const TcState* st, cudaStream_t s, const PropTcParams& p, unsigned long long* launches,
                         char* err, size_t errlen) {
  const int grid = std::min(st->W, num_sms());
  k_prop_tc<CWP><<<grid, kPropThreads, st->pg.smem, s>>>(st->map_vp, st->map_fp, p);
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tensor-core propagation launch: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

}  // namespace

int prop_gemm_stages(int bn) { return std::min(6, (kMaxSmem - 1024 - 256) / (16384 + bn * 128)); }
size_t prop_gemm_smem(int bn) { return 1024 + (size_t)prop_gemm_stages(bn) * (16384 + bn * 128) + 256; }

PropGeom prop_geom(int N, int ncol, bool cplx) {
  PropGeom g{};
  if (N < 1 || ncol < 1) return g;
  if (N > 128 || cplx) {   // large form (a complex E_h has no room beside V in the fused kernel)
    if (ncol > 128) return g;
    g.large = 1;
    g.cplx_f = cplx ? 1 : 0;
    g.npad = (N + 7) / 8 * 8;
    g.kq = (N + 63) / 64 * 64;
    g.ncolp = (ncol + 7) / 8 * 8;
    g.mtiles = (N + 127) / 128;
    g.ok = prop_gemm_stages(2 * g.ncolp) >= 2 ? 1 : 0;
    return g;
  }
  const int npad = (N + 7) / 8 * 8;
  for (int cwmax : {32, 24, 16, 8}) {
    const int nch = (ncol + cwmax - 1) / cwmax;
    const int cw = (ncol + nch - 1) / nch;
    const int cwp = (cw + 7) / 8 * 8;
    PropGeom t{};
    t.npad = npad;
    t.kq = 128;
    t.nk = (N + 15) / 16;
    t.cw = cw;
    t.cwp = cwp;
    t.nch = nch;
    t.off_vlo = npad * 512;
    t.off_fhi = npad * 1024;
    t.off_flo = npad * 1280;
    t.off_b = npad * 1536;
    int end = t.off_b + cwp * 1024;   // 2 K atoms of 4 cwp rows
    // an M = 128 product reads 16 KiB from the start of every A atom, rows npad..127 included
    end = std::max(end, t.off_flo + npad * 128 + 16384);
    t.off_bar = (end + 63) / 64 * 64;
    t.smem = 1024 + t.off_bar + 64;
    if (t.smem <= kMaxSmem) {
      t.ok = 1;
      return t;
    }
  }
  return g;
}

afqmc_status prepare_prop(TcState* st, cudaStream_t s, char* tcbuf, const double* f64, unsigned long long* launches,
                          char* err, size_t errlen) {
  if (!st->pg.ok) return AFQMC_OK;
  const PropGeom& g = st->pg;
  __nv_bfloat16* vp = reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_vp);
  __nv_bfloat16* fp = reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_fp);
  if (cudaMemsetAsync(vp, 0, (size_t)st->W * 4 * g.npad * g.kq * 2, s) != cudaSuccess) {
    snprintf(err, errlen, "tensor-core propagation: clearing the V planes failed");
    return AFQMC_ECUDA;
  }
  k_f_planes<<<64, 256, 0, s>>>(st->N, g.npad, g.kq, f64, fp, g.cplx_f);
  ++*launches;
  const unsigned box = g.large ? 128u : (unsigned)g.npad;   // one 128-row tile, or every row
  if (!make_map(&st->map_vp, vp, (unsigned long long)st->W * 4 * g.npad, g.kq, box) ||
      !make_map(&st->map_fp, fp, (unsigned long long)(g.cplx_f ? 4 : 2) * g.npad, g.kq, box)) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed for the propagation planes");
    return AFQMC_ECUDA;
  }
  if (g.large) {
    for (int i = 0; i < 2; ++i) {
      void* b = tcbuf + st->off_b[i];
      const size_t bytes = (size_t)st->W * 2 * (2 * g.ncolp) * (2 * g.kq) * 2;
      if (cudaMemsetAsync(b, 0, bytes, s) != cudaSuccess ||
          !make_map(&st->map_b[i], b, (unsigned long long)st->W * 2 * 2 * g.ncolp, 2ull * g.kq,
                    (unsigned)(2 * g.ncolp))) {
        snprintf(err, errlen, "tensor-core propagation: term operand buffers");
        return AFQMC_ECUDA;
      }
    }
    if (cudaFuncSetAttribute(k_prop_gemm_t<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_prop_gemm_t<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
            cudaSuccess) {
      snprintf(err, errlen, "tensor-core propagation: cannot reserve shared memory");
      return AFQMC_ECUDA;
    }
  }
  const void* fns[4] = {reinterpret_cast<const void*>(k_prop_tc<8>), reinterpret_cast<const void*>(k_prop_tc<16>),
                        reinterpret_cast<const void*>(k_prop_tc<24>), reinterpret_cast<const void*>(k_prop_tc<32>)};
  for (const void* fn : fns)
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess) {
      snprintf(err, errlen, "tensor-core propagation: cannot reserve shared memory");
      return AFQMC_ECUDA;
    }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tensor-core propagation prepare: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

afqmc_status propagate(TcState* st, cudaStream_t s, char* tcbuf, int order, float2* psi, const double* w,
                       int* status, unsigned long long* launches, char* err, size_t errlen) {
  (void)tcbuf;
  const PropGeom& g = st->pg;
  if (!g.ok) {
    snprintf(err, errlen, "tensor-core propagation is not available for this problem");
    return AFQMC_EINVAL;
  }
  if (g.large) {
    __nv_bfloat16* b[2] = {reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_b[0]),
                           reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_b[1])};
    k_psi_to_b<<<1184, 256, 0, s>>>(PsiToB{st->W, st->N, st->ncol, g.ncolp, g.kq, g.cplx_f, psi, b[0]});
    ++*launches;
    PropGemmParams q{};
    q.cplx_f = g.cplx_f;
    q.N = st->N; q.npad = g.npad; q.kq = g.kq; q.nq = g.kq / 64; q.ncol = st->ncol; q.ncolp = g.ncolp;
    q.bn = 2 * g.ncolp; q.mtiles = g.mtiles; q.W = st->W; q.order = order;
    q.stages = prop_gemm_stages(q.bn);
    q.psi = psi; q.w = w; q.acc = reinterpret_cast<float2*>(tcbuf + st->off_acc); q.status = status;
    const int grid = std::min(st->W * g.mtiles, num_sms());
    const size_t smem = prop_gemm_smem(q.bn);
    for (int m = 0; m <= order + 1; ++m) {   // operand m % 2 in, (m + 1) % 2 out
      q.mode = m;
      q.bnext = b[(m + 1) % 2];
      const bool fmode = m == 0 || m == order + 1;
      k_prop_gemm_t<false><<<grid, 192, smem, s>>>(fmode ? st->map_fp : st->map_vp, st->map_b[m % 2], q,
                                                   PropGroupArgs{});
      ++*launches;
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        snprintf(err, errlen, "tensor-core propagation launch: %s", cudaGetErrorString(e));
        return AFQMC_ECUDA;
      }
    }
    return AFQMC_OK;
  }
  PropTcParams p{};
  p.N = st->N; p.npad = g.npad; p.nk = g.nk; p.ncol = st->ncol; p.cw = g.cw; p.nch = g.nch;
  p.order = order; p.W = st->W;
  p.off_vlo = g.off_vlo; p.off_fhi = g.off_fhi; p.off_flo = g.off_flo;
  p.off_b = g.off_b; p.off_bar = g.off_bar;
  p.tmem_cols = 8 * g.cwp <= 64 ? 64 : (8 * g.cwp <= 128 ? 128 : 256);   // D1 and D2, 4 cwp columns each
  p.psi = psi;
  p.w = w;
  p.status = status;
  switch (g.cwp) {
    case 8: return launch_prop<8>(st, s, p, launches, err, errlen);
    case 16: return launch_prop<16>(st, s, p, launches, err, errlen);
    case 24: return launch_prop<24>(st, s, p, launches, err, errlen);
    default: return launch_prop<32>(st, s, p, launches, err, errlen);
  }
}

// ---------------------------------------------------------------------------------------------
// Grouped propagation of several systems: the small-form systems in one k_prop_tc_group launch, the
// large-form systems in one k_prop_gemm_t<true> launch per product.
namespace {
template <typename T>
afqmc_status to_device_p(const std::vector<T>& v, void** dev, char* err, size_t errlen) {
  *dev = nullptr;
  if (v.empty()) return AFQMC_OK;
  if (cudaMalloc(dev, v.size() * sizeof(T)) != cudaSuccess ||
      cudaMemcpy(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    snprintf(err, errlen, "grouped propagation: device descriptors (%zu bytes)", v.size() * sizeof(T));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}
int tmem_pow2(int cols) {
  int c = 32;
  while (c < cols) c <<= 1;
  return c;
}
}  // namespace

afqmc_status group_prop_plan(const GroupPropSystem* sys, int nsys, int order, GroupProp* gp, char* err,
                             size_t errlen) {
  *gp = GroupProp{};
  gp->order = order;
  std::vector<PropTcProblem> small;
  std::vector<double> cost;   // per small-form walker
  std::vector<PropGemmProblem> large;
  std::vector<PsiToB> psib;
  int items = 0, off_bar = 0, tcols = 32;
  for (int i = 0; i < nsys; ++i) {
    TcState* st = sys[i].st;
    const PropGeom& g = st->pg;
    if (!g.ok) {
      snprintf(err, errlen, "grouped propagation: system %d has no tensor-core propagation", i);
      return AFQMC_EINVAL;
    }
    if (!g.large) {
      PropTcProblem q{};
      q.mapV = st->map_vp;
      q.mapF = st->map_fp;
      PropTcParams& p = q.p;
      p.N = st->N; p.npad = g.npad; p.nk = g.nk; p.ncol = st->ncol; p.cw = g.cw; p.nch = g.nch;
      p.order = order; p.W = st->W;
      p.off_vlo = g.off_vlo; p.off_fhi = g.off_fhi; p.off_flo = g.off_flo; p.off_b = g.off_b; p.off_bar = g.off_bar;
      p.tmem_cols = 8 * g.cwp <= 64 ? 64 : (8 * g.cwp <= 128 ? 128 : 256);
      p.psi = sys[i].psi;
      p.w = sys[i].w;
      p.status = sys[i].status;
      q.cwp = g.cwp;
      q.item0 = items;
      items += st->W;
      off_bar = std::max(off_bar, g.off_bar);
      tcols = std::max(tcols, p.tmem_cols);
      // cost of a walker: per chunk, order + 2 chained products (hand-off ~3k cycles each) and their MMAs
      const double c = (double)g.nch * ((order + 2) * 3000.0 + 55.0 * g.nk * (4.0 + 4.0 * order));
      for (int w = 0; w < st->W; ++w) cost.push_back(c);
      small.push_back(q);
    } else {
      PropGemmProblem q{};
      q.mapV = st->map_vp;
      q.mapF = st->map_fp;
      q.mapB[0] = st->map_b[0];
      q.mapB[1] = st->map_b[1];
      PropGemmParams& p = q.p;
      p.cplx_f = g.cplx_f;
      p.N = st->N; p.npad = g.npad; p.kq = g.kq; p.nq = g.kq / 64; p.ncol = st->ncol; p.ncolp = g.ncolp;
      p.bn = 2 * g.ncolp; p.mtiles = g.mtiles; p.W = st->W; p.order = order;
      p.stages = prop_gemm_stages(p.bn);
      p.psi = sys[i].psi; p.w = sys[i].w; p.status = sys[i].status;
      p.acc = reinterpret_cast<float2*>(sys[i].tcbuf + st->off_acc);
      for (int k = 0; k < 2; ++k) q.b[k] = reinterpret_cast<__nv_bfloat16*>(sys[i].tcbuf + st->off_b[k]);
      large.push_back(q);
      psib.push_back(PsiToB{st->W, st->N, st->ncol, g.ncolp, g.kq, g.cplx_f, sys[i].psi, q.b[0]});
    }
  }
  afqmc_status r;
  if (!small.empty()) {
    // contiguous walker ranges of about equal cost, one per CTA
    const int grid = std::min(items, num_sms());
    double total = 0.0;
    for (double c : cost) total += c;
    std::vector<int> first(grid + 1, items);
    first[0] = 0;
    double acc = 0.0;
    int b = 1;
    for (int it = 0; it < items && b < grid; ++it) {
      acc += cost[it];
      if (acc >= total * b / grid) first[b++] = it + 1;
    }
    for (; b < grid; ++b) first[b] = items;
    gp->nsmall = (int)small.size();
    gp->small_grid = grid;
    gp->small_off_bar = off_bar;
    gp->small_tmem = tcols;
    gp->small_smem = 1024 + (size_t)off_bar + 64;
    if (cudaFuncSetAttribute(k_prop_tc_group, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess) {
      snprintf(err, errlen, "grouped propagation: cannot reserve shared memory");
      return AFQMC_ECUDA;
    }
    if ((r = to_device_p(small, &gp->dev_small, err, errlen)) != AFQMC_OK ||
        (r = to_device_p(first, &gp->dev_cta, err, errlen)) != AFQMC_OK) {
      group_prop_free(gp);
      return r;
    }
  }
  if (!large.empty()) {
    std::stable_sort(large.begin(), large.end(), [](const PropGemmProblem& a, const PropGemmProblem& b) {
      return (long long)a.p.nq * a.p.bn > (long long)b.p.nq * b.p.bn;
    });
    int t = 0, bn = 0;
    for (auto& q : large) {
      q.tile0 = t;
      q.tiles = q.p.W * q.p.mtiles;
      t += q.tiles;
      bn = std::max(bn, q.p.bn);
    }
    gp->nlarge = (int)large.size();
    gp->large_tiles = t;
    gp->large_grid = std::min(t, num_sms());
    gp->large_stages = prop_gemm_stages(bn);
    gp->large_stride = 16384 + bn * 128;
    gp->large_acc = bn;
    gp->large_tmem = tmem_pow2(2 * bn);
    gp->large_smem = prop_gemm_smem(bn);
    if (gp->large_stages < 2 || gp->large_tmem > 512) {
      snprintf(err, errlen, "grouped propagation: no layout fits the widest system");
      group_prop_free(gp);
      return AFQMC_EINVAL;
    }
    if ((r = to_device_p(large, &gp->dev_large, err, errlen)) != AFQMC_OK ||
        (r = to_device_p(psib, &gp->dev_psib, err, errlen)) != AFQMC_OK) {
      group_prop_free(gp);
      return r;
    }
  }
  return AFQMC_OK;
}

afqmc_status group_propagate(const GroupProp& gp, cudaStream_t s, unsigned long long* launches, char* err,
                             size_t errlen, cudaStream_t s2) {
  const cudaStream_t sl = s2 ? s2 : s;   // the large-form launches
  if (gp.nsmall) {
    k_prop_tc_group<<<gp.small_grid, kPropThreads, gp.small_smem, s>>>(
        static_cast<const PropTcProblem*>(gp.dev_small), gp.nsmall, static_cast<const int*>(gp.dev_cta),
        gp.small_off_bar, gp.small_tmem);
    ++*launches;
  }
  if (gp.nlarge) {
    k_psi_to_b_group<<<dim3(296, gp.nlarge), 256, 0, sl>>>(static_cast<const PsiToB*>(gp.dev_psib));
    ++*launches;
    PropGroupArgs ga{};
    ga.probs = static_cast<const PropGemmProblem*>(gp.dev_large);
    ga.nprob = gp.nlarge;
    ga.tiles = gp.large_tiles;
    ga.stages = gp.large_stages;
    ga.stride = gp.large_stride;
    ga.tmem_cols = gp.large_tmem;
    ga.acc_stride = gp.large_acc;
    const CUtensorMap none{};
    const PropGemmParams p0{};
    for (int m = 0; m <= gp.order + 1; ++m) {   // operand m % 2 in, (m + 1) % 2 out
      ga.mode = m;
      k_prop_gemm_t<true><<<gp.large_grid, 192, gp.large_smem, sl>>>(none, none, p0, ga);
      ++*launches;
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "grouped propagation launch: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

void group_prop_free(GroupProp* gp) {
  for (void* p : {gp->dev_small, gp->dev_cta, gp->dev_large, gp->dev_psib})
    if (p) cudaFree(p);
  gp->dev_small = gp->dev_cta = gp->dev_large = gp->dev_psib = nullptr;
}

}  // namespace tc
}  // namespace afq
