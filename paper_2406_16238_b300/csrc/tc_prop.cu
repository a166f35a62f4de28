// Tensor-core propagation for the BF16 forms (Eq. 8 with the mean-field form of h_eff):
//   t = E_h psi,  acc = t,  t <- V t / k and acc += t for k = 1..order,  psi <- E_h acc,
// with E_h = exp(-dt/2 h_eff) applied as psi + F psi, F = E_h - I (F is O(dt), so its split-bf16
// product error is far below that of E_h itself).
//
// Per walker and chunk of cw columns every product is one tcgen05 contraction D = A B^T,
// M = 128 rows p (orbitals), N = 2 cwp (real parts of the chunk's columns, then imaginary
// parts), K = q over two halves:
//   A = [Re V | Im V]  (K = 256: q of Re V, then q of Im V),  A = F for E_h (first half only),
//   B rows c:        [Re t(:,c) | -Im t(:,c)],   B rows cwp + c: [Im t(:,c) | Re t(:,c)],
// so that D[p][c] = Re (V t)[p][c] and D[p][cwp + c] = Im (V t)[p][c].  Operands are split-bf16
// (hi + lo, products hi*hi + lo*hi + hi*lo, fp32 accumulation in tensor memory).
//
// Roles: warp 16 (one thread) loads F once and each walker's V planes by TMA and issues the MMAs;
// warps 0-15 read the accumulator, warp w covering lanes 32 (w % 4) .. + 31 (rows p) and a
// quarter of the chunk's columns: it keeps its part of row p of acc in registers and writes the
// matching entries of column k = p of the next B operand (hi and lo) into shared memory.  V of the
// next walker is fetched as soon as the last Taylor product of the current one has completed.
// Rows p >= N of D (padding, and rows 112-127 which the MMA reads from the following buffer)
// are never used: those threads write zeros into B.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace afq {
namespace tc {

namespace {

struct PropTcParams {
  int N, npad, nk, ncol, cw, nch, order, W;
  int off_vlo, off_fhi, off_flo, off_bhi, off_blo, off_bar;
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

// Columns j0 .. j0 + SW - 1 of column k = p of the next B operand from this thread's slice of
// the term (ur, ui); `both` also writes the second K half (needed by the V products, not by the
// F products).
template <int CWP, int SW>
__device__ __forceinline__ void write_b(uint8_t* bhi, uint8_t* blo, int p, int j0, const float* ur, const float* ui,
                                        bool both) {
  constexpr int ab = 2 * CWP * 128;
#pragma unroll
  for (int jj = 0; jj < SW; ++jj) {
    const int j = j0 + jj;
    const __nv_bfloat16 rh = __float2bfloat16_rn(ur[jj]);
    const __nv_bfloat16 rl = __float2bfloat16_rn(ur[jj] - __bfloat162float(rh));
    const __nv_bfloat16 ih = __float2bfloat16_rn(ui[jj]);
    const __nv_bfloat16 il = __float2bfloat16_rn(ui[jj] - __bfloat162float(ih));
    const uint32_t o_r = sw_off(j, p, ab), o_i = sw_off(CWP + j, p, ab);
    st_bf16(bhi, o_r, rh);
    st_bf16(blo, o_r, rl);
    st_bf16(bhi, o_i, ih);
    st_bf16(blo, o_i, il);
    if (both) {
      const uint32_t o_r2 = sw_off(j, 128 + p, ab), o_i2 = sw_off(CWP + j, 128 + p, ab);
      st_bf16(bhi, o_r2, __hneg(ih));
      st_bf16(blo, o_r2, __hneg(il));
      st_bf16(bhi, o_i2, rh);
      st_bf16(blo, o_i2, rl);
    }
  }
}

// Generic-proxy writes of B become visible to the tensor core; one arrival per warp.
__device__ __forceinline__ void signal_b(uint64_t* bar_b, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(bar_b);
}

// Lane 0 waits, the warp follows its verdict (tcgen05.ld needs the whole warp).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) tc_fence_after();
  return ok != 0;
}

// SW consecutive accumulator columns of this thread's lane (no wait).
template <int SW>
__device__ __forceinline__ void ld_cols(uint32_t taddr, uint32_t* r) {
  if constexpr (SW == 2) {
    tmem_ld2_nowait(taddr, r);
  } else if constexpr (SW == 4) {
    tmem_ld4_nowait(taddr, r);
  } else if constexpr (SW == 6) {
    tmem_ld4_nowait(taddr, r);
    tmem_ld2_nowait(taddr + 4, r + 4);
  } else {
    static_assert(SW == 8, "slice width");
    tmem_ld8_nowait(taddr, r);
  }
}

// This thread's slice of row p of D: dr[jj] = D[p][j0 + jj], di[jj] = D[p][CWP + j0 + jj].
template <int CWP, int SW>
__device__ __forceinline__ void load_d(uint32_t trow, int j0, float* dr, float* di) {
  uint32_t r[SW], q[SW];
  ld_cols<SW>(trow + (uint32_t)j0, r);
  ld_cols<SW>(trow + (uint32_t)(CWP + j0), q);
  tmem_wait();
#pragma unroll
  for (int jj = 0; jj < SW; ++jj) {
    dr[jj] = __uint_as_float(r[jj]);
    di[jj] = __uint_as_float(q[jj]);
  }
}

constexpr int kEpiWarps = 16;                 // 4 lane quadrants x 4 column slices
constexpr int kPropThreads = 32 * kEpiWarps + 32;

template <int CWP>
__global__ void __launch_bounds__(kPropThreads, 1) k_prop_tc(const __grid_constant__ CUtensorMap mapV,
                                                             const __grid_constant__ CUtensorMap mapF,
                                                             const PropTcParams a) {
  constexpr int SW = CWP / 4;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + a.off_bar);
  uint64_t* bar_v = bars;
  uint64_t* bar_f = bars + 1;
  uint64_t* bar_mma = bars + 2;
  uint64_t* bar_b = bars + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(bar_v, 1);
    mbar_init(bar_f, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar_b, kEpiWarps);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto next_live = [&](int from) {
    for (int k = from; k < a.W; k += gridDim.x)
      if (a.w[k] != 0.0) return k;
    return a.W;
  };

  if (warp == kEpiWarps) {
    if (lane == 0) {   // TMA + MMA issue
      const uint32_t s0 = smem_u32(sm);
      const uint32_t vatom = (uint32_t)a.npad * 128u, batom = 2u * CWP * 128u;
      const uint32_t idesc = idesc_bf16(2 * CWP);
      // descriptors are linear in the address: desc(base + off) = desc(base) + off / 16
      const uint64_t dvhi = sw128_desc(s0), dvlo = sw128_desc(s0 + (uint32_t)a.off_vlo);
      const uint64_t dfhi = sw128_desc(s0 + (uint32_t)a.off_fhi), dflo = sw128_desc(s0 + (uint32_t)a.off_flo);
      const uint64_t dbhi = sw128_desc(s0 + (uint32_t)a.off_bhi), dblo = sw128_desc(s0 + (uint32_t)a.off_blo);
      auto issue_v = [&](int wk) {
        mbar_expect_tx(bar_v, 8u * vatom);
        for (int pl = 0; pl < 4; ++pl)
          for (int at = 0; at < 2; ++at) {
            const uint32_t dst = (pl < 2 ? 0u : (uint32_t)a.off_vlo) + (uint32_t)((pl & 1) * 2 + at) * vatom;
            tma_load_2d(sm + dst, &mapV, bar_v, 64 * at, (wk * 4 + pl) * a.npad);
          }
      };
      auto product = [&](bool isv) {
        const uint64_t ah = isv ? dvhi : dfhi, al = isv ? dvlo : dflo;
        uint32_t accf = 0;
        for (int h = 0; h < (isv ? 2 : 1); ++h)
          for (int ks = 0; ks < a.nk; ++ks) {
            const int atom = 2 * h + (ks >> 2);
            const uint32_t ko = (uint32_t)(ks & 3) * 32u;
            const uint64_t ao = ((uint32_t)atom * vatom + ko) >> 4, bo = ((uint32_t)atom * batom + ko) >> 4;
            umma_bf16(tmem, ah + ao, dbhi + bo, idesc, accf);
            accf = 1;
            umma_bf16(tmem, al + ao, dbhi + bo, idesc, 1);
            umma_bf16(tmem, ah + ao, dblo + bo, idesc, 1);
          }
        umma_commit(bar_mma);
      };
      bool go = true;
      uint32_t ph_b = 0, ph_v = 0;
      int wk = next_live(blockIdx.x);
      if (wk < a.W) {
        mbar_expect_tx(bar_f, 4u * vatom);
        for (int pl = 0; pl < 2; ++pl)
          for (int at = 0; at < 2; ++at)
            tma_load_2d(sm + (pl ? a.off_flo : a.off_fhi) + at * vatom, &mapF, bar_f, 64 * at, pl * a.npad);
        issue_v(wk);
      }
      bool f_ready = false;
      while (wk < a.W && go) {
        for (int ch = 0; ch < a.nch && go; ++ch) {
          if (!mbar_wait(bar_b, ph_b, abort_flag)) { go = false; break; }
          ph_b ^= 1u;
          if (!f_ready) {
            if (!mbar_wait(bar_f, 0, abort_flag)) { go = false; break; }
            f_ready = true;
          }
          tc_fence_after();
          product(false);   // F psi
          for (int k = 1; k <= a.order && go; ++k) {
            if (!mbar_wait(bar_b, ph_b, abort_flag)) { go = false; break; }
            ph_b ^= 1u;
            if (ch == 0 && k == 1) {
              if (!mbar_wait(bar_v, ph_v, abort_flag)) { go = false; break; }
              ph_v ^= 1u;
            }
            tc_fence_after();
            product(true);   // V t_{k-1} / k
          }
          if (!go) break;
          if (!mbar_wait(bar_b, ph_b, abort_flag)) { go = false; break; }
          ph_b ^= 1u;
          if (ch == a.nch - 1) {   // every V product of this walker has completed
            const int nxt = next_live(wk + gridDim.x);
            if (nxt < a.W) issue_v(nxt);
          }
          tc_fence_after();
          product(false);   // F acc
        }
        wk = next_live(wk + gridDim.x);
      }
      if (!go) {
        atomicOr(a.status, kStatusTimeout);
        *abort_flag = 1;
      }
    }
  } else {   // epilogue warp: lanes 32 (warp % 4) .. + 31, columns j0 .. j0 + SW - 1 of the chunk
    const int quad = warp & 3, j0 = (warp >> 2) * SW;
    const int p = 32 * quad + lane;
    const bool row = p < a.N;
    const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16);
    uint8_t* bhi = sm + a.off_bhi;
    uint8_t* blo = sm + a.off_blo;
    uint32_t ph_m = 0;
    bool go = true;
    float accr[SW], acci[SW], dr[SW], di[SW];
    for (int wk = next_live(blockIdx.x); wk < a.W && go; wk = next_live(wk + gridDim.x)) {
      for (int ch = 0; ch < a.nch; ++ch) {
        const int c0 = ch * a.cw, cwn = min(a.cw, a.ncol - c0);
        float2* prow = a.psi + ((size_t)wk * a.N + (row ? p : 0)) * a.ncol + c0;
#pragma unroll
        for (int jj = 0; jj < SW; ++jj) {
          float2 v = make_float2(0.f, 0.f);
          if (row && j0 + jj < cwn) v = prow[j0 + jj];
          accr[jj] = dr[jj] = v.x;
          acci[jj] = di[jj] = v.y;
        }
        write_b<CWP, SW>(bhi, blo, p, j0, dr, di, false);
        signal_b(bar_b, lane);
        if (!(go = warp_wait(bar_mma, ph_m, abort_flag, lane))) break;
        ph_m ^= 1u;
        load_d<CWP, SW>(trow, j0, dr, di);   // F psi
#pragma unroll
        for (int jj = 0; jj < SW; ++jj) {   // t_0 = psi + F psi
          accr[jj] = row ? accr[jj] + dr[jj] : 0.f;
          acci[jj] = row ? acci[jj] + di[jj] : 0.f;
        }
        write_b<CWP, SW>(bhi, blo, p, j0, accr, acci, true);
        signal_b(bar_b, lane);
        for (int k = 1; k <= a.order; ++k) {
          if (!(go = warp_wait(bar_mma, ph_m, abort_flag, lane))) break;
          ph_m ^= 1u;
          load_d<CWP, SW>(trow, j0, dr, di);   // t_k
          const float s = 1.f / (float)(k + 1);
#pragma unroll
          for (int jj = 0; jj < SW; ++jj) {
            const float tr = row ? dr[jj] : 0.f, ti = row ? di[jj] : 0.f;
            accr[jj] += tr;
            acci[jj] += ti;
            dr[jj] = tr * s;   // next operand t_k / (k + 1)
            di[jj] = ti * s;
          }
          if (k < a.order) write_b<CWP, SW>(bhi, blo, p, j0, dr, di, true);
          else write_b<CWP, SW>(bhi, blo, p, j0, accr, acci, false);
          signal_b(bar_b, lane);
        }
        if (!go) break;
        if (!(go = warp_wait(bar_mma, ph_m, abort_flag, lane))) break;
        ph_m ^= 1u;
        load_d<CWP, SW>(trow, j0, dr, di);   // F acc
#pragma unroll
        for (int jj = 0; jj < SW; ++jj)
          if (row && j0 + jj < cwn) prow[j0 + jj] = make_float2(accr[jj] + dr[jj], acci[jj] + di[jj]);
      }
    }
    if (!go && lane == 0) {
      atomicOr(a.status, kStatusTimeout);
      *abort_flag = 1;
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
  if (warp == kEpiWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
}

// F = E_h - I (binary64 [N][N]) -> planes [hi, lo][npad][128], zero outside N x N.
__global__ void k_f_planes(int N, int npad, const double* f64, __nv_bfloat16* out) {
  const int per = npad * 128;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * per; idx += gridDim.x * blockDim.x) {
    const int pl = idx / per, rem = idx % per, p = rem / 128, q = rem % 128;
    const double v = (p < N && q < N) ? f64[(size_t)p * N + q] : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(v);
    out[idx] = pl ? __double2bfloat16(v - (double)__bfloat162float(hi)) : hi;
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

PropGeom prop_geom(int N, int ncol) {
  PropGeom g{};
  if (N < 1 || N > 128 || ncol < 1) return g;
  const int npad = (N + 7) / 8 * 8;
  for (int cwmax : {32, 24, 16, 8}) {
    const int nch = (ncol + cwmax - 1) / cwmax;
    const int cw = (ncol + nch - 1) / nch;
    const int cwp = (cw + 7) / 8 * 8;
    PropGeom t{};
    t.npad = npad;
    t.nk = (N + 15) / 16;
    t.cw = cw;
    t.cwp = cwp;
    t.nch = nch;
    t.off_vlo = npad * 512;
    t.off_fhi = npad * 1024;
    t.off_flo = npad * 1280;
    t.off_bhi = npad * 1536;
    t.off_blo = t.off_bhi + cwp * 1024;
    int end = t.off_blo + cwp * 1024;
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
  if (cudaMemsetAsync(vp, 0, (size_t)st->W * 4 * g.npad * 128 * 2, s) != cudaSuccess) {
    snprintf(err, errlen, "tensor-core propagation: clearing the V planes failed");
    return AFQMC_ECUDA;
  }
  k_f_planes<<<64, 256, 0, s>>>(st->N, g.npad, f64, fp);
  ++*launches;
  if (!make_map(&st->map_vp, vp, (unsigned long long)st->W * 4 * g.npad, 128, (unsigned)g.npad) ||
      !make_map(&st->map_fp, fp, (unsigned long long)2 * g.npad, 128, (unsigned)g.npad)) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed for the propagation planes");
    return AFQMC_ECUDA;
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
  PropTcParams p{};
  p.N = st->N; p.npad = g.npad; p.nk = g.nk; p.ncol = st->ncol; p.cw = g.cw; p.nch = g.nch;
  p.order = order; p.W = st->W;
  p.off_vlo = g.off_vlo; p.off_fhi = g.off_fhi; p.off_flo = g.off_flo;
  p.off_bhi = g.off_bhi; p.off_blo = g.off_blo; p.off_bar = g.off_bar;
  p.tmem_cols = 2 * g.cwp <= 32 ? 32 : 64;
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

}  // namespace tc
}  // namespace afq
