// Tensor-core (tcgen05 + TMA) contractions for the BF16 and BF16x3 forms.
//
// One persistent, warp-specialised GEMM kernel D = A B^T (A [M][K], B [Ncols][K],
// both bf16 K-major, fp32 accumulation in tensor memory) with two epilogues:
//   EPI 0 (exchange): the tile holds T^{g}_{ab} for gpt gammas x wpt walkers;
//          the epilogue forms Tr T (force bias) and sum_ab T_ab T_ba (exchange).
//   EPI 1 (store): the tile is written to an fp32 matrix (the VHS build).
// Roles per CTA: warp 0 issues TMA loads into a ring of shared-memory stages,
// warp 1 allocates tensor memory and one of its threads issues tcgen05.mma
// (M = 128, N = bn, K = 16 per instruction) into one of two accumulators,
// warps 2.. read the finished accumulator with tcgen05.ld while the next tile
// is being multiplied.  Every wait is bounded: on timeout the kernel records
// kStatusTimeout, the roles stop, and tensor memory is released.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace afq {
namespace tc {

constexpr int kStageA = kBM * kBK * 2;           // 16 KiB
constexpr int kTailBytes = 512;                  // mbarriers, TMEM slot, abort flag (< 256 B), then the series tables
constexpr int kParamSlot = 384;                  // grouped launch: one epilogue group's copy of its problem's Params

struct Geom {
  int m_tiles, n_tiles, k_blocks;
  int k_steps;              // 16-wide MMA k-steps with data (the last k-block may be partly past K)
  int m_step, n_step;       // TMA row coordinate of tile (mt, nt): mt * m_step, nt * n_step
  int bn;                   // MMA N
  int stages, epi_groups;
  int epi_bytes;            // per epilogue group
  int tmem_cols;
  // il3: split operands stored as [hi | lo] (seg elements each), one operand tile per stage: virtual
  // k-block v takes real k-block v / 3 of (A hi, B hi), (A lo, B hi), (A hi, B lo) for v % 3 = 0, 1, 2
  // (twice the stages of the dual form, for operands streamed from HBM)
  int il3, seg;
  // dual: every stage holds the hi and lo parts of both operands of one real k-block (A hi at column
  // 0, A lo at a_lo, B hi at b_hi, B lo at b_lo, plus kb * 64) and each 16-wide k-step issues the
  // three split products, so each operand byte crosses shared memory once (k_blocks, k_steps: real)
  int dual, a_lo, b_hi, b_lo;
  int stage_bytes;
  // tile order: 0: M tiles fastest; ntg > 0: groups of ntg N tiles, M tiles in turn within a group,
  // N tiles fastest (concurrent CTAs share A tiles; a group's B tiles stay in L2)
  int ntg;
};

__host__ __device__ __forceinline__ void tile_mn(const Geom& g, int t, int* mt, int* nt) {
  if (g.ntg <= 0) {
    *mt = t % g.m_tiles;
    *nt = t / g.m_tiles;
    return;
  }
  const int per = g.m_tiles * g.ntg;
  const int grp = t / per, rem = t - grp * per;
  const int nsz = g.n_tiles - grp * g.ntg < g.ntg ? g.n_tiles - grp * g.ntg : g.ntg;
  *mt = rem / nsz;
  *nt = grp * g.ntg + (rem - (rem / nsz) * nsz);
}

struct Params {
  Geom g;
  int* status;
  // exchange epilogue
  int W, X, n, gpt, wpt, chunk_offset, nchunk;
  int vbias_add;   // staged epilogue: 0 store, 1 add (second spin block), 2 atomic add (grouped launch)
  float smul;
  float2* vbias;
  float2* exch_part;   // binary32 partials (the epilogue's sums are binary32)
  // store epilogue
  float* out;
  long long ldo;
  int out_rows, out_cols;
  // bf16 plane epilogue
  __nv_bfloat16* planes;
  int npad, kq;   // plane rows, plane row pitch (elements)
  const int* pairs;   // packed L^T: p N + q of each packed row (p <= q; -1: a row left out), or NULL
  const int2* blocks; // packed L^T: the (8-row p block, 16-column q block) of each M tile
  // exchange: an extra warp draws the step's normals (nrm.x != nullptr)
  NormalsJob nrm;
  // exchange with the Ltilde tile in tensor memory: segment length and the tensor-memory column of
  // its hi half (the lo half follows kst / 2 columns later)
  int kst, a0;
};


// ----------------------------------------------------------------------------- epilogues
// Exchange epilogue state of one warpgroup: [ok flags 2 x int (16 B)] [buf: the staged tile]
// [diag 128 float2] [red 4 float2].  Each group handles one walker per tile (wpt == groups).
struct EpiSmem {
  float* buf;
  float2* diag;
  float2* red;
  int* ok;
};

// Row pitch of the staged tile, >= 2n + 1 and = 1 (mod 32): thread r's row r and the partner rows
// (g n + b) it reads at column a then fall in distinct banks for the 32 rows of a warp.
__host__ __device__ __forceinline__ int exch_ld(int n) { return 32 * ((2 * n + 31) / 32) + 1; }
__host__ __device__ __forceinline__ int exch_buf_bytes(int n) { return ((128 * exch_ld(n) * 4) + 15) & ~15; }
// Register-row epilogue: rows of complex entries (float2), pitch n | 1 entries.  An odd pitch puts
// the 8-byte entries of 16 consecutive rows (one half-warp access) in distinct bank pairs; partner
// reads whose half-warp spans two gamma blocks may meet 2-way conflicts.  (A pitch with n (ld2 - 1)
// a multiple of 16 removes those, but the larger buffers cost ring stages and measured slower.)
__host__ __device__ __forceinline__ int exch_ld2(int n) { return n | 1; }
__host__ __device__ __forceinline__ int exch_buf2_bytes(int n) { return ((128 * exch_ld2(n) * 8) + 15) & ~15; }

__device__ __forceinline__ EpiSmem epi_smem(uint8_t* base, const Params& p, int group, bool reg) {
  EpiSmem e;
  uint8_t* g = base + (size_t)group * p.g.epi_bytes;
  e.ok = reinterpret_cast<int*>(g);
  e.buf = reinterpret_cast<float*>(g + 16);
  e.diag = reinterpret_cast<float2*>(g + 16 + (reg ? exch_buf2_bytes(p.n) : exch_buf_bytes(p.n)));
  e.red = e.diag + 128;
  return e;
}

// ncols accumulator columns of this thread's row into dst, loads batched 32 + 8 + 2 + 1 under one wait
// per 32-column chunk.
__device__ __forceinline__ void tmem_row_to_smem(uint32_t taddr, int ncols, float* dst) {
  int c = 0;
  for (; c + 32 <= ncols; c += 32) {
    float v[16];
    tmem_ld16(taddr + c, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) dst[c + i] = v[i];
    tmem_ld16(taddr + c + 16, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) dst[c + 16 + i] = v[i];
  }
  const int rem = ncols - c;
  if (rem <= 0) return;
  uint32_t r[32];
  int k = 0;
  if (rem & 16) { uint32_t* q = r + k; float v[16]; tmem_ld16(taddr + c + k, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = __float_as_uint(v[i]);
    k += 16; }
  if (rem & 8) { tmem_ld8_nowait(taddr + c + k, r + k); k += 8; }
  if (rem & 4) { tmem_ld4_nowait(taddr + c + k, r + k); k += 4; }
  if (rem & 2) { tmem_ld2_nowait(taddr + c + k, r + k); k += 2; }
  if (rem & 1) { tmem_ld1_nowait(taddr + c + k, r + k); k += 1; }
  tmem_wait();
  for (int i = 0; i < rem; ++i) dst[c + i] = __uint_as_float(r[i]);
}

// One walker per group and tile: stage its 2n accumulator columns, form the row products,
// then warp 0 of the group writes vbias for the tile's gammas and the exchange partial.
__device__ void exchange_tile(const Params& p, int mt, int nt, uint32_t tacc, const EpiSmem& e, int group,
                              int wig, int r, int lane) {
  const int n = p.n, n2 = 2 * n, ld = exch_ld(n), rows = p.gpt * n;
  const int bar_id = 1 + group;
  for (int v = group; v < p.wpt; v += p.g.epi_groups) {
    tmem_row_to_smem(tacc + (uint32_t)(v * n2), n2, e.buf + r * ld);
    named_bar(bar_id, 128);
    float er = 0.f, ei = 0.f;
    float2 dg = make_float2(0.f, 0.f);
    if (r < rows) {
      const int g = r / n, a = r % n;
      if (mt * p.gpt + g < p.X) {
        const float* rowr = e.buf + r * ld;
        const float* blk = e.buf + (g * n) * ld;
#pragma unroll 4
        for (int b = 0; b < n; ++b) {
          const float tr = rowr[b], ti = rowr[n + b];
          const float ur = blk[b * ld + a], ui = blk[b * ld + n + a];
          er = fmaf(tr, ur, er);
          er = fmaf(-ti, ui, er);
          ei = fmaf(tr, ui, ei);
          ei = fmaf(ti, ur, ei);
        }
        dg = make_float2(rowr[a], rowr[n + a]);
      }
    }
    e.diag[r] = dg;
    er = warp_sum_f(er);
    ei = warp_sum_f(ei);
    if (lane == 0) e.red[wig] = make_float2(er, ei);
    named_bar(bar_id, 128);
    const int w = nt * p.wpt + v;
    if (w < p.W && wig == 0) {
      for (int gl = lane; p.vbias && gl < p.gpt; gl += 32) {   // one gamma per lane, sequential sum over its n rows
        const int gam = mt * p.gpt + gl;
        if (gam >= p.X) continue;
        float sr = 0.f, si = 0.f;
        for (int a = 0; a < n; ++a) {
          const float2 d = e.diag[gl * n + a];
          sr += d.x;
          si += d.y;
        }
        float2* dst = p.vbias + (size_t)w * p.X + gam;
        float2 val = make_float2(p.smul * sr, p.smul * si);
        if (p.vbias_add == 2) {   // grouped launch: both spin blocks run at once, onto a cleared vbias
          atomicAdd(dst, val);
          continue;
        }
        if (p.vbias_add) {
          val.x += dst->x;
          val.y += dst->y;
        }
        *dst = val;
      }
      if (lane < 4) {   // the tile's four partial slots: the sum in the first, zeros in the others
        const float sr = (e.red[0].x + e.red[1].x) + (e.red[2].x + e.red[3].x);
        const float si = (e.red[0].y + e.red[1].y) + (e.red[2].y + e.red[3].y);
        p.exch_part[(size_t)w * p.nchunk + p.chunk_offset + 4 * mt + lane] =
            lane == 0 ? make_float2(p.smul * sr, p.smul * si) : make_float2(0.f, 0.f);
      }
    }
    if (v + p.g.epi_groups < p.wpt) named_bar(bar_id, 128);   // buffers reused by the next walker
  }
}

// NB consecutive accumulator columns of this thread's lane into v (no wait).
template <int NB>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t* v) {
  static_assert(NB % 8 == 0 && NB <= 32, "column count");
  if constexpr (NB >= 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
  }
  if constexpr (NB == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr + 16)
        : "memory");
  }
  if constexpr (NB % 16 == 8) tmem_ld8_nowait(taddr + (NB - 8), v + (NB - 8));
}

// As exchange_tile, with the thread's own row T_ab (b < n <= NB) kept in registers: the real
// parts come from columns [v 2n, v 2n + NB), the imaginary parts from [v 2n + n, v 2n + n + NB)
// (the columns past the walker are read and ignored).  The row goes to shared memory as complex
// entries, and each partner entry T_ba is read back with one 8-byte load.  After that each warp
// works alone: its exchange partial goes to slot 4 mt + (warp in group) of the walker's partials,
// and the per-gamma traces (force bias) are summed by a segmented scan over the warp's rows (the
// diagonal T_aa read back from the thread's staged row) and added to vbias, which the caller has
// zeroed: a gamma block (n <= 32 rows) meets at most two warps, and two additions onto zero give
// the same bits in either order, so the result does not depend on timing.
template <int NB>
__device__ void exchange_tile_reg(const Params& p, int mt, int nt, uint32_t tacc, const EpiSmem& e, int group,
                                  int wig, int r, int lane) {
  const int n = p.n, n2 = 2 * n, ld2 = exch_ld2(n), rows = p.gpt * n;
  const int bar_id = 1 + group;
  const int g = r / n, a = r - (r / n) * n;
  const bool live = r < rows && mt * p.gpt + g < p.X;
  float2* buf = reinterpret_cast<float2*>(e.buf);
  float2* rowp = buf + r * ld2;
  const float2* part = buf + (g * n) * ld2 + a;   // T_ba at part[b ld2]
  for (int v = group; v < p.wpt; v += p.g.epi_groups) {
    uint32_t ur[NB], ui[NB];
    tmem_ld_cols<NB>(tacc + (uint32_t)(v * n2), ur);
    tmem_ld_cols<NB>(tacc + (uint32_t)(v * n2 + n), ui);
    tmem_wait();
    if (v > group) named_bar(bar_id, 128);   // every partner read of the previous walker is done
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < n) rowp[b] = make_float2(__uint_as_float(ur[b]), __uint_as_float(ui[b]));
    named_bar(bar_id, 128);
    float er0 = 0.f, ei0 = 0.f, er1 = 0.f, ei1 = 0.f;
    float2 dg = make_float2(0.f, 0.f);
    if (live) {
#pragma unroll
      for (int b = 0; b < NB; b += 2) {
        if (b < n) {
          const float tr = __uint_as_float(ur[b]), ti = __uint_as_float(ui[b]);
          const float2 q = part[b * ld2];
          er0 = fmaf(tr, q.x, er0);
          er0 = fmaf(-ti, q.y, er0);
          ei0 = fmaf(tr, q.y, ei0);
          ei0 = fmaf(ti, q.x, ei0);
        }
        if (b + 1 < n) {
          const float tr = __uint_as_float(ur[b + 1]), ti = __uint_as_float(ui[b + 1]);
          const float2 q = part[(b + 1) * ld2];
          er1 = fmaf(tr, q.x, er1);
          er1 = fmaf(-ti, q.y, er1);
          ei1 = fmaf(tr, q.y, ei1);
          ei1 = fmaf(ti, q.x, ei1);
        }
      }
      dg = rowp[a];   // T_aa
    }
    // the warp's exchange sum (butterfly) and the inclusive segmented scan of the diagonal over the
    // warp's rows of gamma block g, interleaved
    float er = er0 + er1, ei = ei0 + ei1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      er += __shfl_xor_sync(0xffffffffu, er, 32 / (2 * o));
      ei += __shfl_xor_sync(0xffffffffu, ei, 32 / (2 * o));
      const float tx = __shfl_up_sync(0xffffffffu, dg.x, o), ty = __shfl_up_sync(0xffffffffu, dg.y, o);
      if (lane >= o && r - o >= g * n) {
        dg.x += tx;
        dg.y += ty;
      }
    }
    const int w = nt * p.wpt + v;
    if (lane == 0 && w < p.W)
      p.exch_part[(size_t)w * p.nchunk + p.chunk_offset + 4 * mt + wig] = make_float2(p.smul * er, p.smul * ei);
    if (p.vbias && live && w < p.W && (lane == 31 || a == n - 1))   // last row of the block within this warp
      atomicAdd(p.vbias + (size_t)w * p.X + mt * p.gpt + g, make_float2(p.smul * dg.x, p.smul * dg.y));
  }
}

__device__ void store_tile(const Params& p, int mt, int nt, uint32_t tacc, int group, int r) {
  const int row = mt * p.g.m_step + r;
  const int c0 = nt * p.g.n_step;
  const int ncols = p.g.bn / p.g.epi_groups;     // each group covers a contiguous share of the columns
  const int cbeg = group * ncols;
  float v[16];
  for (int c = cbeg; c < cbeg + ncols; c += 16) {
    tmem_ld16(tacc + (uint32_t)c, v);
    if (row >= p.out_rows) continue;
    float* dst = p.out + (size_t)row * p.ldo + c0 + c;
    const int rem = p.out_cols - (c0 + c);
    if (rem >= 16 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
      for (int i = 0; i < 16; i += 4) *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
      for (int i = 0; i < 16 && i < rem; ++i) dst[i] = v[i];
    }
  }
}

// Tile rows are pq = p N + q (M over N^2), columns are (w, part) = 2 w + part.  Each value is
// split into hi = bf16(v), lo = bf16(v - hi) and written to the plane
// [w][hi re, hi im, lo re, lo im][npad][kq] at (p, q).  Consecutive lanes hold consecutive pq,
// so every store instruction covers a contiguous run of q.
__device__ void store_planes(const Params& p, int mt, int nt, uint32_t tacc, int group, int r) {
  const int pq = mt * kBM + r;
  const bool live = pq < p.out_cols;
  const int pp = live ? pq / p.n : 0, qq = live ? pq - pp * p.n : 0;
  const int ncols = p.g.bn / p.g.epi_groups;   // a multiple of 8
  const int cbeg = group * ncols;
  const size_t plane = (size_t)p.npad * p.kq;
  auto put = [&](int c, int cnt, const float* v) {
    for (int i = 0; i < cnt; ++i) {
      const int col = nt * p.g.n_step + c + i;
      if (col >= p.out_rows) break;
      __nv_bfloat16* dst = p.planes + ((size_t)(col >> 1) * 4 + (col & 1)) * plane + (size_t)pp * p.kq + qq;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v[i]);
      dst[0] = hi;
      dst[2 * plane] = __float2bfloat16_rn(v[i] - __bfloat162float(hi));
    }
  };
  float v[16];
  int c = cbeg;
  for (; c + 16 <= cbeg + ncols; c += 16) {
    tmem_ld16(tacc + (uint32_t)c, v);
    if (live) put(c, 16, v);
  }
  if (c < cbeg + ncols) {   // 8 columns left
    uint32_t r8[8];
    tmem_ld8_nowait(tacc + (uint32_t)c, r8);
    tmem_wait();
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r8[i]);
    if (live) put(c, 8, v);
  }
}

// Packed L^T: each M tile is one block of the symmetric V, p in [8 bi, 8 bi + 8) x q in
// [16 bj, 16 bj + 16) (row r = 16 (p - 8 bi) + q - 16 bj), with 8 bi <= 16 bj + 15.  Entries with
// p <= q are written at (p, q): a warp covers two p rows of 16 q (two full 32-byte sectors).  Entries
// with p < q are also written at (q, p): staged per group in shared memory, eight columns at a time,
// then written as rows of 8 consecutive p (16-byte stores; blocks (bi, bj) and (bi + 1, bj) are
// consecutive tiles, so the other half of each sector follows at once).  stage: 8 columns x 128 rows x
// (hi, lo) bf16 = 4 KiB per group.
__device__ void store_planes_packed(const Params& p, int mt, int nt, uint32_t tacc, int group, int r,
                                    __nv_bfloat16* stage) {
  const int2 blk = p.blocks[mt];
  const int p0 = 8 * blk.x, q0 = 16 * blk.y;
  const int pp = p0 + (r >> 4), qq = q0 + (r & 15);
  const bool direct = pp < p.n && qq < p.n && pp <= qq;
  const bool full = p0 + 7 < q0;   // every entry of the block has p < q
  const int ncols = p.g.bn / p.g.epi_groups;   // a multiple of 8
  const int cbeg = group * ncols;
  const size_t plane = (size_t)p.npad * p.kq;
  const int tid = r;   // 0 .. 127 within the group
  for (int c = cbeg; c < cbeg + ncols; c += 8) {
    uint32_t r8[8];
    tmem_ld8_nowait(tacc + (uint32_t)c, r8);
    tmem_wait();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = __uint_as_float(r8[i]);
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      const int col = nt * p.g.n_step + c + i;
      if (direct && col < p.out_rows) {
        __nv_bfloat16* dst = p.planes + ((size_t)(col >> 1) * 4 + (col & 1)) * plane + (size_t)pp * p.kq + qq;
        dst[0] = hi;
        dst[2 * plane] = lo;
      }
      stage[(i * 2 + 0) * 128 + r] = hi;
      stage[(i * 2 + 1) * 128 + r] = lo;
    }
    named_bar(5 + group, 128);
    // mirrored rows: 8 columns x 2 parts x 16 q rows, 8 consecutive p each
    for (int task = tid; task < 8 * 2 * 16; task += 128) {
      const int i = task >> 5, hl = (task >> 4) & 1, ql = task & 15;
      const int col = nt * p.g.n_step + c + i, q = q0 + ql;
      if (col >= p.out_rows || q >= p.n) continue;
      const __nv_bfloat16* src = stage + (i * 2 + hl) * 128 + ql;   // rows 16 pl + ql
      __nv_bfloat16* dst = p.planes + ((size_t)(col >> 1) * 4 + (col & 1) + 2 * hl) * plane + (size_t)q * p.kq + p0;
      if (full) {
        __align__(16) __nv_bfloat16 row[8];
#pragma unroll
        for (int pl = 0; pl < 8; ++pl) row[pl] = src[16 * pl];
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(row);
      } else {
        for (int pl = 0; pl < 8; ++pl)
          if (p0 + pl < q && p0 + pl < p.n) dst[pl] = src[16 * pl];
      }
    }
    named_bar(5 + group, 128);   // the stage is rewritten by the next columns
  }
}

// The step's normals drawn by one warp per CTA (pairs strided over the grid); tab_mem holds the
// series tables.
__device__ void draw_normals_warp(const NormalsJob& nj, uint8_t* tab_mem, int lane) {
  SeriesTables& tab = *reinterpret_cast<SeriesTables*>(tab_mem);
  if (lane == 0) fill_series_tables(&tab);
  __syncwarp();
  const unsigned long long st = *nj.step;
  const int npairs = (nj.X + 1) / 2;
  const long long total = (long long)nj.W * npairs;
  for (long long i = (long long)blockIdx.x * 32 + lane; i < total; i += (long long)gridDim.x * 32) {
    const int w = (int)(i / npairs), j = (int)(i - (long long)w * npairs);
    double z0, z1;
    normal_pair(nj.seed, (uint32_t)j, (uint32_t)w, st, 0u, tab, &z0, &z1);
    nj.x[(size_t)w * nj.X + 2 * j] = z0;
    if (2 * j + 1 < nj.X) nj.x[(size_t)w * nj.X + 2 * j + 1] = z1;
  }
}

// ----------------------------------------------------------------------------- the kernel
// GROUP: one persistent launch over the tiles of several independent problems (systems, spin
// blocks).  Problem i owns tiles [tile0, tile0 + tiles) of the launch's list (in problem order, each
// CTA's tiles ascending, so a cursor finds the problem); its tensor maps and parameters are read
// from device memory.  The ring of stages, the epilogue buffers and the two accumulators are laid
// out for the largest problem (GroupArgs); each problem's own Geom gives its tiles, K blocks, MMA N
// and the bytes a stage receives.
static_assert(sizeof(Params) <= kParamSlot && sizeof(Params) % 4 == 0, "parameter slot");

struct GroupProblem {   // aligned as its tensor maps
  CUtensorMap mapA, mapB;
  Params p;        // p.g: the problem's own tiles, MMA N, stage bytes, epilogue groups and buffers
  int tile0, tiles;
  int nb;          // exchange: register-row epilogue width (8, 16, 24, 32), 0: the staged epilogue (one per launch)
};
struct GroupArgs {
  const GroupProblem* probs;
  int nprob, tiles;
  int stages, stage_stride, epi_groups, epi_bytes, tmem_cols, acc_stride;
  const NormalsJob* nrm;   // exchange: normals drawn by the spare warp, one job per system
  int nnrm;
};

template <int EPI, int NB = 0, bool GROUP = false>
__global__ void __launch_bounds__(608, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                    const __grid_constant__ CUtensorMap mapB,
                                                    const __grid_constant__ Params p,
                                                    const __grid_constant__ GroupArgs ga) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int stages = GROUP ? ga.stages : p.g.stages;
  const int stride = GROUP ? ga.stage_stride : p.g.stage_bytes;
  const int egroups = GROUP ? ga.epi_groups : p.g.epi_groups;
  const int ebytes = GROUP ? ga.epi_bytes : p.g.epi_bytes;
  const int tmem_cols = GROUP ? ga.tmem_cols : p.g.tmem_cols;
  const uint32_t acc_stride = (uint32_t)(GROUP ? ga.acc_stride : p.g.bn);
  const int tiles = GROUP ? ga.tiles : p.g.m_tiles * p.g.n_tiles;
  uint8_t* epi_base = smem + (size_t)stages * stride;
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_base + (size_t)egroups * ebytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* tfull = bars + 2 * stages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // the problem of tile t: parameters, maps, the tile's index within the problem, epilogue width
  // (grouped: each problem's tiles start at a multiple of the grid, so all CTAs enter a problem at
  // the same turn; the slots between problems are skipped)
  struct Item {
    const Params* p;
    const CUtensorMap* a;
    const CUtensorMap* b;
    int t, nb;
    bool valid;
  };
  auto resolve = [&](int t, int& cur) -> Item {
    if constexpr (GROUP) {
      while (cur + 1 < ga.nprob && t >= ga.probs[cur + 1].tile0) ++cur;
      const GroupProblem& pr = ga.probs[cur];
      return Item{&pr.p, &pr.mapA, &pr.mapB, t - pr.tile0, pr.nb, t - pr.tile0 < pr.tiles};
    } else {
      (void)cur;
      return Item{&p, &mapA, &mapB, t, NB, true};
    }
  };
  auto give_up = [&]() {
    if constexpr (GROUP) {
      for (int i = 0; i < ga.nprob; ++i) atomicOr(ga.probs[i].p.status, kStatusTimeout);
    } else {
      atomicOr(p.status, kStatusTimeout);
    }
    *abort_flag = 1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4 * egroups);
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
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      int stage = 0, cur = 0;
      uint32_t ph = 0;
      bool go = true;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x) {
        const Item it = resolve(t, cur);
        if (!it.valid) continue;
        const Geom g = it.p->g;   // a register copy: the copies' asm would force reloads of a reference
        int mt, nt;
        tile_mn(g, it.t, &mt, &nt);
        for (int kb = 0; kb < g.k_blocks; ++kb) {
          if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag)) { go = false; break; }
          uint8_t* sa = smem + (size_t)stage * stride;
          mbar_expect_tx(&full[stage], (uint32_t)g.stage_bytes);
          if (g.dual) {
            const int kc = kb * kBK, ay = mt * g.m_step, by = nt * g.n_step;
            tma_load_2d(sa, it.a, &full[stage], kc, ay);
            tma_load_2d(sa + kStageA, it.a, &full[stage], g.a_lo + kc, ay);
            tma_load_2d(sa + 2 * kStageA, it.b, &full[stage], g.b_hi + kc, by);
            tma_load_2d(sa + 2 * kStageA + g.bn * 128, it.b, &full[stage], g.b_lo + kc, by);
            if (++stage == stages) { stage = 0; ph ^= 1u; }
            continue;
          }
          int ka = kb * kBK, kbb = kb * kBK;
          if (g.il3) {
            const int j = kb / 3, sv = kb - 3 * j;
            ka = (sv == 1 ? g.seg : 0) + j * kBK;
            kbb = (sv == 2 ? g.seg : 0) + j * kBK;
          }
          tma_load_2d(sa, it.a, &full[stage], ka, mt * g.m_step);
          tma_load_2d(sa + kStageA, it.b, &full[stage], kbb, nt * g.n_step);
          if (++stage == stages) { stage = 0; ph ^= 1u; }
        }
      }
      if (!go) give_up();
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      int stage = 0, n_it = 0, cur = 0;
      uint32_t ph = 0;
      bool go = true;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x) {
        const Item it = resolve(t, cur);
        if (!it.valid) continue;
        const Geom g = it.p->g;   // a register copy (see the producer)
        const uint32_t idesc = idesc_bf16(g.bn);
        const int acc = n_it & 1;
        const uint32_t aph = (uint32_t)(n_it >> 1) & 1u;
        ++n_it;
        if (!mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) { go = false; break; }
        tc_fence_after();
        const uint32_t dtm = tmem_base + (uint32_t)acc * acc_stride;
        for (int kb = 0; kb < g.k_blocks; ++kb) {
          if (!mbar_wait(&full[stage], ph, abort_flag)) { go = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + (size_t)stage * stride);
          if (g.dual) {
            const uint32_t sal = sa + kStageA, sb = sa + 2 * kStageA, sbl = sb + (uint32_t)(g.bn * 128);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              if (kb * (kBK / 16) + k < g.k_steps) {
                const uint64_t ah = sw128_desc(sa + 32 * k), bh = sw128_desc(sb + 32 * k);
                umma_bf16(dtm, ah, bh, idesc, (kb | k) != 0 ? 1u : 0u);                  // A hi B hi
                umma_bf16(dtm, sw128_desc(sal + 32 * k), bh, idesc, 1u);                // A lo B hi
                umma_bf16(dtm, ah, sw128_desc(sbl + 32 * k), idesc, 1u);                // A hi B lo
              }
          } else {
            const uint32_t sb = sa + kStageA;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              if (kb * (kBK / 16) + k < g.k_steps)
                umma_bf16(dtm, sw128_desc(sa + 32 * k), sw128_desc(sb + 32 * k), idesc, (kb | k) != 0 ? 1u : 0u);
          }
          umma_commit(&empty[stage]);
          if (++stage == stages) { stage = 0; ph ^= 1u; }
        }
        if (!go) break;
        umma_commit(&tfull[acc]);
      }
      if (!go) give_up();
    }
  } else if (warp >= 2 + 4 * egroups) {   // spare warp: the step's normals (binary64 pipe)
    if constexpr (GROUP) {
      for (int j = 0; j < ga.nnrm; ++j) draw_normals_warp(ga.nrm[j], reinterpret_cast<uint8_t*>(bars) + 256, lane);
    } else {
      if (EPI == 0 && p.nrm.x) draw_normals_warp(p.nrm, reinterpret_cast<uint8_t*>(bars) + 256, lane);
    }
  } else {   // epilogue warps
    const int ew = warp - 2, group = ew >> 2, wig = ew & 3, q = warp & 3;
    const int r = 32 * q + lane;
    // the group's tile-ready flags: EpiSmem::ok (single problem), or a launch-wide slot in the tail
    // (grouped: each problem lays out its own epilogue buffers)
    int* ok_flags = GROUP ? reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(bars) + 128) + 2 * group
                          : reinterpret_cast<int*>(epi_base + (size_t)group * ebytes);
    const EpiSmem es0 = epi_smem(epi_base, p, group, NB > 0);                      // single problem
    int n_it = 0, cur = 0, loaded = -1;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const Item it = resolve(t, cur);
      if (!it.valid) continue;
      const int acc = n_it & 1;
      const uint32_t aph = (uint32_t)(n_it >> 1) & 1u;
      ++n_it;
      if (wig == 0 && lane == 0) {   // slot acc is rewritten two tiles later, after this group's next barrier
        const bool ok = mbar_wait(&tfull[acc], aph, abort_flag);
        if (!ok) give_up();
        ok_flags[acc] = ok ? 1 : 0;
      }
      named_bar(1 + group, 128);   // also: every thread of the group is done with the previous tile's buffers
      const int ok = ok_flags[acc];
      if (!ok) break;
      tc_fence_after();
      const Params* ppp = it.p;
      if constexpr (GROUP) {   // the problem's parameters into the group's shared-memory slot
        Params* slot = reinterpret_cast<Params*>(reinterpret_cast<uint8_t*>(bars) + kTailBytes + group * kParamSlot);
        if (cur != loaded) {   // every thread of the group is past the previous tile (barrier above)
          const int* src = reinterpret_cast<const int*>(it.p);
          int* dst = reinterpret_cast<int*>(slot);
          for (int i = r; i < (int)(sizeof(Params) / 4); i += 128) dst[i] = src[i];
          named_bar(1 + group, 128);
          loaded = cur;
        }
        ppp = slot;
      }
      const Params& pp = *ppp;
      const uint32_t tacc = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)acc * acc_stride;
      int mt, nt;
      tile_mn(pp.g, it.t, &mt, &nt);
      if (GROUP && group >= pp.g.epi_groups) {
        // a problem with fewer epilogue groups than the launch: this group idles for the tile
      } else if constexpr (EPI == 0 && !GROUP) {
        if constexpr (NB > 0) exchange_tile_reg<NB>(pp, mt, nt, tacc, es0, group, wig, r, lane);
        else exchange_tile(pp, mt, nt, tacc, es0, group, wig, r, lane);
      } else if constexpr (EPI == 0) {   // grouped: every problem of the launch has the epilogue width NB
        const EpiSmem es = epi_smem(epi_base, pp, group, NB > 0);
        if constexpr (NB > 0) exchange_tile_reg<NB>(pp, mt, nt, tacc, es, group, wig, r, lane);
        else exchange_tile(pp, mt, nt, tacc, es, group, wig, r, lane);
      } else if constexpr (EPI == 1) {
        store_tile(pp, mt, nt, tacc, group, r);
      } else if (pp.blocks) {
        store_planes_packed(pp, mt, nt, tacc, group, r,
                            reinterpret_cast<__nv_bfloat16*>(epi_base + (size_t)group * pp.g.epi_bytes + 16));
      } else {
        store_planes(pp, mt, nt, tacc, group, r);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols) : "memory");
}


// ----------------------------------------------------------------------------- exchange, Ltilde resident
// The exchange contraction with its A operand, the Ltilde tile of gpt gammas (hi and lo halves), held
// in tensor memory.  Each CTA takes a contiguous range of tiles in M-major order, so the tile is
// staged through the shared-memory ring and copied into tensor memory (tcgen05.cp) once or twice per
// CTA; Theta of the tile's walkers streams through the ring as [hi | lo] K blocks, and each 16-wide
// k-step issues A_hi B_hi, A_lo B_hi and A_hi B_lo with A read from tensor memory.  Shared memory
// then carries each B byte once (TMA write, MMA read) plus the epilogue's transposition, against
// three copies of every operand in the streamed form (K-concatenated [hi | lo | hi] x [hi | hi | lo]).
// Tensor memory: accumulators [0, bn) and [bn, 2 bn), A hi [a0, a0 + kst / 2), A lo up to 512.
// Roles, epilogue and bounded waits as in k_tc_gemm.
__host__ __device__ __forceinline__ int tm_stage_bytes(int bn) { return 2 * (kStageA > bn * 128 ? kStageA : bn * 128); }

template <int NB>
__global__ void __launch_bounds__(608, 1) k_exch_tm(const __grid_constant__ CUtensorMap mapA,
                                                    const __grid_constant__ CUtensorMap mapB, const Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const Geom& g = p.g;
  const int stage_bytes = tm_stage_bytes(g.bn);
  uint8_t* epi_base = smem + (size_t)g.stages * stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_base + (size_t)g.epi_groups * g.epi_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + g.stages;
  uint64_t* tfull = bars + 2 * g.stages;
  uint64_t* tempty = tfull + 2;
  uint64_t* adone = tempty + 2;   // MMAs done with the resident tile before it is replaced
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(adone + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles = (long long)g.m_tiles * g.n_tiles;
  const int t_beg = (int)(tiles * blockIdx.x / gridDim.x), t_end = (int)(tiles * (blockIdx.x + 1) / gridDim.x);
  const int nks = p.kst / 16, nkb = (p.kst + kBK - 1) / kBK, half = p.kst / 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < g.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4 * g.epi_groups);
    }
    mbar_init(adone, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer: the A tile (hi, lo) on every change of mt, then B (hi, lo) per tile
      int stage = 0;
      uint32_t ph = 0;
      bool go = true;
      int mt_prev = -1;
      for (int t = t_beg; t < t_end && go; ++t) {
        const int mt = t / g.n_tiles, nt = t - (t / g.n_tiles) * g.n_tiles;
        for (int part = (mt != mt_prev ? 0 : 1); part < 2 && go; ++part)
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&empty[stage], ph ^ 1u, abort_flag)) { go = false; break; }
            uint8_t* st = smem + (size_t)stage * stage_bytes;
            if (part == 0) {
              mbar_expect_tx(&full[stage], 2u * kStageA);
              tma_load_2d(st, &mapA, &full[stage], kb * kBK, mt * g.m_step);
              tma_load_2d(st + kStageA, &mapA, &full[stage], p.kst + kb * kBK, mt * g.m_step);
            } else {
              mbar_expect_tx(&full[stage], (uint32_t)(2 * g.bn * 128));
              tma_load_2d(st, &mapB, &full[stage], kb * kBK, nt * g.n_step);
              tma_load_2d(st + g.bn * 128, &mapB, &full[stage], 2 * p.kst + kb * kBK, nt * g.n_step);
            }
            if (++stage == g.stages) { stage = 0; ph ^= 1u; }
          }
        mt_prev = mt;
      }
      if (!go) { atomicOr(p.status, kStatusTimeout); *abort_flag = 1; }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      int stage = 0;
      uint32_t ph = 0, ph_a = 0;
      int it = 0, mt_prev = -1;
      bool go = true;
      const uint32_t idesc = idesc_bf16(g.bn);
      const uint32_t a_hi = tmem_base + (uint32_t)p.a0, a_lo = a_hi + (uint32_t)half;
      for (int t = t_beg; t < t_end && go; ++t, ++it) {
        const int mt = t / g.n_tiles;
        if (mt != mt_prev) {   // replace the resident tile once the MMAs reading it have completed
          if (mt_prev >= 0) {
            umma_commit(adone);
            if (!mbar_wait(adone, ph_a, abort_flag)) { go = false; break; }
            ph_a ^= 1u;
          }
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&full[stage], ph, abort_flag)) { go = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + (size_t)stage * stage_bytes);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
              const int ks = kb * (kBK / 16) + k;
              if (ks < nks) {
                tmem_cp_128x256b(a_hi + (uint32_t)(ks * 8), sw128_desc(sa + 32 * k));
                tmem_cp_128x256b(a_lo + (uint32_t)(ks * 8), sw128_desc(sa + kStageA + 32 * k));
              }
            }
            umma_commit(&empty[stage]);
            if (++stage == g.stages) { stage = 0; ph ^= 1u; }
          }
          if (!go) break;
          mt_prev = mt;
        }
        const int acc = it & 1;
        const uint32_t aph = (uint32_t)(it >> 1) & 1u;
        if (!mbar_wait(&tempty[acc], aph ^ 1u, abort_flag)) { go = false; break; }
        tc_fence_after();
        const uint32_t dtm = tmem_base + (uint32_t)(acc * g.bn);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&full[stage], ph, abort_flag)) { go = false; break; }
          tc_fence_after();
          const uint32_t sb = smem_u32(smem + (size_t)stage * stage_bytes);
          const uint64_t dbh = sw128_desc(sb), dbl = sw128_desc(sb + (uint32_t)(g.bn * 128));
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const int ks = kb * (kBK / 16) + k;
            if (ks < nks) {
              const uint32_t ah = a_hi + (uint32_t)(ks * 8), al = a_lo + (uint32_t)(ks * 8);
              umma_bf16_ts(dtm, ah, dbh + (uint64_t)(2 * k), idesc, ks > 0 ? 1u : 0u);   // A hi B hi
              umma_bf16_ts(dtm, al, dbh + (uint64_t)(2 * k), idesc, 1u);                 // A lo B hi
              umma_bf16_ts(dtm, ah, dbl + (uint64_t)(2 * k), idesc, 1u);                 // A hi B lo
            }
          }
          umma_commit(&empty[stage]);
          if (++stage == g.stages) { stage = 0; ph ^= 1u; }
        }
        if (!go) break;
        umma_commit(&tfull[acc]);
      }
      if (!go) { atomicOr(p.status, kStatusTimeout); *abort_flag = 1; }
    }
  } else if (warp >= 2 + 4 * g.epi_groups) {   // spare warp: the step's normals (binary64 pipe)
    if (p.nrm.x) draw_normals_warp(p.nrm, reinterpret_cast<uint8_t*>(bars) + 256, lane);
  } else {   // epilogue warps
    const int ew = warp - 2, group = ew >> 2, wig = ew & 3, q = warp & 3;
    const int r = 32 * q + lane;
    const EpiSmem es = epi_smem(epi_base, p, group, true);
    int it = 0;
    for (int t = t_beg; t < t_end; ++t, ++it) {
      const int acc = it & 1;
      const uint32_t aph = (uint32_t)(it >> 1) & 1u;
      if (wig == 0 && lane == 0) {   // slot it & 1 is rewritten two tiles later, after this group's next barrier
        const bool ok = mbar_wait(&tfull[acc], aph, abort_flag);
        if (!ok) { atomicOr(p.status, kStatusTimeout); *abort_flag = 1; }
        es.ok[it & 1] = ok ? 1 : 0;
      }
      named_bar(1 + group, 128);   // also: every thread of the group is done with the previous tile's buffers
      const int ok = es.ok[it & 1];
      if (!ok) break;
      tc_fence_after();
      const uint32_t tacc = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * g.bn);
      const int mt = t / g.n_tiles, nt = t - (t / g.n_tiles) * g.n_tiles;
      exchange_tile_reg<NB>(p, mt, nt, tacc, es, group, wig, r, lane);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(g.tmem_cols) : "memory");
}

// ----------------------------------------------------------------------------- operand conversion
// Theta^T complex64 [W][ncol][N] -> per block rows (w, part, b) of nseg * kst bf16: B = [hi | hi | lo].
// Row block w holds walker src.
__device__ __forceinline__ void theta_bf16_rows(int w, int src, int N, int ncol, int c0, int n, int kst, int nseg,
                                                const float2* thetaT, __nv_bfloat16* out, int kst0) {
  const int rowlen = nseg * kst;
  for (int idx = threadIdx.x; idx < 2 * n * kst; idx += blockDim.x) {
    const int row = idx / kst, k = idx % kst;
    const int part = row / n, b = row % n;
    // complex Hamiltonian (kst0 > 0): row (w, 0, b) = [Re | Im], row (w, 1, b) = [Im | -Re]
    const int half = kst0 ? k / kst0 : 0, pp = kst0 ? k - half * kst0 : k;
    float v = 0.f;
    if (pp < N) {
      const float2 t = thetaT[((size_t)src * ncol + c0 + b) * N + pp];
      if (!kst0) v = part ? t.y : t.x;
      else if (part == 0) v = half ? t.y : t.x;
      else v = half ? -t.x : t.y;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16* dst = out + ((size_t)w * 2 * n + row) * rowlen + k;
    dst[0] = hi;
    if (nseg == 3) {
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      dst[kst] = hi;
      dst[2 * kst] = lo;
    }
  }
}

__global__ void k_theta_bf16(int W, int N, int ncol, int c0, int n, int kst, int nseg, const float2* thetaT,
                             __nv_bfloat16* out, const int* widx, int kst0 = 0) {
  (void)W;
  const int w = blockIdx.x;   // output row block
  theta_bf16_rows(w, widx ? widx[w] : w, N, ncol, c0, n, kst, nseg, thetaT, out, kst0);
}

// The bf16 Theta^T operands of several (system, spin block) jobs, one block per walker.
struct ThetaJob {
  int N, ncol, c0, n, kst, nseg, kst0;
  const float2* thetaT;
  __nv_bfloat16* out;
};
__global__ void k_theta_bf16_group(const ThetaJob* __restrict__ jobs, const int* __restrict__ first, int njobs) {
  const int j = group_of(first, njobs, blockIdx.x);
  const ThetaJob& a = jobs[j];
  const int w = blockIdx.x - first[j];
  theta_bf16_rows(w, w, a.N, a.ncol, a.c0, a.n, a.kst, a.nseg, a.thetaT, a.out, a.kst0);
}

// Ltilde [ng][ncol][N] (gammas g0 .. g0 + ng - 1, binary64 or binary32) -> block rows (g, a) of
// nseg * kst bf16: A = [hi | lo | hi].
template <typename T>
__global__ void k_lrot_bf16(int g0, int ng, int N, int ncol, int c0, int n, int kst, int nseg, const T* lrot,
                            __nv_bfloat16* out) {
  const int rowlen = nseg * kst;
  const size_t total = (size_t)ng * n * kst;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t row = idx / kst;
    const int pp = (int)(idx % kst);
    const int g = (int)(row / n), a = (int)(row % n);
    const double v = pp < N ? (double)lrot[((size_t)g * ncol + c0 + a) * N + pp] : 0.0;
    const __nv_bfloat16 hi = __double2bfloat16(v);
    __nv_bfloat16* dst = out + ((size_t)g0 * n + row) * rowlen + pp;
    dst[0] = hi;
    if (nseg == 3) {
      dst[kst] = __double2bfloat16(v - (double)__bfloat162float(hi));
      dst[2 * kst] = hi;
    }
  }
}

// L [ng][NN] (gammas g0 .. g0 + ng - 1) -> columns g0 .. g0 + ng - 1 of the Lt rows, each row
// [hi | lo] (kx elements per part; hi only when nseg = 1).  Rows are pq, or with packed L^T the
// pairs p <= q listed in `pairs`.  A 32-gamma x 64-pq tile is transposed
// through shared memory so that both the reads (pq contiguous) and the writes (gamma contiguous)
// are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) k_lt_bf16(int g0, int ng, size_t NN, size_t nrows, const int* pairs, int kx,
                                                 int nseg, const T* chol, __nv_bfloat16* out) {
  __shared__ float tile[32][65];
  const int nparts = nseg == 3 ? 2 : 1;
  const size_t rowlen = (size_t)nparts * kx;
  const size_t pq0 = (size_t)blockIdx.x * 64;
  const int gt = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * 64; i += 256) {
    const int gl = i / 64, c = i % 64;
    const size_t row = pq0 + c;
    const long long src = row < nrows ? (pairs ? (long long)pairs[row] : (long long)row) : -1;
    tile[gl][c] = (gt + gl < ng && src >= 0) ? (float)chol[(size_t)(gt + gl) * NN + (size_t)src] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * 64; i += 256) {
    const int c = i / 32, gl = i % 32;
    const size_t pq = pq0 + c;
    if (gt + gl >= ng || pq >= nrows) continue;
    const float v = tile[gl][c];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16* dst = out + pq * rowlen + g0 + gt + gl;
    dst[0] = hi;
    if (nseg == 3) dst[kx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// Complex Hamiltonian, exchange A: Ltilde complex [nf][ncol][N] (fields f0 ..) -> block rows (f, a) of
// nseg * kst bf16, each segment [Re (kst0) | -Im (kst0)], segments [hi | lo | hi].
template <typename G>
__global__ void k_lrot_bf16_c(int f0, int nf, int N, int ncol, int c0, int n, int kst, int kst0, int nseg,
                              const G* lrot, __nv_bfloat16* out) {
  const int rowlen = nseg * kst;
  const size_t total = (size_t)nf * n * kst;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t row = idx / kst;
    const int k = (int)(idx % kst), part = k / kst0, pp = k - part * kst0;
    const int g = (int)(row / n), a = (int)(row % n);
    double v = 0.0;
    if (pp < N) {
      const size_t e = 2 * (((size_t)g * ncol + c0 + a) * N + pp);
      v = part ? -(double)lrot[e + 1] : (double)lrot[e];
    }
    const __nv_bfloat16 hi = __double2bfloat16(v);
    __nv_bfloat16* dst = out + ((size_t)f0 * n + row) * rowlen + k;
    dst[0] = hi;
    if (nseg == 3) {
      dst[kst] = __double2bfloat16(v - (double)__bfloat162float(hi));
      dst[2 * kst] = hi;
    }
  }
}

// Complex Hamiltonian, VHS A: fields complex [nf][NN] (f0 ..) -> columns f0 + f (real part) and
// kx0 + f0 + f (imaginary part) of the Lt rows pq, each row [hi | lo] of kx.
template <typename G>
__global__ void __launch_bounds__(256) k_lt_bf16_c(int f0, int nf, size_t NN, int kx, int kx0, int nseg,
                                                   const G* fields, __nv_bfloat16* out) {
  __shared__ float tile[2][32][65];
  const size_t rowlen = (size_t)(nseg == 3 ? 2 : 1) * kx;
  const size_t pq0 = (size_t)blockIdx.x * 64;
  const int gt = blockIdx.y * 32;
  for (int i = threadIdx.x; i < 32 * 64; i += 256) {
    const int gl = i / 64, c = i % 64;
    const size_t pq = pq0 + c;
    const bool ok = gt + gl < nf && pq < NN;
    const size_t e = 2 * ((size_t)(gt + gl) * NN + pq);
    tile[0][gl][c] = ok ? (float)fields[e] : 0.f;
    tile[1][gl][c] = ok ? (float)fields[e + 1] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * 32 * 64; i += 256) {
    const int part = i / 2048, rem = i % 2048, c = rem / 32, gl = rem % 32;
    const size_t pq = pq0 + c;
    if (gt + gl >= nf || pq >= NN) continue;
    const float v = tile[part][gl][c];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16* dst = out + pq * rowlen + (size_t)part * kx0 + f0 + gt + gl;
    dst[0] = hi;
    if (nseg == 3) dst[kx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// VHS coefficients complex64 [W][X] -> rows (w, part) of [hi | lo] bf16 (kx elements per part; hi
// only when nseg = 1).  Complex Hamiltonian (kx0 > 0): row (w, 0) = [Re c | -Im c], row (w, 1) =
// [Im c | Re c], each real part kx0 long.
__global__ void k_coef_bf16(int W, int X, int kx, int nseg, const float2* coef, __nv_bfloat16* out, int kx0 = 0) {
  const int w = blockIdx.x;
  const int rowlen = (nseg == 3 ? 2 : 1) * kx;
  for (int idx = threadIdx.x; idx < 2 * kx; idx += blockDim.x) {
    const int part = idx / kx, k = idx % kx;
    const int half = kx0 ? k / kx0 : 0, g = kx0 ? k - half * kx0 : k;
    float v = 0.f;
    if (g < X) {
      const float2 c = coef[(size_t)w * X + g];
      if (!kx0) v = part ? c.y : c.x;
      else if (part == 0) v = half ? -c.y : c.x;
      else v = half ? c.x : c.y;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16* dst = out + ((size_t)w * 2 + part) * rowlen + k;
    dst[0] = hi;
    if (nseg == 3) dst[kx] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// ----------------------------------------------------------------------------- host side
namespace {

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int epi_bytes_exchange(int n, bool reg) {
  return 16 + (reg ? exch_buf2_bytes(n) : exch_buf_bytes(n)) + 128 * 8 + 4 * 8;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

bool make_map(CUtensorMap* m, const void* base, unsigned long long rows, unsigned long long kcols, unsigned box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {kcols, rows};
  const cuuint64_t strides[1] = {kcols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

namespace {

int tmem_cols_for(int bn) {
  int c = 32;
  while (c < 2 * bn) c <<= 1;
  return c;
}

// The register-row exchange epilogue applies when n <= 32 and the imaginary-part loads of the last
// walker of the second accumulator stay inside tensor memory.
bool exchange_reg(int n, int wpt, int bn) {
  const int nb = (n + 7) / 8 * 8;
  return nb <= 32 && bn + (wpt - 1) * 2 * n + n + nb <= tmem_cols_for(bn);
}

// Tile order of the streamed exchange.  The dual form (long K), or any Ltilde block too large to stay
// in L2, takes groups of walker tiles whose Theta operand (~32 MB) stays in L2, the M tiles in turn
// within a group: each Ltilde tile then streams from HBM once per group, not once per walker tile.
int exchange_ntg(const TcState* st, const BlockMaps& bm, const Geom& g) {
  const long long a_bytes = (long long)st->X * bm.n * st->nseg * st->kst * 2;
  if (!g.dual && a_bytes <= (24LL << 20)) return 0;
  const long long bt = (long long)g.bn * (g.dual ? 2 : st->nseg) * st->kst * 2;   // Theta bytes per tile
  return (int)std::max(1LL, std::min<long long>(g.n_tiles, (32LL << 20) / bt));
}

// Pick the stage count for a given B box height and epilogue footprint.
bool finish_geom(Geom* g, int epi_bytes_per_group, int epi_groups) {
  g->epi_groups = epi_groups;
  g->epi_bytes = (epi_bytes_per_group + 15) & ~15;
  const int stage_bytes = g->dual ? 2 * kStageA + 2 * g->bn * kBK * 2 : kStageA + g->bn * kBK * 2;
  g->stage_bytes = stage_bytes;
  const int fixed = 1024 + epi_groups * g->epi_bytes + kTailBytes;
  int st = (kMaxSmem - fixed) / stage_bytes;
  if (st > 4) st = 4;
  if (st < 2) return false;
  g->stages = st;
  g->tmem_cols = tmem_cols_for(g->bn);
  return g->tmem_cols <= 512;
}

size_t smem_bytes(const Geom& g) {
  return 1024 + (size_t)g.stages * g.stage_bytes + (size_t)g.epi_groups * g.epi_bytes + kTailBytes;
}

template <int EPI, int NB = 0>
afqmc_status launch(const Geom& g, const CUtensorMap& a, const CUtensorMap& b, const Params& p, cudaStream_t s,
                    unsigned long long* launches, char* err, size_t errlen) {
  const size_t sm = smem_bytes(g);
  if (sm > (size_t)kMaxSmem) {
    snprintf(err, errlen, "tcgen05 GEMM: %zu bytes of shared memory exceed the limit", sm);
    return AFQMC_EINVAL;
  }
  const int tiles = g.m_tiles * g.n_tiles;
  const int grid = std::min(tiles, num_sms());
  k_tc_gemm<EPI, NB><<<grid, 64 + 128 * g.epi_groups + (p.nrm.x ? 32 : 0), sm, s>>>(a, b, p, GroupArgs{});
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tcgen05 GEMM launch: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

template <int NB>
afqmc_status launch_tm(const Geom& g, const CUtensorMap& a, const CUtensorMap& b, const Params& p, cudaStream_t s,
                       unsigned long long* launches, char* err, size_t errlen) {
  const size_t sm = 1024 + (size_t)g.stages * tm_stage_bytes(g.bn) + (size_t)g.epi_groups * g.epi_bytes + kTailBytes;
  if (sm > (size_t)kMaxSmem) {
    snprintf(err, errlen, "tcgen05 exchange: %zu bytes of shared memory exceed the limit", sm);
    return AFQMC_EINVAL;
  }
  const int tiles = g.m_tiles * g.n_tiles;
  const int grid = std::min(tiles, num_sms());
  k_exch_tm<NB><<<grid, 64 + 128 * g.epi_groups + (p.nrm.x ? 32 : 0), sm, s>>>(a, b, p);
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tcgen05 exchange launch: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

}  // namespace

// Largest epilogue group count (<= 4, <= walkers per tile) whose buffers fit beside two stages of
// the tile it implies (walkers per tile = the largest multiple of the group count <= wpt0).
int exchange_groups(int n, int wpt0) {
  for (int g = std::min(4, wpt0); g > 1; --g) {
    const int wpt = wpt0 / g * g;
    const int bn = (wpt * 2 * n + 15) / 16 * 16;
    const int stage_bytes = kStageA + bn * kBK * 2;
    const int need =
        1024 + g * ((epi_bytes_exchange(n, exchange_reg(n, wpt, bn)) + 15) & ~15) + kTailBytes + 2 * stage_bytes;
    if (need <= kMaxSmem) return g;
  }
  return 1;
}

// Walker tiling of one block: epilogue groups, walkers per tile, MMA N and form.  The resident-A
// form (k_exch_tm, BF16x3 only) needs the register-row epilogue (n <= 32), 2 bn + kst <= 512 tensor-memory
// columns and two ring stages beside the epilogue buffers; it takes the largest group count (at
// most `groups` when that is > 0) for which some multiple of it walkers fits, and the most walkers,
// provided the tile holds at least 3/4 of the streamed form's walkers (for large N the tensor-memory
// budget leaves too few columns and the narrow products run below the tensor pipe's rate).
// Otherwise (or with form 1) the streamed form with the largest group count that fits.
namespace {
void exchange_config(TcState* st, BlockMaps& bm, int groups, int form) {
  const int n = bm.n, wpt0 = 256 / (2 * n);
  int gs = exchange_groups(n, wpt0);
  if (groups > 0) gs = std::max(1, std::min(gs, groups));
  const int wpt_streamed = wpt0 / gs * gs;
  if (form != 1 && st->nseg == 3 && (n + 7) / 8 * 8 <= 32) {
    for (int g = std::min(4, wpt0); g >= 1; --g) {
      if (groups > 0 && g > groups) continue;
      int wpt = 0;
      for (int w = g; w <= wpt0; w += g)
        if (2 * ((w * 2 * n + 15) / 16 * 16) + st->kst <= 512) wpt = w;
      if (wpt == 0 || 4 * wpt < 3 * wpt_streamed) continue;
      const int bn = (wpt * 2 * n + 15) / 16 * 16;
      const int need = 1024 + g * ((epi_bytes_exchange(n, true) + 15) & ~15) + kTailBytes + 2 * tm_stage_bytes(bn);
      if (need > kMaxSmem) continue;
      bm.groups = g;
      bm.wpt = wpt;
      bm.bn = bn;
      bm.form = 1;
      bm.n_tiles = (st->W + wpt - 1) / wpt;
      return;
    }
  }
  bm.dual = 0;
  if (st->nseg == 3 && st->kst >= 512) {
    // long K (large N): load each k-block's hi and lo parts once (dual stages); the most walkers per
    // tile, then the most epilogue groups, whose buffers fit beside two stages
    for (int wpt = wpt0; wpt >= 1 && !bm.dual; --wpt)
      for (int g = std::min(4, wpt); g >= 1; --g) {
        if (wpt % g || (groups > 0 && g > groups)) continue;
        const int bn = (wpt * 2 * n + 15) / 16 * 16;
        const int stage = 2 * kStageA + 2 * bn * 128;
        const int need = 1024 + g * ((epi_bytes_exchange(n, exchange_reg(n, wpt, bn)) + 15) & ~15) + kTailBytes +
                         2 * stage;
        if (need > kMaxSmem) continue;
        bm.dual = 1;
        bm.groups = g;
        bm.wpt = wpt;
        bm.bn = bn;
        break;
      }
    if (bm.dual) {
      bm.form = 0;
      bm.n_tiles = (st->W + bm.wpt - 1) / bm.wpt;
      return;
    }
  }
  bm.groups = gs;
  bm.wpt = wpt_streamed;
  bm.bn = (bm.wpt * 2 * n + 15) / 16 * 16;
  bm.form = 0;
  bm.n_tiles = (st->W + bm.wpt - 1) / bm.wpt;
}
}  // namespace

size_t plan(TcState* st, int prec, int W, int N, int X, int ncol, const int* c0, const int* nb, int nblk,
            bool cplx) {
  if (prec != AFQMC_PREC_BF16 && prec != AFQMC_PREC_BF16X3) return 0;
  st->prec = prec;
  st->W = W; st->N = N; st->X = X; st->ncol = ncol; st->nblk = nblk;
  st->cplx = cplx ? 1 : 0;
  st->nseg = prec == AFQMC_PREC_BF16X3 ? 3 : 1;
  // segments padded to the MMA k-step only; the last TMA box reads past K.  A complex Hamiltonian
  // realifies every contraction along K: exchange A rows [Re Ltilde | -Im Ltilde], B rows
  // [Re Theta | Im Theta] and [Im Theta | -Re Theta]; VHS A rows [Re M | Im M] over the fields, B rows
  // [Re c | -Im c] and [Im c | Re c]; each real part padded to kst0 / kx0
  st->kst0 = (N + 15) / 16 * 16;
  st->kst = cplx ? 2 * st->kst0 : st->kst0;
  st->kx0 = (X + kBK - 1) / kBK * kBK;
  st->kx = cplx ? 2 * st->kx0 : st->kx0;
  size_t cur = 0;
  st->nchunk = 0;
  for (int s = 0; s < nblk; ++s) {
    BlockMaps& b = st->blk[s];
    b.n = nb[s];
    b.c0 = c0[s];
    if (b.n == 0) { b.m_tiles = b.n_tiles = 0; continue; }
    b.gpt = kBM / b.n;
    exchange_config(st, b, 0, 0);   // every epilogue group takes the same number of walkers
    b.m_tiles = (X + b.gpt - 1) / b.gpt;
    b.off_l = cur;
    cur = align256(cur + (size_t)X * b.n * st->nseg * st->kst * 2);
    b.off_th = cur;
    cur = align256(cur + (size_t)W * 2 * b.n * st->nseg * st->kst * 2);
    st->nchunk += 4 * b.m_tiles;   // four exchange partial slots per M tile (one per epilogue warp)
  }
  st->vparts = st->nseg == 3 ? 2 : 1;   // VHS operands stored [hi | lo] (see Geom::dual)
  st->pg = prop_geom(N, ncol, cplx);
  // packed L^T (the upper triangle p <= q only) where the large-form propagation consumes the V
  // planes: the VHS GEMM then reads half of L and its epilogue writes each V_pq at (p, q) and (q, p)
  // (V symmetric: real symmetric L; a complex Hamiltonian's V is not, so it keeps every row)
  st->packed = (st->pg.ok && st->pg.large && !cplx) ? 1 : 0;
  st->lt_rows = (long long)N * N;
  st->nblocks = 0;
  if (st->packed) {   // blocks of 8 p x 16 q touching the upper triangle, 128 rows each
    const int bi = (N + 7) / 8, bj = (N + 15) / 16;
    long long nb = 0;
    for (int j = 0; j < bj; ++j) nb += std::min(bi, (16 * j + 15) / 8 + 1);
    st->nblocks = nb;
    st->lt_rows = nb * 128;
    st->off_pairs = cur;
    cur = align256(cur + (size_t)st->lt_rows * 4);
    st->off_blocks = cur;
    cur = align256(cur + (size_t)nb * 8);
  }
  st->off_lt = cur;
  cur = align256(cur + (size_t)st->lt_rows * st->vparts * st->kx * 2);
  st->off_coef = cur;
  cur = align256(cur + (size_t)W * 2 * st->vparts * st->kx * 2);
  st->vhs_m_tiles = (2 * W + kBM - 1) / kBM;
  st->vhs_n_tiles = (N * N + 255) / 256;
  // VHS planes GEMM width: M tiles x N tiles spread over the SMs; a tile costs about 48 + bn units
  // (measured at N = 108, X = 432, W = 640 over bn = 128 .. 256: 7.3, 8.8, 10.0, 11.7 and 12.8 us
  // per wave of tiles); the width with the smallest busiest-SM cost (the last wave of a wide
  // tiling can be nearly empty, a ragged last column tile costs a full one)
  {
    const long long mt = (st->lt_rows + kBM - 1) / kBM;
    const int sms = num_sms();
    long long best = -1;
    for (int bn : {256, 224, 192, 160, 128}) {
      const long long tiles = mt * ((2LL * W + bn - 1) / bn);
      const long long cost = ((tiles + sms - 1) / sms) * (48 + bn);
      if (best < 0 || cost < best) { best = cost; st->vhs_bn = bn; }
    }
  }
  if (st->pg.ok) {
    const PropGeom& pg = st->pg;
    st->off_vp = cur;
    cur = align256(cur + (size_t)W * 4 * pg.npad * pg.kq * 2);
    st->off_fp = cur;
    cur = align256(cur + (size_t)(pg.cplx_f ? 4 : 2) * pg.npad * pg.kq * 2);
    if (pg.large) {   // term operands (two, ping-pong) and the Taylor sum
      for (int i = 0; i < 2; ++i) {
        st->off_b[i] = cur;
        cur = align256(cur + (size_t)W * 2 * (2 * pg.ncolp) * (2 * pg.kq) * 2);
      }
      st->off_acc = cur;
      cur = align256(cur + (size_t)W * pg.npad * pg.ncolp * 8);
    }
  }
  return cur;
}

int set_exchange_groups(TcState* st, char* tcbuf, int groups, int form) {
  int used = 0;
  for (int b = 0; b < st->nblk; ++b) {
    BlockMaps& bm = st->blk[b];
    if (bm.n == 0) continue;
    exchange_config(st, bm, groups, form);
    const int g = bm.groups;
    if (tcbuf)
      make_map(&bm.map_th, tcbuf + bm.off_th, (unsigned long long)st->W * 2 * bm.n,
               (unsigned long long)st->nseg * st->kst, (unsigned)bm.bn);
    if (!used) used = g;
  }
  return used;
}

afqmc_status begin(TcState* st, cudaStream_t s, char* tcbuf, char* err, size_t errlen) {
  if (!encode_fn()) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled is not available from the driver");
    return AFQMC_ECUDA;
  }
  // every operand's K padding stays zero (the overlap and fields kernels, and the chunked loads
  // below, write only the data columns): clear the exchange operands, L^T and the coefficients once
  if (cudaMemsetAsync(tcbuf, 0, st->off_coef + (size_t)st->W * 2 * st->vparts * st->kx * 2, s) != cudaSuccess) {
    snprintf(err, errlen, "tc set-up: clearing the operand buffers failed");
    return AFQMC_ECUDA;
  }
  if (st->packed) {   // blocks in q-block order, p blocks ascending; p N + q per row, -1 where left out
    const int N = st->N, bi = (N + 7) / 8, bj = (N + 15) / 16;
    std::vector<int> pairs((size_t)st->lt_rows);
    std::vector<int2> blocks((size_t)st->nblocks);
    size_t b = 0;
    for (int j = 0; j < bj; ++j)
      for (int i = 0; i < std::min(bi, (16 * j + 15) / 8 + 1); ++i, ++b) {
        blocks[b] = make_int2(i, j);
        for (int r = 0; r < 128; ++r) {
          const int pp = 8 * i + r / 16, qq = 16 * j + r % 16;
          pairs[b * 128 + r] = (pp < N && qq < N && pp <= qq) ? pp * N + qq : -1;
        }
      }
    if (cudaMemcpyAsync(tcbuf + st->off_pairs, pairs.data(), pairs.size() * 4, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(tcbuf + st->off_blocks, blocks.data(), blocks.size() * 8, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      snprintf(err, errlen, "tc set-up: the packed pair table copy failed");
      return AFQMC_ECUDA;
    }
  }
  return AFQMC_OK;
}

template <typename T, typename TL>
afqmc_status load_chunk(TcState* st, cudaStream_t s, char* tcbuf, int g0, int ng, const T* chol, const TL* lrot,
                        unsigned long long* launches, char* err, size_t errlen) {
  for (int b = 0; b < st->nblk; ++b) {
    const BlockMaps& bm = st->blk[b];
    if (bm.n == 0) continue;
    k_lrot_bf16<TL><<<592, 256, 0, s>>>(g0, ng, st->N, st->ncol, bm.c0, bm.n, st->kst, st->nseg, lrot,
                                         reinterpret_cast<__nv_bfloat16*>(tcbuf + bm.off_l));
    ++*launches;
  }
  const size_t NN = (size_t)st->N * st->N, nrows = (size_t)st->lt_rows;
  const dim3 grid((unsigned)((nrows + 63) / 64), (unsigned)((ng + 31) / 32));
  k_lt_bf16<T><<<grid, 256, 0, s>>>(g0, ng, NN, nrows, st->packed ? reinterpret_cast<const int*>(tcbuf + st->off_pairs)
                                                                   : nullptr,
                                     st->kx, st->nseg, chol, reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_lt));
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tc set-up chunk: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}
template afqmc_status load_chunk<double, double>(TcState*, cudaStream_t, char*, int, int, const double*,
                                                 const double*, unsigned long long*, char*, size_t);
template afqmc_status load_chunk<float, float>(TcState*, cudaStream_t, char*, int, int, const float*, const float*,
                                               unsigned long long*, char*, size_t);
template afqmc_status load_chunk<double, float>(TcState*, cudaStream_t, char*, int, int, const double*, const float*,
                                                unsigned long long*, char*, size_t);
template afqmc_status load_chunk<float, double>(TcState*, cudaStream_t, char*, int, int, const float*, const double*,
                                                unsigned long long*, char*, size_t);

template <typename G>
afqmc_status load_chunk_c(TcState* st, cudaStream_t s, char* tcbuf, int f0, int nf, const G* fields, const G* lrot,
                          unsigned long long* launches, char* err, size_t errlen) {
  for (int b = 0; b < st->nblk; ++b) {
    const BlockMaps& bm = st->blk[b];
    if (bm.n == 0) continue;
    k_lrot_bf16_c<G><<<592, 256, 0, s>>>(f0, nf, st->N, st->ncol, bm.c0, bm.n, st->kst, st->kst0, st->nseg, lrot,
                                          reinterpret_cast<__nv_bfloat16*>(tcbuf + bm.off_l));
    ++*launches;
  }
  const size_t NN = (size_t)st->N * st->N;
  const dim3 grid((unsigned)((NN + 63) / 64), (unsigned)((nf + 31) / 32));
  k_lt_bf16_c<G><<<grid, 256, 0, s>>>(f0, nf, NN, st->kx, st->kx0, st->nseg, fields,
                                       reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_lt));
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tc set-up chunk (complex): %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}
template afqmc_status load_chunk_c<double>(TcState*, cudaStream_t, char*, int, int, const double*, const double*,
                                           unsigned long long*, char*, size_t);
template afqmc_status load_chunk_c<float>(TcState*, cudaStream_t, char*, int, int, const float*, const float*,
                                          unsigned long long*, char*, size_t);

afqmc_status finish(TcState* st, char* tcbuf, char* err, size_t errlen) {
  for (int b = 0; b < st->nblk; ++b) {
    BlockMaps& bm = st->blk[b];
    if (bm.n == 0) continue;
    if (!make_map(&bm.map_l, tcbuf + bm.off_l, (unsigned long long)st->X * bm.n,
                  (unsigned long long)st->nseg * st->kst, kBM) ||
        !make_map(&bm.map_th, tcbuf + bm.off_th, (unsigned long long)st->W * 2 * bm.n,
                  (unsigned long long)st->nseg * st->kst, (unsigned)bm.bn)) {
      snprintf(err, errlen, "cuTensorMapEncodeTiled failed for the exchange operands");
      return AFQMC_ECUDA;
    }
  }
  __nv_bfloat16* lt = reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_lt);
  const unsigned long long vk = (unsigned long long)st->vparts * st->kx;
  if (!make_map(&st->map_lt, lt, (unsigned long long)st->lt_rows, vk, 256) ||
      !make_map(&st->map_coef, tcbuf + st->off_coef, (unsigned long long)st->W * 2, vk, kBM)) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed for the VHS operands");
    return AFQMC_ECUDA;
  }
  if (st->pg.ok &&
      (!make_map(&st->map_lt_a, lt, (unsigned long long)st->lt_rows, vk, kBM) ||
       !make_map(&st->map_coef_b, tcbuf + st->off_coef, (unsigned long long)st->W * 2, vk, (unsigned)st->vhs_bn))) {
    snprintf(err, errlen, "cuTensorMapEncodeTiled failed for the VHS plane operands");
    return AFQMC_ECUDA;
  }
  // reserve the kernels' shared memory now (not while a stream is being captured)
  if (cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 24, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<2, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_tc_gemm<0, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_exch_tm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_exch_tm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_exch_tm<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_exch_tm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess) {
    snprintf(err, errlen, "tcgen05 GEMM: cannot reserve shared memory");
    return AFQMC_ECUDA;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "tc set-up: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  st->ready = true;
  return AFQMC_OK;
}

afqmc_status exchange(TcState* st, cudaStream_t s, char* tcbuf, double smul, const float2* thetaT, float2* vbias,
                      float2* exch_part, int* status, const int* widx, int nw, unsigned long long* launches,
                      char* err, size_t errlen, const NormalsJob* nj, bool theta_ready) {
  int chunk = 0;
  bool first = true;
  if (nw <= 0) return AFQMC_OK;
  // the register-row epilogue adds its per-gamma traces onto vbias
  if (vbias && cudaMemsetAsync(vbias, 0, (size_t)nw * st->X * sizeof(float2), s) != cudaSuccess) {
    snprintf(err, errlen, "tcgen05 exchange: clearing vbias failed");
    return AFQMC_ECUDA;
  }
  for (int b = 0; b < st->nblk; ++b) {
    BlockMaps& bm = st->blk[b];
    if (bm.n == 0) continue;
    if (!theta_ready || widx) {
      k_theta_bf16<<<nw, 256, 0, s>>>(nw, st->N, st->ncol, bm.c0, bm.n, st->kst, st->nseg, thetaT,
                                      reinterpret_cast<__nv_bfloat16*>(tcbuf + bm.off_th), widx,
                                      st->cplx ? st->kst0 : 0);
      ++*launches;
    }
    Geom g{};
    g.m_tiles = bm.m_tiles;
    g.n_tiles = (nw + bm.wpt - 1) / bm.wpt;
    g.k_blocks = (st->nseg * st->kst + kBK - 1) / kBK;
    g.k_steps = st->nseg * st->kst / 16;
    g.m_step = bm.gpt * bm.n;
    g.n_step = bm.wpt * 2 * bm.n;
    g.bn = bm.bn;
    if (bm.form == 0 && bm.dual) {   // A = [hi | lo | hi], B = [hi | hi | lo]: parts at 0 / kst / 2 kst
      g.dual = 1;
      g.k_blocks = (st->kst + kBK - 1) / kBK;
      g.k_steps = st->kst / 16;
      g.a_lo = st->kst;
      g.b_hi = 0;
      g.b_lo = 2 * st->kst;
    }
    if (bm.form == 0) g.ntg = exchange_ntg(st, bm, g);
    const bool reg = bm.form == 1 || exchange_reg(bm.n, bm.wpt, g.bn);
    const int epb = epi_bytes_exchange(bm.n, reg);
    if (bm.form == 0 && !finish_geom(&g, epb, bm.groups)) {
      snprintf(err, errlen, "tcgen05 exchange: n = %d does not fit shared memory", bm.n);
      return AFQMC_EINVAL;
    }
    Params p{};
    if (bm.form == 1) {   // Ltilde resident in tensor memory: its own ring and tensor-memory plan
      g.epi_groups = bm.groups;
      g.epi_bytes = (epi_bytes_exchange(bm.n, true) + 15) & ~15;
      g.stages = std::min(4, (kMaxSmem - 1024 - g.epi_groups * g.epi_bytes - kTailBytes) / tm_stage_bytes(g.bn));
      g.tmem_cols = 512;
      if (g.stages < 2 || 2 * g.bn + st->kst > 512) {
        snprintf(err, errlen, "tcgen05 exchange: resident form does not fit (n = %d)", bm.n);
        return AFQMC_EINVAL;
      }
      p.kst = st->kst;
      p.a0 = 512 - st->kst;
    }
    p.g = g;
    p.status = status;
    p.W = nw; p.X = st->X; p.n = bm.n; p.gpt = bm.gpt; p.wpt = bm.wpt;
    p.chunk_offset = chunk; p.nchunk = st->nchunk; p.vbias_add = first ? 0 : 1;
    p.smul = (float)smul;
    p.vbias = vbias;
    p.exch_part = exch_part;
    if (first && nj) p.nrm = *nj;
    const int nb = (bm.n + 7) / 8 * 8;
    afqmc_status r;
    if (bm.form == 1) {
      if (nb == 8) r = launch_tm<8>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
      else if (nb == 16) r = launch_tm<16>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
      else if (nb == 24) r = launch_tm<24>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
      else r = launch_tm<32>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    } else if (!reg) r = launch<0>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    else if (nb == 8) r = launch<0, 8>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    else if (nb == 16) r = launch<0, 16>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    else if (nb == 24) r = launch<0, 24>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    else r = launch<0, 32>(g, bm.map_l, bm.map_th, p, s, launches, err, errlen);
    if (r != AFQMC_OK) return r;
    chunk += 4 * bm.m_tiles;
    first = false;
  }
  return AFQMC_OK;
}

// The VHS operands' form: dual stages (each operand byte once through shared memory) while L^T is
// small enough to stay in L2; the interleaved single-tile stages (twice the ring depth) when L^T
// streams from HBM, where hiding its latency matters more (measured at N = 1512: 19 vs 22 ms).
bool vhs_dual(const TcState* st) { return (double)st->lt_rows * st->vparts * st->kx * 2 < 1e9; }

afqmc_status vhs_planes(TcState* st, cudaStream_t s, char* tcbuf, const float2* coef, int* status,
                        unsigned long long* launches, char* err, size_t errlen, bool coef_ready) {
  if (!st->pg.ok) {
    snprintf(err, errlen, "tensor-core propagation is not available for this problem");
    return AFQMC_EINVAL;
  }
  if (!coef_ready) {
    k_coef_bf16<<<st->W, 256, 0, s>>>(st->W, st->X, st->kx, st->nseg, coef,
                                      reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_coef), st->cplx ? st->kx0 : 0);
    ++*launches;
  }
  Geom g{};
  g.m_tiles = (int)((st->lt_rows + kBM - 1) / kBM);
  g.n_tiles = (2 * st->W + st->vhs_bn - 1) / st->vhs_bn;
  g.k_blocks = st->nseg * st->kx / kBK;
  g.k_steps = st->nseg * st->kx / 16;
  if (st->nseg == 3 && vhs_dual(st)) {   // A = L^T [hi | lo], B = the coefficients [hi | lo]
    g.dual = 1;
    g.k_blocks = st->kx / kBK;
    g.k_steps = st->kx / 16;
    g.a_lo = st->kx;
    g.b_hi = 0;
    g.b_lo = st->kx;
  } else if (st->nseg == 3) {
    g.il3 = 1;
    g.seg = st->kx;
  }
  g.m_step = kBM;
  g.n_step = st->vhs_bn;
  g.bn = st->vhs_bn;
  if (!finish_geom(&g, 16 + (st->packed ? 4096 : 0), 4)) {
    snprintf(err, errlen, "tcgen05 VHS: shared memory plan failed");
    return AFQMC_EINVAL;
  }
  Params p{};
  p.g = g;
  p.status = status;
  p.n = st->N;
  p.out_rows = 2 * st->W;
  p.out_cols = (int)st->lt_rows;
  p.pairs = st->packed ? reinterpret_cast<const int*>(tcbuf + st->off_pairs) : nullptr;
  p.blocks = st->packed ? reinterpret_cast<const int2*>(tcbuf + st->off_blocks) : nullptr;
  p.planes = reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_vp);
  p.npad = st->pg.npad;
  p.kq = st->pg.kq;
  return launch<2>(g, st->map_lt_a, st->map_coef_b, p, s, launches, err, errlen);
}

afqmc_status vhs(TcState* st, cudaStream_t s, char* tcbuf, const float2* coef, float* out, int* status,
                 unsigned long long* launches, char* err, size_t errlen) {
  if (st->packed) {
    snprintf(err, errlen, "tcgen05 VHS: packed L^T feeds only the tensor-core propagation");
    return AFQMC_EINVAL;
  }
  k_coef_bf16<<<st->W, 256, 0, s>>>(st->W, st->X, st->kx, st->nseg, coef,
                                    reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_coef), st->cplx ? st->kx0 : 0);
  ++*launches;
  Geom g{};
  g.m_tiles = st->vhs_m_tiles;
  g.n_tiles = st->vhs_n_tiles;
  g.k_blocks = st->nseg * st->kx / kBK;
  g.k_steps = st->nseg * st->kx / 16;
  if (st->nseg == 3 && vhs_dual(st)) {   // A = the coefficients [hi | lo], B = L^T [hi | lo]
    g.dual = 1;
    g.k_blocks = st->kx / kBK;
    g.k_steps = st->kx / 16;
    g.a_lo = st->kx;
    g.b_hi = 0;
    g.b_lo = st->kx;
  } else if (st->nseg == 3) {
    g.il3 = 1;
    g.seg = st->kx;
  }
  g.m_step = kBM;
  g.n_step = 256;
  g.bn = 256;
  if (!finish_geom(&g, 16, 4)) {
    snprintf(err, errlen, "tcgen05 VHS: shared memory plan failed");
    return AFQMC_EINVAL;
  }
  Params p{};
  p.g = g;
  p.status = status;
  p.out = out;
  p.ldo = (long long)st->N * st->N;
  p.out_rows = 2 * st->W;
  p.out_cols = st->N * st->N;
  return launch<1>(g, st->map_coef, st->map_lt, p, s, launches, err, errlen);
}

// ----------------------------------------------------------------------------- grouped launches
namespace {

template <typename T>
afqmc_status to_device(const std::vector<T>& v, void** dev, char* err, size_t errlen) {
  *dev = nullptr;
  if (v.empty()) return AFQMC_OK;
  if (cudaMalloc(dev, v.size() * sizeof(T)) != cudaSuccess ||
      cudaMemcpy(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    snprintf(err, errlen, "grouped launch: device descriptors (%zu bytes)", v.size() * sizeof(T));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

// Problems in order of the cost of one tile (K blocks x MMA N x products per k-step), the most
// expensive first (the CTAs take tiles in turn), and their tile ranges; returns the tile count.
// Each problem's first tile is rounded up to a multiple of the SM count, so that the CTAs (one per
// SM, taking every SM-count-th tile) enter each problem at the same turn: at most one problem's
// operands compete for L2 at a time.
int order_problems(std::vector<GroupProblem>& pr) {
  auto cost = [](const GroupProblem& q) { return (long long)q.p.g.k_blocks * q.p.g.bn * (q.p.g.dual ? 3 : 1); };
  std::stable_sort(pr.begin(), pr.end(), [&](const GroupProblem& a, const GroupProblem& b) { return cost(a) > cost(b); });
  const int sms = num_sms();
  int t = 0;
  for (auto& q : pr) {
    t = (t + sms - 1) / sms * sms;
    q.tile0 = t;
    q.tiles = q.p.g.m_tiles * q.p.g.n_tiles;
    t += q.tiles;
  }
  return t;
}

int stage_bytes_of(const Geom& g) { return g.dual ? 2 * kStageA + 2 * g.bn * kBK * 2 : kStageA + g.bn * kBK * 2; }

// The launch layout for the problems, each with its own epilogue groups and buffers (p.g.epi_groups,
// p.g.epi_bytes): the stage stride, the epilogue region (the largest problem's), ring depth and
// accumulators.  The launch runs the most groups any problem uses; a problem's surplus groups idle.
bool group_layout(std::vector<GroupProblem>& pr, GroupLaunch* gg) {
  int stride = 0, acc = 0, groups = 1, region = 0;
  for (auto& q : pr) {
    q.p.g.epi_bytes = (q.p.g.epi_bytes + 15) & ~15;
    stride = std::max(stride, q.p.g.stage_bytes);
    acc = std::max(acc, q.p.g.bn);
    groups = std::max(groups, q.p.g.epi_groups);
    region = std::max(region, q.p.g.epi_groups * q.p.g.epi_bytes);
  }
  const int per = ((region + groups - 1) / groups + 15) & ~15;   // the kernel sizes the region as groups x per
  const int st = std::min(4, (kMaxSmem - 1024 - groups * per - kTailBytes - 4 * kParamSlot) / std::max(1, stride));
  if (st < 2) return false;
  gg->stages = st;
  gg->stage_stride = stride;
  gg->epi_groups = groups;
  gg->epi_bytes = per;
  gg->acc_stride = acc;
  gg->tmem_cols = tmem_cols_for(acc);
  if (gg->tmem_cols > 512) return false;
  for (auto& q : pr) {
    q.p.g.stages = st;
    q.p.g.tmem_cols = gg->tmem_cols;
  }
  gg->smem = 1024 + (size_t)st * stride + (size_t)groups * per + kTailBytes + 4 * kParamSlot;
  return gg->smem <= (size_t)kMaxSmem;
}

}  // namespace

namespace {
int first_block(const TcState* st) {
  for (int b = 0; b < st->nblk; ++b)
    if (st->blk[b].n > 0) return b;
  return 0;
}
// Ring depth of a launch whose largest stage is `stride` bytes and largest epilogue region `region`.
int group_stages(int stride, int region) {
  return std::min(4, (kMaxSmem - 1024 - region - kTailBytes - 4 * kParamSlot) / std::max(1, stride));
}
int epi_region(const GroupProblem& q) { return q.p.g.epi_groups * ((q.p.g.epi_bytes + 15) & ~15); }

// Problem (system i, block b) of the grouped exchange in the streamed form with at most cap
// epilogue groups; the register-row epilogue where its loads stay within `acc` accumulator
// columns of a launch whose tensor memory is laid out for MMA N <= acc.
bool exchange_problem(const GroupSystem& sy, int b, int cap, int acc_min, GroupProblem* out, char* err,
                      size_t errlen) {
  TcState* st = sy.st;
  BlockMaps bm = st->blk[b];   // a copy: the system's own exchange keeps its form
  exchange_config(st, bm, cap, 1);
  int chunk = 0;   // exchange partial slots of the earlier blocks
  for (int b0 = 0; b0 < b; ++b0) chunk += 4 * st->blk[b0].m_tiles;
  GroupProblem q{};
  Geom& g = q.p.g;
  g.m_tiles = bm.m_tiles;
  g.n_tiles = (st->W + bm.wpt - 1) / bm.wpt;
  g.k_blocks = (st->nseg * st->kst + kBK - 1) / kBK;
  g.k_steps = st->nseg * st->kst / 16;
  g.m_step = bm.gpt * bm.n;
  g.n_step = bm.wpt * 2 * bm.n;
  g.bn = bm.bn;
  g.epi_groups = bm.groups;
  if (bm.dual) {
    g.dual = 1;
    g.k_blocks = (st->kst + kBK - 1) / kBK;
    g.k_steps = st->kst / 16;
    g.a_lo = st->kst;
    g.b_hi = 0;
    g.b_lo = 2 * st->kst;
  }
  g.ntg = exchange_ntg(st, bm, g);
  g.stage_bytes = stage_bytes_of(g);
  q.mapA = bm.map_l;
  if (!make_map(&q.mapB, sy.tcbuf + bm.off_th, (unsigned long long)st->W * 2 * bm.n,
                (unsigned long long)st->nseg * st->kst, (unsigned)bm.bn)) {
    snprintf(err, errlen, "grouped exchange: tensor map of the Theta operand");
    return false;
  }
  Params& p = q.p;
  p.status = sy.status;
  p.W = st->W; p.X = st->X; p.n = bm.n; p.gpt = bm.gpt; p.wpt = bm.wpt;
  p.chunk_offset = chunk; p.nchunk = st->nchunk;
  p.vbias_add = 2;
  p.smul = (float)sy.smul;
  p.vbias = sy.vbias;
  p.exch_part = sy.exch_part;
  const int acc = std::max(acc_min, g.bn), nb = (bm.n + 7) / 8 * 8;
  const bool reg = nb <= 32 && exchange_reg(p.n, p.wpt, g.bn) && acc + (p.wpt - 1) * 2 * p.n + p.n + nb <= tmem_cols_for(acc);
  q.nb = reg ? nb : 0;
  g.epi_bytes = epi_bytes_exchange(p.n, reg);
  *out = q;
  return true;
}
}  // namespace

afqmc_status group_exchange_plan(const GroupSystem* sys, int nsys, int groups, GroupGemm* gg, char* err,
                                 size_t errlen) {
  *gg = GroupGemm{};
  gg->epi = 0;
  std::vector<ThetaJob> th;
  std::vector<int> th_first(1, 0);
  // 1. every (system, block) in its own configuration: at most `groups` epilogue groups (0: the
  //    system's tuned count where its exchange is streamed), fewer until two ring stages fit
  struct Cand { int sys, blk, cap, stages; GroupProblem q; };
  std::vector<Cand> cands;
  for (int i = 0; i < nsys; ++i)
    for (int b = 0; b < sys[i].st->nblk; ++b) {
      const BlockMaps& bm = sys[i].st->blk[b];
      if (bm.n == 0) continue;
      Cand c{i, b, groups > 0 ? std::min(groups, 4) : (bm.form == 0 ? std::max(1, bm.groups) : 4), 0, GroupProblem{}};
      for (;;) {
        if (!exchange_problem(sys[i], b, c.cap, 0, &c.q, err, errlen)) return AFQMC_ECUDA;
        c.stages = group_stages(c.q.p.g.stage_bytes, epi_region(c.q));
        if (c.stages >= 2 || c.q.p.g.epi_groups <= 1) break;
        c.cap = c.q.p.g.epi_groups - 1;
      }
      if (c.stages < 2) {
        snprintf(err, errlen, "grouped exchange: system %d does not fit shared memory", i);
        return AFQMC_EINVAL;
      }
      cands.push_back(c);
    }
  // 2. classes: a problem joins the first class whose merged layout keeps its ring depth (and the
  //    class's), else opens a class of its own
  struct Cls { std::vector<int> mem; int stride = 0, region = 0, bn = 0, stages = 0, nb = 0; };
  // a register-row problem keeps its epilogue under a launch whose accumulators are `acc` wide
  auto reg_fits = [&](const Cand& c, int acc) {
    const Params& p = c.q.p;
    return c.q.nb == 0 || acc + (p.wpt - 1) * 2 * p.n + p.n + c.q.nb <= tmem_cols_for(acc);
  };
  std::vector<Cls> cls;
  std::vector<int> order(cands.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cands[x].stages > cands[y].stages; });
  for (int k : order) {
    const Cand& c = cands[k];
    int pick = -1;
    for (int j = 0; j < (int)cls.size(); ++j) {
      if (cls[j].nb != c.q.nb) continue;   // one epilogue width per launch
      const int acc = std::max(cls[j].bn, c.q.p.g.bn);
      bool fits = reg_fits(c, acc);
      for (int m : cls[j].mem) fits = fits && reg_fits(cands[m], acc);
      if (!fits) continue;
      const int d = group_stages(std::max(cls[j].stride, c.q.p.g.stage_bytes), std::max(cls[j].region, epi_region(c.q)));
      if (d == c.stages && d == cls[j].stages) { pick = j; break; }
    }
    if (pick < 0) {
      cls.push_back(Cls{});
      pick = (int)cls.size() - 1;
      cls[pick].nb = c.q.nb;
    }
    Cls& L = cls[pick];
    L.mem.push_back(k);
    L.stride = std::max(L.stride, c.q.p.g.stage_bytes);
    L.region = std::max(L.region, epi_region(c.q));
    L.bn = std::max(L.bn, c.q.p.g.bn);
    L.stages = group_stages(L.stride, L.region);
  }
  // 3. one launch per class, the register-row epilogues decided against the class's accumulators
  for (const Cls& L : cls) {
    std::vector<GroupProblem> pr;
    std::vector<NormalsJob> nrm;   // drawn by this launch's spare warp: its systems' first blocks
    for (int k : L.mem)
      if (sys[cands[k].sys].nj.x && cands[k].blk == first_block(sys[cands[k].sys].st)) nrm.push_back(sys[cands[k].sys].nj);
    for (int k : L.mem) {
      GroupProblem q;
      if (!exchange_problem(sys[cands[k].sys], cands[k].blk, cands[k].cap, L.bn, &q, err, errlen)) {
        group_free(gg);
        return AFQMC_ECUDA;
      }
      pr.push_back(q);
    }
    gg->part.emplace_back();
    GroupLaunch& gl = gg->part.back();
    gl.nb = L.nb;
    for (const auto& q : pr)
      if (q.nb != L.nb) {
        snprintf(err, errlen, "grouped exchange: mixed epilogue widths in one launch");
        group_free(gg);
        return AFQMC_EINVAL;
      }
    if (!group_layout(pr, &gl)) {
      snprintf(err, errlen, "grouped exchange: no shared-memory layout fits every system");
      group_free(gg);
      return AFQMC_EINVAL;
    }
    gl.tiles = order_problems(pr);
    gl.nprob = (int)pr.size();
    gl.grid = std::min(gl.tiles, num_sms());
    gl.nnrm = (int)nrm.size();
    afqmc_status r;
    if ((r = to_device(pr, &gl.dev_probs, err, errlen)) != AFQMC_OK ||
        (r = to_device(nrm, &gl.dev_nrm, err, errlen)) != AFQMC_OK) {
      group_free(gg);
      return r;
    }
    ++gg->nparts;
  }
  for (int i = 0; i < nsys; ++i) {
    TcState* st = sys[i].st;
    for (int b = 0; b < st->nblk; ++b) {
      const BlockMaps& bm = st->blk[b];
      if (bm.n == 0) continue;
      ThetaJob j{st->N, st->ncol, bm.c0, bm.n, st->kst, st->nseg, st->cplx ? st->kst0 : 0, sys[i].thetaT,
                 reinterpret_cast<__nv_bfloat16*>(sys[i].tcbuf + bm.off_th)};
      th.push_back(j);
      th_first.push_back(th_first.back() + st->W);
    }
  }
  gg->ntheta = (int)th.size();
  gg->theta_blocks = th_first.back();
  afqmc_status r;
  if ((r = to_device(th, &gg->dev_theta, err, errlen)) != AFQMC_OK ||
      (r = to_device(th_first, &gg->dev_theta_first, err, errlen)) != AFQMC_OK) {
    group_free(gg);
    return r;
  }
  return AFQMC_OK;
}

afqmc_status group_vhs_plan(const GroupSystem* sys, int nsys, GroupGemm* gg, char* err, size_t errlen) {
  *gg = GroupGemm{};
  gg->epi = 2;
  std::vector<GroupProblem> pr;
  for (int i = 0; i < nsys; ++i) {
    TcState* st = sys[i].st;
    char* tcbuf = sys[i].tcbuf;
    if (!st->pg.ok) {
      snprintf(err, errlen, "grouped VHS: system %d has no tensor-core propagation", i);
      return AFQMC_EINVAL;
    }
    GroupProblem q{};
    Geom& g = q.p.g;
    g.m_tiles = (int)((st->lt_rows + kBM - 1) / kBM);
    g.n_tiles = (2 * st->W + st->vhs_bn - 1) / st->vhs_bn;
    g.k_blocks = st->nseg * st->kx / kBK;
    g.k_steps = st->nseg * st->kx / 16;
    if (st->nseg == 3 && vhs_dual(st)) {
      g.dual = 1;
      g.k_blocks = st->kx / kBK;
      g.k_steps = st->kx / 16;
      g.a_lo = st->kx;
      g.b_hi = 0;
      g.b_lo = st->kx;
    } else if (st->nseg == 3) {
      g.il3 = 1;
      g.seg = st->kx;
    }
    g.m_step = kBM;
    g.n_step = st->vhs_bn;
    g.bn = st->vhs_bn;
    g.stage_bytes = stage_bytes_of(g);
    q.mapA = st->map_lt_a;
    q.mapB = st->map_coef_b;
    Params& p = q.p;
    p.status = sys[i].status;
    p.n = st->N;
    p.out_rows = 2 * st->W;
    p.out_cols = (int)st->lt_rows;
    p.pairs = st->packed ? reinterpret_cast<const int*>(tcbuf + st->off_pairs) : nullptr;
    p.blocks = st->packed ? reinterpret_cast<const int2*>(tcbuf + st->off_blocks) : nullptr;
    p.planes = reinterpret_cast<__nv_bfloat16*>(tcbuf + st->off_vp);
    p.npad = st->pg.npad;
    p.kq = st->pg.kq;
    g.epi_groups = 4;
    g.epi_bytes = 16 + (st->packed ? 4096 : 0);   // packed: the mirrored rows' staging
    pr.push_back(q);
  }
  gg->part.assign(1, GroupLaunch{});
  GroupLaunch& gl = gg->part[0];
  if (pr.empty() || !group_layout(pr, &gl)) {
    snprintf(err, errlen, "grouped VHS: no shared-memory layout fits every system");
    return AFQMC_EINVAL;
  }
  gl.tiles = order_problems(pr);
  gl.nprob = (int)pr.size();
  gl.grid = std::min(gl.tiles, num_sms());
  gg->nparts = 1;
  return to_device(pr, &gl.dev_probs, err, errlen);
}

afqmc_status group_gemm(const GroupGemm& gg, cudaStream_t s, bool normals, unsigned long long* launches, char* err,
                        size_t errlen, cudaStream_t s2) {
  for (int k = 0; k < gg.nparts; ++k) {
    const GroupLaunch& gl = gg.part[k];
    const cudaStream_t sk = (s2 && (k & 1)) ? s2 : s;
    GroupArgs ga{};
    ga.probs = static_cast<const GroupProblem*>(gl.dev_probs);
    ga.nprob = gl.nprob;
    ga.tiles = gl.tiles;
    ga.stages = gl.stages;
    ga.stage_stride = gl.stage_stride;
    ga.epi_groups = gl.epi_groups;
    ga.epi_bytes = gl.epi_bytes;
    ga.tmem_cols = gl.tmem_cols;
    ga.acc_stride = gl.acc_stride;
    const bool draw = normals && gl.nnrm > 0;   // each launch draws the normals of its systems
    ga.nrm = draw ? static_cast<const NormalsJob*>(gl.dev_nrm) : nullptr;
    ga.nnrm = draw ? gl.nnrm : 0;
    const int threads = 64 + 128 * gl.epi_groups + (ga.nnrm ? 32 : 0);
    const CUtensorMap none{};
    const Params p0{};
    if (gg.epi == 2) k_tc_gemm<2, 0, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    else if (gl.nb == 8) k_tc_gemm<0, 8, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    else if (gl.nb == 16) k_tc_gemm<0, 16, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    else if (gl.nb == 24) k_tc_gemm<0, 24, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    else if (gl.nb == 32) k_tc_gemm<0, 32, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    else k_tc_gemm<0, 0, true><<<gl.grid, threads, gl.smem, sk>>>(none, none, p0, ga);
    ++*launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      snprintf(err, errlen, "grouped tcgen05 GEMM launch: %s", cudaGetErrorString(e));
      return AFQMC_ECUDA;
    }
  }
  return AFQMC_OK;
}

afqmc_status group_theta(const GroupGemm& gg, cudaStream_t s, unsigned long long* launches, char* err, size_t errlen) {
  if (gg.ntheta == 0) return AFQMC_OK;
  k_theta_bf16_group<<<gg.theta_blocks, 256, 0, s>>>(static_cast<const ThetaJob*>(gg.dev_theta),
                                                     static_cast<const int*>(gg.dev_theta_first), gg.ntheta);
  ++*launches;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(err, errlen, "grouped Theta conversion: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

void group_free(GroupGemm* gg) {
  for (auto& gl : gg->part) {
    if (gl.dev_probs) cudaFree(gl.dev_probs);
    if (gl.dev_nrm) cudaFree(gl.dev_nrm);
    gl.dev_probs = gl.dev_nrm = nullptr;
  }
  for (void* p : {gg->dev_theta, gg->dev_theta_first})
    if (p) cudaFree(p);
  gg->dev_theta = gg->dev_theta_first = nullptr;
  gg->part.clear();
  gg->nparts = 0;
}

// ----------------------------------------------------------------------------- general fp32 GEMM
// One operand (rows x K, element (i, k) at src[i si + k sk]) as split bf16 K-major rows [hi | lo] of
// kx (K padded to the k-block) each, zeros in the padding.
__global__ void k_split_rows(int rows, int K, int kx, const float* src, long long si, long long sk,
                             __nv_bfloat16* out) {
  const size_t total = (size_t)rows * kx;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / kx), k = (int)(idx % kx);
    const float v = k < K ? src[(size_t)i * si + (size_t)k * sk] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16* row = out + (size_t)i * 2 * kx;
    row[k] = hi;
    row[kx + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

afqmc_status gemm_f32_prepare(char* err, size_t errlen) {
  if (cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem) != cudaSuccess) {
    snprintf(err, errlen, "tcgen05 fp32 GEMM: cannot reserve shared memory");
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

size_t gemm_f32_scratch(int M, int N, int K) {
  const size_t kx = ((size_t)K + kBK - 1) / kBK * kBK;
  return align256((size_t)M * 2 * kx * 2) + align256((size_t)N * 2 * kx * 2);
}

afqmc_status gemm_f32(cudaStream_t s, int M, int N, int K, const float* A, long long sAm, long long sAk,
                      const float* B, long long sBk, long long sBn, float* C, long long ldc, char* scratch,
                      size_t scratch_bytes, int* status, unsigned long long* launches, char* err, size_t errlen) {
  if (M < 1 || N < 1 || K < 1 || N % 16 != 0) {
    snprintf(err, errlen, "tcgen05 fp32 GEMM: shape %d x %d x %d (N a multiple of 16)", M, N, K);
    return AFQMC_EINVAL;
  }
  if (gemm_f32_scratch(M, N, K) > scratch_bytes) {
    snprintf(err, errlen, "tcgen05 fp32 GEMM: scratch too small for %d x %d x %d", M, N, K);
    return AFQMC_EINVAL;
  }
  const int kx = (K + kBK - 1) / kBK * kBK;
  __nv_bfloat16* a = reinterpret_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(scratch + align256((size_t)M * 2 * kx * 2));
  const int ga = (int)std::min<size_t>(1184, ((size_t)M * kx + 255) / 256);
  const int gb = (int)std::min<size_t>(1184, ((size_t)N * kx + 255) / 256);
  k_split_rows<<<ga, 256, 0, s>>>(M, K, kx, A, sAm, sAk, a);
  k_split_rows<<<gb, 256, 0, s>>>(N, K, kx, B, sBn, sBk, b);
  *launches += 2;
  Geom g{};
  g.bn = std::min(256, N);
  g.m_tiles = (M + kBM - 1) / kBM;
  g.n_tiles = (N + g.bn - 1) / g.bn;
  g.il3 = 1;   // A [hi | lo] x B [hi | lo]: hi hi, lo hi, hi lo per k-block
  g.seg = kx;
  g.k_blocks = 3 * kx / kBK;
  g.k_steps = 3 * kx / 16;
  g.m_step = kBM;
  g.n_step = g.bn;
  int groups = 4;   // each epilogue group stores a multiple of 16 columns
  while (g.bn % (16 * groups)) --groups;
  if (!finish_geom(&g, 16, groups)) {
    snprintf(err, errlen, "tcgen05 fp32 GEMM: shared memory plan failed");
    return AFQMC_EINVAL;
  }
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, (unsigned long long)M, 2ull * kx, kBM) ||
      !make_map(&mb, b, (unsigned long long)N, 2ull * kx, (unsigned)g.bn)) {
    snprintf(err, errlen, "tcgen05 fp32 GEMM: tensor maps");
    return AFQMC_ECUDA;
  }
  Params p{};
  p.g = g;
  p.status = status;
  p.out = C;
  p.ldo = ldc;
  p.out_rows = M;
  p.out_cols = N;
  return launch<1>(g, ma, mb, p, s, launches, err, errlen);
}

}  // namespace tc
}  // namespace afq
