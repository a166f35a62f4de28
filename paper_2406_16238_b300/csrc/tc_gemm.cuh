// Tensor-core (tcgen05 + TMA) contractions for the BF16 and BF16x3 forms.
//
// Operands are bf16, K-major (the contracted index contiguous), rows padded to a
// multiple of 64 elements with zeros.  BF16x3 stores the split operands
// concatenated along K, A = [hi | lo | hi] and B = [hi | hi | lo], so one
// bf16 GEMM with three times the K accumulates hi*hi + lo*hi + hi*lo in fp32.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "afqmc.h"

namespace afq {
namespace tc {

struct BlockMaps {
  int n;             // occupied orbitals of this spin block
  int c0;            // first stored column of the block
  int gpt, wpt;      // gammas per M tile (gpt * n <= 128), walkers per N tile (wpt * 2n <= 256)
  int bn;            // MMA N (multiple of 16, >= wpt * 2n)
  int groups;        // epilogue warpgroups of the exchange kernel (wpt is a multiple of it)
  int m_tiles, n_tiles;
  size_t off_l, off_th;   // byte offsets of the bf16 Ltilde / Theta^T copies in the tc buffer
  CUtensorMap map_l, map_th;
};

struct TcState {
  int prec = 0, W = 0, N = 0, X = 0, ncol = 0, nblk = 0;
  int kst = 0;        // padded length of one K segment of the exchange operands (multiple of 64)
  int nseg = 1;       // 1 (BF16) or 3 (BF16x3)
  int nchunk = 0;     // exchange partials per walker (sum of m_tiles over blocks)
  BlockMaps blk[2];
  // VHS build
  int kx = 0;         // padded naux (multiple of 64)
  size_t off_lt = 0, off_coef = 0;
  int vhs_m_tiles = 0, vhs_n_tiles = 0;
  CUtensorMap map_lt, map_coef;
  bool ready = false;
};

// Fills the geometry of st (no device work) and returns the bytes of the tc buffer.
size_t plan(TcState* st, int prec, int W, int N, int X, int ncol, const int* c0, const int* nb, int nblk);

// Caps the exchange epilogue warpgroups at `groups` (0: largest that fits) and re-derives the walker
// tiling and the Theta tensor map; returns the groups in use for block 0.
int set_exchange_groups(TcState* st, char* tcbuf, int groups);

// One-time bf16 copies of Ltilde (from binary64 [X][ncol][N]) and of L^T (from binary64 [X][N][N]),
// and the TMA descriptors over the tc buffer.
afqmc_status prepare(TcState* st, cudaStream_t s, char* tcbuf, const double* chol64, const double* lrot64,
                     unsigned long long* launches, char* err, size_t errlen);

// vbias[w][g] = smul sum_s Tr T^{g s}, exch_part[w][chunk] = smul sum over the chunk's gammas of
// sum_ab T_ab T_ba, with T^{g s} = Ltilde^{g s} Theta^s; Theta^T complex64 [W][ncol][N].
// widx (optional, nw entries): the kernel works on walkers widx[0..nw) and writes their partials
// to rows 0..nw of exch_part; vbias may be NULL (not written).
afqmc_status exchange(TcState* st, cudaStream_t s, char* tcbuf, double smul, const float2* thetaT, float2* vbias,
                      double2* exch_part, int* status, const int* widx, int nw, unsigned long long* launches,
                      char* err, size_t errlen);

// VHS planar fp32: out[w][0][pq] + i out[w][1][pq] = sum_g coef[w][g] L^g_pq, coef complex64 [W][X].
afqmc_status vhs(TcState* st, cudaStream_t s, char* tcbuf, const float2* coef, float* out, int* status,
                 unsigned long long* launches, char* err, size_t errlen);

}  // namespace tc
}  // namespace afq
