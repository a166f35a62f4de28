// Tensor-core (tcgen05 + TMA) contractions for the BF16 and BF16x3 forms.
//
// Operands are bf16, K-major (the contracted index contiguous), rows padded to a
// multiple of 64 elements with zeros.  BF16x3 accumulates hi*hi + lo*hi + hi*lo
// in fp32: the exchange operands are stored concatenated along K, A = [hi | lo |
// hi] and B = [hi | hi | lo], so one bf16 GEMM with three times the K forms the
// sum; the VHS operands (L^T, the coefficients) are stored once as [hi | lo] and
// the kernel's producer picks the part of each operand per K block.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "afqmc.h"

namespace afq {
namespace tc {

struct BlockMaps {
  int n;             // occupied orbitals of this spin block
  int c0;            // first stored column of the block
  int gpt, wpt;      // gammas per M tile (gpt * n <= 128), walkers per N tile (wpt * 2n <= 256)
  int bn;            // MMA N (multiple of 16, >= wpt * 2n)
  int groups;        // epilogue warpgroups of the exchange kernel (wpt is a multiple of it)
  int form;          // 1: the Ltilde tile stays in tensor memory (k_exch_tm), 0: both operands streamed
  int dual;          // streamed form: each stage holds the hi and lo parts of both operands (long K)
  int m_tiles, n_tiles;
  size_t off_l, off_th;   // byte offsets of the bf16 Ltilde / Theta^T copies in the tc buffer
  CUtensorMap map_l, map_th;
};

// Geometry of the tensor-core propagation kernel (N <= 128).  Per walker and column chunk the
// kernel forms t = E_h psi, the Taylor terms V t / k and E_h acc as D = A B^T with A = V or
// F = E_h - I (rows p, K = q) and B = the current term, both split into bf16 hi + lo.
// Shared memory, from a 1024-byte aligned base: V hi | V lo (4 swizzle atoms of npad rows:
// Re V q < 64, Re V q >= 64, Im V q < 64, Im V q >= 64) | F hi | F lo (2 atoms) | B (2 atoms of
// 4 cwp rows: the term's hi parts, then its lo parts) | mbarriers.
struct PropGeom {
  int ok = 0;
  int large = 0;       // 1: N > 128 (or a complex Hamiltonian), the batched form (V streamed per product,
                       // one launch per product)
  int cplx_f = 0;      // complex E_h: F = E_h - I as four planes [Re hi, Im hi, Re lo, Im lo], F products
                       // over two K halves like the V products
  int npad = 0;        // N rounded up to 8: rows of the V and F planes
  int kq = 0;          // row pitch of the planes: 128 (N <= 128) or N rounded up to 64
  int ncolp = 0;       // large form: walker columns rounded up to 8 (B operand rows 2 ncolp)
  int mtiles = 0;      // large form: 128-row tiles per walker
  int nk = 0;          // 16-wide k-steps per K half, ceil(N / 16)
  int cw = 0, cwp = 0; // columns per chunk and its padding to a multiple of 8
  int nch = 0;         // chunks per walker
  int off_vlo = 0, off_fhi = 0, off_flo = 0, off_b = 0, off_bar = 0;
  int smem = 0;        // dynamic shared memory bytes including the alignment slack
};
PropGeom prop_geom(int N, int ncol, bool cplx = false);

struct TcState {
  int prec = 0, W = 0, N = 0, X = 0, ncol = 0, nblk = 0;
  int cplx = 0;       // complex Hamiltonian: operands realified along K (see plan)
  int kst0 = 0, kx0 = 0;   // complex: the padded length of one real part (exchange: N, VHS: fields)
  int kst = 0;        // padded length of one K segment of the exchange operands (multiple of 16)
  int nseg = 1;       // 1 (BF16) or 3 (BF16x3)
  int nchunk = 0;     // exchange partial slots per walker (four per M tile, summed over blocks)
  BlockMaps blk[2];
  // VHS build
  int kx = 0;         // padded naux (multiple of 64)
  int vparts = 1;     // stored parts of the VHS operands: [hi | lo] (BF16x3) or hi (BF16)
  int packed = 0;     // L^T holds only blocks touching the upper triangle (large-form propagation; see plan)
  long long lt_rows = 0;   // rows of L^T: N^2, or 128 per packed block
  long long nblocks = 0;   // packed: 8 x 16 (p, q) blocks, one M tile each
  size_t off_pairs = 0;    // packed: int32 p N + q per row (-1: a row left out)
  size_t off_blocks = 0;   // packed: int2 (p block, q block) per M tile
  size_t off_lt = 0, off_coef = 0;
  int vhs_m_tiles = 0, vhs_n_tiles = 0;
  int vhs_bn = 256;   // N tile of the VHS planes GEMM (multiple of 32)
  CUtensorMap map_lt, map_coef;
  // tensor-core propagation
  PropGeom pg;
  size_t off_vp = 0, off_fp = 0;   // V planes [W][4][npad][kq], F planes [2][npad][kq] (bf16)
  size_t off_b[2] = {0, 0};        // large form: term operands [W][hi, lo][2 ncolp][2 kq] (bf16)
  size_t off_acc = 0;              // large form: Taylor sum [W][npad][ncolp] complex64
  CUtensorMap map_vp, map_fp, map_lt_a, map_coef_b, map_b[2];
  bool ready = false;
};

// Fills the geometry of st (no device work) and returns the bytes of the tc buffer.
size_t plan(TcState* st, int prec, int W, int N, int X, int ncol, const int* c0, const int* nb, int nblk,
            bool cplx = false);

// Caps the exchange epilogue warpgroups at `groups` (0: largest that fits), selects the form (0: the
// Ltilde tile resident in tensor memory where it fits, else streamed; 1: streamed) and re-derives
// the walker tiling and the Theta tensor map; returns the groups in use for block 0.
int set_exchange_groups(TcState* st, char* tcbuf, int groups, int form = 0);

// Set-up of the tensor-core operands, which arrive in chunks of Cholesky vectors: begin clears the
// operand buffers (their K padding must stay zero); load_chunk writes the bf16 copies of Ltilde
// (from [ng][ncol][N]) and of L^T (from [ng][N][N]) for gammas g0 .. g0 + ng - 1; finish builds the
// TMA descriptors over the tc buffer and reserves the kernels' shared memory.
afqmc_status begin(TcState* st, cudaStream_t s, char* tcbuf, char* err, size_t errlen);
template <typename T, typename TL>
afqmc_status load_chunk(TcState* st, cudaStream_t s, char* tcbuf, int g0, int ng, const T* chol, const TL* lrot,
                        unsigned long long* launches, char* err, size_t errlen);
// Complex Hamiltonian: fields f0 .. f0 + nf - 1 (complex [nf][N][N], interleaved) and their Ltilde
// (complex [nf][ncol][N]) into the realified operands.
template <typename G>
afqmc_status load_chunk_c(TcState* st, cudaStream_t s, char* tcbuf, int f0, int nf, const G* fields, const G* lrot,
                          unsigned long long* launches, char* err, size_t errlen);
afqmc_status finish(TcState* st, char* tcbuf, char* err, size_t errlen);

// N(0,1) fields of the step counter *step (stream 0) for W walker slots x X into x[w][g]; drawn by
// a spare warp of the exchange kernel, whose binary64 pipe is otherwise idle.
struct NormalsJob {
  double* x;
  unsigned long long seed;
  const unsigned long long* step;
  int W, X;
};

// vbias[w][g] = smul sum_s Tr T^{g s} (vbias is cleared first), exch_part[w][slot]: the slots of each
// M tile hold partial sums (one per epilogue warp, or the tile's sum and zeros) of smul sum over the
// tile's gammas of sum_ab T_ab T_ba, with T^{g s} = Ltilde^{g s} Theta^s; Theta^T complex64 [W][ncol][N].
// widx (optional, nw entries): the kernel works on walkers widx[0..nw) and writes their partials
// to rows 0..nw of exch_part; vbias may be NULL (not written).
// nj (optional): the first launch also draws those normals.  theta_ready: the bf16 operand copy of
// Theta^T (every walker, in walker order) is already current, so it is not rebuilt (ignored with widx).
afqmc_status exchange(TcState* st, cudaStream_t s, char* tcbuf, double smul, const float2* thetaT, float2* vbias,
                      float2* exch_part, int* status, const int* widx, int nw, unsigned long long* launches,
                      char* err, size_t errlen, const NormalsJob* nj = nullptr, bool theta_ready = false);

// VHS planar fp32: out[w][0][pq] + i out[w][1][pq] = sum_g coef[w][g] L^g_pq, coef complex64 [W][X].
afqmc_status vhs(TcState* st, cudaStream_t s, char* tcbuf, const float2* coef, float* out, int* status,
                 unsigned long long* launches, char* err, size_t errlen);

// Tensor-core propagation: one-time F = E_h - I planes from binary64 f64 [N][N], zeroed V planes
// and the tensor maps.  Only when st->pg.ok.
afqmc_status prepare_prop(TcState* st, cudaStream_t s, char* tcbuf, const double* f64, unsigned long long* launches,
                          char* err, size_t errlen);

// VHS into the bf16 hi/lo planes read by the tensor-core propagation.
// coef_ready: the split-bf16 coefficients were written by the fields kernel (not rebuilt from coef).
afqmc_status vhs_planes(TcState* st, cudaStream_t s, char* tcbuf, const float2* coef, int* status,
                        unsigned long long* launches, char* err, size_t errlen, bool coef_ready = false);

// psi <- E_h sum_{k<=order} V^k / k! E_h psi for every walker with w != 0 (psi complex64 [W][N][ncol]).
afqmc_status propagate(TcState* st, cudaStream_t s, char* tcbuf, int order, float2* psi, const double* w,
                       int* status, unsigned long long* launches, char* err, size_t errlen);

// C[M][N] (row pitch ldc) = A B in fp32 with split-bf16 tensor-core products (hi hi + lo hi + hi lo,
// fp32 accumulation): A element (i, k) at A[i sAm + k sAk], B element (k, j) at B[k sBk + j sBn]; N a
// multiple of 16.  The operands are first split into bf16 K-major rows in `scratch`
// (gemm_f32_scratch(M, N, K) bytes, 256-byte aligned).
size_t gemm_f32_scratch(int M, int N, int K);
afqmc_status gemm_f32_prepare(char* err, size_t errlen);   // once, outside stream capture
afqmc_status gemm_f32(cudaStream_t s, int M, int N, int K, const float* A, long long sAm, long long sAk,
                      const float* B, long long sBk, long long sBn, float* C, long long ldc, char* scratch,
                      size_t scratch_bytes, int* status, unsigned long long* launches, char* err, size_t errlen);

// ------------------------------------------------------------------ grouped launches (uneven batches)
// One persistent launch of the exchange (or the VHS planes) contraction over the tiles of several
// systems and spin blocks (a work list ordered by tile cost), with the problems' tensor maps and
// parameters in device memory.
struct GroupSystem {
  TcState* st;
  char* tcbuf;
  double smul;
  const float2* thetaT;   // exchange: Theta^T complex64 [W][ncol][N]
  float2* vbias;          // exchange: cleared before the launch, every block adds its traces
  float2* exch_part;      // exchange: binary32 partials
  int* status;
  NormalsJob nj;          // exchange: the step's normals (nj.x == nullptr: none)
};
struct GroupLaunch {   // one persistent launch over several problems
  int nprob = 0, tiles = 0, grid = 0;
  int stages = 0, stage_stride = 0, epi_groups = 0, epi_bytes = 0, tmem_cols = 0, acc_stride = 0;
  int nb = 0;                          // exchange: the launch's register-row epilogue width (0: staged)
  size_t smem = 0;
  void* dev_probs = nullptr;           // the problems (device)
  void* dev_nrm = nullptr;             // exchange: NormalsJob of the systems whose first block is here
  int nnrm = 0;
};
struct GroupGemm {
  int epi = 0;              // 0: exchange and force bias, 2: VHS planes
  int nparts = 0;           // exchange: one launch per class of problems with one ring depth
  std::vector<GroupLaunch> part;
  void* dev_theta = nullptr;           // exchange: Theta^T conversion jobs, one per (system, block)
  void* dev_theta_first = nullptr;     // their first block in the grid
  int ntheta = 0, theta_blocks = 0;
};
// Exchange over every (system, block) in the streamed form, each with its own walker tiling and
// epilogue warpgroups (at most `groups`; 0: the system's own tuned count), in as few launches as keep
// every problem's own ring depth: problems whose largest stage and epilogue buffers leave the same
// number of stages share a launch.  The systems' own exchange forms are left as
// they are.
afqmc_status group_exchange_plan(const GroupSystem* sys, int nsys, int groups, GroupGemm* gg, char* err,
                                 size_t errlen);
afqmc_status group_vhs_plan(const GroupSystem* sys, int nsys, GroupGemm* gg, char* err, size_t errlen);
// normals: the exchange launch also draws every system's normals of the current step counter.
// s2 (optional): every second launch goes there (the caller orders s2 after s before the call and s
// after s2 afterwards), so that one launch's last wave overlaps the next one's first.
afqmc_status group_gemm(const GroupGemm& gg, cudaStream_t s, bool normals, unsigned long long* launches, char* err,
                        size_t errlen, cudaStream_t s2 = nullptr);
// The bf16 Theta^T operands of every (system, block) from Theta^T (when the copies are stale).
afqmc_status group_theta(const GroupGemm& gg, cudaStream_t s, unsigned long long* launches, char* err,
                         size_t errlen);
void group_free(GroupGemm* gg);

// The tensor-core propagation of several systems: the small-form systems (N <= 128) in one launch
// over all their walkers (contiguous walker ranges per CTA, balanced by cost), the large-form ones
// in one launch per product over all their (walker, row tile) pairs.  Every system takes the same
// Taylor order.
struct GroupPropSystem {
  TcState* st;
  char* tcbuf;
  float2* psi;
  const double* w;
  int* status;
};
struct GroupProp {
  int order = 0;
  int nsmall = 0, small_grid = 0, small_off_bar = 0, small_tmem = 0;
  size_t small_smem = 0;
  void* dev_small = nullptr;   // small-form systems (device)
  void* dev_cta = nullptr;     // first walker of each CTA (device, small_grid + 1)
  int nlarge = 0, large_tiles = 0, large_grid = 0, large_stages = 0, large_stride = 0, large_tmem = 0,
      large_acc = 0;
  size_t large_smem = 0;
  void* dev_large = nullptr;   // large-form systems (device)
  void* dev_psib = nullptr;    // their first-operand jobs (device)
};
afqmc_status group_prop_plan(const GroupPropSystem* sys, int nsys, int order, GroupProp* gp, char* err,
                             size_t errlen);
// s2 (optional, ordered by the caller as for group_gemm): the large-form launches go there, beside
// the small-form one.
afqmc_status group_propagate(const GroupProp& gp, cudaStream_t s, unsigned long long* launches, char* err,
                             size_t errlen, cudaStream_t s2 = nullptr);
void group_prop_free(GroupProp* gp);

}  // namespace tc
}  // namespace afq
