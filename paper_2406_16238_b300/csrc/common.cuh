// Shared device helpers of the AFQMC library: complex arithmetic on (re, im)
// pairs, block reductions, and the bit-reproducible Gaussian field draw.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace afq {

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };
template <typename R> using cplx_t = typename Cplx<R>::T;

__host__ __device__ __forceinline__ double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__host__ __device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
template <typename R> __host__ __device__ __forceinline__ cplx_t<R> from_d2(double2 v);
template <> __host__ __device__ __forceinline__ double2 from_d2<double>(double2 v) { return v; }
template <> __host__ __device__ __forceinline__ float2 from_d2<float>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm (scaled division, avoids overflow of |b|^2)
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return mk((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  }
  double r = b.x / b.y, den = b.x * r + b.y;
  return mk((a.x * r + a.y) / den, (a.y * r - a.x) / den);
}

// Grouped launches over several systems: block b of the flattened grid belongs to the system s with
// first[s] <= b < first[s + 1] (first[0] = 0, first[nsys] = the grid size).
__device__ __forceinline__ int group_of(const int* __restrict__ first, int nsys, int b) {
  int lo = 0, hi = nsys;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(first + mid) <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of one double (fixed shuffle tree + fixed warp order).
// scratch: >= 32 doubles of shared memory.  All threads must call it.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < nw ? scratch[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) scratch[0] = t;
  }
  __syncthreads();
  t = scratch[0];
  __syncthreads();
  return t;
}

// NQ deterministic block sums at once for a 256-thread block: a fixed-order shared-memory tree
// down to 32 values per quantity, then one warp per quantity.  Binary64 additions on few warps:
// on B300 an FP64 warp instruction costs an issue slot of the slow FP64 pipe whatever its active
// lanes, so this uses about a third of the FP64 instructions of NQ separate block_sum calls.
// part: NQ * 256 doubles of shared memory; the sums land in out[0..NQ) (shared); all threads call.
template <int NQ>
__device__ __forceinline__ void block_sum_multi(const double* v, double* part, double* out) {
  static_assert(NQ >= 1 && NQ <= 8, "at most one warp per quantity");
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < NQ; ++q) part[q * 256 + tid] = v[q];
  for (int stride = 128; stride >= 32; stride >>= 1) {
    __syncthreads();
    if (tid < stride)
#pragma unroll
      for (int q = 0; q < NQ; ++q) part[q * 256 + tid] += part[q * 256 + tid + stride];
  }
  __syncthreads();
  const int wid = tid >> 5, lane = tid & 31;
  if (wid < NQ) {
    const double s = warp_sum(part[wid * 256 + lane]);
    if (lane == 0) out[wid] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ double2 block_sum2(double2 v, double* scratch) {
  double a = block_sum(v.x, scratch);
  double b = block_sum(v.y, scratch);
  return mk(a, b);
}

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Box-Muller field
// draw.  Every floating-point step is one binary64 operation rounded to
// nearest with no contraction (explicit __d*_rn intrinsics), so the draws are
// reproducible bit for bit by any IEEE-754 implementation that performs the
// same operations in the same order.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// u = (m + 1/2) 2^-52, m = top 52 bits of hi:lo; exact, strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint32_t hi, uint32_t lo) {
  const unsigned long long word = ((unsigned long long)hi << 32) | lo;
  const unsigned long long m = word >> 12;
  return __dmul_rn(__dadd_rn(__ull2double_rn(m), 0.5), 0x1p-52);
}

constexpr int kLogTerms = 12;   // odd atanh series: 1, 1/3, ..., 1/23
constexpr int kTrigTerms = 9;   // sin to degree 17, cos to degree 16

struct SeriesTables {
  double lg[kLogTerms];
  double sn[kTrigTerms];
  double cs[kTrigTerms];
};

// Coefficients by exact-integer divisions in a fixed order.
__device__ __forceinline__ void fill_series_tables(SeriesTables* t) {
  for (int k = 0; k < kLogTerms; ++k) t->lg[k] = __ddiv_rn(1.0, (double)(2 * k + 1));
  t->sn[0] = 1.0;
  t->cs[0] = 1.0;
  for (int k = 1; k < kTrigTerms; ++k) {
    t->sn[k] = __ddiv_rn(t->sn[k - 1], -(double)((2 * k) * (2 * k + 1)));
    t->cs[k] = __ddiv_rn(t->cs[k - 1], -(double)((2 * k - 1) * (2 * k)));
  }
}

// log u for normal u in (0, 1]: u = m 2^e, m in [sqrt(1/2), sqrt(2)), log m = 2 atanh((m-1)/(m+1)).
__device__ __forceinline__ double series_log(double u, const SeriesTables& t) {
  const long long bits = __double_as_longlong(u);
  int e = (int)((bits >> 52) & 0x7ff) - 1022;
  double m = __longlong_as_double((bits & 0x800fffffffffffffLL) | (1022LL << 52));  // [0.5, 1)
  if (m < 0.7071067811865476) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double z = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z2 = __dmul_rn(z, z);
  double s = t.lg[kLogTerms - 1];
#pragma unroll
  for (int k = kLogTerms - 2; k >= 0; --k) s = __dadd_rn(__dmul_rn(s, z2), t.lg[k]);
  return __dadd_rn(__dmul_rn((double)e, 0.6931471805599453), __dmul_rn(2.0, __dmul_rn(z, s)));
}

// cos and sin of 2 pi u2 for u2 in [0, 1): quarter-turn reduction, reflection to [0, pi/4].
__device__ __forceinline__ void series_sincos_turn(double u2, const SeriesTables& t, double* c_out,
                                                   double* s_out) {
  const double q = __dmul_rn(4.0, u2);
  const double kq = floor(q);
  const double f = __dsub_rn(q, kq);
  const bool flip = f > 0.5;
  const double r = __dmul_rn(flip ? __dsub_rn(1.0, f) : f, 1.5707963267948966);
  const double r2 = __dmul_rn(r, r);
  double ps = t.sn[kTrigTerms - 1];
#pragma unroll
  for (int j = kTrigTerms - 2; j >= 1; --j) ps = __dadd_rn(__dmul_rn(ps, r2), t.sn[j]);
  const double sin_r = __dadd_rn(r, __dmul_rn(__dmul_rn(r, r2), ps));
  double pc = t.cs[kTrigTerms - 1];
#pragma unroll
  for (int j = kTrigTerms - 2; j >= 1; --j) pc = __dadd_rn(__dmul_rn(pc, r2), t.cs[j]);
  const double cos_r = __dadd_rn(1.0, __dmul_rn(r2, pc));
  const double ct = flip ? sin_r : cos_r;
  const double st = flip ? cos_r : sin_r;
  const int k = (int)kq;
  double c, s;
  switch (k) {
    case 0: c = ct; s = st; break;
    case 1: c = -st; s = ct; break;
    case 2: c = -ct; s = -st; break;
    default: c = st; s = -ct; break;
  }
  *c_out = c;
  *s_out = s;
}

__device__ __forceinline__ uint4 field_counter(uint32_t pair, uint32_t slot, unsigned long long step,
                                               uint32_t stream) {
  return make_uint4(pair, slot, (uint32_t)(step & 0xffffffffull),
                    (uint32_t)((step >> 32) & 0xffffull) | (stream << 16));
}

// Two N(0,1) draws (x_{2j}, x_{2j+1}) of walker slot w at a step.
__device__ __forceinline__ void normal_pair(unsigned long long seed, uint32_t pair, uint32_t slot,
                                            unsigned long long step, uint32_t stream,
                                            const SeriesTables& t, double* z0, double* z1) {
  const uint4 r = philox4x32_10(field_counter(pair, slot, step, stream), (uint32_t)(seed & 0xffffffffull),
                                (uint32_t)(seed >> 32));
  const double u1 = uniform52(r.x, r.y);
  const double u2 = uniform52(r.z, r.w);
  const double rho = __dsqrt_rn(__dmul_rn(-2.0, series_log(u1, t)));
  double c, s;
  series_sincos_turn(u2, t, &c, &s);
  *z0 = __dmul_rn(rho, c);
  *z1 = __dmul_rn(rho, s);
}

// Device status bits (sticky until read by the host).
enum : int { kStatusSingular = 1, kStatusNonFinite = 2, kStatusNoWalkers = 4, kStatusTimeout = 8 };

}  // namespace afq
