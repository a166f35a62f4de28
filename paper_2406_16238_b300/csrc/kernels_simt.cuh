// CUDA-core kernels of the AFQMC step, templated on the real type R (double for
// the FP64 form, float for the reduced forms).  Overlap inverses and
// log-determinants, weights, QR and all energy reductions are binary64 in both.
#pragma once
#include <type_traits>

#include <cuda_bf16.h>

#include "common.cuh"
#include "ff.cuh"

namespace afq {

// ============================================================================
// Batched strided GEMM on CUDA cores:  out = alpha * A[b] (M x K) * B[b] (K x Nc)
// A, B real or complex (interleaved); the output is complex if either is.
// C (optional) is stored; D (optional) is stored or accumulated.  Batches whose
// skip[b] == 0.0 are left untouched (frozen walkers).
// ============================================================================
struct GemmDesc {
  int M, Nc, K, batch;
  const void* A; long long sAb, sAm, sAk;
  const void* B; long long sBb, sBk, sBn;
  void* C; long long sCb, sCm, sCn;
  void* D; long long sDb, sDm, sDn;
  int d_add;
  double alpha_re, alpha_im;
  const double* skip;
  int a_planar;          // complex A stored as separate real and imaginary planes
  long long a_im_off;    // element offset of the imaginary plane (a_planar)
  int conj_a;            // complex A enters conjugated (A^+ with the transposing strides)
};

// Block tile BM x BN = 16 TM x 16 TN, each of the 256 threads owns a TM x TN register tile.
template <typename R, bool CA, bool CB, int TM, int TN>
__global__ void __launch_bounds__(256) k_gemm(GemmDesc g) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  constexpr bool CC = CA || CB;
  using R2 = cplx_t<R>;
  __shared__ R As_re[BK][BM], As_im[CA ? BK : 1][CA ? BM : 1];
  __shared__ R Bs_re[BK][BN], Bs_im[CB ? BK : 1][CB ? BN : 1];
  const int b = blockIdx.z;
  if (g.skip != nullptr && g.skip[b] == 0.0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const char* Ab = (const char*)g.A + (size_t)b * g.sAb * ((CA && !g.a_planar) ? sizeof(R2) : sizeof(R));
  const char* Bb = (const char*)g.B + (size_t)b * g.sBb * (CB ? sizeof(R2) : sizeof(R));
  R acc_re[TM][TN], acc_im[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_re[i][j] = acc_im[i][j] = R(0);
  const bool a_kfast = g.sAk == 1;
  const bool b_nfast = g.sBn == 1 || g.sBk != 1;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int l = 0; l < (BM * BK) / 256; ++l) {
      const int e = tid + 256 * l;
      int mm, kk;
      if (a_kfast) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      const int m = m0 + mm, k = k0 + kk;
      R vr = R(0), vi = R(0);
      if (m < g.M && k < g.K) {
        const long long idx = (long long)m * g.sAm + (long long)k * g.sAk;
        if (CA) {
          if (g.a_planar) { vr = ((const R*)Ab)[idx]; vi = ((const R*)Ab)[idx + g.a_im_off]; }
          else { R2 v = ((const R2*)Ab)[idx]; vr = v.x; vi = v.y; }
          if (g.conj_a) vi = -vi;
        } else vr = ((const R*)Ab)[idx];
      }
      As_re[kk][mm] = vr;
      if (CA) As_im[kk][mm] = vi;
    }
#pragma unroll
    for (int l = 0; l < (BN * BK) / 256; ++l) {
      const int e = tid + 256 * l;
      int nn, kk;
      if (b_nfast) { kk = e / BN; nn = e % BN; } else { nn = e / BK; kk = e % BK; }
      const int n = n0 + nn, k = k0 + kk;
      R vr = R(0), vi = R(0);
      if (n < g.Nc && k < g.K) {
        const long long idx = (long long)k * g.sBk + (long long)n * g.sBn;
        if (CB) { R2 v = ((const R2*)Bb)[idx]; vr = v.x; vi = v.y; }
        else vr = ((const R*)Bb)[idx];
      }
      Bs_re[kk][nn] = vr;
      if (CB) Bs_im[kk][nn] = vi;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R ar[TM], ai[TM], br[TN], bi[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) { ar[i] = As_re[kk][ty + 16 * i]; ai[i] = CA ? As_im[kk][ty + 16 * i] : R(0); }
#pragma unroll
      for (int j = 0; j < TN; ++j) { br[j] = Bs_re[kk][tx + 16 * j]; bi[j] = CB ? Bs_im[kk][tx + 16 * j] : R(0); }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if (!CA && !CB) {
            acc_re[i][j] += ar[i] * br[j];
          } else if (CA && !CB) {
            acc_re[i][j] += ar[i] * br[j];
            acc_im[i][j] += ai[i] * br[j];
          } else if (!CA && CB) {
            acc_re[i][j] += ar[i] * br[j];
            acc_im[i][j] += ar[i] * bi[j];
          } else {
            acc_re[i][j] += ar[i] * br[j] - ai[i] * bi[j];
            acc_im[i][j] += ar[i] * bi[j] + ai[i] * br[j];
          }
        }
    }
    __syncthreads();
  }
  const R al_r = (R)g.alpha_re, al_i = (R)g.alpha_im;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.Nc) continue;
      if (CC) {
        R2 v;
        v.x = al_r * acc_re[i][j] - al_i * acc_im[i][j];
        v.y = al_r * acc_im[i][j] + al_i * acc_re[i][j];
        if (g.C) ((R2*)g.C)[(size_t)b * g.sCb + (size_t)m * g.sCm + (size_t)n * g.sCn] = v;
        if (g.D) {
          R2* d = (R2*)g.D + (size_t)b * g.sDb + (size_t)m * g.sDm + (size_t)n * g.sDn;
          if (g.d_add) { R2 o = *d; o.x += v.x; o.y += v.y; *d = o; } else *d = v;
        }
      } else {
        const R v = al_r * acc_re[i][j];
        if (g.C) ((R*)g.C)[(size_t)b * g.sCb + (size_t)m * g.sCm + (size_t)n * g.sCn] = v;
        if (g.D) {
          R* d = (R*)g.D + (size_t)b * g.sDb + (size_t)m * g.sDm + (size_t)n * g.sDn;
          *d = g.d_add ? *d + v : v;
        }
      }
    }
  }
}

// ============================================================================
// Arguments of the overlap / Theta / weight-update kernel (k_overlap_gj below).
// mode 0: write log O; mode 1: weight update (Eqs. 13-16) from the stored
// log O, c_mf and sum(x xbar - xbar^2/2); mode 2: Theta only.
// ============================================================================
template <typename R>
struct OverlapArgs {
  int N, ncol, nblk, c0[2], nb[2];
  double smul;                    // 2 for a restricted (one stored spin block) context, else 1
  const cplx_t<R>* psi;           // [W][N][ncol]
  const double* phi;              // [N][ncol]
  const R* phi_r;                 // [N][ncol] at the walkers' precision
  const cplx_t<R>* phi_c;         // complex trial [N][ncol] (complex Hamiltonians; A = Phi^+ psi)
  cplx_t<R>* thetaT;              // [W][ncol][N]
  double2* logO;                  // [W]
  double* w;                      // [W]
  int* status;
  int mode;
  const double2* cmf;             // [W]
  const double2* xxbar;           // [W]
  double dt, e_trial, e_c;
  double eshift;                  // exp(dt (E_T - E_c)), the same factor for every walker
  const double* etr;              // non-null: E_T = etr[0] on the device (updated at each comb), eshift unused
  unsigned long long* step;       // incremented once (mode 1) if non-null
  double* wph;                    // free projection (mode 1): weight phases [W]; null: phaseless
  // optional: Theta^T also as the tensor-core exchange operand of each spin block s, rows
  // (w, part, b) of nseg * kst bf16 = [hi | hi | lo] (hi only when nseg = 1)
  __nv_bfloat16* thb[2];
  int kst, nseg;
  int kst0;                       // complex Hamiltonian: the realified operand layout (0: real)
};

// Theta^T entry (b, p) of walker w as the split-bf16 exchange operand of its block.
template <typename R2>
__device__ __forceinline__ void store_theta_bf16(__nv_bfloat16* out, int kst, int nseg, int n, int w, int b, int p,
                                                 R2 v, int kst0 = 0) {
  const size_t rowlen = (size_t)nseg * kst;
  __nv_bfloat16* re = out + ((size_t)w * 2 * n + b) * rowlen + p;
  __nv_bfloat16* im = re + (size_t)n * rowlen;
  const float fx = (float)v.x, fy = (float)v.y;
  const __nv_bfloat16 hr = __float2bfloat16_rn(fx), hi = __float2bfloat16_rn(fy);
  const __nv_bfloat16 lr = __float2bfloat16_rn(fx - __bfloat162float(hr));
  const __nv_bfloat16 li = __float2bfloat16_rn(fy - __bfloat162float(hi));
  re[0] = hr;
  im[0] = hi;
  if (nseg == 3) {
    re[kst] = hr;
    im[kst] = hi;
    re[2 * kst] = lr;
    im[2 * kst] = li;
  }
  if (kst0) {   // complex Hamiltonian: rows [Re | Im] and [Im | -Re] (each real part kst0 long)
    re[kst0] = hi;
    im[kst0] = __hneg(hr);
    if (nseg == 3) {
      re[kst + kst0] = hi;
      im[kst + kst0] = __hneg(hr);
      re[2 * kst + kst0] = li;
      im[2 * kst + kst0] = __hneg(lr);
    }
  }
}

// t mapped to (-pi, pi] by subtracting a multiple of 2 pi (few binary64 operations; the slow FP64
// units make atan2(sin t, cos t) a long serial chain).
__device__ __forceinline__ double wrap_angle(double t) {
  const double twopi = 6.283185307179586, pi = 3.141592653589793;
  double r = fma(-twopi, rint(t * (1.0 / twopi)), t);
  if (r > pi) r -= twopi;
  else if (r <= -pi) r += twopi;
  return r;
}

// ============================================================================
// Local energy pieces on CUDA cores.  CTA (chunk, walker): for gamma in the
// chunk, T^{g s} = Ltilde^{g s} Theta^s (n x n), vbias_g = smul sum_s Tr T,
// exchange partial = smul sum_{g in chunk, s} sum_ab T_ab T_ba.
// ============================================================================
template <typename R>
struct ExchangeArgs {
  int N, X, ncol, nblk, c0[2], nb[2];
  double smul;
  int gchunk, nchunk;
  const cplx_t<R>* thetaT;   // [W][ncol][N]
  const R* lrot;             // [X][ncol][N]
  const cplx_t<R>* lrot_c;   // complex Ltilde [X][ncol][N] (complex Hamiltonians), used by k_exchange<R, true>
  cplx_t<R>* vbias;          // [W][X]
  double2* exch_part;        // [rows][nchunk]
  int with_exchange;
  const int* widx;           // optional: CTA row y works on walker widx[y] (its partials go to row y)
  int with_vbias;
};

template <typename R, bool CL = false>
__global__ void __launch_bounds__(256) k_exchange(ExchangeArgs<R> a) {
  using R2 = cplx_t<R>;
  using LT = typename std::conditional<CL, R2, R>::type;
  extern __shared__ __align__(16) unsigned char sm_ex[];
  __shared__ double red[32];
  const int chunk = blockIdx.x, row = blockIdx.y, tid = threadIdx.x;
  const int w = a.widx ? a.widx[row] : row;
  const int cn = a.ncol * a.N;
  R2* th = (R2*)sm_ex;                                // [ncol][N]
  LT* lr = (LT*)(th + cn);                            // [ncol][N]
  const int nmax = max(a.nb[0], a.nblk > 1 ? a.nb[1] : 0);
  R2* T = (R2*)((R*)lr + (CL ? 2 * cn : cn + (cn & 1)));   // [nmax][nmax]
  const LT* lsrc = CL ? reinterpret_cast<const LT*>(a.lrot_c) : reinterpret_cast<const LT*>(a.lrot);
  for (int i = tid; i < cn; i += blockDim.x) th[i] = a.thetaT[(size_t)w * cn + i];
  double2 exx = mk(0.0, 0.0);
  const int g0 = chunk * a.gchunk, g1 = min(a.X, g0 + a.gchunk);
  for (int g = g0; g < g1; ++g) {
    __syncthreads();
    for (int i = tid; i < cn; i += blockDim.x) lr[i] = lsrc[(size_t)g * cn + i];
    __syncthreads();
    double2 vb = mk(0.0, 0.0);
    for (int s = 0; s < a.nblk; ++s) {
      const int c0 = a.c0[s], n = a.nb[s];
      if (n == 0) continue;
      for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int ia = idx / n, ib = idx % n;
        const LT* lrow = lr + (size_t)(c0 + ia) * a.N;
        const R2* trow = th + (size_t)(c0 + ib) * a.N;
        R sr = R(0), si = R(0);
        for (int p = 0; p < a.N; ++p) {
          const R2 t = trow[p];
          if constexpr (CL) {
            const R2 l = lrow[p];
            sr += l.x * t.x - l.y * t.y;
            si += l.x * t.y + l.y * t.x;
          } else {
            const R l = lrow[p];
            sr += l * t.x;
            si += l * t.y;
          }
        }
        R2 v;
        v.x = sr;
        v.y = si;
        T[idx] = v;
      }
      __syncthreads();
      if (a.with_exchange) {
        for (int idx = tid; idx < n * n; idx += blockDim.x) {
          const int ia = idx / n, ib = idx % n;
          const double2 tab = to_d2(T[ia * n + ib]), tba = to_d2(T[ib * n + ia]);
          exx = cadd(exx, cmul(tab, tba));
        }
      }
      if (tid < 32) {
        double dr = 0.0, di = 0.0;
        for (int ia = tid; ia < n; ia += 32) {
          const double2 t = to_d2(T[ia * n + ia]);
          dr += t.x;
          di += t.y;
        }
        dr = warp_sum(dr);
        di = warp_sum(di);
        vb = cadd(vb, mk(dr, di));
      }
      __syncthreads();
    }
    if (tid == 0 && a.with_vbias) a.vbias[(size_t)w * a.X + g] = from_d2<R>(cscale(vb, a.smul));
  }
  if (!a.with_exchange) return;
  const double2 tot = block_sum2(exx, red);
  if (tid == 0) a.exch_part[(size_t)row * a.nchunk + chunk] = cscale(tot, a.smul);
}

// Per-walker local energy from the pieces: E1 = smul sum htilde . Theta^T,
// J = 1/2 sum_g vbias_g^2, K = 1/2 sum exchange partials.  eloc[w] = (E, E0+E1, J-K).
// The last CTA to finish (completion counter `done`, reset by it) forms the weighted estimator
// sums (ENumer, EDenom, E1Body, E2Body) over all walkers in a fixed order (free projection, wph
// non-null: Re and Im of sum w e^{i phi} E_L, Re and Im of sum w e^{i phi}); with a slot counter
// they go to out + 4 * (*slot) and the counter advances (graph-replayable history).
template <typename R>
struct EnergyArgs {
  int N, X, ncol;
  double smul, ecore;
  int nchunk;
  const cplx_t<R>* thetaT;
  const void* hrot;           // htilde: real [ncol][N] at the walkers' precision, or complex (CH)
  const cplx_t<R>* vbias;
  const double2* exch_part;   // binary64 partials (CUDA-core exchange), or
  const float2* exch_part_f;  // binary32 partials (tensor-core exchange), when non-null
  double2* eloc;
  int W;
  const double* wgt;
  const double* wph;
  double* out;
  int* slot;
  unsigned int* done;
  double* etacc;              // non-null: ENumer and EDenom also added to etacc[1], etacc[2] (running sums of E_T)
};

template <typename R, bool CH>
__device__ __forceinline__ void energy_walker(const EnergyArgs<R> A, const int w) {
  const int N = A.N, X = A.X, ncol = A.ncol, nchunk = A.nchunk, W = A.W;
  const double smul = A.smul, ecore = A.ecore;
  const cplx_t<R>* thetaT = A.thetaT;
  const void* hrot_v = A.hrot;
  const cplx_t<R>* vbias = A.vbias;
  const double2* exch_part = A.exch_part;
  const float2* exch_part_f = A.exch_part_f;
  double2* eloc = A.eloc;
  const double* wgt = A.wgt;
  const double* wph = A.wph;
  double* out = A.out;
  int* slot = A.slot;
  unsigned int* done = A.done;
  __shared__ double red[32];
  __shared__ double part[6 * 256];
  __shared__ int last_s;
  const int tid = threadIdx.x;
  const int cn = ncol * N;
  const cplx_t<R>* th = thetaT + (size_t)w * cn;
  // per-thread partials at the walkers' precision (four independent chains), summed in binary64
  R ar[4] = {R(0), R(0), R(0), R(0)}, ai[4] = {R(0), R(0), R(0), R(0)};
  int i = tid;
  const R* hrot_r = static_cast<const R*>(hrot_v);
  if constexpr (CH) {   // complex htilde: sum htilde Theta^T, complex products
    const cplx_t<R>* hc = static_cast<const cplx_t<R>*>(hrot_v);
    for (; i < cn; i += 256) {
      const cplx_t<R> t = th[i], h = hc[i];
      ar[0] += t.x * h.x - t.y * h.y;
      ai[0] += t.x * h.y + t.y * h.x;
    }
  }
  for (; i + 3 * 256 < cn; i += 4 * 256) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const cplx_t<R> t = th[i + u * 256];
      const R h = hrot_r[i + u * 256];
      ar[u] += t.x * h;
      ai[u] += t.y * h;
    }
  }
  for (; i < cn; i += 256) {
    const cplx_t<R> t = th[i];
    const R h = hrot_r[i];
    ar[0] += t.x * h;
    ai[0] += t.y * h;
  }
  double v[6];
  v[0] = (double)((ar[0] + ar[1]) + (ar[2] + ar[3]));
  v[1] = (double)((ai[0] + ai[1]) + (ai[2] + ai[3]));
  double jr = 0.0, ji = 0.0;
  for (int g = tid; g < X; g += 256) {   // vbias_g^2
    const double2 vb = to_d2(vbias[(size_t)w * X + g]);
    jr = fma(vb.x, vb.x, fma(-vb.y, vb.y, jr));
    ji = fma(2.0 * vb.x, vb.y, ji);
  }
  v[2] = jr;
  v[3] = ji;
  double kr = 0.0, ki = 0.0;
  for (int c = tid; c < nchunk; c += 256) {
    const double2 e = exch_part_f ? to_d2(exch_part_f[(size_t)w * nchunk + c]) : exch_part[(size_t)w * nchunk + c];
    kr += e.x;
    ki += e.y;
  }
  v[4] = kr;
  v[5] = ki;
  block_sum_multi<6>(v, part, red);
  if (tid == 0) {
    const double2 one = mk(ecore + smul * red[0], smul * red[1]);
    const double2 two = mk(0.5 * (red[2] - red[4]), 0.5 * (red[3] - red[5]));
    eloc[3 * w + 0] = cadd(one, two);
    eloc[3 * w + 1] = one;
    eloc[3 * w + 2] = two;
    __threadfence();
    last_s = atomicAdd(done, 1u) == (unsigned int)(W - 1);
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (wph) {   // free projection: complex weights w e^{i phi}; (Re, Im) of sum w e^{i phi} E_L and of sum w e^{i phi}
    for (int u = tid; u < W; u += blockDim.x) {
      const double wi = wgt[u];
      if (wi == 0.0) continue;
      double sn, cs;
      sincos(wph[u], &sn, &cs);
      const double2 e = __ldcg(&eloc[3 * u]);
      const double wr = wi * cs, wim = wi * sn;
      s0 += wr * e.x - wim * e.y;
      s1 += wr * e.y + wim * e.x;
      s2 += wr;
      s3 += wim;
    }
  } else {
    for (int u = tid; u < W; u += blockDim.x) {
      const double wi = wgt[u];
      if (wi == 0.0) continue;
      s0 += wi * __ldcg(&eloc[3 * u].x);
      s1 += wi;
      s2 += wi * __ldcg(&eloc[3 * u + 1].x);
      s3 += wi * __ldcg(&eloc[3 * u + 2].x);
    }
  }
  const double s4[4] = {s0, s1, s2, s3};
  __syncthreads();   // part[] and red[] are reused
  block_sum_multi<4>(s4, part, red);
  if (tid == 0) {
    double* o = slot ? out + 4 * (size_t)(*slot) : out;
    o[0] = red[0]; o[1] = red[1]; o[2] = red[2]; o[3] = red[3];
    if (slot) *slot += 1;
    if (A.etacc) {
      A.etacc[1] += red[0];
      A.etacc[2] += red[1];
    }
    *done = 0u;
  }
}

template <typename R, bool CH = false>
__global__ void __launch_bounds__(256) k_energy(EnergyArgs<R> a) {
  energy_walker<R, CH>(a, blockIdx.x);
}
// Several systems in one launch, one block per walker (each system's last block forms its sums).
template <typename R, bool CH = false>
__global__ void __launch_bounds__(256) k_energy_group(const EnergyArgs<R>* __restrict__ args,
                                                      const int* __restrict__ first, int nsys) {
  const int s = group_of(first, nsys, blockIdx.x);
  energy_walker<R, CH>(args[s], blockIdx.x - first[s]);
}

// ============================================================================
// Fields (Eq. 8, 10, 12): x ~ N(0,1) (Philox), xbar = -i sqrt(dt)(vbias - lbar)
// capped, xs = x - xbar, VHS coefficient -i sqrt(dt) xs, c_mf = i sqrt(dt) xs.lbar,
// sum(x xbar - xbar^2/2).  One CTA per walker.
// ============================================================================
template <typename R>
struct FieldArgs {
  int X;
  double sdt, cap;
  unsigned long long seed;
  const unsigned long long* step;
  const cplx_t<R>* vbias;   // [W][X]
  const double* lbar;       // [X]
  const double* slbar;      // [X] sqrt(dt) lbar
  double* x;                // [W][X]
  double2* xbar;            // [W][X]
  cplx_t<R>* coef;          // [W][X]
  __nv_bfloat16* coefb;     // optional: rows (w, part) of bf16 [hi | lo] (kx each; hi only if nseg = 1)
  int kx, nseg;
  int kx0;                  // complex Hamiltonian: rows (w, 0) = [Re c | -Im c], (w, 1) = [Im c | Re c] (kx0 each)
  double2* cmf;             // [W]
  double2* xxbar;           // [W]
  int free_proj;            // free projection: no force-bias shift (xbar = 0)
};

// The N(0,1) fields of every walker slot at the current step counter (stream 0) into x[w][g],
// one thread per pair (2j, 2j+1), grid-stride.
__device__ __forceinline__ void normals_grid(unsigned long long seed, const unsigned long long* step, int W, int X,
                                             double* x, const SeriesTables& tab) {
  const unsigned long long st = *step;
  const int npairs = (X + 1) / 2;
  const long long total = (long long)W * npairs;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(i / npairs), j = (int)(i - (long long)w * npairs);
    double z0, z1;
    normal_pair(seed, (uint32_t)j, (uint32_t)w, st, 0u, tab, &z0, &z1);
    x[(size_t)w * X + 2 * j] = z0;
    if (2 * j + 1 < X) x[(size_t)w * X + 2 * j + 1] = z1;
  }
}
__global__ void __launch_bounds__(128) k_normals(unsigned long long seed, const unsigned long long* step, int W,
                                                 int X, double* x) {
  __shared__ SeriesTables tab;
  if (threadIdx.x == 0) fill_series_tables(&tab);
  __syncthreads();
  normals_grid(seed, step, W, X, x, tab);
}
// Several systems: blockIdx.y is the system.
struct NormalsArgs {
  unsigned long long seed;
  const unsigned long long* step;
  int W, X;
  double* x;
};
__global__ void __launch_bounds__(128) k_normals_group(const NormalsArgs* __restrict__ args) {
  __shared__ SeriesTables tab;
  if (threadIdx.x == 0) fill_series_tables(&tab);
  __syncthreads();
  const NormalsArgs a = args[blockIdx.y];
  normals_grid(a.seed, a.step, a.W, a.X, a.x, tab);
}

// Zeroes n[s] float2 at p[s] for system s = blockIdx.y.
struct ZeroArgs {
  float2* p;
  size_t n;
};
__global__ void k_zero_group(const ZeroArgs* __restrict__ args) {
  const ZeroArgs a = args[blockIdx.y];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x)
    a.p[i] = make_float2(0.f, 0.f);
}

// Fields of one walker per CTA from the normals x[w][g] drawn by k_normals.  Registers held for
// 5 CTAs per SM: W = 640 walkers in one wave on 148 SMs.
template <typename R>
__device__ __forceinline__ void fields_walker(const FieldArgs<R> a, const int w) {
  __shared__ double red[32];
  const int tid = threadIdx.x;
  // c_mf = i sdt sum lbar_g xs_g; sum (x xbar - xbar^2 / 2) = sum (a x - (a^2 - b^2) / 2) +
  // i sum b (x - a) for xbar = a + i b, kept as sum a x, sum (a^2 - b^2) and sum b (x - a)
  double2 cm = mk(0.0, 0.0);
  double s_ax = 0.0, s_q = 0.0, s_im = 0.0;
  const int npairs = (a.X + 1) / 2;
  for (int j = tid; j < npairs; j += blockDim.x) {
    for (int t = 0; t < 2; ++t) {
      const int g = 2 * j + t;
      if (g >= a.X) break;
      const double x = a.x[(size_t)w * a.X + g];
      double2 xb = mk(0.0, 0.0);
      const double sl = a.slbar[g];
      if (!a.free_proj) {   // xbar = -i sdt (vbias - lbar)
        const double2 vb = to_d2(a.vbias[(size_t)w * a.X + g]);
        xb = mk(a.sdt * vb.y, fma(-a.sdt, vb.x, sl));
        if (a.cap > 0.0) {   // |xb| > cap, tested on the squares (the square root only when capping)
          const double m2 = xb.x * xb.x + xb.y * xb.y;
          if (m2 > a.cap * a.cap) {
            const double m = sqrt(m2);
            if (m > a.cap) xb = cscale(xb, a.cap / m);
          }
        }
      }
      const double2 xs = mk(x - xb.x, -xb.y);
      cplx_t<R> cf;   // -i sdt xs (binary32 forms: the product in binary32)
      if constexpr (sizeof(R) == 4) {
        const float sf = (float)a.sdt;
        cf.x = sf * (float)xs.y;
        cf.y = -sf * (float)xs.x;
      } else {
        cf = from_d2<R>(mk(a.sdt * xs.y, -a.sdt * xs.x));
      }
      a.coef[(size_t)w * a.X + g] = cf;
      if (a.coefb) {
        const size_t rowlen = (size_t)(a.nseg == 3 ? 2 : 1) * a.kx;
        __nv_bfloat16* re = a.coefb + (size_t)w * 2 * rowlen + g;
        __nv_bfloat16* im = re + rowlen;
        const float fx = (float)cf.x, fy = (float)cf.y;
        const __nv_bfloat16 hr = __float2bfloat16_rn(fx), hi = __float2bfloat16_rn(fy);
        const __nv_bfloat16 lr = __float2bfloat16_rn(fx - __bfloat162float(hr));
        const __nv_bfloat16 li = __float2bfloat16_rn(fy - __bfloat162float(hi));
        re[0] = hr;
        im[0] = hi;
        if (a.nseg == 3) {
          re[a.kx] = lr;
          im[a.kx] = li;
        }
        if (a.kx0) {   // the second real part of each complex row
          re[a.kx0] = __hneg(hi);
          im[a.kx0] = hr;
          if (a.nseg == 3) {
            re[a.kx + a.kx0] = __hneg(li);
            im[a.kx + a.kx0] = lr;
          }
        }
      }
      cm.x = fma(-sl, xs.y, cm.x);
      cm.y = fma(sl, xs.x, cm.y);
      s_ax = fma(xb.x, x, s_ax);
      s_q = fma(xb.x, xb.x, fma(-xb.y, xb.y, s_q));
      s_im = fma(xb.y, xs.x, s_im);
      a.xbar[(size_t)w * a.X + g] = xb;
    }
  }
  __shared__ double part[4 * 256];
  const double v4[4] = {cm.x, cm.y, fma(-0.5, s_q, s_ax), s_im};
  block_sum_multi<4>(v4, part, red);
  if (tid == 0) {
    a.cmf[w] = mk(red[0], red[1]);
    a.xxbar[w] = mk(red[2], red[3]);
  }
}
template <typename R>
__global__ void __launch_bounds__(256, 5) k_fields(FieldArgs<R> a) {
  fields_walker<R>(a, blockIdx.x);
}
template <typename R>
__global__ void __launch_bounds__(256, 5) k_fields_group(const FieldArgs<R>* __restrict__ args,
                                                         const int* __restrict__ first, int nsys) {
  const int s = group_of(first, nsys, blockIdx.x);
  fields_walker<R>(args[s], blockIdx.x - first[s]);
}

// Standalone draw (C-ABI afqmc_draw_normals): grid over walker slots.
__global__ void __launch_bounds__(256) k_draw_normals(unsigned long long seed, unsigned long long step,
                                                      uint32_t stream, int W, int X, double* out) {
  __shared__ SeriesTables tab;
  if (threadIdx.x == 0) fill_series_tables(&tab);
  __syncthreads();
  const int w = blockIdx.x;
  const int npairs = (X + 1) / 2;
  for (int j = threadIdx.x; j < npairs; j += blockDim.x) {
    double z0, z1;
    normal_pair(seed, (uint32_t)j, (uint32_t)w, step, stream, tab, &z0, &z1);
    out[(size_t)w * X + 2 * j] = z0;
    if (2 * j + 1 < X) out[(size_t)w * X + 2 * j + 1] = z1;
  }
}

// ============================================================================
// Comb population control.  One CTA: sequential (index-order) binary64 prefix
// of the weights, xi from Philox stream 1, tooth search.  Then a gather.
// ============================================================================
// et (optional): E_T and its running sums {E_T, sum ENumer, sum EDenom}; E_T becomes the running mixed
// estimate sum ENumer / sum EDenom once a measurement has been made.
__device__ __forceinline__ void comb_plan(int W, unsigned long long seed, const unsigned long long* step,
                                          const double* w, double* cum, int* src, double* neww, int* status,
                                          double* et = nullptr) {
  constexpr int kTile = 2048;
  __shared__ double ws[kTile];
  __shared__ double total_s, xi_s;
  __shared__ int last_s, ok_s;
  double t = 0.0;
  int last = -1;
  for (int base = 0; base < W; base += kTile) {   // weights staged per tile, summed by one thread in index order
    const int len = min(kTile, W - base);
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) ws[i] = w[base + i];
    __syncthreads();
    if (threadIdx.x == 0) {   // eight weights loaded ahead of their additions (the chain of sums stays in order)
      // "w > 0" as a signed integer compare of the bit patterns (the same answer for every value but
      // NaN, which makes the total non-finite anyway), which leaves the binary64 pipe to the chain of
      // additions
      int i = 0;
      for (; i + 8 <= len; i += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = ws[i + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          t = t + v[u];
          ws[i + u] = t;
          if (__double_as_longlong(v[u]) > 0) last = base + i + u;
        }
      }
      for (; i < len; ++i) {
        const double wi = ws[i];
        t = t + wi;
        ws[i] = t;
        if (__double_as_longlong(wi) > 0) last = base + i;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) cum[base + i] = ws[i];
  }
  if (threadIdx.x == 0) {
    total_s = t;
    last_s = last;
    ok_s = (t > 0.0) && isfinite(t) && last >= 0;
    const uint4 r = philox4x32_10(field_counter(0u, 0u, *step, 1u), (uint32_t)(seed & 0xffffffffull),
                                  (uint32_t)(seed >> 32));
    xi_s = uniform52(r.x, r.y);
    if (!ok_s) atomicOr(status, kStatusNoWalkers);
    *neww = ok_s ? t / (double)W : -1.0;
    if (et && et[2] > 0.0) et[0] = et[1] / et[2];
  }
  __syncthreads();
  const double total = total_s, xi = xi_s;
  const double* cs = W <= kTile ? ws : cum;   // the prefix sums (still in shared memory for one tile)
  for (int k = threadIdx.x; k < W; k += blockDim.x) {
    if (!ok_s) { src[k] = k; continue; }
    const double tooth = __ddiv_rn(__dmul_rn(__dadd_rn((double)k, xi), total), (double)W);
    int lo = 0, hi = W;   // first i with cum[i] > tooth
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cs[mid] > tooth) hi = mid; else lo = mid + 1;
    }
    src[k] = lo < W ? lo : last_s;
  }
}

__global__ void __launch_bounds__(256) k_comb_plan(int W, unsigned long long seed, const unsigned long long* step,
                                                   const double* w, double* cum, int* src, double* neww,
                                                   int* status, double* et) {
  comb_plan(W, seed, step, w, cum, src, neww, status, et);
}

// The comb of several systems (one launch per phase): the plans (one block per system), the gather of
// every system's walkers into its spare buffers (one block per walker), and the copy back.
template <typename R>
struct CombArgs {
  int W, psi_elems;
  unsigned long long seed;
  const unsigned long long* step;
  double* cum;
  int* src;
  double* neww;
  int* status;
  cplx_t<R>* psi;
  cplx_t<R>* psi_tmp;
  cplx_t<R>* th;
  cplx_t<R>* th_tmp;
  double2* logO;
  double2* logO_tmp;
  double* w;
  double* w_tmp;
  double* et;
};
template <typename R>
__global__ void __launch_bounds__(256) k_comb_plan_group(const CombArgs<R>* __restrict__ args) {
  const CombArgs<R> a = args[blockIdx.x];
  comb_plan(a.W, a.seed, a.step, a.w, a.cum, a.src, a.neww, a.status, a.et);
}

template <typename R>
__device__ __forceinline__ void comb_gather(int k, int psi_elems, int th_elems, const int* src, const double* neww,
                                            const cplx_t<R>* psi, cplx_t<R>* psi_out, const cplx_t<R>* th,
                                            cplx_t<R>* th_out, const double2* logO, double2* logO_out,
                                            const double* w, double* w_out) {
  const int s = src[k];
  const double nw = *neww;
  for (int i = threadIdx.x; i < psi_elems; i += blockDim.x) psi_out[(size_t)k * psi_elems + i] = psi[(size_t)s * psi_elems + i];
  for (int i = threadIdx.x; i < th_elems; i += blockDim.x) th_out[(size_t)k * th_elems + i] = th[(size_t)s * th_elems + i];
  if (threadIdx.x == 0) {
    logO_out[k] = logO[s];
    w_out[k] = nw >= 0.0 ? nw : w[s];
  }
}
template <typename R>
__global__ void __launch_bounds__(256) k_comb_gather(int W, int psi_elems, int th_elems, const int* src,
                                                     const double* neww, const cplx_t<R>* psi, cplx_t<R>* psi_out,
                                                     const cplx_t<R>* th, cplx_t<R>* th_out, const double2* logO,
                                                     double2* logO_out, const double* w, double* w_out) {
  (void)W;
  comb_gather<R>(blockIdx.x, psi_elems, th_elems, src, neww, psi, psi_out, th, th_out, logO, logO_out, w, w_out);
}
template <typename R>
__global__ void __launch_bounds__(256) k_comb_gather_group(const CombArgs<R>* __restrict__ args,
                                                           const int* __restrict__ first, int nsys) {
  const int s = group_of(first, nsys, blockIdx.x);
  const CombArgs<R> a = args[s];
  comb_gather<R>(blockIdx.x - first[s], a.psi_elems, a.psi_elems, a.src, a.neww, a.psi, a.psi_tmp, a.th, a.th_tmp,
                 a.logO, a.logO_tmp, a.w, a.w_tmp);
}
// The gathered walkers back into place (walker k of system s per block).
template <typename R>
__global__ void __launch_bounds__(256) k_comb_back_group(const CombArgs<R>* __restrict__ args,
                                                         const int* __restrict__ first, int nsys) {
  const int s = group_of(first, nsys, blockIdx.x);
  const CombArgs<R> a = args[s];
  const int k = blockIdx.x - first[s];
  const size_t off = (size_t)k * a.psi_elems;
  for (int i = threadIdx.x; i < a.psi_elems; i += blockDim.x) {
    a.psi[off + i] = a.psi_tmp[off + i];
    a.th[off + i] = a.th_tmp[off + i];
  }
  if (threadIdx.x == 0) {
    a.logO[k] = a.logO_tmp[k];
    a.w[k] = a.w_tmp[k];
  }
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init_walkers(int W, int N, int ncol, const double* phi, cplx_t<R>* psi, double* w, int cplx) {
  const size_t total = (size_t)W * N * ncol;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t k = i % ((size_t)N * ncol);
    psi[i] = from_d2<R>(cplx ? mk(phi[2 * k], phi[2 * k + 1]) : mk(phi[k], 0.0));
    if (i < (size_t)W) w[i] = 1.0;
  }
}

template <typename R>
__global__ void k_convert(size_t n, const double* in, R* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (R)in[i];
}

// sum over gamma of the batched products L^g L^g: out[pq] = sum_g in[g][pq] (fixed order)
__global__ void k_sum_batches(int nb, size_t len, const double* in, double* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += in[(size_t)b * len + i];
    out[i] = s;
  }
}

}  // namespace afq

namespace afq {

// ============================================================================
// Fused propagation for the fp32 forms, one CTA per walker, everything staged
// in shared memory:  t = E_h psi;  acc = t;  t <- VHS t / k, acc += t  (k = 1..p);
// psi = E_h acc.  VHS and E_h are symmetric, so row q of each is also column q.
// Thread tile: 4 rows x 2 columns of the N x ncol block.
// ============================================================================
struct PropArgs {
  int N, ncol, order, ldv, ldc;
  const float* eh;        // [N][N]
  const void* vhs;        // planar [W][2][N*N] or interleaved complex [W][N*N]
  int planar;
  float2* psi;            // [W][N][ncol]
  const double* w;
  int W;
  int* status;
};

__host__ __device__ inline size_t prop_smem_floats(int N, int ncol, int* ldv_out, int* ldc_out) {
  // V rows padded to a multiple of 4 (float4 loads; the last float4 of an 8-row tile may read 4
  // floats past a row, which stay inside the next shared-memory array and feed rows >= N only)
  const int ldv = (N + 3) / 4 * 4;
  const int ldc = (ncol + 3) / 4 * 4;   // columns padded for 4-column register tiles
  if (ldv_out) *ldv_out = ldv;
  if (ldc_out) *ldc_out = ldc;
  return (size_t)3 * N * ldv + (size_t)6 * N * ldc + 8;
}

// Out = scale * V T (V real if REALV); acc_mode 0: none, 1: Acc = Out, 2: Acc += Out.
// Thread tile: TM rows (TM/4 float4 of V per part) x TC columns (TC/2 float2 of T per part).
template <bool REALV, int TM, int TC>
__device__ __forceinline__ void prop_product(int N, int ldv, int ldc, int ncol, const float* Vr, const float* Vi,
                                             const float* Tr, const float* Ti, float* Or, float* Oi, float* Ar,
                                             float* Ai, float scale, int acc_mode) {
  const int ptiles = (N + TM - 1) / TM, ctiles = ldc / TC;
  for (int tile = threadIdx.x; tile < ptiles * ctiles; tile += blockDim.x) {
    const int p0 = TM * (tile / ctiles), c0 = TC * (tile % ctiles);
    float accr[TM][TC], acci[TM][TC];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) accr[i][j] = acci[i][j] = 0.f;
    for (int q = 0; q < N; ++q) {
      float ar[TM], ai[TM], br[TC], bi[TC];
#pragma unroll
      for (int i = 0; i < TM; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(Vr + (size_t)q * ldv + p0 + i);
        ar[i] = v.x; ar[i + 1] = v.y; ar[i + 2] = v.z; ar[i + 3] = v.w;
        if (!REALV) {
          const float4 u = *reinterpret_cast<const float4*>(Vi + (size_t)q * ldv + p0 + i);
          ai[i] = u.x; ai[i + 1] = u.y; ai[i + 2] = u.z; ai[i + 3] = u.w;
        }
      }
#pragma unroll
      for (int j = 0; j < TC; j += 2) {
        const float2 t = *reinterpret_cast<const float2*>(Tr + (size_t)q * ldc + c0 + j);
        const float2 u = *reinterpret_cast<const float2*>(Ti + (size_t)q * ldc + c0 + j);
        br[j] = t.x; br[j + 1] = t.y; bi[j] = u.x; bi[j + 1] = u.y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) {
          accr[i][j] = fmaf(ar[i], br[j], accr[i][j]);
          acci[i][j] = fmaf(ar[i], bi[j], acci[i][j]);
          if (!REALV) {
            accr[i][j] = fmaf(-ai[i], bi[j], accr[i][j]);
            acci[i][j] = fmaf(ai[i], br[j], acci[i][j]);
          }
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int p = p0 + i;
      if (p >= N) continue;
#pragma unroll
      for (int j = 0; j < TC; ++j) {
        const int c = c0 + j;
        if (c >= ncol) continue;
        const float orv = scale * accr[i][j], oiv = scale * acci[i][j];
        const size_t o = (size_t)p * ldc + c;
        if (Or) { Or[o] = orv; Oi[o] = oiv; }
        if (acc_mode == 1) { Ar[o] = orv; Ai[o] = oiv; }
        else if (acc_mode == 2) { Ar[o] += orv; Ai[o] += oiv; }
      }
    }
  }
}

__device__ __forceinline__ uint32_t smem_addr_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bulk global->shared copy completing on an mbarrier (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr_u32(dst)),
               "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_addr_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr_u32(bar);
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (it == 0) t0 = t;
    else if (t - t0 > 2000000000ull) return false;
  }
}

// Persistent: each CTA loads E_h once and loops over walkers; with planar VHS and N % 4 == 0
// the walker's VHS (re and im planes) arrives by two bulk copies, the next walker's copy
// being issued as soon as the Taylor terms of the current one are done.
template <int TM, int TC>
__global__ void __launch_bounds__(512) k_propagate_smem(PropArgs a) {
  extern __shared__ __align__(16) float sm_pr[];
  const int N = a.N, ldv = a.ldv, ldc = a.ldc;
  const size_t NN = (size_t)N * N;
  float* Vr = sm_pr;
  float* Vi = Vr + (size_t)N * ldv;
  float* E = Vi + (size_t)N * ldv;
  float* T0r = E + (size_t)N * ldv;
  float* T0i = T0r + (size_t)N * ldc;
  float* T1r = T0i + (size_t)N * ldc;
  float* T1i = T1r + (size_t)N * ldc;
  float* Ar = T1i + (size_t)N * ldc;
  float* Ai = Ar + (size_t)N * ldc;
  __shared__ __align__(8) uint64_t vbar;
  __shared__ int go_s;
  const bool bulk = a.planar && ldv == N && ((NN * 4) % 16 == 0);   // rows are contiguous in smem
  for (size_t i = threadIdx.x; i < (size_t)N * ldv; i += blockDim.x) {
    const int q = (int)(i / ldv), p = (int)(i % ldv);
    E[i] = p < N ? a.eh[(size_t)q * N + p] : 0.f;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr_u32(&vbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto next_live = [&](int from) {
    for (int k = from; k < a.W; k += gridDim.x)
      if (a.w[k] != 0.0) return k;
    return a.W;
  };
  auto issue = [&](int wk) {   // thread 0 only
    const float* v = reinterpret_cast<const float*>(a.vhs) + (size_t)wk * 2 * NN;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr_u32(&vbar)),
                 "r"((uint32_t)(2 * NN * 4))
                 : "memory");
    bulk_g2s(Vr, v, (uint32_t)(NN * 4), &vbar);
    bulk_g2s(Vi, v + NN, (uint32_t)(NN * 4), &vbar);
  };
  uint32_t phase = 0;
  int wk = next_live(blockIdx.x);
  if (bulk && threadIdx.x == 0 && wk < a.W) issue(wk);
  while (wk < a.W) {
    if (bulk) {
      if (threadIdx.x == 0) {
        go_s = mbar_wait_bounded(&vbar, phase) ? 1 : 0;
        if (!go_s) atomicOr(a.status, kStatusTimeout);
      }
    } else {
      for (size_t i = threadIdx.x; i < (size_t)N * ldv; i += blockDim.x) {
        const int q = (int)(i / ldv), p = (int)(i % ldv);
        float vr = 0.f, vi = 0.f;
        if (p < N) {
          const size_t o = (size_t)q * N + p;
          if (a.planar) {
            const float* v = reinterpret_cast<const float*>(a.vhs) + (size_t)wk * 2 * NN;
            vr = v[o];
            vi = v[NN + o];
          } else {
            const float2 v = reinterpret_cast<const float2*>(a.vhs)[(size_t)wk * NN + o];
            vr = v.x;
            vi = v.y;
          }
        }
        Vr[i] = vr;
        Vi[i] = vi;
      }
      if (threadIdx.x == 0) go_s = 1;
    }
    for (int i = threadIdx.x; i < N * ldc; i += blockDim.x) {
      const int p = i / ldc, c = i % ldc;
      float2 v = make_float2(0.f, 0.f);
      if (c < a.ncol) v = a.psi[((size_t)wk * N + p) * a.ncol + c];
      T0r[i] = v.x;
      T0i[i] = v.y;
      T1r[i] = 0.f;
      T1i[i] = 0.f;
      Ar[i] = 0.f;
      Ai[i] = 0.f;
    }
    __syncthreads();
    if (!go_s) break;
    phase ^= 1u;
    prop_product<true, TM, TC>(N, ldv, ldc, a.ncol, E, nullptr, T0r, T0i, T1r, T1i, Ar, Ai, 1.f, 1);
    __syncthreads();
    float *tin_r = T1r, *tin_i = T1i, *tout_r = T0r, *tout_i = T0i;
    for (int k = 1; k <= a.order; ++k) {
      prop_product<false, TM, TC>(N, ldv, ldc, a.ncol, Vr, Vi, tin_r, tin_i, k < a.order ? tout_r : nullptr,
                          k < a.order ? tout_i : nullptr, Ar, Ai, 1.f / (float)k, 2);
      __syncthreads();
      float* t = tin_r; tin_r = tout_r; tout_r = t;
      t = tin_i; tin_i = tout_i; tout_i = t;
    }
    const int nxt = next_live(wk + gridDim.x);
    if (bulk && threadIdx.x == 0 && nxt < a.W) issue(nxt);   // VHS buffer is free from here on
    prop_product<true, TM, TC>(N, ldv, ldc, a.ncol, E, nullptr, Ar, Ai, tout_r, tout_i, nullptr, nullptr, 1.f, 0);
    __syncthreads();
    for (int i = threadIdx.x; i < N * a.ncol; i += blockDim.x) {
      const int p = i / a.ncol, c = i % a.ncol;
      a.psi[((size_t)wk * N + p) * a.ncol + c] =
          make_float2(tout_r[(size_t)p * ldc + c], tout_i[(size_t)p * ldc + c]);
    }
    __syncthreads();
    wk = nxt;
  }
  if (threadIdx.x == 0 && bulk && !go_s) {   // a copy may still be in flight after a timeout: let it land
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do { asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); } while (t - t0 < 2000000ull);
  }
}

// ============================================================================
// Overlap, Theta and weight update (Eqs. 13-16), one CTA per walker.  Per spin
// block: A = Phi^T psi is formed at the walkers' precision R (an R accumulator;
// binary64 in the FP64 form) and stored in binary64; LU with partial pivoting
// P A = L U in binary64 gives log det A = sum log U_kk (+ i pi for an odd
// number of row swaps); Theta = psi A^-1 = psi U^-1 L^-1 P is applied row by
// row by forward (U) and backward (unit L) substitution at the walkers'
// precision with the factors rounded once to R.  mode 0: log O only;
// mode 1: also the weight update; mode 2: Theta and log det, no weights.
// ============================================================================
// STAGE: psi rows, Phi and the substitution vectors live in shared memory (Y); otherwise the
// vectors live in Theta^T itself (row perm[k] holds y_k throughout, so no final permutation).
// Shared memory: A [n][lda] binary64 | pivots, 1 / pivots [n] binary64 | perm [n] | F [n][n] R |
// (STAGE) Y [N][ldy] R complex | Phi [N][n] R.
template <typename R>
__host__ __device__ inline size_t overlap_lu_smem(int N, int nmax, bool stage, bool cphi = false) {
  const int lda = nmax + 1, ldy = nmax | 1;
  const size_t fixed = (size_t)nmax * lda * 16 + (size_t)nmax * 32 + ((size_t)nmax * 4 + 15) / 16 * 16 +
                       (size_t)nmax * nmax * 2 * sizeof(R);
  return fixed + (stage ? (size_t)N * ldy * 2 * sizeof(R) + (size_t)N * nmax * sizeof(R) * (cphi ? 2 : 1) : 0) + 16;
}

// Complex product with the larger component renormalised to [1, 2) (exact power of two); e
// accumulates the exponent removed.
__device__ __forceinline__ double2 cmul_renorm(double2 a, double2 b, int* e) {
  double2 q = mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
  const long long big = __double_as_longlong(fmax(fabs(q.x), fabs(q.y)));
  const int ex = (int)((big >> 52) & 0x7ff) - 1023;
  if (ex > -1000 && ex < 1000) {
    const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
    q = mk(q.x * sc, q.y * sc);
    *e += ex;
  }
  return q;
}

// One element (4, 8 or 16 bytes, aligned to its size) from global to shared memory without a
// register round trip (cp.async); cp_async_wait_all waits for the thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// acc -= a b (complex)
template <typename R>
__device__ __forceinline__ void csub(cplx_t<R>& acc, const cplx_t<R>& a, const cplx_t<R>& b) {
  acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
}

// Theta rows of one spin block from the staged psi rows: thread p solves row p in place in
// Y[p] (z U = psi_p forward, then y L = z with unit lower L backward), four columns at a time
// (the block's earlier entries are subtracted by a compact loop with four independent
// accumulators, then the 4 x 4 triangle), and writes Theta^T[perm[i]][p] = y_i and its split-bf16
// copy.  Loops stay rolled: the kernel runs between large tensor-core kernels, so straight-line
// code would be fetched cold from L2 on every launch.
template <typename R>
__device__ __forceinline__ void subst_rows_blocked(cplx_t<R>* Y, int ldy, const cplx_t<R>* F, const int* perm, int n,
                                                   int N, cplx_t<R>* thw, __nv_bfloat16* thb, int kst, int nseg, int w,
                                                   int kst0 = 0) {
  using R2 = cplx_t<R>;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    R2* y = Y + (size_t)p * ldy;
    for (int j0 = 0; j0 < n; j0 += 4) {   // z U = psi_p
      const int nb = min(4, n - j0);
      R2 acc[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[t].x = R(0);
        acc[t].y = R(0);
        if (t < nb) acc[t] = y[j0 + t];
      }
      for (int k = 0; k < j0; ++k) {
        const R2 z = y[k];
        const R2* f = F + k * n + j0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nb) csub<R>(acc[t], z, f[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t < nb) {
          const R2 d = F[(j0 + t) * n + j0 + t];   // 1 / U_jj
          const R2 z = acc[t];
          acc[t].x = z.x * d.x - z.y * d.y;
          acc[t].y = z.x * d.y + z.y * d.x;
#pragma unroll
          for (int t2 = t + 1; t2 < 4; ++t2)
            if (t2 < nb) csub<R>(acc[t2], acc[t], F[(j0 + t) * n + j0 + t2]);
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nb) y[j0 + t] = acc[t];
    }
    for (int j0 = ((n - 1) / 4) * 4; j0 >= 0; j0 -= 4) {   // y L = z, blocks in descending order
      const int nb = min(4, n - j0);
      R2 acc[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[t].x = R(0);
        acc[t].y = R(0);
        if (t < nb) acc[t] = y[j0 + t];
      }
      for (int k = j0 + nb; k < n; ++k) {
        const R2 yk = y[k];
        const R2* f = F + k * n + j0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (t < nb) csub<R>(acc[t], yk, f[t]);
      }
#pragma unroll
      for (int t = 3; t >= 1; --t)
        if (t < nb) {
#pragma unroll
          for (int t2 = 0; t2 < t; ++t2) csub<R>(acc[t2], acc[t], F[(j0 + t) * n + j0 + t2]);
        }
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nb) y[j0 + t] = acc[t];
    }
    for (int i = 0; i < n; ++i) {   // Theta^T[perm[i]][p] = y_i (consecutive p: coalesced)
      const R2 v = y[i];
      const int b = perm[i];
      thw[(size_t)b * N + p] = v;
      if (thb) store_theta_bf16(thb, kst, nseg, n, w, b, p, v, kst0);
    }
  }
}

// 5 CTAs per SM: the W = 640 walkers of the benchmark shape run in one wave on 148 SMs.
template <typename R, bool STAGE, bool CPHI>
__device__ __forceinline__ void overlap_walker(const OverlapArgs<R> a, const int w) {
  using R2 = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char sm_lu[];
  __shared__ int piv_s, sing_s, swaps_s, exp_s;
  __shared__ double2 inv_s, prod_s;
  __shared__ double ld_im_s;   // imaginary part of log det (its atan2 runs in a second warp)
  const int tid = threadIdx.x, N = a.N;
  if (tid == 32) ld_im_s = 0.0;
  if (a.mode == 1 && a.step != nullptr && w == 0 && tid == 0) *a.step += 1ull;
  if (a.mode == 1 && a.w[w] == 0.0) return;
  const int nmax = max(a.nb[0], a.nblk > 1 ? a.nb[1] : 0);
  const int lda = nmax + 1, ldy = nmax | 1;
  double2* A = reinterpret_cast<double2*>(sm_lu);           // [n][lda] binary64, becomes L\U
  double2* pivv = A + (size_t)nmax * lda;                   // pivots U_kk
  double2* dinv = pivv + nmax;                              // 1 / U_kk
  int* perm = reinterpret_cast<int*>(dinv + nmax);
  R2* F = reinterpret_cast<R2*>(reinterpret_cast<unsigned char*>(perm) + ((size_t)nmax * 4 + 15) / 16 * 16);
  R2* Y = F + (size_t)nmax * nmax;                          // [N][ldy]: psi rows, then Theta rows
  R* PH = reinterpret_cast<R*>(Y + (size_t)N * ldy);        // [N][n] Phi block
  double ld_re = 0.0;
  bool singular = false;
  for (int s = 0; s < a.nblk; ++s) {
    const int c0 = a.c0[s], n = a.nb[s];
    if (n == 0) continue;
    __syncthreads();
    const R2* psw = a.psi + (size_t)w * N * a.ncol + c0;
    if (STAGE) {   // asynchronous copies into shared memory, all of the block's in flight at once
      for (int idx = tid; idx < N * n; idx += blockDim.x) {
        const int p = idx / n, j = idx - p * n;
        cp_async_elem<sizeof(R2)>(&Y[(size_t)p * ldy + j], &psw[(size_t)p * a.ncol + j]);
        if (CPHI) cp_async_elem<sizeof(R2)>(&reinterpret_cast<R2*>(PH)[idx], &a.phi_c[(size_t)p * a.ncol + c0 + j]);
        else cp_async_elem<sizeof(R)>(&PH[idx], &a.phi_r[(size_t)p * a.ncol + c0 + j]);
      }
      cp_async_wait_all();
    }
    if (tid < n) perm[tid] = tid;
    if (tid == 0) { sing_s = 0; swaps_s = 0; }
    __syncthreads();
    // A = Phi^T psi (Phi^+ psi for a complex trial): 2 x 2 register tiles
    const int nt = (n + 1) / 2;
    for (int t = tid; t < nt * nt; t += blockDim.x) {
      const int i0 = 2 * (t / nt), j0 = 2 * (t % nt);
      const bool i1ok = i0 + 1 < n, j1ok = j0 + 1 < n;
      R acc[2][2][2] = {};
      if (CPHI) {
        const R2* PHc = reinterpret_cast<const R2*>(PH);
        for (int p = 0; p < N; ++p) {
          R2 f[2], g[2];
          f[0] = STAGE ? PHc[p * n + i0] : a.phi_c[(size_t)p * a.ncol + c0 + i0];
          f[1] = i1ok ? (STAGE ? PHc[p * n + i0 + 1] : a.phi_c[(size_t)p * a.ncol + c0 + i0 + 1]) : R2{R(0), R(0)};
          g[0] = STAGE ? Y[(size_t)p * ldy + j0] : psw[(size_t)p * a.ncol + j0];
          g[1] = j1ok ? (STAGE ? Y[(size_t)p * ldy + j0 + 1] : psw[(size_t)p * a.ncol + j0 + 1]) : g[0];
#pragma unroll
          for (int di = 0; di < 2; ++di)
#pragma unroll
            for (int dj = 0; dj < 2; ++dj) {   // conj(f) g
              acc[di][dj][0] += f[di].x * g[dj].x + f[di].y * g[dj].y;
              acc[di][dj][1] += f[di].x * g[dj].y - f[di].y * g[dj].x;
            }
        }
      } else {
        auto fetch = [&](int p, R& ph0, R& ph1, R2& ps0, R2& ps1) {
          if (STAGE) {
            ph0 = PH[p * n + i0];
            ph1 = i1ok ? PH[p * n + i0 + 1] : R(0);
            ps0 = Y[(size_t)p * ldy + j0];
            ps1 = j1ok ? Y[(size_t)p * ldy + j0 + 1] : ps0;
          } else {
            ph0 = a.phi_r[(size_t)p * a.ncol + c0 + i0];
            ph1 = i1ok ? a.phi_r[(size_t)p * a.ncol + c0 + i0 + 1] : R(0);
            ps0 = psw[(size_t)p * a.ncol + j0];
            ps1 = j1ok ? psw[(size_t)p * a.ncol + j0 + 1] : ps0;
          }
        };
        auto mac = [&](R ph0, R ph1, R2 ps0, R2 ps1) {
          acc[0][0][0] += ph0 * ps0.x; acc[0][0][1] += ph0 * ps0.y;
          acc[0][1][0] += ph0 * ps1.x; acc[0][1][1] += ph0 * ps1.y;
          acc[1][0][0] += ph1 * ps0.x; acc[1][0][1] += ph1 * ps0.y;
          acc[1][1][0] += ph1 * ps1.x; acc[1][1][1] += ph1 * ps1.y;
        };
        int p = 0;
        for (; p + 4 <= N; p += 4) {   // four rows of loads in flight, then their products in order
          R f0[4], f1[4];
          R2 g0[4], g1[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) fetch(p + u, f0[u], f1[u], g0[u], g1[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u) mac(f0[u], f1[u], g0[u], g1[u]);
        }
        for (; p < N; ++p) {
          R f0, f1;
          R2 g0, g1;
          fetch(p, f0, f1, g0, g1);
          mac(f0, f1, g0, g1);
        }
      }
      for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
          if ((di == 0 || i1ok) && (dj == 0 || j1ok))
            A[(i0 + di) * lda + j0 + dj] = mk((double)acc[di][dj][0], (double)acc[di][dj][1]);
    }
    __syncthreads();
    if (n <= 32) {
      // One warp takes the pivot step: every lane holds its row's column-k entry and its
      // reciprocal (formed while the pivot is being chosen), then swaps the rows and writes the
      // multipliers; one barrier before and one after the trailing update.
      const int lane = tid & 31;
      for (int k = 0; k < n; ++k) {
        if (tid < 32) {
          const bool own = lane >= k && lane < n;
          const double2 v = own ? A[lane * lda + k] : mk(0.0, 0.0);
          // largest |re| + |im| (non-negative doubles order like their bit patterns), lowest row on ties
          long long best = own ? __double_as_longlong(fabs(v.x) + fabs(v.y)) : -1ll;
          int bi = own ? lane : 64;
          // 1 / v = conj(v) / |v|^2 (lanes without a row divide 1 by 1, not by 0)
          const double2 vr = own ? v : mk(1.0, 0.0);
          const double r = 1.0 / fma(vr.x, vr.x, vr.y * vr.y);
          double2 inv = mk(vr.x * r, -vr.y * r);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          // zero, NaN or infinity: the sum's bit pattern is 0 or has every exponent bit set
          if (best <= 0 || best >= 0x7ff0000000000000LL) {
            if (lane == 0) sing_s = 1;
          } else {
            inv = mk(__shfl_sync(0xffffffffu, inv.x, bi), __shfl_sync(0xffffffffu, inv.y, bi));
            const double2 pk = mk(__shfl_sync(0xffffffffu, v.x, bi), __shfl_sync(0xffffffffu, v.y, bi));
            const double2 vk = mk(__shfl_sync(0xffffffffu, v.x, k), __shfl_sync(0xffffffffu, v.y, k));
            if (bi != k && lane < n && lane != k) {   // rows k and bi trade places (column k below)
              const double2 t = A[k * lda + lane];
              A[k * lda + lane] = A[bi * lda + lane];
              A[bi * lda + lane] = t;
            }
            if (lane == k) A[k * lda + k] = pk;
            if (lane > k && lane < n) {   // multiplier of the row now at `lane` (old row k if lane == bi)
              const double2 src = lane == bi ? vk : v;
              A[lane * lda + k] = mk(fma(src.x, inv.x, -src.y * inv.y), fma(src.x, inv.y, src.y * inv.x));
            }
            if (lane == 0) {
              dinv[k] = inv;
              pivv[k] = pk;
              if (bi != k) {
                swaps_s ^= 1;
                const int t = perm[k];
                perm[k] = perm[bi];
                perm[bi] = t;
              }
            }
          }
        }
        __syncthreads();
        if (sing_s) break;
        const int rem = n - k - 1;
        // (i, j) of a flat index: the single-precision quotient is exact here (idx < 1024, rem <= 31)
        const float frem = __frcp_rn((float)max(rem, 1));
        for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
          const int io = (int)(((float)idx + 0.5f) * frem);
          const int i = k + 1 + io, j = k + 1 + idx - io * rem;
          const double2 l = A[i * lda + k], u = A[k * lda + j];
          double2 v = A[i * lda + j];
          v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
          v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
          A[i * lda + j] = v;
        }
        __syncthreads();
      }
    } else
    for (int k = 0; k < n; ++k) {
      if (tid < 32) {   // pivot: largest |re| + |im| in column k, lowest row on ties
        // non-negative doubles order like their bit patterns: compare as integers
        long long best = -1;
        int bi = k;
        for (int i = k + tid; i < n; i += 32) {
          const double2 v = A[i * lda + k];
          const long long m = __double_as_longlong(fabs(v.x) + fabs(v.y));
          if (m > best) { best = m; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          piv_s = bi;
          // zero, NaN or infinity: the sum's bit pattern is 0 or has every exponent bit set
          if (best <= 0 || best >= 0x7ff0000000000000LL) sing_s = 1;
          if (!sing_s) {
            const double2 pk = A[bi * lda + k];
            const double r = 1.0 / fma(pk.x, pk.x, pk.y * pk.y);   // 1 / pk = conj(pk) / |pk|^2
            const double2 inv = mk(pk.x * r, -pk.y * r);
            inv_s = inv;
            dinv[k] = inv;
            pivv[k] = pk;
            if (bi != k) {
              swaps_s ^= 1;
              const int t = perm[k];
              perm[k] = perm[bi];
              perm[bi] = t;
            }
          }
        }
      }
      __syncthreads();
      if (sing_s) break;
      const int pv = piv_s;
      if (pv != k)
        for (int j = tid; j < n; j += blockDim.x) {
          const double2 t = A[k * lda + j];
          A[k * lda + j] = A[pv * lda + j];
          A[pv * lda + j] = t;
        }
      __syncthreads();
      const double2 inv = inv_s;
      for (int i = k + 1 + tid; i < n; i += blockDim.x) {
        const double2 v = A[i * lda + k];
        A[i * lda + k] = mk(fma(v.x, inv.x, -v.y * inv.y), fma(v.x, inv.y, v.y * inv.x));
      }
      __syncthreads();
      const int rem = n - k - 1;
      for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
        const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
        const double2 l = A[i * lda + k], u = A[k * lda + j];
        double2 v = A[i * lda + j];
        v.x = fma(-l.x, u.x, fma(l.y, u.y, v.x));
        v.y = fma(-l.x, u.y, fma(-l.y, u.x, v.y));
        A[i * lda + j] = v;
      }
      __syncthreads();
    }
    if (sing_s) {
      singular = true;
      for (int idx = tid; idx < n * N; idx += blockDim.x) {
        const int b = idx / N, p = idx % N;
        const R2 z = from_d2<R>(mk(0.0, 0.0));
        a.thetaT[((size_t)w * a.ncol + c0 + b) * N + p] = z;
        if (a.thb[s]) store_theta_bf16(a.thb[s], a.kst, a.nseg, n, w, b, p, z, a.kst0);
      }
      continue;
    }
    if (tid < 32) {   // det U = product of the pivots: butterfly with exact renormalisation
      double2 q = tid < n ? pivv[tid] : mk(1.0, 0.0);
      int e = 0;
      for (int i = tid + 32; i < n; i += 32) q = cmul_renorm(q, pivv[i], &e);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double2 oq = mk(__shfl_xor_sync(0xffffffffu, q.x, o), __shfl_xor_sync(0xffffffffu, q.y, o));
        const int oe = __shfl_xor_sync(0xffffffffu, e, o);
        q = cmul_renorm(q, oq, &e);
        e += oe;
      }
      if (tid == 0) { prod_s = q; exp_s = e; }
    }
    // one rounding of each factor entry to R, by the warps other than the determinant's
    for (int idx = tid - 32; idx < n * n; idx += (int)blockDim.x - 32) {
      if (idx < 0) break;
      const int i = idx / n, j = idx % n;
      F[idx] = from_d2<R>(i == j ? dinv[i] : A[i * lda + j]);
    }
    __syncthreads();
    R2* thw = a.thetaT + ((size_t)w * a.ncol + c0) * N;
    if (STAGE) {
      subst_rows_blocked<R>(Y, ldy, F, perm, n, N, thw, a.thb[s], a.kst, a.nseg, w, a.kst0);
    } else {   // row perm[k] of Theta^T holds y_k of every psi row throughout (no final permutation)
      for (int p = tid; p < N; p += blockDim.x) {
        auto at = [&](int k) -> R2& { return thw[(size_t)perm[k] * N + p]; };
        for (int j = 0; j < n; ++j) at(j) = psw[(size_t)p * a.ncol + j];
        for (int j = 0; j < n; ++j) {   // z U = psi_p (two independent partial sums)
          R sr0 = at(j).x, si0 = at(j).y, sr1 = R(0), si1 = R(0);
          int k = 0;
          for (; k + 1 < j; k += 2) {
            const R2 z0 = at(k), u0 = F[k * n + j], z1 = at(k + 1), u1 = F[(k + 1) * n + j];
            sr0 -= z0.x * u0.x - z0.y * u0.y;
            si0 -= z0.x * u0.y + z0.y * u0.x;
            sr1 -= z1.x * u1.x - z1.y * u1.y;
            si1 -= z1.x * u1.y + z1.y * u1.x;
          }
          if (k < j) {
            const R2 z0 = at(k), u0 = F[k * n + j];
            sr0 -= z0.x * u0.x - z0.y * u0.y;
            si0 -= z0.x * u0.y + z0.y * u0.x;
          }
          const R sr = sr0 + sr1, si = si0 + si1;
          const R2 d = F[j * n + j];
          R2 o;
          o.x = sr * d.x - si * d.y;
          o.y = sr * d.y + si * d.x;
          at(j) = o;
        }
        for (int j = n - 2; j >= 0; --j) {   // y L = z (unit lower L)
          R sr0 = at(j).x, si0 = at(j).y, sr1 = R(0), si1 = R(0);
          int k = j + 1;
          for (; k + 1 < n; k += 2) {
            const R2 z0 = at(k), l0 = F[k * n + j], z1 = at(k + 1), l1 = F[(k + 1) * n + j];
            sr0 -= z0.x * l0.x - z0.y * l0.y;
            si0 -= z0.x * l0.y + z0.y * l0.x;
            sr1 -= z1.x * l1.x - z1.y * l1.y;
            si1 -= z1.x * l1.y + z1.y * l1.x;
          }
          if (k < n) {
            const R2 z0 = at(k), l0 = F[k * n + j];
            sr0 -= z0.x * l0.x - z0.y * l0.y;
            si0 -= z0.x * l0.y + z0.y * l0.x;
          }
          R2 o;
          o.x = sr0 + sr1;
          o.y = si0 + si1;
          at(j) = o;
        }
      }
      __syncthreads();
      if (a.thb[s])
        for (int idx = tid; idx < n * N; idx += blockDim.x) {
          const int b = idx / N, p = idx % N;
          store_theta_bf16(a.thb[s], a.kst, a.nseg, n, w, b, p, thw[(size_t)b * N + p], a.kst0);
        }
    }
    // log det = log(prod) + exp ln 2 (+ i pi for an odd number of row swaps); the real and
    // imaginary parts in two warps
    if (tid == 0) {
      const double2 pr = prod_s;
      ld_re += 0.5 * log(fma(pr.x, pr.x, pr.y * pr.y)) + exp_s * 0.6931471805599453;   // |pr| in [1, 2 sqrt 2)
    } else if (tid == 32) {
      const double2 pr = prod_s;
      ld_im_s += atan2(pr.y, pr.x) + (swaps_s ? 3.141592653589793 : 0.0);
    }
    __syncthreads();
  }
  if (tid != 0) return;
  if (singular) {
    if (a.mode != 2) a.w[w] = 0.0;
    atomicOr(a.status, kStatusSingular);
    return;
  }
  const double2 lo_new = mk(a.smul * ld_re, wrap_angle(a.smul * ld_im_s));
  if (a.mode == 0) {
    a.logO[w] = lo_new;
  } else if (a.mode == 1) {
    const double2 lo_old = a.logO[w];
    const double2 c = a.cmf[w];
    const double2 xx = a.xxbar[w];
    const double ls_re = lo_new.x - lo_old.x + c.x;
    const double theta = lo_new.y - lo_old.y + c.y;
    const double eshift = a.etr ? exp(a.dt * (a.etr[0] - a.e_c)) : a.eshift;
    double wn;
    if (a.wph) {   // free projection: the whole ratio (O'/O) e^{c_mf}, its phase kept with the weight
      wn = a.w[w] * exp(ls_re) * eshift;
      a.wph[w] = wrap_angle(a.wph[w] + theta);
    } else {
      const double li_re = ls_re + xx.x;
      wn = a.w[w] * exp(li_re) * fmax(0.0, cos(theta)) * eshift;
    }
    if (!isfinite(wn)) {
      wn = 0.0;
      atomicOr(a.status, kStatusNonFinite);
    }
    a.w[w] = wn;
    a.logO[w] = lo_new;
  }
}
template <typename R, bool STAGE, bool CPHI = false>
__global__ void __launch_bounds__(128, 5) k_overlap_lu(OverlapArgs<R> a) {
  overlap_walker<R, STAGE, CPHI>(a, blockIdx.x);
}
// Large N (psi and Phi read in place, few walkers per SM): one wide CTA per walker.
template <typename R, bool CPHI = false>
__global__ void __launch_bounds__(512, 1) k_overlap_lu_wide(OverlapArgs<R> a) {
  overlap_walker<R, false, CPHI>(a, blockIdx.x);
}
// Several systems in one launch, one block per walker (block b is walker b + base of the list);
// stage[s]: system s stages psi and Theta in shared memory (the launch's shared memory covers the
// largest need among its systems).
template <typename R, bool CPHI = false>
__global__ void __launch_bounds__(128, 5) k_overlap_group(const OverlapArgs<R>* __restrict__ args,
                                                          const int* __restrict__ first,
                                                          const int* __restrict__ stage, int nsys, int base) {
  const int b = blockIdx.x + base, s = group_of(first, nsys, b);
  if (stage[s]) overlap_walker<R, true, CPHI>(args[s], b - first[s]);
  else overlap_walker<R, false, CPHI>(args[s], b - first[s]);
}

// ============================================================================
// Cholesky QR, one CTA per walker: G = psi^H psi accumulated in binary64
// (Hermitian; products of walker-precision entries are exact in binary64; for
// binary32 walkers the sums are compensated binary32 dot products (Dot2), as
// accurate as binary64 accumulation here and several times cheaper on this
// GPU, then rounded once to binary64),
// G = R^H R in binary64 with R upper triangular and diag R > 0, then
// psi <- psi R^-1 (= Q with diag R > 0, the unique thin QR) by forward
// substitution on each row at the walkers' precision with R rounded once, and
// log O -= smul sum log R_ii.  stage_psi: the block's columns are staged in
// shared memory as binary64 rows P[j][p] with an odd row pitch.
// In the factorisation one warp forms R_kk, 1 / R_kk and row k, and the whole
// CTA takes the trailing update, walking the packed upper triangle in a table
// ordered by decreasing row, so the pairs of step k are its first m (m + 1) / 2
// entries (m = n - k - 1).
// Shared memory: G [nmax^2] binary64 complex | 1 / R_kk [nmax] | pair table
// [nmax (nmax + 1) / 2] (row, column bytes) | a region holding P during the
// Gram product and R at the walkers' precision afterwards.
// ============================================================================
__host__ __device__ inline int qr_pitch(int N) { return N | 1; }
__host__ __device__ inline size_t qr_off_rinv(int nmax) { return (size_t)nmax * nmax * 16; }
__host__ __device__ inline size_t qr_off_tri(int nmax) { return qr_off_rinv(nmax) + ((size_t)nmax * 8 + 15) / 16 * 16; }
__host__ __device__ inline size_t qr_off_region(int nmax) {
  return qr_off_tri(nmax) + ((size_t)nmax * (nmax + 1) + 15) / 16 * 16;
}
template <typename R>
__host__ __device__ inline size_t qr_smem_bytes(int N, int nmax, bool stage) {
  const size_t pst = stage ? (size_t)nmax * qr_pitch(N) * 16 : 0, rl = (size_t)nmax * nmax * sizeof(cplx_t<R>);
  return qr_off_region(nmax) + (pst > rl ? pst : rl);
}

template <typename R>
struct QrArgs {
  int N, ncol, nblk, c00, n0, c01, n1;
  double smul;
  cplx_t<R>* psi;
  double2* logO;
  const double* wgt;
  int* status;
  int stage_psi;
};

template <typename R>
__device__ __forceinline__ void qr_walker(const QrArgs<R> A, const int w) {
  const int N = A.N, ncol = A.ncol, nblk = A.nblk, c00 = A.c00, n0 = A.n0, c01 = A.c01, n1 = A.n1;
  const double smul = A.smul;
  cplx_t<R>* psi = A.psi;
  double2* logO = A.logO;
  const double* wgt = A.wgt;
  int* status = A.status;
  const int stage_psi = A.stage_psi;
  using R2 = cplx_t<R>;
  extern __shared__ double2 sm_cq[];
  __shared__ double logsum_s;
  __shared__ int bad_s;
  const int tid = threadIdx.x;
  if (wgt[w] == 0.0) return;
  if (tid == 0) { logsum_s = 0.0; bad_s = 0; }
  const int ldp = qr_pitch(N), nmax = max(n0, nblk > 1 ? n1 : 0);
  unsigned char* base = reinterpret_cast<unsigned char*>(sm_cq);
  double2* G = sm_cq;                                                        // [n][n], becomes R (upper)
  double* rinv = reinterpret_cast<double*>(base + qr_off_rinv(nmax));
  uchar2* tri = reinterpret_cast<uchar2*>(base + qr_off_tri(nmax));
  double2* P = reinterpret_cast<double2*>(base + qr_off_region(nmax));      // [n][ldp] during the Gram product
  R2* Rl = reinterpret_cast<R2*>(base + qr_off_region(nmax));               // R at the walkers' precision, diagonal 1 / R_kk
  for (int s = 0; s < nblk; ++s) {
    const int c0 = s == 0 ? c00 : c01, n = s == 0 ? n0 : n1;
    if (n == 0) continue;
    R2* pw = psi + (size_t)w * N * ncol + c0;
    __syncthreads();
    if (tid < n) {   // pair table: rows n - 1, n - 2, ..., each with its columns j >= i
      const int m = n - 1 - tid;
      for (int j = tid; j < n; ++j) tri[m * (m + 1) / 2 + (j - tid)] = make_uchar2((unsigned char)tid, (unsigned char)j);
    }
    constexpr bool kDot2 = std::is_same<R, float>::value;
    float2* Pf = reinterpret_cast<float2*>(P);   // binary32 staging (Dot2 Gram)
    if (stage_psi) {
      for (int idx = tid; idx < n * N; idx += blockDim.x) {
        const int p = idx / n, j = idx % n;
        if (kDot2) Pf[(size_t)j * ldp + p] = make_float2((float)pw[(size_t)p * ncol + j].x, (float)pw[(size_t)p * ncol + j].y);
        else P[(size_t)j * ldp + p] = to_d2(pw[(size_t)p * ncol + j]);
      }
    }
    __syncthreads();
    const int npk = n * (n + 1) / 2;
    for (int e = tid; e < npk; e += blockDim.x) {   // packed upper triangle
      const int i = tri[e].x, j = tri[e].y;
      double re = 0.0, im = 0.0;      // (psi^H psi)_ij = sum_p conj(psi_pi) psi_pj
      if (kDot2 && stage_psi) {
        const float2* u = Pf + (size_t)i * ldp;
        const float2* v = Pf + (size_t)j * ldp;
        dot2 sr{0.f, 0.f}, si{0.f, 0.f};
        for (int p = 0; p < N; ++p) {
          const float2 a = u[p], b = v[p];
          dot2_add(sr, a.x, b.x);
          dot2_add(sr, a.y, b.y);
          dot2_add(si, a.x, b.y);
          dot2_add(si, -a.y, b.x);
        }
        re = dot2_value(sr);
        im = dot2_value(si);
      } else if (stage_psi) {
        const double2* u = P + (size_t)i * ldp;
        const double2* v = P + (size_t)j * ldp;
        for (int p = 0; p < N; ++p) {   // four fused multiply-adds per term (no separate products)
          re = fma(u[p].x, v[p].x, re);
          re = fma(u[p].y, v[p].y, re);
          im = fma(u[p].x, v[p].y, im);
          im = fma(-u[p].y, v[p].x, im);
        }
      } else if (kDot2) {   // binary32 walkers read in place (large N)
        dot2 sr{0.f, 0.f}, si{0.f, 0.f};
        for (int p = 0; p < N; ++p) {
          const R2 a = pw[(size_t)p * ncol + i], b = pw[(size_t)p * ncol + j];
          dot2_add(sr, (float)a.x, (float)b.x);
          dot2_add(sr, (float)a.y, (float)b.y);
          dot2_add(si, (float)a.x, (float)b.y);
          dot2_add(si, -(float)a.y, (float)b.x);
        }
        re = dot2_value(sr);
        im = dot2_value(si);
      } else {
        for (int p = 0; p < N; ++p) {
          const double2 u = to_d2(pw[(size_t)p * ncol + i]);
          const double2 v = to_d2(pw[(size_t)p * ncol + j]);
          re = fma(u.x, v.x, re);
          re = fma(u.y, v.y, re);
          im = fma(u.x, v.y, im);
          im = fma(-u.y, v.x, im);
        }
      }
      G[i * n + j] = mk(re, im);
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle: G_kk -> R_kk and row k -> R_kj in one warp,
    // the trailing update G_ij -= conj(R_ki) R_kj (k < i <= j) by the whole CTA.  The one-warp
    // part runs in warp (blockIdx.x / 148) % 4: CTAs resident on one SM are usually 148 blocks
    // apart, so their serial binary64 chains land on different sub-partitions.
    {
      const int sw = (blockIdx.x / 148) % 4, lane = tid & 31;
      for (int k = 0; k < n; ++k) {
        if ((tid >> 5) == sw) {
          const double d = G[k * n + k].x;
          __syncwarp();   // every lane has read G_kk before lane 0 overwrites it
          // 1 / R_kk from one reciprocal square root and R_kk = G_kk / R_kk (no division)
          const double dd = fmax(d, 1e-300), ri = rsqrt(dd), r = dd * ri;
          for (int j = k + 1 + lane; j < n; j += 32) G[k * n + j] = cscale(G[k * n + j], ri);
          if (lane == 0) {
            if (!(d > 0.0) || !isfinite(d)) bad_s = 1;
            G[k * n + k] = mk(r, 0.0);
            rinv[k] = ri;
          }
        }
        __syncthreads();
        const int m = n - k - 1, tot = m * (m + 1) / 2;
        for (int e = tid; e < tot; e += blockDim.x) {
          const int i = tri[e].x, j = tri[e].y;
          const double2 rki = G[k * n + i], rkj = G[k * n + j];
          double2 g = G[i * n + j];
          g.x = fma(-rki.x, rkj.x, fma(-rki.y, rkj.y, g.x));
          g.y = fma(-rki.x, rkj.y, fma(rki.y, rkj.x, g.y));
          G[i * n + j] = g;
        }
        __syncthreads();
      }
      if (tid < 32) {
        double ls = 0.0;   // sum_k log R_kk, one lane per diagonal entry
        for (int k = tid; k < n; k += 32) ls += log(G[k * n + k].x);
        ls = warp_sum(ls);
        if (tid == 0) logsum_s += ls;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += blockDim.x) {   // one rounding of each entry of R to R (P is dead)
      const int i = idx / n, j = idx % n;
      Rl[idx] = from_d2<R>(i == j ? mk(rinv[i], 0.0) : (j > i ? G[idx] : mk(0.0, 0.0)));
    }
    __syncthreads();
    // row p of Q: x R = psi_p, x_j = (psi_pj - sum_{k<j} x_k R_kj) / R_jj, in place on the row
    for (int p = tid; p < N; p += blockDim.x) {
      R2* row = pw + (size_t)p * ncol;
      for (int j = 0; j < n; ++j) {
        R sr = row[j].x, si = row[j].y;
        for (int k = 0; k < j; ++k) {
          const R2 z = row[k], r = Rl[k * n + j];
          sr -= z.x * r.x - z.y * r.y;
          si -= z.x * r.y + z.y * r.x;
        }
        const R d = Rl[j * n + j].x;
        R2 o;
        o.x = sr * d;
        o.y = si * d;
        row[j] = o;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (bad_s) atomicOr(status, kStatusSingular);
    logO[w].x -= smul * logsum_s;
  }
}
template <typename R>
__global__ void __launch_bounds__(256) k_qr_chol(QrArgs<R> a) {
  qr_walker<R>(a, blockIdx.x);
}
// Large N (psi read in place, few walkers per SM): one wide CTA per walker.
template <typename R>
__global__ void __launch_bounds__(1024, 1) k_qr_chol_wide(QrArgs<R> a) {
  qr_walker<R>(a, blockIdx.x);
}
template <typename R>
__global__ void __launch_bounds__(256) k_qr_group(const QrArgs<R>* __restrict__ args, const int* __restrict__ first,
                                                  int nsys, int base) {
  const int b = blockIdx.x + base, s = group_of(first, nsys, b);
  qr_walker<R>(args[s], b - first[s]);
}

}  // namespace afq
