// CUDA-core kernels of the AFQMC step, templated on the real type R (double for
// the FP64 form, float for the reduced forms).  Overlap inverses and
// log-determinants, weights, QR and all energy reductions are binary64 in both.
#pragma once

#include "common.cuh"

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
};

template <typename R, bool CA, bool CB>
__global__ void __launch_bounds__(256) k_gemm(GemmDesc g) {
  constexpr int BM = 64, BN = 64, BK = 16;
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
  R acc_re[4][4], acc_im[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc_re[i][j] = acc_im[i][j] = R(0);
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
      R ar[4], ai[4], br[4], bi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { ar[i] = As_re[kk][ty + 16 * i]; ai[i] = CA ? As_im[kk][ty + 16 * i] : R(0); }
#pragma unroll
      for (int j = 0; j < 4; ++j) { br[j] = Bs_re[kk][tx + 16 * j]; bi[j] = CB ? Bs_im[kk][tx + 16 * j] : R(0); }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
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
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
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
// Overlap, Theta and (optionally) the weight update, one CTA per walker.
//   A^s = Phi^sT psi^s (binary64), LU with partial pivoting (binary64), log det,
//   (A^s)^-1 by triangular solves, Theta^sT = (psi^s (A^s)^-1)^T.
// mode 0: write log O; mode 1: weight update (Eqs. 13-16) from the stored
// log O, c_mf and sum(x xbar - xbar^2/2); mode 2: Theta only.
// ============================================================================
template <typename R>
struct OverlapArgs {
  int N, ncol, nblk, c0[2], nb[2];
  double smul;                    // 2 for a restricted (one stored spin block) context, else 1
  const cplx_t<R>* psi;           // [W][N][ncol]
  const double* phi;              // [N][ncol]
  cplx_t<R>* thetaT;              // [W][ncol][N]
  double2* logO;                  // [W]
  double* w;                      // [W]
  int* status;
  int mode;
  const double2* cmf;             // [W]
  const double2* xxbar;           // [W]
  double dt, e_trial, e_c;
  unsigned long long* step;       // incremented once (mode 1) if non-null
};

__device__ __forceinline__ double wrap_angle(double t) { return atan2(sin(t), cos(t)); }

template <typename R>
__global__ void __launch_bounds__(256) k_overlap(OverlapArgs<R> a) {
  using R2 = cplx_t<R>;
  extern __shared__ double2 sm_ov[];
  __shared__ int perm_s[64];
  __shared__ int piv_s, sing_s;
  __shared__ double2 logdet_s;
  const int w = blockIdx.x, tid = threadIdx.x;
  if (a.mode == 1 && a.step != nullptr && w == 0 && tid == 0) *a.step += 1ull;
  if (a.mode == 1 && a.w[w] == 0.0) return;          // frozen walker: psi unchanged, Theta still valid
  const int nmax = max(a.nb[0], a.nblk > 1 ? a.nb[1] : 0);
  double2* A = sm_ov;
  double2* Ai = sm_ov + nmax * nmax;
  double ld_re = 0.0, ld_im = 0.0;
  bool singular = false;
  for (int s = 0; s < a.nblk; ++s) {
    const int c0 = a.c0[s], n = a.nb[s];
    if (n == 0) continue;
    // A = Phi^T psi
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      double2 acc = mk(0.0, 0.0);
      for (int p = 0; p < a.N; ++p) {
        const double ph = a.phi[(size_t)p * a.ncol + c0 + i];
        const double2 ps = to_d2(a.psi[((size_t)w * a.N + p) * a.ncol + c0 + j]);
        acc.x += ph * ps.x;
        acc.y += ph * ps.y;
      }
      A[i * n + j] = acc;
    }
    if (tid == 0) { sing_s = 0; logdet_s = mk(0.0, 0.0); }
    __syncthreads();
    int swaps = 0;
    for (int k = 0; k < n; ++k) {
      if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += 32) {
          const double2 v = A[i * n + k];
          const double m = fabs(v.x) + fabs(v.y);
          if (m > best) { best = m; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) {
          piv_s = bi;
          perm_s[k] = bi;
          if (!(best > 0.0) || !isfinite(best)) sing_s = 1;
        }
      }
      __syncthreads();
      if (sing_s) break;
      const int pv = piv_s;
      if (pv != k) {
        for (int j = tid; j < n; j += blockDim.x) {
          const double2 t = A[k * n + j];
          A[k * n + j] = A[pv * n + j];
          A[pv * n + j] = t;
        }
        ++swaps;
      }
      __syncthreads();
      const double2 inv = cdiv(mk(1.0, 0.0), A[k * n + k]);
      for (int i = k + 1 + tid; i < n; i += blockDim.x) A[i * n + k] = cmul(A[i * n + k], inv);
      __syncthreads();
      const int rem = n - k - 1;
      for (int idx = tid; idx < rem * rem; idx += blockDim.x) {
        const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
        A[i * n + j] = csub(A[i * n + j], cmul(A[i * n + k], A[k * n + j]));
      }
      __syncthreads();
    }
    if (sing_s) {
      singular = true;
      for (int idx = tid; idx < n * a.N; idx += blockDim.x) {
        const int b = idx / a.N, p = idx % a.N;
        a.thetaT[((size_t)w * a.ncol + c0 + b) * a.N + p] = from_d2<R>(mk(0.0, 0.0));
      }
      __syncthreads();
      continue;
    }
    if (tid == 0) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < n; ++k) {
        const double2 u = A[k * n + k];
        re += log(hypot(u.x, u.y));
        im += atan2(u.y, u.x);
      }
      im += (swaps & 1) ? 3.141592653589793 : 0.0;
      logdet_s = mk(re, im);
    }
    // A^-1: column j solves L U x = P e_j (one thread per column, x kept in Ai[:, j])
    for (int j = tid; j < n; j += blockDim.x) {
      for (int i = 0; i < n; ++i) Ai[i * n + j] = mk(i == j ? 1.0 : 0.0, 0.0);
      for (int k = 0; k < n; ++k) {
        const int pk = perm_s[k];
        if (pk != k) { double2 t = Ai[k * n + j]; Ai[k * n + j] = Ai[pk * n + j]; Ai[pk * n + j] = t; }
      }
      for (int i = 0; i < n; ++i) {
        double2 y = Ai[i * n + j];
        for (int k = 0; k < i; ++k) y = csub(y, cmul(A[i * n + k], Ai[k * n + j]));
        Ai[i * n + j] = y;
      }
      for (int i = n - 1; i >= 0; --i) {
        double2 y = Ai[i * n + j];
        for (int k = i + 1; k < n; ++k) y = csub(y, cmul(A[i * n + k], Ai[k * n + j]));
        Ai[i * n + j] = cdiv(y, A[i * n + i]);
      }
    }
    __syncthreads();
    // Theta^T[b][p] = sum_j psi[p][j] Ainv[j][b]
    for (int idx = tid; idx < n * a.N; idx += blockDim.x) {
      const int b = idx / a.N, p = idx % a.N;
      const R2* prow = a.psi + ((size_t)w * a.N + p) * a.ncol + c0;
      R accr = R(0), acci = R(0);
      for (int j = 0; j < n; ++j) {
        const R2 ps = prow[j];
        const double2 iv = Ai[j * n + b];
        const R ivr = (R)iv.x, ivi = (R)iv.y;
        accr += ps.x * ivr - ps.y * ivi;
        acci += ps.x * ivi + ps.y * ivr;
      }
      R2 out;
      out.x = accr;
      out.y = acci;
      a.thetaT[((size_t)w * a.ncol + c0 + b) * a.N + p] = out;
    }
    ld_re += logdet_s.x;
    ld_im += logdet_s.y;
    __syncthreads();
  }
  if (tid != 0) return;
  if (singular) {
    if (a.mode != 2) a.w[w] = 0.0;
    atomicOr(a.status, kStatusSingular);
    return;
  }
  const double2 lo_new = mk(a.smul * ld_re, wrap_angle(a.smul * ld_im));
  if (a.mode == 0) {
    a.logO[w] = lo_new;
  } else if (a.mode == 1) {
    const double2 lo_old = a.logO[w];
    const double2 c = a.cmf[w];
    const double2 xx = a.xxbar[w];
    const double ls_re = lo_new.x - lo_old.x + c.x;
    const double theta = lo_new.y - lo_old.y + c.y;
    const double li_re = ls_re + xx.x;
    double wn = a.w[w] * exp(li_re) * fmax(0.0, cos(theta)) * exp(a.dt * (a.e_trial - a.e_c));
    if (!isfinite(wn)) {
      wn = 0.0;
      atomicOr(a.status, kStatusNonFinite);
    }
    a.w[w] = wn;
    a.logO[w] = lo_new;
  }
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
  cplx_t<R>* vbias;          // [W][X]
  double2* exch_part;        // [W][nchunk]
  int with_exchange;
};

template <typename R>
__global__ void __launch_bounds__(256) k_exchange(ExchangeArgs<R> a) {
  using R2 = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char sm_ex[];
  __shared__ double red[32];
  const int chunk = blockIdx.x, w = blockIdx.y, tid = threadIdx.x;
  const int cn = a.ncol * a.N;
  R2* th = (R2*)sm_ex;                                // [ncol][N]
  R* lr = (R*)(th + cn);                              // [ncol][N]
  const int nmax = max(a.nb[0], a.nblk > 1 ? a.nb[1] : 0);
  R2* T = (R2*)(lr + cn + (cn & 1));                  // [nmax][nmax]
  for (int i = tid; i < cn; i += blockDim.x) th[i] = a.thetaT[(size_t)w * cn + i];
  double2 exx = mk(0.0, 0.0);
  const int g0 = chunk * a.gchunk, g1 = min(a.X, g0 + a.gchunk);
  for (int g = g0; g < g1; ++g) {
    __syncthreads();
    for (int i = tid; i < cn; i += blockDim.x) lr[i] = a.lrot[(size_t)g * cn + i];
    __syncthreads();
    double2 vb = mk(0.0, 0.0);
    for (int s = 0; s < a.nblk; ++s) {
      const int c0 = a.c0[s], n = a.nb[s];
      if (n == 0) continue;
      for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int ia = idx / n, ib = idx % n;
        const R* lrow = lr + (size_t)(c0 + ia) * a.N;
        const R2* trow = th + (size_t)(c0 + ib) * a.N;
        R sr = R(0), si = R(0);
        for (int p = 0; p < a.N; ++p) {
          const R l = lrow[p];
          const R2 t = trow[p];
          sr += l * t.x;
          si += l * t.y;
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
    if (tid == 0) a.vbias[(size_t)w * a.X + g] = from_d2<R>(cscale(vb, a.smul));
  }
  if (!a.with_exchange) return;
  const double2 tot = block_sum2(exx, red);
  if (tid == 0) a.exch_part[(size_t)w * a.nchunk + chunk] = cscale(tot, a.smul);
}

// Per-walker local energy from the pieces: E1 = smul sum htilde . Theta^T,
// J = 1/2 sum_g vbias_g^2, K = 1/2 sum exchange partials.  eloc[w] = (E, E0+E1, J-K).
template <typename R>
__global__ void __launch_bounds__(256) k_energy_walker(int N, int X, int ncol, double smul, double ecore,
                                                         int nchunk, const cplx_t<R>* thetaT, const double* hrot,
                                                         const cplx_t<R>* vbias, const double2* exch_part,
                                                         double2* eloc) {
  __shared__ double red[32];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int cn = ncol * N;
  double2 e1 = mk(0.0, 0.0);
  for (int i = tid; i < cn; i += blockDim.x) e1 = cadd(e1, cscale(to_d2(thetaT[(size_t)w * cn + i]), hrot[i]));
  double2 j = mk(0.0, 0.0);
  for (int g = tid; g < X; g += blockDim.x) {
    const double2 v = to_d2(vbias[(size_t)w * X + g]);
    j = cadd(j, cmul(v, v));
  }
  double2 k = mk(0.0, 0.0);
  for (int c = tid; c < nchunk; c += blockDim.x) k = cadd(k, exch_part[(size_t)w * nchunk + c]);
  e1 = block_sum2(e1, red);
  j = block_sum2(j, red);
  k = block_sum2(k, red);
  if (tid == 0) {
    const double2 one = mk(ecore + smul * e1.x, smul * e1.y);
    const double2 two = mk(0.5 * (j.x - k.x), 0.5 * (j.y - k.y));
    eloc[3 * w + 0] = cadd(one, two);
    eloc[3 * w + 1] = one;
    eloc[3 * w + 2] = two;
  }
}

// Weighted estimator sums (ENumer, EDenom, E1Body, E2Body), fixed reduction order.
__global__ void __launch_bounds__(256) k_energy_sums(int W, const double* w, const double2* eloc, double* out) {
  __shared__ double red[32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double wi = w[i];
    if (wi == 0.0) continue;
    s0 += wi * eloc[3 * i].x;
    s1 += wi;
    s2 += wi * eloc[3 * i + 1].x;
    s3 += wi * eloc[3 * i + 2].x;
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  s3 = block_sum(s3, red);
  if (threadIdx.x == 0) { out[0] = s0; out[1] = s1; out[2] = s2; out[3] = s3; }
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
  double* x;                // [W][X]
  double2* xbar;            // [W][X]
  cplx_t<R>* coef;          // [W][X]
  double2* cmf;             // [W]
  double2* xxbar;           // [W]
};

template <typename R>
__global__ void __launch_bounds__(256) k_fields(FieldArgs<R> a) {
  __shared__ SeriesTables tab;
  __shared__ double red[32];
  const int w = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) fill_series_tables(&tab);
  __syncthreads();
  const unsigned long long step = *a.step;
  double2 cm = mk(0.0, 0.0), xx = mk(0.0, 0.0);
  const int npairs = (a.X + 1) / 2;
  for (int j = tid; j < npairs; j += blockDim.x) {
    double z[2];
    normal_pair(a.seed, (uint32_t)j, (uint32_t)w, step, 0u, tab, &z[0], &z[1]);
    for (int t = 0; t < 2; ++t) {
      const int g = 2 * j + t;
      if (g >= a.X) break;
      const double x = z[t];
      const double2 vb = to_d2(a.vbias[(size_t)w * a.X + g]);
      const double dre = vb.x - a.lbar[g], dim = vb.y;
      double2 xb = mk(a.sdt * dim, -a.sdt * dre);
      if (a.cap > 0.0) {
        const double m = sqrt(xb.x * xb.x + xb.y * xb.y);
        if (m > a.cap) xb = cscale(xb, a.cap / m);
      }
      const double2 xs = mk(x - xb.x, -xb.y);
      a.coef[(size_t)w * a.X + g] = from_d2<R>(mk(a.sdt * xs.y, -a.sdt * xs.x));
      const double l = a.lbar[g];
      cm = cadd(cm, mk(-a.sdt * l * xs.y, a.sdt * l * xs.x));
      xx = cadd(xx, mk(x * xb.x - 0.5 * (xb.x * xb.x - xb.y * xb.y), x * xb.y - xb.x * xb.y));
      a.x[(size_t)w * a.X + g] = x;
      a.xbar[(size_t)w * a.X + g] = xb;
    }
  }
  cm = block_sum2(cm, red);
  xx = block_sum2(xx, red);
  if (tid == 0) {
    a.cmf[w] = cm;
    a.xxbar[w] = xx;
  }
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
// QR stabilisation (classical Gram-Schmidt with one reorthogonalisation pass,
// binary64), one CTA per walker.  diag(R) > 0 by construction.
// ============================================================================
template <typename R>
__global__ void __launch_bounds__(256) k_qr(int N, int ncol, int nblk, int c00, int n0, int c01, int n1, double smul,
                                            cplx_t<R>* psi, double2* logO, const double* wgt) {
  extern __shared__ double2 sm_qr[];
  __shared__ double red[32];
  __shared__ double2 rcoef[64];
  const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  if (wgt[w] == 0.0) return;
  double logsum = 0.0;
  for (int s = 0; s < nblk; ++s) {
    const int c0 = s == 0 ? c00 : c01, n = s == 0 ? n0 : n1;
    if (n == 0) continue;
    double2* Q = sm_qr;   // column-major [n][N]
    for (int idx = tid; idx < n * N; idx += blockDim.x) {
      const int p = idx / n, j = idx % n;
      Q[(size_t)j * N + p] = to_d2(psi[((size_t)w * N + p) * ncol + c0 + j]);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      double2* v = Q + (size_t)j * N;
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = wid; i < j; i += nwarp) {
          const double2* q = Q + (size_t)i * N;
          double re = 0.0, im = 0.0;
          for (int p = lane; p < N; p += 32) {   // conj(q) . v
            re += q[p].x * v[p].x + q[p].y * v[p].y;
            im += q[p].x * v[p].y - q[p].y * v[p].x;
          }
          re = warp_sum(re);
          im = warp_sum(im);
          if (lane == 0) rcoef[i] = mk(re, im);
        }
        __syncthreads();
        for (int p = tid; p < N; p += blockDim.x) {
          double2 acc = v[p];
          for (int i = 0; i < j; ++i) acc = csub(acc, cmul(Q[(size_t)i * N + p], rcoef[i]));
          v[p] = acc;
        }
        __syncthreads();
      }
      double nrm = 0.0;
      for (int p = tid; p < N; p += blockDim.x) nrm += v[p].x * v[p].x + v[p].y * v[p].y;
      nrm = sqrt(block_sum(nrm, red));
      const double inv = 1.0 / nrm;
      for (int p = tid; p < N; p += blockDim.x) v[p] = cscale(v[p], inv);
      logsum += log(nrm);
      __syncthreads();
    }
    for (int idx = tid; idx < n * N; idx += blockDim.x) {
      const int p = idx / n, j = idx % n;
      psi[((size_t)w * N + p) * ncol + c0 + j] = from_d2<R>(Q[(size_t)j * N + p]);
    }
    __syncthreads();
  }
  if (tid == 0) logO[w].x -= smul * logsum;
}

// ============================================================================
// Comb population control.  One CTA: sequential (index-order) binary64 prefix
// of the weights, xi from Philox stream 1, tooth search.  Then a gather.
// ============================================================================
__global__ void __launch_bounds__(256) k_comb_plan(int W, unsigned long long seed, const unsigned long long* step,
                                                   const double* w, double* cum, int* src, double* neww,
                                                   int* status) {
  __shared__ double total_s, xi_s;
  __shared__ int last_s, ok_s;
  if (threadIdx.x == 0) {
    double t = 0.0;
    int last = -1;
    for (int i = 0; i < W; ++i) {
      t = t + w[i];
      cum[i] = t;
      if (w[i] > 0.0) last = i;
    }
    total_s = t;
    last_s = last;
    ok_s = (t > 0.0) && isfinite(t) && last >= 0;
    const uint4 r = philox4x32_10(field_counter(0u, 0u, *step, 1u), (uint32_t)(seed & 0xffffffffull),
                                  (uint32_t)(seed >> 32));
    xi_s = uniform52(r.x, r.y);
    if (!ok_s) atomicOr(status, kStatusNoWalkers);
    *neww = ok_s ? t / (double)W : -1.0;
  }
  __syncthreads();
  const double total = total_s, xi = xi_s;
  for (int k = threadIdx.x; k < W; k += blockDim.x) {
    if (!ok_s) { src[k] = k; continue; }
    const double tooth = __ddiv_rn(__dmul_rn(__dadd_rn((double)k, xi), total), (double)W);
    int lo = 0, hi = W;   // first i with cum[i] > tooth
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cum[mid] > tooth) hi = mid; else lo = mid + 1;
    }
    src[k] = lo < W ? lo : last_s;
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_comb_gather(int W, int psi_elems, int th_elems, const int* src,
                                                     const double* neww, const cplx_t<R>* psi, cplx_t<R>* psi_out,
                                                     const cplx_t<R>* th, cplx_t<R>* th_out, const double2* logO,
                                                     double2* logO_out, const double* w, double* w_out) {
  const int k = blockIdx.x;
  const int s = src[k];
  const double nw = *neww;
  for (int i = threadIdx.x; i < psi_elems; i += blockDim.x) psi_out[(size_t)k * psi_elems + i] = psi[(size_t)s * psi_elems + i];
  for (int i = threadIdx.x; i < th_elems; i += blockDim.x) th_out[(size_t)k * th_elems + i] = th[(size_t)s * th_elems + i];
  if (threadIdx.x == 0) {
    logO_out[k] = logO[s];
    w_out[k] = nw >= 0.0 ? nw : w[s];
  }
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_init_walkers(int W, int N, int ncol, const double* phi, cplx_t<R>* psi, double* w) {
  const size_t total = (size_t)W * N * ncol;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    psi[i] = from_d2<R>(mk(phi[i % ((size_t)N * ncol)], 0.0));
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
