// Kernels of the learned control variate for the exchange energy.
//
// The mixed energy of Eq. 9 splits per walker into A = Re(E0 + E1 + J) (cheap) and
// K = Re(1/2 sum_{g s} Tr T T) (the exchange).  An MLP f(z) of per-walker features z
// predicts K; exact K on a uniformly drawn subsample S of m walkers (without replacement,
// inclusion probability m / W) corrects it:
//   ENumer_CV = sum_i w_i (A_i - f_i) - (W / m) sum_{i in S} w_i (K_i - f_i),
// which has the expectation sum_i w_i (A_i - K_i) over the draw of S for any f.
#pragma once

#include "common.cuh"

namespace afq {

constexpr int kCvHidden = 256;

// z = [diag Re G^a (N), diag Re G^b (N), mean, var, skew, kurt of Re vbias, same of Im vbias],
// standardised with (mean, std) when zmean is given.  G_pp = sum_a Re(Theta_pa) Phi_pa per block.
template <typename R>
__global__ void __launch_bounds__(256) k_cv_features(int N, int X, int ncol, int nblk, int c00, int n0, int c01,
                                                     int n1, int restricted, const cplx_t<R>* thetaT, const R* phi_r,
                                                     const cplx_t<R>* vbias, const float* zmean, const float* zstd,
                                                     float* Z) {
  __shared__ double red[32];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int D = 2 * N + 8;
  float* z = Z + (size_t)w * D;
  for (int p = tid; p < N; p += blockDim.x) {
    double ga = 0.0, gb = 0.0;
    for (int a = 0; a < n0; ++a)
      ga += (double)thetaT[((size_t)w * ncol + c00 + a) * N + p].x * (double)phi_r[(size_t)p * ncol + c00 + a];
    if (restricted) gb = ga;
    else if (nblk > 1)
      for (int a = 0; a < n1; ++a)
        gb += (double)thetaT[((size_t)w * ncol + c01 + a) * N + p].x * (double)phi_r[(size_t)p * ncol + c01 + a];
    z[p] = (float)ga;
    z[N + p] = (float)gb;
  }
  for (int part = 0; part < 2; ++part) {
    double s = 0.0;
    for (int g = tid; g < X; g += blockDim.x) {
      const cplx_t<R> v = vbias[(size_t)w * X + g];
      s += part ? (double)v.y : (double)v.x;
    }
    const double mean = block_sum(s, red) / X;
    double s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (int g = tid; g < X; g += blockDim.x) {
      const cplx_t<R> v = vbias[(size_t)w * X + g];
      const double c = (part ? (double)v.y : (double)v.x) - mean;
      s2 += c * c;
      s3 += c * c * c;
      s4 += c * c * c * c;
    }
    const double var = block_sum(s2, red) / X;
    const double m3 = block_sum(s3, red) / X;
    const double m4 = block_sum(s4, red) / X;
    if (tid == 0) {
      const double sd = sqrt(var);
      z[2 * N + 4 * part + 0] = (float)mean;
      z[2 * N + 4 * part + 1] = (float)var;
      z[2 * N + 4 * part + 2] = sd > 0.0 ? (float)(m3 / (sd * sd * sd)) : 0.f;
      z[2 * N + 4 * part + 3] = sd > 0.0 ? (float)(m4 / (var * var)) : 0.f;
    }
  }
  if (zmean) {
    __syncthreads();
    for (int i = tid; i < D; i += blockDim.x) z[i] = (z[i] - zmean[i]) / zstd[i];
  }
}

// Column mean and standard deviation of rows x cols (one block per column), binary64 sums.
__global__ void __launch_bounds__(256) k_col_stats(int rows, int cols, const float* A, float* mean, float* stdv) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s += A[(size_t)r * cols + c];
  const double m = block_sum(s, red) / rows;
  double s2 = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const double d = A[(size_t)r * cols + c] - m;
    s2 += d * d;
  }
  const double var = block_sum(s2, red) / rows;
  if (threadIdx.x == 0) {
    mean[c] = (float)m;
    stdv[c] = var > 1e-20 ? (float)sqrt(var) : 1.f;
  }
}

__global__ void k_standardize(size_t rows, int cols, float* A, const float* mean, const float* stdv) {
  const size_t total = rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    A[i] = (A[i] - mean[c]) / stdv[c];
  }
}

__global__ void k_bias_tanh(int rows, int cols, float* H, const float* b) {
  const size_t total = (size_t)rows * cols;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    H[i] = tanhf(H[i] + b[i % cols]);
}

__global__ void k_bias_add(int rows, float* out, const float* b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) out[i] += b[0];
}

// dout = 2 (out - y) / B and the summed squared residual (one block, fixed order).
__global__ void __launch_bounds__(256) k_mse(int B, const float* out, const float* y, float* dout, float* loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float r = out[i] - y[i];
    dout[i] = 2.f * r / (float)B;
    s += (double)r * r;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) *loss += (float)(s / B);
}

// dZ = dA * (1 - A^2), in place on dA.
__global__ void k_tanh_backward(size_t n, float* dA, const float* A) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dA[i] *= 1.f - A[i] * A[i];
}

// db[j] = sum_b dZ[b][j] (one thread per column, sequential rows).
__global__ void k_colsum(int rows, int cols, const float* dZ, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dZ[(size_t)r * cols + j];
  db[j] = s;
}

// Adam (Kingma & Ba 2015), bias-corrected, t >= 1.
__global__ void k_adam(size_t n, float* P, const float* G, float* M, float* V, int t, float lr, float b1, float b2,
                       float eps) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

__global__ void k_gather_rows(int B, int D, const int* idx, const float* src, float* dst, const float* ysrc,
                              float* ydst) {
  const int b = blockIdx.x;
  const int r = idx[b];
  for (int i = threadIdx.x; i < D; i += blockDim.x) dst[(size_t)b * D + i] = src[(size_t)r * D + i];
  if (threadIdx.x == 0) ydst[b] = ysrc[r];
}

// Exactly m walkers of W chosen uniformly without replacement: the m smallest Philox keys
// (stream 2, counter (0, walker, step)), ties by index.  One block, bitonic sort in shared memory.
__global__ void __launch_bounds__(1024) k_cv_select(int W, int m, unsigned long long seed,
                                                    const unsigned long long* step, int* sel) {
  extern __shared__ unsigned long long keys[];   // [P] packed (key << 16 | index) with P a power of two >= W
  int P = 1;
  while (P < W) P <<= 1;
  const unsigned long long st = *step;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long k = ~0ull;
    if (i < W) {
      const uint4 r = philox4x32_10(field_counter(0u, (uint32_t)i, st, 2u), (uint32_t)(seed & 0xffffffffull),
                                    (uint32_t)(seed >> 32));
      k = ((unsigned long long)(r.x >> 16) << 32 | (unsigned long long)r.y) << 16 | (unsigned long long)i;
    }
    keys[i] = k;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = keys[i], b = keys[j];
          if ((a > b) == up) { keys[i] = b; keys[j] = a; }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < m; i += blockDim.x) sel[i] = (int)(keys[i] & 0xffffull);
}

// Per walker: A = Re(E0 + E1 + J) and Re(E0 + E1) (binary64 reductions).
template <typename R>
__global__ void __launch_bounds__(256) k_cv_walker(int N, int X, int ncol, double smul, double ecore,
                                                   const cplx_t<R>* thetaT, const R* hrot_r, const cplx_t<R>* vbias,
                                                   double* a_out, double* e1_out) {
  __shared__ double red[32];
  const int w = blockIdx.x, tid = threadIdx.x;
  const int cn = ncol * N;
  R e1r = R(0);
  for (int i = tid; i < cn; i += blockDim.x) e1r += thetaT[(size_t)w * cn + i].x * hrot_r[i];
  double jr = 0.0;
  for (int g = tid; g < X; g += blockDim.x) {
    const double2 v = to_d2(vbias[(size_t)w * X + g]);
    jr += v.x * v.x - v.y * v.y;
  }
  const double e1 = block_sum((double)e1r, red);
  jr = block_sum(jr, red);
  if (tid == 0) {
    e1_out[w] = ecore + smul * e1;
    a_out[w] = ecore + smul * e1 + 0.5 * jr;
  }
}

// Estimator sums of the control-variate form:
// out = {ENumer_CV, EDenom, E1Body, ENumer_CV - E1Body}, fixed reduction order, optional history slot
// and running sums of E_T (etacc[1], etacc[2]).
__global__ void __launch_bounds__(256) k_cv_sums(int W, int m, int nchunk, const double* w, const double* a,
                                                 const double* e1, const float* f, const int* sel,
                                                 const double2* exch_part, const float2* exch_part_f, double* out,
                                                 int* slot,
                                                 double* etacc) {
  __shared__ double red[32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, sc = 0.0;
  for (int i = threadIdx.x; i < W; i += blockDim.x) {
    const double wi = w[i];
    if (wi == 0.0) continue;
    s0 += wi * (a[i] - (double)f[i]);
    s1 += wi;
    s2 += wi * e1[i];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const int i = sel[j];
    const double wi = w[i];
    if (wi == 0.0) continue;
    double k = 0.0;
    for (int c = 0; c < nchunk; ++c)
      k += exch_part_f ? (double)exch_part_f[(size_t)j * nchunk + c].x : exch_part[(size_t)j * nchunk + c].x;
    sc += wi * (0.5 * k - (double)f[i]);
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  sc = block_sum(sc, red);
  if (threadIdx.x == 0) {
    double* o = slot ? out + 4 * (size_t)(*slot) : out;
    const double num = s0 - ((double)W / (double)m) * sc;
    o[0] = num; o[1] = s1; o[2] = s2; o[3] = num - s2;
    if (slot) *slot += 1;
    if (etacc) {   // running sums of E_T
      etacc[1] += num;
      etacc[2] += s1;
    }
  }
}

// Exact K = Re(1/2 sum of exchange partials) of every walker (training targets).
__global__ void k_exact_k(int W, int nchunk, const double2* exch_part, const float2* exch_part_f, float* k_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= W) return;
  double k = 0.0;
  for (int c = 0; c < nchunk; ++c)
    k += exch_part_f ? (double)exch_part_f[(size_t)i * nchunk + c].x : exch_part[(size_t)i * nchunk + c].x;
  k_out[i] = (float)(0.5 * k);
}

// f = out * ystd + ymean (un-standardise the network output)
__global__ void k_unscale(int n, const float* out, const float* ystat, float* f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    f[i] = out[i] * ystat[1] + ystat[0];
}

}  // namespace afq

namespace afq {

// Host-side state of the learned control variate (buffers inside a caller-provided device block).
struct CvState {
  bool attached = false, enabled = false, scaled = false;
  int D = 0, H = kCvHidden, cap = 0, B = 0, m = 0, ndata = 0, adam_t = 0;
  double frac = 0.125;
  size_t nparams = 0, bytes = 0;
  unsigned long long seed = 0;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  float *dataZ = nullptr, *dataY = nullptr, *zmean = nullptr, *zstd = nullptr, *ystat = nullptr;
  float *X = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr, *out = nullptr, *dout = nullptr, *yb = nullptr;
  float *dA = nullptr, *dB = nullptr, *loss = nullptr;
  float *Zw = nullptr, *WA1 = nullptr, *WA2 = nullptr, *WA3 = nullptr, *wout = nullptr, *fw = nullptr;
  int *perm = nullptr, *sel = nullptr;
  double *a = nullptr, *e1 = nullptr;
  char* tc_scratch = nullptr;   // split-bf16 operands of the tensor-core GEMMs
  size_t tc_bytes = 0;
  // parameter blocks inside P (and the same offsets inside G, Mo, Vo)
  size_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, oW4 = 0, ob4 = 0;
};

}  // namespace afq
