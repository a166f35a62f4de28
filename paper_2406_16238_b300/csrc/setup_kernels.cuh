// Set-up kernels of the Hamiltonian store (Section "Theory of AFQMC", Eqs. 4-6 and the mean-field
// shift of Eq. 12).  The Cholesky vectors arrive in chunks of gammas, binary64 or binary32, so
// the store of a Hamiltonian whose L does not fit a binary64 copy on the device is built one
// chunk at a time:
//   lbar_g = Tr(L^g P_T)                       (k_chunk_lbar, P_T = P_alpha + P_beta, symmetric)
//   lsum  += sum_g lbar_g L^g                  (k_chunk_lsum)
//   msum  += sum_g L^g L^g                     (one GEMM per chunk, in afqmc.cu)
//   h_eff  = h - 1/2 msum + lsum,  A = -dt/2 h_eff (symmetrised)   (k_heff)
//   exp(A) by scaling and squaring of its Taylor series in Horner form (k_identity_plus, GEMMs)
#pragma once
#include "common.cuh"

namespace afq {

constexpr int kSetupNonFinite = 1, kSetupAsymmetric = 2;

// flags |= kSetupNonFinite for a non-finite entry and kSetupAsymmetric where
// |L_pq - L_qp| > 1e-12 max(1, |L_pq|, |L_qp|), over ng gammas of [ng][N][N].
template <typename T>
__global__ void __launch_bounds__(256) k_chol_check(int ng, int N, const T* chol, int* flags) {
  const size_t NN = (size_t)N * N, total = (size_t)ng * NN;
  int f = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t g = i / NN, r = i - g * NN;
    const int p = (int)(r / N), q = (int)(r - (size_t)p * N);
    const double v = (double)chol[i];
    if (!isfinite(v)) f |= kSetupNonFinite;
    if (q > p) {
      const double u = (double)chol[g * NN + (size_t)q * N + p];
      if (fabs(v - u) > 1e-12 * fmax(1.0, fmax(fabs(v), fabs(u)))) f |= kSetupAsymmetric;
    }
  }
  f = __reduce_or_sync(0xffffffffu, f);
  if (f && (threadIdx.x & 31) == 0) atomicOr(flags, f);
}

// lbar[g] = sum_pq L^g_pq P_pq for the chunk's gammas (one CTA per gamma, binary64 sums).
template <typename T>
__global__ void __launch_bounds__(256) k_chunk_lbar(int N, const T* chol, const double* P, double* lbar) {
  __shared__ double part[8];
  const size_t NN = (size_t)N * N;
  const T* L = chol + (size_t)blockIdx.x * NN;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x) acc = fma((double)L[i], P[i], acc);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    lbar[blockIdx.x] = t;
  }
}

// lsum[i] += sum_g lbar[g] L^g_i over the chunk's ng gammas (in gamma order).
template <typename T>
__global__ void __launch_bounds__(256) k_chunk_lsum(int ng, size_t NN, const T* chol, const double* lbar,
                                                    double* lsum) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = 0; g < ng; ++g) acc = fma(lbar[g], (double)chol[(size_t)g * NN + i], acc);
    lsum[i] += acc;
  }
}

// out[i] += (double) in[i]  (binary32 partial sums of one chunk into the binary64 total).
__global__ void k_add_f32_to_f64(size_t n, const float* in, double* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] += (double)in[i];
}

template <typename Ti, typename To>
__global__ void k_cast(size_t n, const Ti* in, To* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

// A = scale * h_eff, h_eff = h - 1/2 msum + lsum, symmetrised: A_pq = scale (x_pq + x_qp) / 2.
__global__ void k_heff(int N, double scale, const double* h, const double* msum, const double* lsum, double* A) {
  const size_t NN = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / N), q = (int)(i - (size_t)p * N);
    const size_t j = (size_t)q * N + p;
    const double xpq = h[i] - 0.5 * msum[i] + lsum[i];
    const double xqp = h[j] - 0.5 * msum[j] + lsum[j];
    A[i] = scale * (0.5 * (xpq + xqp));
  }
}

// out[0] = max_j sum_i |A_ij| (the 1-norm), one CTA.
__global__ void __launch_bounds__(1024) k_norm1(int N, const double* A, double* out) {
  __shared__ double part[32];
  double m = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += fabs(A[(size_t)i * N + j]);
    m = fmax(m, s);
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, part[k]);
    out[0] = t;
  }
}

// T = alpha B + diag I  (in place allowed: T == B).
__global__ void k_identity_plus(int N, double alpha, double diag, const double* B, double* T) {
  const size_t NN = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / N), q = (int)(i - (size_t)p * N);
    T[i] = alpha * B[i] + (p == q ? diag : 0.0);
  }
}

}  // namespace afq
