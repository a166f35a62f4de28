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

// ---- complex Hamiltonians (Section "Support of complex Cholesky vectors") -----------------------
// X complex Cholesky vectors L^g (g_psqr = sum_g L^g_ps conj(L^g_rq)) become 2X Hermitian field
// matrices A^g = (L^g + L^g+) / 2 and B^g = i (L^g - L^g+) / 2, which then play the part of the
// real symmetric L^g of the real case.  Complex arrays are interleaved (re, im).
namespace afq {

// flags |= kSetupNonFinite for a non-finite entry of the complex chunk [ng][N][N].
template <typename T>
__global__ void __launch_bounds__(256) k_chol_check_c(int ng, int N, const T* chol, int* flags) {
  const size_t total = (size_t)ng * N * N * 2;
  int f = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite((double)chol[i])) f |= kSetupNonFinite;
  f = __reduce_or_sync(0xffffffffu, f);
  if (f && (threadIdx.x & 31) == 0) atomicOr(flags, f);
}

// fields [2 ng][N][N] (type G, interleaved) from the complex chunk L [ng][N][N] (type T).
template <typename T, typename G>
__global__ void __launch_bounds__(256) k_hermitian_fields(int ng, int N, const T* chol, G* fields) {
  const size_t NN = (size_t)N * N, total = (size_t)ng * NN;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t g = i / NN, r = i - g * NN;
    const int p = (int)(r / N), q = (int)(r - (size_t)p * N);
    const size_t t = g * NN + (size_t)q * N + p;
    const double lr = (double)chol[2 * i], li = (double)chol[2 * i + 1];     // L_pq
    const double tr = (double)chol[2 * t], ti = -(double)chol[2 * t + 1];   // conj(L_qp) = (L^+)_pq
    G* a = fields + 2 * ((2 * g) * NN + r);
    G* b = fields + 2 * ((2 * g + 1) * NN + r);
    a[0] = (G)(0.5 * (lr + tr));
    a[1] = (G)(0.5 * (li + ti));
    // i (L - L^+) / 2 = (-(Im L - Im L^+), Re L - Re L^+) / 2
    b[0] = (G)(-0.5 * (li - ti));
    b[1] = (G)(0.5 * (lr - tr));
  }
}

// lbar[g] = Re Tr(M^g P) = sum_pq Re(M_pq conj(P_pq)) (M, P Hermitian), one CTA per field.
template <typename G>
__global__ void __launch_bounds__(256) k_chunk_lbar_c(int N, const G* fields, const double* P, double* lbar) {
  __shared__ double part[8];
  const size_t NN = (size_t)N * N;
  const G* M = fields + 2 * (size_t)blockIdx.x * NN;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < NN; i += blockDim.x)
    acc = fma((double)M[2 * i], P[2 * i], fma((double)M[2 * i + 1], P[2 * i + 1], acc));
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    lbar[blockIdx.x] = t;
  }
}

// A = scale * h_eff made Hermitian: A_pq = scale (x_pq + conj(x_qp)) / 2, x = h - 1/2 msum + lsum.
__global__ void k_heff_c(int N, double scale, const double* h, const double* msum, const double* lsum, double* A) {
  const size_t NN = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / N), q = (int)(i - (size_t)p * N);
    const size_t j = (size_t)q * N + p;
    const double xr = h[2 * i] - 0.5 * msum[2 * i] + lsum[2 * i];
    const double xi = h[2 * i + 1] - 0.5 * msum[2 * i + 1] + lsum[2 * i + 1];
    const double yr = h[2 * j] - 0.5 * msum[2 * j] + lsum[2 * j];
    const double yi = h[2 * j + 1] - 0.5 * msum[2 * j + 1] + lsum[2 * j + 1];
    A[2 * i] = scale * (0.5 * (xr + yr));
    A[2 * i + 1] = scale * (0.5 * (xi - yi));
  }
}

// out[0] = max_j sum_i |A_ij| of a complex matrix, one CTA.
__global__ void __launch_bounds__(1024) k_norm1_c(int N, const double* A, double* out) {
  __shared__ double part[32];
  double m = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) s += hypot(A[2 * ((size_t)i * N + j)], A[2 * ((size_t)i * N + j) + 1]);
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

// T = alpha B + diag I on complex matrices (alpha, diag real; in place allowed).
__global__ void k_identity_plus_c(int N, double alpha, double diag, const double* B, double* T) {
  const size_t NN = (size_t)N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / N), q = (int)(i - (size_t)p * N);
    T[2 * i] = alpha * B[2 * i] + (p == q ? diag : 0.0);
    T[2 * i + 1] = alpha * B[2 * i + 1];
  }
}

}  // namespace afq
