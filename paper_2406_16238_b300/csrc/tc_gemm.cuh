// Tensor-core (tcgen05) contractions for the BF16 and BF16x3 forms.
#pragma once
#include <cuda_runtime.h>
#include "afqmc.h"

namespace afq {
namespace tc {

// Bytes of operand staging the BF16 forms need inside the workspace (0 for the other forms).
size_t operand_bytes(int prec, int W, int N, int X, int ncol, const int* c0, const int* nb, int nblk);

// One-time conversion of the binary64 L and Ltilde into the tensor-core operand layouts.
afqmc_status prepare(int prec, cudaStream_t s, char* tcbuf, int W, int N, int X, int ncol, const int* c0,
                     const int* nb, int nblk, const double* chol64, const double* lrot64,
                     unsigned long long* launches);

// vbias and exchange partials from Theta^T (complex64) -- see k_exchange for the definitions.
afqmc_status exchange(int prec, cudaStream_t s, char* tcbuf, int W, int N, int X, int ncol, const int* c0,
                      const int* nb, int nblk, double smul, const float2* thetaT, float2* vbias,
                      double2* exch_part, int nchunk, unsigned long long* launches);

afqmc_status force_bias(int prec, cudaStream_t s, char* tcbuf, int W, int N, int X, int ncol, double smul,
                        const float2* thetaT, float2* vbias, unsigned long long* launches);

// VHS[w][pq] = sum_g coef[w][g] L[g][pq] (complex64 out).
afqmc_status vhs(int prec, cudaStream_t s, char* tcbuf, int W, int N, int X, const float2* coef, float2* out,
                 unsigned long long* launches);

}  // namespace tc
}  // namespace afq
