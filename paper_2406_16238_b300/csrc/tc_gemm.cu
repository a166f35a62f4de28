// Tensor-core (tcgen05) contractions for the BF16 and BF16x3 forms.
#include "tc_gemm.cuh"

namespace afq {
namespace tc {

size_t operand_bytes(int prec, int, int, int, int, const int*, const int*, int) {
  (void)prec;
  return 0;
}

static afqmc_status not_built() { return AFQMC_EINVAL; }

afqmc_status prepare(int, cudaStream_t, char*, int, int, int, int, const int*, const int*, int, const double*,
                     const double*, unsigned long long*) { return not_built(); }
afqmc_status exchange(int, cudaStream_t, char*, int, int, int, int, const int*, const int*, int, double,
                      const float2*, float2*, double2*, int, unsigned long long*) { return not_built(); }
afqmc_status force_bias(int, cudaStream_t, char*, int, int, int, int, double, const float2*, float2*,
                        unsigned long long*) { return not_built(); }
afqmc_status vhs(int, cudaStream_t, char*, int, int, int, const float2*, float2*, unsigned long long*) {
  return not_built();
}

}  // namespace tc
}  // namespace afq
