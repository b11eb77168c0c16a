// Orders 3 and 4 on curves and triangles: the element-major two-pass path
// (each element once into the local-matrix buffer, then each CSR slot sums its
// list), with the Jacobian in the general form J = sum_a (x_a - x_0) grad^phi_a^T,
// and the element stages at these orders.
#include "dispatch.cuh"

namespace lfem {

lfem_status run_twopass_high(int D, int NA, int P, bool mixed, const TwoPassArgs& a, int sms, cudaStream_t st) {
  const FastBankTet unused{};
#define LFEM_HIGH_CASE(DD, NN, PP)                                                    \
  if (D == DD && NA == NN && P == PP)                                                 \
    return mixed ? launch_twopass<DD, NN, PP, float>(a, false, unused, sms, st)       \
                 : launch_twopass<DD, NN, PP, double>(a, false, unused, sms, st);
  LFEM_HIGH_CASE(1, 1, 3)
  LFEM_HIGH_CASE(1, 1, 4)
  LFEM_HIGH_CASE(1, 2, 3)
  LFEM_HIGH_CASE(1, 2, 4)
  LFEM_HIGH_CASE(1, 3, 3)
  LFEM_HIGH_CASE(1, 3, 4)
  LFEM_HIGH_CASE(2, 2, 3)
  LFEM_HIGH_CASE(2, 2, 4)
  LFEM_HIGH_CASE(2, 3, 3)
  LFEM_HIGH_CASE(2, 3, 4)
#undef LFEM_HIGH_CASE
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

// The element stages (points, geometry, local matrices; FP64) at orders 3, 4.
lfem_status run_stage_high(int D, int NA, int P, int kind, const StageArgs& s, cudaStream_t st) {
#define LFEM_HIGH_STAGE(DD, NN, PP) \
  if (D == DD && NA == NN && P == PP) return launch_stage<DD, NN, PP>(kind, s, st);
  LFEM_HIGH_STAGE(1, 1, 3)
  LFEM_HIGH_STAGE(1, 1, 4)
  LFEM_HIGH_STAGE(1, 2, 3)
  LFEM_HIGH_STAGE(1, 2, 4)
  LFEM_HIGH_STAGE(1, 3, 3)
  LFEM_HIGH_STAGE(1, 3, 4)
  LFEM_HIGH_STAGE(2, 2, 3)
  LFEM_HIGH_STAGE(2, 2, 4)
  LFEM_HIGH_STAGE(2, 3, 3)
  LFEM_HIGH_STAGE(2, 3, 4)
#undef LFEM_HIGH_STAGE
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_high(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
