// Kernels for elements of dimension 3 (all supported ambient dimensions, orders 1 and 2).
#include "dispatch.cuh"

namespace lfem {

lfem_status run_stage_d3(int NA, int P, int kind, const StageArgs& s, cudaStream_t st) {
  LFEM_DEFINE_CASE_STAGE(3, 3, 1)
  LFEM_DEFINE_CASE_STAGE(3, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status run_adjoint_d3(int NA, int P, const AdjArgs& a, int64_t T, int pos_bytes, cudaStream_t st) {
  LFEM_DEFINE_CASE_ADJ(3, 3, 1)
  LFEM_DEFINE_CASE_ADJ(3, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status run_pipe_d3(int NA, int P, bool mixed, const PipeArgs& a, int ent_bytes, bool fast, const FastBank& fb,
                        int sms, cudaStream_t st) {
  LFEM_DEFINE_CASE_PIPE(3, 3, 1)
  LFEM_DEFINE_CASE_PIPE(3, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status run_twopass_d3(int P, bool mixed, bool fast, const FastBankTet& fb, const TwoPassArgs& a, int sms,
                           cudaStream_t st) {
  if (P == 1)
    return mixed ? launch_twopass<3, 3, 1, float>(a, fast, fb, sms, st) : launch_twopass<3, 3, 1, double>(a, false, fb, sms, st);
  if (P == 2)
    return mixed ? launch_twopass<3, 3, 2, float>(a, fast, fb, sms, st) : launch_twopass<3, 3, 2, double>(a, false, fb, sms, st);
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_d3(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
