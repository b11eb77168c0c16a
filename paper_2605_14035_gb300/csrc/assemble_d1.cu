// Kernels for elements of dimension 1 (all supported ambient dimensions, orders 1 and 2).
#include "dispatch.cuh"

namespace lfem {

lfem_status run_stage_d1(int NA, int P, int kind, const StageArgs& s, cudaStream_t st) {
  LFEM_DEFINE_CASE_STAGE(1, 1, 1)
  LFEM_DEFINE_CASE_STAGE(1, 1, 2)
  LFEM_DEFINE_CASE_STAGE(1, 2, 1)
  LFEM_DEFINE_CASE_STAGE(1, 2, 2)
  LFEM_DEFINE_CASE_STAGE(1, 3, 1)
  LFEM_DEFINE_CASE_STAGE(1, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status run_adjoint_d1(int NA, int P, const AdjArgs& a, int64_t T, int pos_bytes, cudaStream_t st) {
  LFEM_DEFINE_CASE_ADJ(1, 1, 1)
  LFEM_DEFINE_CASE_ADJ(1, 1, 2)
  LFEM_DEFINE_CASE_ADJ(1, 2, 1)
  LFEM_DEFINE_CASE_ADJ(1, 2, 2)
  LFEM_DEFINE_CASE_ADJ(1, 3, 1)
  LFEM_DEFINE_CASE_ADJ(1, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status run_pipe_d1(int NA, int P, bool mixed, const PipeArgs& a, int ent_bytes, bool fast, const FastBank& fb,
                        int sms, cudaStream_t st) {
  LFEM_DEFINE_CASE_PIPE(1, 1, 1)
  LFEM_DEFINE_CASE_PIPE(1, 1, 2)
  LFEM_DEFINE_CASE_PIPE(1, 2, 1)
  LFEM_DEFINE_CASE_PIPE(1, 2, 2)
  LFEM_DEFINE_CASE_PIPE(1, 3, 1)
  LFEM_DEFINE_CASE_PIPE(1, 3, 2)
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_d1(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
