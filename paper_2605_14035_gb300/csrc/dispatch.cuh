// Per-dimension entry points into the templated kernels (one translation unit per D).
#pragma once

#include "adjoint_impl.cuh"
#include "assemble_impl.cuh"
#include "assemble_pipe.cuh"
#include "assemble_twopass.cuh"

namespace lfem {

#define LFEM_DECLARE_DIM(DD)                                                                                      \
  lfem_status run_stage_d##DD(int NA, int P, int kind, const StageArgs& s, cudaStream_t st);                     \
  lfem_status run_adjoint_d##DD(int NA, int P, const AdjArgs& a, int64_t T, int pos_bytes, cudaStream_t st);     \
  lfem_status bank_upload_d##DD(const void* src, size_t bytes, size_t offset);                                 \
  lfem_status run_pipe_d##DD(int NA, int P, bool mixed, const PipeArgs& a, int ent_bytes, bool fast,             \
                             const FastBank& fb, int sms, cudaStream_t st);

LFEM_DECLARE_DIM(1)
LFEM_DECLARE_DIM(2)
LFEM_DECLARE_DIM(3)
lfem_status run_twopass_d3(int P, bool mixed, bool fast, const FastBankTet& fb, const TwoPassArgs& a, int sms,
                           cudaStream_t st);
lfem_status bank_upload_batch(const void* src, size_t bytes, size_t offset);
lfem_status bank_upload_vec(const void* src, size_t bytes, size_t offset);
lfem_status bank_upload_high(const void* src, size_t bytes, size_t offset);
lfem_status run_twopass_high(int D, int NA, int P, bool mixed, const TwoPassArgs& a, int sms, cudaStream_t st);
lfem_status bank_upload_tet_high(const void* src, size_t bytes, size_t offset);
lfem_status bank_upload_adj_high(const void* src, size_t bytes, size_t offset);
lfem_status run_stage_high(int D, int NA, int P, int kind, const StageArgs& s, cudaStream_t st);
// Orders 3, 4: the adjoint (FP64, warp per element); scratch holds
// adjoint_high_scratch_bytes(...) bytes.
size_t adjoint_high_scratch_bytes(int dim, int P, int Q, int ambient, int64_t n_elem);
lfem_status run_adjoint_high(int dim, int NA, int P, const AdjArgs& a, int pos_bytes, void* scratch, int sms,
                             cudaStream_t st);
lfem_status run_tet_high(int P, bool mixed, const TwoPassArgs& a, void* scratch, int sms, cudaStream_t st);
size_t tet_high_scratch_bytes(int P, int Q, int64_t n_elem);
lfem_status run_tet_high_load(int P, const VecArgs& a, void* scratch, int sms, cudaStream_t st);
lfem_status run_vec_gather(const VecArgs& a, int ref, int nc, cudaStream_t st);
lfem_status run_vectors(int D, int NA, int P, int kind, const VecArgs& a, cudaStream_t st);
lfem_status run_mcf_solve(int nc, const McfSolveArgs& s, cudaStream_t st, int* iterations);

// Body of one dimension's dispatch functions over (NA, P).
#define LFEM_DEFINE_CASE_STAGE(DD, NN, PP) \
  if (NA == NN && P == PP) return launch_stage<DD, NN, PP>(kind, s, st);
#define LFEM_DEFINE_CASE_ADJ(DD, NN, PP) \
  if (NA == NN && P == PP) return launch_adjoint<DD, NN, PP>(a, T, pos_bytes, st);

#define LFEM_DEFINE_CASE_PIPE(DD, NN, PP)                                                          \
  if (NA == NN && P == PP)                                                                         \
    return mixed ? launch_pipe<DD, NN, PP, float>(a, ent_bytes, fast, fb, sms, st)                 \
                 : launch_pipe<DD, NN, PP, double>(a, ent_bytes, false, fb, sms, st);

}  // namespace lfem
