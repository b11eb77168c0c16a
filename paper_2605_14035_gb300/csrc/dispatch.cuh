// Per-dimension entry points into the templated kernels (one translation unit per D).
#pragma once

#include "adjoint_impl.cuh"
#include "assemble_impl.cuh"

namespace lfem {

#define LFEM_DECLARE_DIM(DD)                                                                                      \
  lfem_status run_tiles_d##DD(int NA, int P, bool mixed, const AsmArgs& a, int64_t T, int threads, int pos_bytes, \
                              cudaStream_t st);                                                                   \
  lfem_status run_stage_d##DD(int NA, int P, int kind, const StageArgs& s, cudaStream_t st);                     \
  lfem_status run_adjoint_d##DD(int NA, int P, const AdjArgs& a, int64_t T, int pos_bytes, cudaStream_t st);     \
  size_t tile_smem_d##DD(int NA, int P, bool mixed, int nm, int slots, int chunk);                             \
  lfem_status bank_upload_d##DD(const void* src, size_t bytes, size_t offset);

LFEM_DECLARE_DIM(1)
LFEM_DECLARE_DIM(2)
LFEM_DECLARE_DIM(3)

// Body of one dimension's dispatch functions over (NA, P).
#define LFEM_DEFINE_CASE_TILES(DD, NN, PP)                                                              \
  if (NA == NN && P == PP)                                                                              \
    return mixed ? launch_tiles<DD, NN, PP, float>(a, T, threads, pos_bytes, st)                        \
                 : launch_tiles<DD, NN, PP, double>(a, T, threads, pos_bytes, st);
#define LFEM_DEFINE_CASE_STAGE(DD, NN, PP) \
  if (NA == NN && P == PP) return launch_stage<DD, NN, PP>(kind, s, st);
#define LFEM_DEFINE_CASE_ADJ(DD, NN, PP) \
  if (NA == NN && P == PP) return launch_adjoint<DD, NN, PP>(a, T, pos_bytes, st);
#define LFEM_DEFINE_CASE_SMEM(DD, NN, PP)                                               \
  if (NA == NN && P == PP)                                                              \
    return mixed ? tile_smem_bytes<DD, NN, PP, float>(nm, slots, chunk)                 \
                 : tile_smem_bytes<DD, NN, PP, double>(nm, slots, chunk);

}  // namespace lfem
