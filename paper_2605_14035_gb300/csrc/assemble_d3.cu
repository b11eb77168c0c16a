// Kernels for elements of dimension 3 (all supported ambient dimensions, orders 1 and 2).
#include "assemble_tet2.cuh"
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
  if (P == 2) {
    if (mixed && fast) {
      Tet2Pack pk;
      tet2_pack_host(fb.v + FastBankTet::OFF32, pk);
      return launch_tet2(a, pk, sms, st);
    }
    return mixed ? launch_twopass<3, 3, 2, float>(a, false, fb, sms, st) : launch_twopass<3, 3, 2, double>(a, false, fb, sms, st);
  }
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

void tet2_pack_host(const float* fl, Tet2Pack& out) {
  using L = FastLayout<3, 2>;
  using T = Tet2Pack;
  for (int i = 0; i < T::SIZE; ++i) out.v[i] = 0.f;
  for (int q = 0; q < T::Q; ++q) {
    float* o = out.v + q * T::PER_Q;
    for (int k = 0; k < T::NE; ++k)
      for (int m = 0; m < 3; ++m) o[T::DPS + 2 * (3 * k + m)] = o[T::DPS + 2 * (3 * k + m) + 1] = fl[L::dpsi(q, k, m)];
    for (int b = 0; b < T::REF; ++b)
      for (int m = 0; m < 3; ++m) o[T::DPD + 2 * (3 * b + m)] = o[T::DPD + 2 * (3 * b + m) + 1] = fl[L::dphi(q, b, m)];
    for (int j = 0; j < T::NJ; ++j)
      for (int n = 0; n < 3; ++n) {
        o[T::DPP + 2 * (3 * j + n)] = fl[L::dphi(q, 2 * j, n)];
        o[T::DPP + 2 * (3 * j + n) + 1] = fl[L::dphi(q, 2 * j + 1, n)];
      }
    o[T::WQ] = fl[L::w(q)];
    for (int u = 0; u < T::U; ++u) out.v[T::TM2 + 2 * q * T::UH + u] = fl[L::tm(q, u)];
  }
}

lfem_status bank_upload_d3(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
