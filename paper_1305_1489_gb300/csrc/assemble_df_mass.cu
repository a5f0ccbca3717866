// K1 of the HDG_MIXED_BF16 assembly: the double-float condensation of assemble_df.cuh with the
// volume masses M_{kappa^-1}, M_c and f^K read formed (FP32, from the split-BF16 tensor-core
// contraction of tc_mass.cu) instead of summed in the kernel; every other step, the launch
// shapes and the outputs are those of HDG_DF32.  A translation unit of its own, so that its
// instantiations compile beside the HDG_DF32 ones.
#include <cstdlib>

#include "assemble_df.cuh"

namespace hdg {

template <int K, bool CONV>
static cudaError_t launch_mass_kc(hdg_mesh* M, const AsmDfArgs& a) {
  int v = M->k1_variant;
  if (const char* ev = std::getenv("HDG_K1_VARIANT")) v = std::atoi(ev);
  if (v == 1) return launch_df_shape<K, 1, CONV, true>(M, a);
  if (K >= 2 && v == 2) return launch_df_shape<K, (K >= 2 ? 2 : 0), CONV, true>(M, a);
  return launch_df_shape<K, 0, CONV, true>(M, a);
}

template <int K>
static cudaError_t launch_mass_k(hdg_mesh* M, const AsmDfArgs& a) {
  return a.beta_q ? launch_mass_kc<K, true>(M, a) : launch_mass_kc<K, false>(M, a);
}

cudaError_t launch_assemble_df_mass(hdg_mesh* M, const float* mass3, int stride) {
  M->rec_df = true;
  AsmDfArgs a = df_args(M);
  a.mass3 = mass3;
  a.m3stride = stride;
  switch (M->k) {
    case 1: return launch_mass_k<1>(M, a);
    case 2: return launch_mass_k<2>(M, a);
    case 3: return launch_mass_k<3>(M, a);
    case 4: return launch_mass_k<4>(M, a);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hdg
