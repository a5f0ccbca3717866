// K1 in double-float arithmetic (precision HDG_DF32): the launchers of the kernel in
// assemble_df.cuh (its launch shapes per degree, with and without convection) and the
// per-mesh element geometry.
#include <cstdlib>

#include "assemble_df.cuh"

namespace hdg {

template <int K, bool CONV>
static cudaError_t launch_df_kc(hdg_mesh* M, const AsmDfArgs& a) {
  // HDG_K1_VARIANT overrides the tuned shape (tests of every shape, profiling)
  int v = M->k1_variant;
  if (const char* ev = std::getenv("HDG_K1_VARIANT")) v = std::atoi(ev);
  if (v == 1) return launch_df_shape<K, 1, CONV>(M, a);
  if (K >= 2 && v == 2) return launch_df_shape<K, (K >= 2 ? 2 : 0), CONV>(M, a);
  return launch_df_shape<K, 0, CONV>(M, a);
}

template <int K>
static cudaError_t launch_df_k(hdg_mesh* M, const AsmDfArgs& a) {
  return a.beta_q ? launch_df_kc<K, true>(M, a) : launch_df_kc<K, false>(M, a);
}

int k1_variants(int k) { return k == 0 ? 1 : k >= 2 ? 3 : 2; }
int k1_threads(int k, int variant) {
  switch (k) {
    case 0: return K1Occupancy<0>::NT;  // k = 0 runs the FP64 kernel
    case 1: return variant ? K1Shape<1, 1>::NT : K1Shape<1, 0>::NT;
    case 2: return variant == 2 ? K1Shape<2, 2>::NT : variant ? K1Shape<2, 1>::NT : K1Shape<2, 0>::NT;
    case 3: return variant == 2 ? K1Shape<3, 2>::NT : variant ? K1Shape<3, 1>::NT : K1Shape<3, 0>::NT;
    default: return variant == 2 ? K1Shape<4, 2>::NT : variant ? K1Shape<4, 1>::NT : K1Shape<4, 0>::NT;
  }
}

// Element geometry of the mesh, once (it depends on the vertices only): per element
// [a (9, row-major) | normals (4 x 3) | areas (4) | vol], FP64.
__global__ void geometry_kernel(const double* __restrict__ vx, int64_t nelt, double* __restrict__ geo) {
  const int64_t K = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nelt) return;
  Geo g;
  element_geometry(vx, nelt, K, g);
  double* o = geo + K * kGeoStride;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o[3 * i + j] = g.a[i][j];
  for (int l = 0; l < 4; ++l) {
    for (int d = 0; d < 3; ++d) o[9 + 3 * l + d] = g.nrm[l][d];
    o[21 + l] = g.area[l];
  }
  o[25] = g.vol;
  o[26] = g.det;
  o[27] = 0.0;
}

cudaError_t launch_geometry(hdg_mesh* M) {
  const unsigned nb = (unsigned)((M->nelt + 127) / 128);
  geometry_kernel<<<nb, 128, 0, M->stream>>>(M->d_vx, M->nelt, M->d_geo);
  M->launches++;
  return cudaGetLastError();
}

AsmDfArgs df_args(hdg_mesh* M) {
  AsmDfArgs a;
  a.geo = M->d_geo;
  a.perm = M->d_perm;
  a.kappa = M->kappa;
  a.c = M->c;
  a.f = M->f;
  a.tau = M->tau;
  a.P = reinterpret_cast<const df*>(M->dt.P_df);
  a.Chat = reinterpret_cast<const df*>(M->dt.Chat_df);
  a.S = reinterpret_cast<const df*>(M->dt.S_df);
  a.E = reinterpret_cast<const df*>(M->dt.E_df);
  a.AA = reinterpret_cast<const df*>(M->dt.sfAA_df);
  a.BB = reinterpret_cast<const df*>(M->dt.sfBB_df);
  a.CC = reinterpret_cast<const df*>(M->dt.sfCC_df);
  a.p2to1 = M->dt.sfp2to1;
  a.p3to2 = M->dt.sfp3to2;
  a.beta_q = M->beta_q;
  a.beta_f = M->beta_f;
  a.Pd = reinterpret_cast<const df*>(M->dt.Pd_df);
  a.Pl = reinterpret_cast<const df*>(M->dt.Pl_df);
  a.Dmu = reinterpret_cast<const df*>(M->dt.Dmu_df);
  a.wf = M->dt.face_w;
  a.w_df = reinterpret_cast<const df*>(M->dt.vol_w_df);
  a.wf_df = reinterpret_cast<const df*>(M->dt.face_w_df);
  a.w = M->dt.vol_w;
  a.pairs_n = M->dt.pairs_n;
  a.pairs_m = M->dt.pairs_m;
  a.C = M->d_C;
  a.Cf = M->d_Cf;
  a.rec = M->d_rec;
  a.nu = M->method == HDG_METHOD_BDM ? M->tab.n - M->tab.d2 : M->tab.n;
  a.status = M->d_status;
  a.nelt = M->nelt;
  a.mass3 = nullptr;
  a.m3stride = 0;
  a.e0 = 0;
  a.count = M->nelt;
  return a;
}

// the condensation of elements e0 .. e0 + count - 1 only (pipelined host-input assembly)
cudaError_t launch_assemble_df_range(hdg_mesh* M, int64_t e0, int64_t count) {
  if (M->k == 0 || count <= 0) return cudaErrorInvalidValue;
  M->rec_df = true;
  AsmDfArgs a = df_args(M);
  a.e0 = e0;
  a.count = count;
  switch (M->k) {
    case 1: return launch_df_k<1>(M, a);
    case 2: return launch_df_k<2>(M, a);
    case 3: return launch_df_k<3>(M, a);
    case 4: return launch_df_k<4>(M, a);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_assemble_df(hdg_mesh* M) {
  if (M->k == 0) return launch_assemble(M);  // k = 0: the FP64 kernel (d3 = 1, nothing to gain)
  M->rec_df = true;
  const AsmDfArgs a = df_args(M);
  switch (M->k) {
    case 1: return launch_df_k<1>(M, a);
    case 2: return launch_df_k<2>(M, a);
    case 3: return launch_df_k<3>(M, a);
    case 4: return launch_df_k<4>(M, a);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hdg
