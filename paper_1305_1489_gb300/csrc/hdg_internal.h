// Internal declarations of libhdg (host tables, mesh handle, kernel launchers).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hdg.h"

namespace hdg {

struct Coarse;

// ------------------------------------------------------------------ reference tables
// Host copies, row-major.  Built once per degree k (tables.cpp).
struct Tables {
  int k = 0, n = 0, d2 = 0, m = 0, nq = 0, nf = 0, n1 = 0;
  int rule = 0;  // volume rule: 0 conical product ((k+2)^3 nodes), 1 symmetric (Grundmann-Moller)
  std::vector<double> vol_pts;  // [nq][3]   p_hat_q                      (eq. 3.1)
  std::vector<double> vol_w;    // [nq]      omega_hat_q, sum = 1         (eq. 3.1)
  std::vector<double> lam;      // [nq][4]   barycentrics Lambda          (eq. 3.4)
  std::vector<double> P;        // [nq][n]   P_hat_j(p_hat_q)             (eq. 3.5)
  std::vector<double> Pd;       // [3][nq][n] d_* P_hat_j(p_hat_q)        (eq. 3.66)
  std::vector<double> Chat;     // [3][n][n] C_hat^*                      (eq. 3.7)
  std::vector<double> face_pts; // [nf][2]   q_hat_r = (s, t)
  std::vector<double> face_w;   // [nf]      varpi_r, sum = 1
  std::vector<double> xi;       // [nf][3]   barycentrics Xi              (eq. 6.2)
  std::vector<double> Pl;       // [4][nf][n] P_hat_i(q_hat_r^l)          (eq. 4.4)
  std::vector<double> D;        // [nf][d2]  D_hat_i(q_hat_r)             (eq. 4.7)
  std::vector<double> Dmu;      // [6][nf][d2] D_hat_i(F_mu(q_hat_r))     (Section 4, type (c))
  std::vector<double> S;        // [4][n][n] (varpi . P^l)^T P^l          (eq. 4.5)
  std::vector<double> E;        // [4][6][d2][n] (varpi . D^mu)^T P^l     (eq. 4.10)
  std::vector<double> P1;       // [nq][n1]  degree-(k+1) basis at the volume nodes
  std::vector<double> G1;       // [3][nq][n1] its reference gradients
  std::vector<double> Shat1;    // [6][n1][n1] (1/6) sum_q w d_# P'_i d_% P'_j, (#,%) in
                                //   xx, xy, xz, yy, yz, zz  (stiffness of eq. 9.11)
  // Sum factorisation of the volume masses: P_a at the conical node (i, j, l) is
  // A_pa(l) B_(pa,qa)(j) C_a(i), so sum_q g_q P_a P_b = sum_i CC_ab(i) sum_j BB(j) sum_l g AA(l).
  // Pair lists: 1-D (pa <= pb) over 0..k; 2-D (a2 <= b2) over the (p, q), p + q <= k, listed
  // p-major from (0, 0); 3-D the (a <= b) pairs of P_k(K) in row-major order (pairs_n).
  int np1 = 0, np2 = 0;
  std::vector<double> sfAA;       // [np1][k+2]  A_pa(l) A_pb(l)
  std::vector<double> sfBB;       // [np2][k+2]  B_a2(j) B_b2(j)
  std::vector<double> sfCC;       // [n(n+1)/2][k+2]  C_a(i) C_b(i)
  std::vector<int16_t> sfp2to1;   // [np2]  1-D pair (p_a2, p_b2) of each 2-D pair
  std::vector<int16_t> sfp3to2;   // [n(n+1)/2]  2-D pair ((pa, qa), (pb, qb)) of each 3-D pair
};

bool build_tables(int k, Tables* t, std::string* err, int rule = 0);
int symmetric_rule_nodes(int k);  // nodes of the symmetric volume rule of degree k
int d3_of(int k);
int d2_of(int k);

// ------------------------------------------------------------------ device table copies
struct DevTables {
  double *P = nullptr, *Pd = nullptr, *Chat = nullptr, *S = nullptr, *E = nullptr;
  double *vol_w = nullptr, *lam = nullptr, *face_w = nullptr, *xi = nullptr, *D = nullptr;
  double *P1 = nullptr, *G1 = nullptr, *Shat1 = nullptr, *Pl = nullptr, *Dmu = nullptr, *face_pts = nullptr;
  // double-float (hi, lo) float pairs of P, C_hat, S, E for the HDG_DF32 assembly
  float *P_df = nullptr, *Chat_df = nullptr, *S_df = nullptr, *E_df = nullptr;
  float *sfAA_df = nullptr, *sfBB_df = nullptr, *sfCC_df = nullptr;  // sum-factorisation tables
  float *G1_df = nullptr, *Shat1_df = nullptr;  // double-float postprocess tables
  float *Pd_df = nullptr, *Pl_df = nullptr, *Dmu_df = nullptr;  // double-float convection tables
  float *vol_w_df = nullptr, *face_w_df = nullptr;  // double-float quadrature weights
  int16_t *sfp2to1 = nullptr, *sfp3to2 = nullptr;
  int16_t* pairs_n = nullptr;   // [n(n+1)/2][2]  (i <= j) pairs of P_k(K) indices
  int16_t* pairs_m = nullptr;   // [m(m+1)/2][2]  (r <= s) pairs of R_k(dK) indices
  int16_t* pairs_n1 = nullptr;  // [(n1-1) n1 / 2][2] pairs of 1..n1-1 (postprocess)
};

}  // namespace hdg

// ------------------------------------------------------------------ mesh handle
struct hdg_mesh {
  int k = 0;
  hdg::Tables tab;
  hdg::DevTables dt;
  int64_t nelt = 0, nfc = 0, nver = 0, ndir = 0, nneu = 0;
  cudaStream_t stream = nullptr;
  int64_t launches = 0;

  // host expanded mesh
  std::vector<int32_t> h_faces;      // [nfc][4]
  std::vector<int32_t> h_facebyele;  // [nelt][4]
  std::vector<int32_t> h_perm;       // [nelt][4] in 1..6

  // device mesh
  double* d_vx = nullptr;         // [12][nelt] SoA: x1..x4, y1..y4, z1..z4
  double* d_geo = nullptr;        // [nelt][kGeoStride] cofactors a (9), normals (12), areas (4), vol
  double* d_fvx = nullptr;        // [9][nfc]   SoA: sorted face vertices x1..x3, y1..y3, z1..z3
  int32_t* d_fverts = nullptr;    // [nfc][3]   sorted face vertex numbers (coarse prolongation)
  double* d_Tproj = nullptr;      // [d2][3]    (varpi . D)^T Xi: linear face data -> face basis
  int32_t* d_facebyele = nullptr; // [nelt][4]
  int32_t* d_perm = nullptr;      // [nelt][4]
  int32_t* d_owner = nullptr;     // [nfc][2]   4*K + l of the (up to) two elements, -1 if none
  int32_t* d_fslot = nullptr;     // [nelt][4]  2 f + side (which owner of face f the element is)
  int32_t* d_ftype = nullptr;     // [nfc]      0 interior, 1 Dirichlet, 2 Neumann

  // borrowed coefficient / data pointers (device)
  const double *kappa = nullptr, *c = nullptr, *f = nullptr, *tau = nullptr;
  const double *beta_q = nullptr;  // [3][nelt][nq] convection at the volume nodes, or NULL
  const double *beta_f = nullptr;  // [3][nelt][4][nf] convection at the element face nodes
  const double *uD = nullptr, *gN = nullptr;

  // products of hdg_assemble_condense (library-owned)
  bool assembled = false;
  double* d_C = nullptr;    // [nelt][m][m] condensed C^K, row-major (eq. 5.5)
  double* d_Cf = nullptr;   // [nelt][m]    C_f^K (eq. 5.6)
  double* d_rec = nullptr;  // [nelt][rec_stride] recovery operators (eq. 5.3)
  int64_t rec_stride = 0;
  bool rec_df = false;      // the record holds double-float pairs (written by the double-float K1)
  int method = 0;           // HDG_METHOD_HDG or HDG_METHOD_BDM (hdg_set_method)
  int32_t* d_status = nullptr;  // [8] error counters written by kernels
  double* d_norm = nullptr;     // partial sums of the error norms (allocated on first use)

  // trace-solve workspace (library-owned, allocated on first solve)
  bool rhs_ready = false;
  bool bj64_ready = false, bj32_ready = false;  // block-Jacobi inverses of the current system
  bool c32_ready = false;                       // FP32 copy of C^K of the current assembly
  double bnorm = 0.0;  // ||b||_2 of the current right-hand side (host copy)
  double inner_rtol = 1e-4;  // relative tolerance of each FP32 inner solve (mixed precision)
  double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr,
         *d_q = nullptr, *d_uhatD = nullptr, *d_BJ = nullptr, *d_red = nullptr,
         *d_scal = nullptr;
  unsigned int* d_counter = nullptr;
  float *d_C32 = nullptr, *d_BJ32 = nullptr, *d_r32 = nullptr, *d_x32 = nullptr,
        *d_z32 = nullptr, *d_p32 = nullptr, *d_q32 = nullptr;
  int red_blocks = 0;
  cudaGraphExec_t graph64 = nullptr, graph32 = nullptr, graph_bicg = nullptr;
  double* d_bicg = nullptr;  // [4][nfc][d2] extra BiCGStab vectors (s, t, ph, sh)
  float* d_bicg32 = nullptr; // the same for the FP32 inner BiCGStab of the mixed solve
  cudaGraphExec_t graph_bicg32 = nullptr, wgraph_bicg = nullptr, wgraph_bicg32 = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  cudaGraphExec_t wgraph64 = nullptr, wgraph32 = nullptr;  // device-driven (conditional WHILE) PCG loops
  bool no_cond_graphs = false;  // the driver refused conditional nodes: host-driven loop
  int graph_iters = 0;
  int face_blocks = 1216;         // persistent grid of the face kernels (hdg_autotune)
  int face_blocks32 = 1216;       // the same for the FP32 inner iterations
  int grid_cap = 0;               // > 0: cap on the grids of the coarse-level kernels (HDG_FACE_BLOCKS)
  // form of the operator H x in the solve loops: element-major pass + face sum (true) or one
  // face-major pass (false), per precision; hdg_autotune measures both unless HDG_MATVEC fixed it.
  // FP64 defaults to the face-major form, the one its residual checks use (the FP64 product is
  // bound by the FP64 pipe, where the element pass gains nothing), FP32 to the element pass
  bool em64 = false, em32 = true;
  bool em_forced = false;
  int graphs_em = -1;             // (em64, em32) of the cached graphs
  double* d_Y = nullptr;          // [2][nvp] element-pass output per face side, FP64 ...
  float* d_Y32 = nullptr;         // ... and FP32 (nvp = nfc d2 rounded up to 4)
  // HDG_MIXED_BF16 assembly: the split pair-product table of the tensor-core contraction (for
  // the volume rule mass3_rule) and the per-element FP32 masses [nelt][mass3_stride(k)]
  void* d_mass3B = nullptr;
  int mass3_rule = -1;
  float* d_mass3 = nullptr;
  // library-owned device copies of host inputs (hdg_assemble_condense_host) and outputs
  // (hdg_recover_host), and the stream that moves them beside the kernels
  double *in_kappa = nullptr, *in_c = nullptr, *in_f = nullptr, *in_beta = nullptr, *in_betaf = nullptr,
         *in_tau = nullptr, *in_uD = nullptr, *in_gN = nullptr, *out_q = nullptr, *out_u = nullptr;
  cudaStream_t copy_stream = nullptr;
  int k1_variant = 0;             // launch shape of the double-float K1 (hdg_autotune)
  int asm_prec = -1;              // precision of the last hdg_assemble_condense
  hdg::Coarse* coarse = nullptr;  // two-level preconditioner (hdg_set_coarse_space), or NULL
  bool graphs_tl = false;         // the cached PCG graphs include the coarse correction
  int coarse_gen = 0;             // incremented by every hdg_set_coarse_space
};

namespace hdg {
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define HDG_CUDA_TRY(expr)                                                               \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return ::hdg::fail(HDG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// kernel launchers (defined in the .cu files); return cudaGetLastError()
cudaError_t launch_qnodes(hdg_mesh* M, double* X, double* Y, double* Z, double* FX, double* FY,
                          double* FZ);
cudaError_t launch_assemble(hdg_mesh* M);
cudaError_t launch_assemble_df(hdg_mesh* M);
cudaError_t launch_assemble_df_mass(hdg_mesh* M, const float* mass3, int stride);
cudaError_t launch_assemble_df_range(hdg_mesh* M, int64_t e0, int64_t count);
cudaError_t launch_recover_range(hdg_mesh* M, const double* uhat, double* q, double* u, int64_t e0, int64_t count);
int mass3_contraction(hdg_mesh* M, float* out);  // tc_mass.cu
int mass3_stride(int k);
cudaError_t launch_projection(hdg_mesh* M, const double* q_vol, const double* u_vol, const double* q_face,
                              const double* u_face, double* Pq, double* Pu);
cudaError_t launch_face_projection(hdg_mesh* M, const double* vals, double* Pu);
cudaError_t launch_volume_norm2(hdg_mesh* M, int degree, const double* coef, const double* vals, double* out_host);
cudaError_t launch_face_norm2(hdg_mesh* M, const double* coef, const double* vals, double* out_host);
constexpr int kGeoStride = 28;  // doubles per element of d_geo (26 used; 224 bytes, 32-byte aligned rows)
cudaError_t launch_geometry(hdg_mesh* M);
cudaError_t launch_recover(hdg_mesh* M, const double* uhat, double* q, double* u);
cudaError_t launch_element_face_nodes(hdg_mesh* M, double* X, double* Y, double* Z);
cudaError_t launch_postprocess(hdg_mesh* M, const double* q, const double* u, double* ustar);
int solve_trace(hdg_mesh* M, int precision, double rtol, int maxit, const double* x0,
                double* uhat, int* iters, double* relres);
int trace_residual(hdg_mesh* M, const double* x, double* r, double* rnorm, double* bnorm);
int trace_apply(hdg_mesh* M, const double* x, double* y);
int batch_record_group(hdg_mesh* M, cudaGraph_t graph, int asm_precision, int solve_precision, const int32_t* face_prob, int np,
                       double* norms, double rtol, int maxit, double* q, double* u, double* uhat, cudaGraphNode_t* last);
int batch_group_iterations(hdg_mesh* M, int* iters, int* status);
int build_mesh(hdg_mesh* M, const double* coords, const int32_t* elems, const int32_t* dir, const int32_t* neu);
int ensure_face_verts(hdg_mesh* M);   // d_fverts and d_Tproj (coarse prolongation)
int coarse_build(hdg_mesh* M);        // Galerkin hierarchy of the two-level preconditioner
int coarse_launch_build(hdg_mesh* M); // the same, enqueued on M->stream without synchronising
void coarse_free(hdg_mesh* M);
void coarse_invalidate(hdg_mesh* M);  // the Galerkin values must be rebuilt (new assembly)
int coarse_precond_apply(hdg_mesh* M, const double* r, double* z);
int autotune_face_grid(hdg_mesh* M, hdg_tuning* out);
int k1_variants(int k);              // launch shapes of the double-float K1 for degree k
int k1_threads(int k, int variant);  // threads per element of a shape
// the double-float K1 over every shape of the mesh (assemble_df_lean.cu): the shapes of
// assemble_df.cu first, then those of the kernel that streams W_* (reaction-diffusion, k = 4)
int k1_shape_count(const hdg_mesh* M);
int k1_shape_threads(const hdg_mesh* M, int variant);
cudaError_t launch_k1(hdg_mesh* M);
cudaError_t launch_k1_range(hdg_mesh* M, int64_t e0, int64_t count);
}  // namespace hdg
