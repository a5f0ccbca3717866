// C ABI of libhdg (declared in include/hdg.h): argument checking, ownership, dispatch.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include <algorithm>

#include "hdg_internal.h"

namespace hdg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int build_mesh(hdg_mesh* M, const double* coords, const int32_t* elems, const int32_t* dir,
               const int32_t* neu);
int build_mesh_host(hdg_mesh* M, const double* coords, const int32_t* elems, const int32_t* dir,
                    const int32_t* neu, std::vector<int32_t>* owner_out);
int64_t rec_stride_of(int k);

template <typename T>
static int upload(T** d, const std::vector<T>& h) {
  HDG_CUDA_TRY(cudaMalloc(d, sizeof(T) * (h.empty() ? 1 : h.size())));
  if (!h.empty()) HDG_CUDA_TRY(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

static std::vector<int16_t> pair_list(int n, int first) {
  std::vector<int16_t> v;
  for (int i = first; i < n; ++i)
    for (int j = i; j < n; ++j) {
      v.push_back((int16_t)(i - first));
      v.push_back((int16_t)(j - first));
    }
  return v;
}

// split each double into the float pair hi + lo (hi = nearest float, lo = nearest float of
// the remainder) for the double-float kernels
static std::vector<float> split_df(const std::vector<double>& v) {
  std::vector<float> o(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float hi = (float)v[i];
    o[2 * i] = hi;
    o[2 * i + 1] = (float)(v[i] - (double)hi);
  }
  return o;
}

static int upload_tables(hdg_mesh* M) {
  const Tables& T = M->tab;
  DevTables& D = M->dt;
  int rc;
  if ((rc = upload(&D.P, T.P)) || (rc = upload(&D.Pd, T.Pd)) || (rc = upload(&D.Chat, T.Chat)) ||
      (rc = upload(&D.S, T.S)) || (rc = upload(&D.E, T.E)) || (rc = upload(&D.vol_w, T.vol_w)) ||
      (rc = upload(&D.lam, T.lam)) || (rc = upload(&D.face_w, T.face_w)) || (rc = upload(&D.xi, T.xi)) ||
      (rc = upload(&D.D, T.D)) || (rc = upload(&D.P1, T.P1)) || (rc = upload(&D.G1, T.G1)) ||
      (rc = upload(&D.Shat1, T.Shat1)) || (rc = upload(&D.Pl, T.Pl)) || (rc = upload(&D.Dmu, T.Dmu)) ||
      (rc = upload(&D.face_pts, T.face_pts)))
    return rc;
  if ((rc = upload(&D.P_df, split_df(T.P))) || (rc = upload(&D.Chat_df, split_df(T.Chat))) ||
      (rc = upload(&D.S_df, split_df(T.S))) || (rc = upload(&D.E_df, split_df(T.E))) ||
      (rc = upload(&D.sfAA_df, split_df(T.sfAA))) || (rc = upload(&D.sfBB_df, split_df(T.sfBB))) ||
      (rc = upload(&D.sfCC_df, split_df(T.sfCC))) || (rc = upload(&D.sfp2to1, T.sfp2to1)) ||
      (rc = upload(&D.sfp3to2, T.sfp3to2)) || (rc = upload(&D.G1_df, split_df(T.G1))) ||
      (rc = upload(&D.Shat1_df, split_df(T.Shat1))) || (rc = upload(&D.Pd_df, split_df(T.Pd))) ||
      (rc = upload(&D.Pl_df, split_df(T.Pl))) || (rc = upload(&D.Dmu_df, split_df(T.Dmu))) ||
      (rc = upload(&D.vol_w_df, split_df(T.vol_w))) || (rc = upload(&D.face_w_df, split_df(T.face_w))))
    return rc;
  if ((rc = upload(&D.pairs_n, pair_list(T.n, 0))) || (rc = upload(&D.pairs_m, pair_list(T.m, 0))) ||
      (rc = upload(&D.pairs_n1, pair_list(T.n1, 1))))
    return rc;
  return HDG_OK;
}

// the device copies of the reference tables
static void free_tables(hdg_mesh* M) {
  DevTables& D = M->dt;
  void* ptrs[] = {D.P, D.Pd, D.Chat, D.S, D.E, D.vol_w, D.lam, D.face_w, D.xi, D.D, D.P1, D.G1, D.Shat1, D.pairs_n,
                  D.pairs_m, D.pairs_n1, D.Pl, D.Dmu, D.face_pts, D.P_df, D.Chat_df, D.S_df, D.E_df, D.sfAA_df,
                  D.sfBB_df, D.sfCC_df, D.sfp2to1, D.sfp3to2, D.G1_df, D.Shat1_df, D.Pd_df, D.Pl_df, D.Dmu_df,
                  D.vol_w_df, D.face_w_df};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  D = DevTables();
}

static void release(hdg_mesh* M) {
  coarse_free(M);
  free_tables(M);
  void* ptrs[] = {M->d_vx, M->d_geo, M->d_fvx, M->d_facebyele, M->d_perm, M->d_owner, M->d_ftype, M->d_C, M->d_Cf,
                  M->d_rec, M->d_status, M->d_b, M->d_x, M->d_r, M->d_z, M->d_p, M->d_q, M->d_uhatD, M->d_BJ,
                  M->d_red, M->d_scal, M->d_counter, M->d_C32, M->d_BJ32, M->d_r32, M->d_x32, M->d_z32,
                  M->d_p32, M->d_q32, M->d_bicg, M->d_fverts, M->d_Tproj, M->d_norm, M->d_bicg32, M->d_Y,
                  M->d_mass3B, M->d_mass3, M->d_fslot, M->d_Y32, M->in_kappa, M->in_c, M->in_f, M->in_beta,
                  M->in_betaf, M->in_tau, M->in_uD, M->in_gN, M->out_q, M->out_u};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (M->graph64) cudaGraphExecDestroy(M->graph64);
  if (M->graph32) cudaGraphExecDestroy(M->graph32);
  if (M->graph_bicg) cudaGraphExecDestroy(M->graph_bicg);
  if (M->graph_bicg32) cudaGraphExecDestroy(M->graph_bicg32);
  if (M->wgraph_bicg) cudaGraphExecDestroy(M->wgraph_bicg);
  if (M->wgraph_bicg32) cudaGraphExecDestroy(M->wgraph_bicg32);
  if (M->wgraph64) cudaGraphExecDestroy(M->wgraph64);
  if (M->wgraph32) cudaGraphExecDestroy(M->wgraph32);
  if (M->cap_stream) cudaStreamDestroy(M->cap_stream);
  if (M->copy_stream) cudaStreamDestroy(M->copy_stream);
}

static int check_status(hdg_mesh* M) {
  int32_t st[8];
  HDG_CUDA_TRY(cudaMemcpyAsync(st, M->d_status, sizeof(st), cudaMemcpyDeviceToHost, M->stream));
  HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
  if (st[7]) {  // counted by the element pass of the trace operator; reported once
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 7, 0, sizeof(int32_t), M->stream));
    return fail(HDG_ERR_CUDA, std::to_string(st[7]) + " element-pass block(s) whose C^K copies did not complete "
                                                      "within the wait limit (the solution is not valid)");
  }
  if (st[4]) {  // counted by the double-float recovery kernel; reported once
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 4, 0, sizeof(int32_t), M->stream));
    return fail(HDG_ERR_CUDA, std::to_string(st[4]) + " element(s) whose recovery record copy did not complete (q, u set to NaN)");
  }
  if (st[1]) return fail(HDG_ERR_COEFF, std::to_string(st[1]) + " element(s) with kappa <= 0, c < 0 or non-finite data");
  if (st[0]) return fail(HDG_ERR_LOCAL_SINGULAR, std::to_string(st[0]) + " element(s) with a non-positive local pivot");
  if (st[2]) return fail(HDG_ERR_LOCAL_SINGULAR, std::to_string(st[2]) + " element(s) with a singular postprocess system");
  if (st[3]) return fail(HDG_ERR_LOCAL_SINGULAR, std::to_string(st[3]) + " face block(s) not positive definite");
  return HDG_OK;
}

}  // namespace hdg

using namespace hdg;

extern "C" {

int hdg_mesh_create(const double* coords, int64_t nver, const int32_t* elems, int64_t nelt, const int32_t* dir,
                    int64_t ndir, const int32_t* neu, int64_t nneu, int k, void* stream, hdg_mesh** out) {
  if (!out) return fail(HDG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!coords || !elems || nver < 4 || nelt < 1 || ndir < 0 || nneu < 0 || (ndir && !dir) || (nneu && !neu))
    return fail(HDG_ERR_ARG, "invalid mesh arrays or sizes");
  if (k < 0 || k > 4) return fail(HDG_ERR_UNSUPPORTED, "degree k must be in 0..4");
  if (nelt > (int64_t)1 << 30) return fail(HDG_ERR_ARG, "too many elements");
  hdg_mesh* M = new (std::nothrow) hdg_mesh();
  if (!M) return fail(HDG_ERR_ARG, "out of host memory");
  M->k = k;
  M->nver = nver;
  M->nelt = nelt;
  M->ndir = ndir;
  M->nneu = nneu;
  M->stream = (cudaStream_t)stream;
  // HDG_HOST_LOOP=1: drive the PCG loop from the host (replays of a plain captured graph)
  // instead of the device-side conditional loop, e.g. for profilers that list graph kernels.
  if (const char* hl = std::getenv("HDG_HOST_LOOP")) M->no_cond_graphs = hl[0] == '1';
  // HDG_FACE_BLOCKS=n: persistent grid of n blocks for the trace-solve kernels (both
  // precisions) and a grid cap of n blocks for the coarse-level kernels, so that small meshes
  // take the multi-tile loops and multi-block reductions that large meshes take.
  if (const char* fb = std::getenv("HDG_FACE_BLOCKS")) {
    const int v = std::atoi(fb);
    if (v > 0) M->face_blocks = M->face_blocks32 = M->grid_cap = v;
  }
  // HDG_MATVEC=face|element: the form of the solve loops' operator products, fixed (the
  // autotuner then leaves it alone)
  if (const char* mv = std::getenv("HDG_MATVEC")) {
    if (std::strcmp(mv, "face") == 0 || std::strcmp(mv, "element") == 0) {
      M->em64 = M->em32 = mv[0] == 'e';
      M->em_forced = true;
    }
  }
  std::string err;
  int rc = HDG_OK;
  if (!build_tables(k, &M->tab, &err)) rc = fail(HDG_ERR_ARG, err);
  if (!rc) rc = build_mesh(M, coords, elems, dir, neu);
  if (!rc) rc = upload_tables(M);
  if (!rc) {
    const int m = M->tab.m;
    M->rec_stride = rec_stride_of(k);
    cudaError_t e = cudaMalloc(&M->d_C, sizeof(double) * nelt * m * m);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_Cf, sizeof(double) * nelt * m);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_rec, sizeof(double) * nelt * M->rec_stride);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_status, sizeof(int32_t) * 8);
    if (e == cudaSuccess) e = cudaMemset(M->d_status, 0, sizeof(int32_t) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&M->d_geo, sizeof(double) * nelt * kGeoStride);
    if (e == cudaSuccess) e = launch_geometry(M);  // the mesh's element geometry, once
    if (e != cudaSuccess) rc = fail(HDG_ERR_CUDA, std::string("device allocation: ") + cudaGetErrorString(e));
  }
  if (rc) {
    release(M);
    delete M;
    return rc;
  }
  *out = M;
  return HDG_OK;
}

int hdg_mesh_destroy(hdg_mesh* M) {
  if (!M) return HDG_OK;
  if (M->stream) cudaStreamSynchronize(M->stream);
  release(M);
  delete M;
  return HDG_OK;
}

int hdg_mesh_get_info(const hdg_mesh* M, hdg_mesh_info* info) {
  if (!M || !info) return fail(HDG_ERR_ARG, "NULL argument");
  info->nelt = M->nelt;
  info->nfc = M->nfc;
  info->ndir = M->ndir;
  info->nneu = M->nneu;
  info->nver = M->nver;
  info->k = M->k;
  info->n = M->tab.n;
  info->d2 = M->tab.d2;
  info->m = M->tab.m;
  info->n1 = M->tab.n1;
  info->nq = M->tab.nq;
  info->nf = M->tab.nf;
  info->has_convection = M->beta_q != nullptr;
  return HDG_OK;
}

int hdg_mesh_get_faces(const hdg_mesh* M, int32_t* faces, int32_t* facebyele, int32_t* perm) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if (faces) std::memcpy(faces, M->h_faces.data(), sizeof(int32_t) * M->h_faces.size());
  if (facebyele) std::memcpy(facebyele, M->h_facebyele.data(), sizeof(int32_t) * M->h_facebyele.size());
  if (perm) std::memcpy(perm, M->h_perm.data(), sizeof(int32_t) * M->h_perm.size());
  return HDG_OK;
}

int hdg_quadrature_nodes(hdg_mesh* M, double* X, double* Y, double* Z, double* FX, double* FY, double* FZ) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if ((X && (!Y || !Z)) || (FX && (!FY || !FZ))) return fail(HDG_ERR_ARG, "incomplete node triple");
  HDG_CUDA_TRY(launch_qnodes(M, X, Y, Z, FX, FY, FZ));
  return HDG_OK;
}

int hdg_set_coefficients(hdg_mesh* M, const double* kappa, const double* c, const double* beta, const double* f,
                         const double* tau) {
  if (!M || !kappa || !c || !f) return fail(HDG_ERR_ARG, "kappa, c and f are required");
  if ((beta != nullptr) != (M->beta_q != nullptr)) {  // switching symmetric <-> non-symmetric
    if (M->graph64) { cudaGraphExecDestroy(M->graph64); M->graph64 = nullptr; }
    if (M->wgraph64) { cudaGraphExecDestroy(M->wgraph64); M->wgraph64 = nullptr; }
  }
  M->beta_q = beta;
  if (!beta) M->beta_f = nullptr;
  M->kappa = kappa;
  M->c = c;
  M->f = f;
  M->tau = tau;
  M->assembled = false;
  M->rhs_ready = false;
  return HDG_OK;
}

int hdg_element_face_nodes(hdg_mesh* M, double* X, double* Y, double* Z) {
  if (!M || !X || !Y || !Z) return fail(HDG_ERR_ARG, "NULL argument");
  HDG_CUDA_TRY(launch_element_face_nodes(M, X, Y, Z));
  return HDG_OK;
}

int hdg_set_face_convection(hdg_mesh* M, const double* beta_f) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  M->beta_f = beta_f;
  M->assembled = false;
  M->rhs_ready = false;
  return HDG_OK;
}

int hdg_set_boundary_data(hdg_mesh* M, const double* uD, const double* gN) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  M->uD = uD;
  M->gN = gN;
  M->rhs_ready = false;
  return HDG_OK;
}

}  // extern "C"

namespace hdg {

// the checks of an assembly request (shared by the device- and host-input entry points)
static int check_assembly(hdg_mesh* M, int precision) {
  if (!M->kappa) return fail(HDG_ERR_STATE, "hdg_set_coefficients was not called");
  if (precision != HDG_FP64 && precision != HDG_DF32 && precision != HDG_MIXED_BF16)
    return fail(HDG_ERR_UNSUPPORTED, "assembly precision must be HDG_FP64, HDG_DF32 or HDG_MIXED_BF16");
  if (M->beta_q && !M->beta_f) return fail(HDG_ERR_STATE, "convection set without hdg_set_face_convection");
  if (M->beta_q && M->method == HDG_METHOD_BDM)
    return fail(HDG_ERR_UNSUPPORTED, "the BDM element is built for reaction-diffusion (beta = 0)");
  if (precision == HDG_DF32 && M->tab.rule != HDG_RULE_CONICAL)
    return fail(HDG_ERR_UNSUPPORTED, "the double-float assembly sums the masses by sum factorisation, which needs "
                                     "the conical volume rule");
  if (precision == HDG_MIXED_BF16 && (M->tab.rule != HDG_RULE_CONICAL || M->k < 1))
    return fail(HDG_ERR_UNSUPPORTED, "the split-BF16 assembly is built for k >= 1 on the conical volume rule");
  if (M->k == 0 && (M->beta_q || M->method == HDG_METHOD_BDM))
    return fail(HDG_ERR_UNSUPPORTED, "k = 0 is built for the HDG method without convection");
  return HDG_OK;
}

// after every assembly: what depended on the previous one is stale; the status is read
static int finish_assembly(hdg_mesh* M, int precision) {
  M->assembled = true;
  M->asm_prec = precision;
  M->c32_ready = false;
  M->bj64_ready = M->bj32_ready = false;
  if (M->coarse) coarse_invalidate(M);
  M->rhs_ready = false;
  return check_status(M);
}

// First element of range ch of nch over nelt elements, the ranges growing by the factor g
// (g = 1: equal ranges).  In the host-input assembly the first range's copy is the only one
// nothing overlaps; a range's copy takes about 0.6 of its condensation at the bench workload
// (208 GB/s against 40 ns per element), so ranges that grow by 1.25 keep the copies ahead
// while the first one shrinks to 0.7 % of the elements at 16 ranges.
static int64_t range_start(int64_t nelt, int nch, int ch, double g) {
  if (ch <= 0) return 0;
  if (ch >= nch) return nelt;
  const double frac = g == 1.0 ? (double)ch / nch : (std::pow(g, ch) - 1.0) / (std::pow(g, nch) - 1.0);
  return std::min<int64_t>(nelt, std::max<int64_t>(0, (int64_t)std::llround(frac * (double)nelt)));
}
constexpr double kAsmRangeGrowth = 1.25;

static int ensure_buffer(double** p, int64_t n) {
  if (!*p) HDG_CUDA_TRY(cudaMalloc(p, sizeof(double) * (n > 0 ? n : 1)));
  return HDG_OK;
}

}  // namespace hdg

extern "C" {

int hdg_assemble_condense(hdg_mesh* M, int precision) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  int rc = check_assembly(M, precision);
  if (rc) return rc;
  HDG_CUDA_TRY(cudaMemsetAsync(M->d_status, 0, sizeof(int32_t) * 4, M->stream));
  if (precision == HDG_MIXED_BF16) {
    const int stride = mass3_stride(M->k);
    if (!M->d_mass3) HDG_CUDA_TRY(cudaMalloc(&M->d_mass3, sizeof(float) * M->nelt * stride));
    rc = mass3_contraction(M, M->d_mass3);
    if (rc) return rc;
    int32_t st6 = 0;
    HDG_CUDA_TRY(cudaMemcpyAsync(&st6, M->d_status + 6, sizeof(int32_t), cudaMemcpyDeviceToHost, M->stream));
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    if (st6) return fail(HDG_ERR_CUDA, "tensor-core contraction: an MMA did not complete within the wait limit");
    HDG_CUDA_TRY(launch_assemble_df_mass(M, M->d_mass3, stride));
  } else {
    HDG_CUDA_TRY(precision == HDG_DF32 ? launch_k1(M) : launch_assemble(M));
  }
  return finish_assembly(M, precision);
}

int hdg_assemble_condense_host(hdg_mesh* M, int precision, const hdg_host_inputs* in, int chunks) {
  if (!M || !in || !in->kappa || !in->c || !in->f) return fail(HDG_ERR_ARG, "kappa, c and f are required");
  if ((in->beta == nullptr) != (in->beta_f == nullptr))
    return fail(HDG_ERR_ARG, "beta and beta_f are given together or not at all");
  const int64_t nelt = M->nelt, nq = M->tab.nq, nf = M->tab.nf, nfc = M->nfc;
  int rc;
  if ((rc = ensure_buffer(&M->in_kappa, nelt * nq)) || (rc = ensure_buffer(&M->in_c, nelt * nq)) ||
      (rc = ensure_buffer(&M->in_f, nelt * nq)))
    return rc;
  if (in->beta && ((rc = ensure_buffer(&M->in_beta, 3 * nelt * nq)) || (rc = ensure_buffer(&M->in_betaf, 12 * nelt * nf))))
    return rc;
  if (in->tau && (rc = ensure_buffer(&M->in_tau, 4 * nelt))) return rc;
  if (in->uD && (rc = ensure_buffer(&M->in_uD, nfc * nf))) return rc;
  if (in->gN && (rc = ensure_buffer(&M->in_gN, 3 * nfc * nf))) return rc;
  // from here on the mesh reads its inputs from the library's copies
  if ((rc = hdg_set_coefficients(M, M->in_kappa, M->in_c, in->beta ? M->in_beta : nullptr, M->in_f,
                                 in->tau ? M->in_tau : nullptr)))
    return rc;
  if (in->beta && (rc = hdg_set_face_convection(M, M->in_betaf))) return rc;
  if ((in->uD || in->gN) &&
      (rc = hdg_set_boundary_data(M, in->uD ? M->in_uD : nullptr, in->gN ? M->in_gN : nullptr)))
    return rc;
  if ((rc = check_assembly(M, precision))) return rc;
  if (!M->copy_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->copy_stream, cudaStreamNonBlocking));
  cudaStream_t cs = M->copy_stream;
  const size_t d = sizeof(double);
  // the copy stream starts after the work already queued on the mesh stream (which may read
  // the buffers being refilled)
  cudaEvent_t ev0;
  HDG_CUDA_TRY(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  HDG_CUDA_TRY(cudaEventRecord(ev0, M->stream));
  HDG_CUDA_TRY(cudaStreamWaitEvent(cs, ev0, 0));
  cudaEventDestroy(ev0);
  if (in->tau) HDG_CUDA_TRY(cudaMemcpyAsync(M->in_tau, in->tau, d * 4 * nelt, cudaMemcpyHostToDevice, cs));
  // pipelined: the double-float condensation of each chunk of elements starts as soon as the
  // chunk's inputs have landed, while the next chunk is copied
  const bool pipe = precision == HDG_DF32 && M->k >= 1;
  const int nch = pipe ? std::max(1, std::min<int>(chunks, (int)std::min<int64_t>(nelt, 1024))) : 1;
  if (pipe) HDG_CUDA_TRY(cudaMemsetAsync(M->d_status, 0, sizeof(int32_t) * 4, M->stream));
  std::vector<cudaEvent_t> evs(nch, nullptr);
  for (int ch = 0; ch < nch; ++ch) {
    const int64_t e0 = range_start(nelt, nch, ch, kAsmRangeGrowth);
    const int64_t ne = range_start(nelt, nch, ch + 1, kAsmRangeGrowth) - e0;
    if (ne <= 0) continue;
    HDG_CUDA_TRY(cudaMemcpyAsync(M->in_kappa + e0 * nq, in->kappa + e0 * nq, d * ne * nq, cudaMemcpyHostToDevice, cs));
    HDG_CUDA_TRY(cudaMemcpyAsync(M->in_c + e0 * nq, in->c + e0 * nq, d * ne * nq, cudaMemcpyHostToDevice, cs));
    HDG_CUDA_TRY(cudaMemcpyAsync(M->in_f + e0 * nq, in->f + e0 * nq, d * ne * nq, cudaMemcpyHostToDevice, cs));
    if (in->beta)
      for (int st = 0; st < 3; ++st) {
        HDG_CUDA_TRY(cudaMemcpyAsync(M->in_beta + (st * nelt + e0) * nq, in->beta + (st * nelt + e0) * nq,
                                     d * ne * nq, cudaMemcpyHostToDevice, cs));
        HDG_CUDA_TRY(cudaMemcpyAsync(M->in_betaf + (st * nelt + e0) * 4 * nf, in->beta_f + (st * nelt + e0) * 4 * nf,
                                     d * ne * 4 * nf, cudaMemcpyHostToDevice, cs));
      }
    if (pipe) {
      HDG_CUDA_TRY(cudaEventCreateWithFlags(&evs[ch], cudaEventDisableTiming));
      HDG_CUDA_TRY(cudaEventRecord(evs[ch], cs));
      HDG_CUDA_TRY(cudaStreamWaitEvent(M->stream, evs[ch], 0));
      HDG_CUDA_TRY(launch_k1_range(M, e0, ne));
    }
  }
  // the boundary data (read by the trace solve) behind the element data
  if (in->uD) HDG_CUDA_TRY(cudaMemcpyAsync(M->in_uD, in->uD, d * nfc * nf, cudaMemcpyHostToDevice, cs));
  if (in->gN) HDG_CUDA_TRY(cudaMemcpyAsync(M->in_gN, in->gN, d * 3 * nfc * nf, cudaMemcpyHostToDevice, cs));
  cudaEvent_t evl;
  HDG_CUDA_TRY(cudaEventCreateWithFlags(&evl, cudaEventDisableTiming));
  HDG_CUDA_TRY(cudaEventRecord(evl, cs));
  HDG_CUDA_TRY(cudaStreamWaitEvent(M->stream, evl, 0));
  cudaEventDestroy(evl);
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (!pipe) return hdg_assemble_condense(M, precision);
  return finish_assembly(M, precision);
}

int hdg_recover_host(hdg_mesh* M, const double* uhat, double* q, double* u, int chunks) {
  if (!M || !uhat || !q || !u) return fail(HDG_ERR_ARG, "NULL argument");
  if (!M->assembled) return fail(HDG_ERR_STATE, "recover before hdg_assemble_condense");
  const int64_t nelt = M->nelt, n = M->tab.n;
  int rc;
  if ((rc = ensure_buffer(&M->out_q, 3 * nelt * n)) || (rc = ensure_buffer(&M->out_u, nelt * n))) return rc;
  if (!M->copy_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->copy_stream, cudaStreamNonBlocking));
  cudaStream_t cs = M->copy_stream;
  const int nch = std::max(1, std::min<int>(chunks, (int)std::min<int64_t>(nelt, 1024)));
  std::vector<cudaEvent_t> evs(nch, nullptr);
  int err = HDG_OK;
  for (int ch = 0; ch < nch && !err; ++ch) {
    const int64_t e0 = range_start(nelt, nch, ch, 1.0), ne = range_start(nelt, nch, ch + 1, 1.0) - e0;
    if (ne <= 0) continue;
    cudaError_t e = launch_recover_range(M, uhat, M->out_q, M->out_u, e0, ne);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[ch], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(evs[ch], M->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, evs[ch], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(q + e0 * 3 * n, M->out_q + e0 * 3 * n, sizeof(double) * ne * 3 * n, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(u + e0 * n, M->out_u + e0 * n, sizeof(double) * ne * n, cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) err = fail(HDG_ERR_CUDA, std::string("pipelined recovery: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(cs);
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (err) return err;
  if (e != cudaSuccess) return fail(HDG_ERR_CUDA, std::string("pipelined recovery: ") + cudaGetErrorString(e));
  return check_status(M);
}

int hdg_set_volume_rule(hdg_mesh* M, int rule) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if (rule != HDG_RULE_CONICAL && rule != HDG_RULE_SYMMETRIC) return fail(HDG_ERR_ARG, "unknown volume rule");
  if (M->tab.rule == rule) return HDG_OK;
  Tables T;
  std::string err;
  if (!build_tables(M->k, &T, &err, rule)) return fail(HDG_ERR_UNSUPPORTED, err);
  if (M->stream) HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
  free_tables(M);
  M->tab = std::move(T);
  int rc = upload_tables(M);
  if (rc) return rc;
  // every array at the volume nodes changes size: the caller sets the coefficients again
  M->kappa = M->c = M->f = nullptr;
  M->beta_q = M->beta_f = nullptr;
  M->assembled = false;
  M->rhs_ready = false;
  M->c32_ready = false;
  M->bj64_ready = M->bj32_ready = false;
  return HDG_OK;
}

int hdg_set_method(hdg_mesh* M, int method) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if (method != HDG_METHOD_HDG && method != HDG_METHOD_BDM) return fail(HDG_ERR_ARG, "unknown method");
  M->method = method;
  return HDG_OK;
}

int hdg_get_condensed(const hdg_mesh* M, double* C, double* Cf) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if (!M->assembled) return fail(HDG_ERR_STATE, "not assembled");
  const int m = M->tab.m;
  if (C)  // stored row-major [K][r][s], the layout of the output
    HDG_CUDA_TRY(cudaMemcpyAsync(C, M->d_C, sizeof(double) * M->nelt * m * m, cudaMemcpyDeviceToDevice, M->stream));
  if (Cf) HDG_CUDA_TRY(cudaMemcpyAsync(Cf, M->d_Cf, sizeof(double) * M->nelt * m, cudaMemcpyDeviceToDevice, M->stream));
  HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
  return HDG_OK;
}

int hdg_solve_trace(hdg_mesh* M, int precision, double rtol, int maxit, const double* x0, double* uhat, int* iters,
                    double* relres) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  int rc = solve_trace(M, precision, rtol, maxit, x0, uhat, iters, relres);
  if (rc == HDG_OK) rc = check_status(M);
  return rc;
}

int hdg_set_inner_tolerance(hdg_mesh* M, double rtol) {
  if (!M || !(rtol > 0) || !(rtol < 1)) return fail(HDG_ERR_ARG, "inner tolerance must be in (0, 1)");
  M->inner_rtol = rtol;
  return HDG_OK;
}

int hdg_trace_apply(hdg_mesh* M, const double* x, double* y) {
  if (!M || !x || !y) return fail(HDG_ERR_ARG, "NULL argument");
  return trace_apply(M, x, y);
}

int hdg_autotune(hdg_mesh* M, hdg_tuning* out) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  hdg_tuning t = {};
  int rc = autotune_face_grid(M, &t);
  if (rc) return rc;
  // launch shapes of the double-float K1: two timed launches each
  float best_t = 1e30f;
  int best = 0;
  {
    cudaEvent_t a, b;
    HDG_CUDA_TRY(cudaEventCreate(&a));
    HDG_CUDA_TRY(cudaEventCreate(&b));
    for (int v = 0; v < k1_shape_count(M); ++v) {
      M->k1_variant = v;
      HDG_CUDA_TRY(launch_k1(M));  // warm-up (sets the launch attributes)
      HDG_CUDA_TRY(cudaEventRecord(a, M->stream));
      HDG_CUDA_TRY(launch_k1(M));
      HDG_CUDA_TRY(launch_k1(M));
      HDG_CUDA_TRY(cudaEventRecord(b, M->stream));
      HDG_CUDA_TRY(cudaEventSynchronize(b));
      float ms = 0.f;
      HDG_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
      if (ms < best_t) {
        best_t = ms;
        best = v;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    M->k1_variant = best;
    // restore the system of the caller's last assembly
    rc = hdg_assemble_condense(M, M->asm_prec >= 0 ? M->asm_prec : HDG_FP64);
    if (rc) return rc;
  }
  t.k1_threads = k1_shape_threads(M, M->k1_variant);
  t.k1_streamed = M->k1_variant >= k1_variants(M->k) ? 1 : 0;
  t.k1_ms = best_t < 1e29f ? best_t / 2.0 : 0.0;
  if (out) *out = t;
  return HDG_OK;
}

int hdg_trace_residual(hdg_mesh* M, const double* x, double* r, double* rnorm, double* bnorm) {
  if (!M || !x || !r) return fail(HDG_ERR_ARG, "NULL argument");
  return trace_residual(M, x, r, rnorm, bnorm);
}

int hdg_recover(hdg_mesh* M, const double* uhat, double* q, double* u) {
  if (!M || !uhat || !q || !u) return fail(HDG_ERR_ARG, "NULL argument");
  if (!M->assembled) return fail(HDG_ERR_STATE, "hdg_recover before hdg_assemble_condense");
  HDG_CUDA_TRY(launch_recover(M, uhat, q, u));
  return HDG_OK;
}

int hdg_postprocess(hdg_mesh* M, const double* q, const double* u, double* ustar) {
  if (!M || !q || !u || !ustar) return fail(HDG_ERR_ARG, "NULL argument");
  if (!M->kappa) return fail(HDG_ERR_STATE, "hdg_set_coefficients was not called");
  HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 2, 0, sizeof(int32_t), M->stream));
  HDG_CUDA_TRY(launch_postprocess(M, q, u, ustar));
  return HDG_OK;
}

int hdg_projection(hdg_mesh* M, const double* q_vol, const double* u_vol, const double* q_face,
                   const double* u_face, double* Pq, double* Pu) {
  if (!M || !q_vol || !u_vol || !q_face || !u_face || !Pq || !Pu) return fail(HDG_ERR_ARG, "NULL argument");
  HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 5, 0, sizeof(int32_t), M->stream));
  HDG_CUDA_TRY(launch_projection(M, q_vol, u_vol, q_face, u_face, Pq, Pu));
  int32_t bad = 0;
  HDG_CUDA_TRY(cudaMemcpyAsync(&bad, M->d_status + 5, sizeof(int32_t), cudaMemcpyDeviceToHost, M->stream));
  HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
  if (bad) return fail(HDG_ERR_LOCAL_SINGULAR, std::to_string(bad) + " element(s) with a singular projection system");
  return HDG_OK;
}

int hdg_face_projection(hdg_mesh* M, const double* vals, double* Pu) {
  if (!M || !vals || !Pu) return fail(HDG_ERR_ARG, "NULL argument");
  HDG_CUDA_TRY(launch_face_projection(M, vals, Pu));
  return HDG_OK;
}

int hdg_volume_norm2(hdg_mesh* M, int degree, const double* coef, const double* vals, double* out) {
  if (!M || !out) return fail(HDG_ERR_ARG, "NULL argument");
  if (degree != M->k && degree != M->k + 1) return fail(HDG_ERR_ARG, "degree must be k or k + 1");
  HDG_CUDA_TRY(launch_volume_norm2(M, degree, coef, vals, out));
  return HDG_OK;
}

int hdg_face_norm2(hdg_mesh* M, const double* coef, const double* vals, double* out) {
  if (!M || !out) return fail(HDG_ERR_ARG, "NULL argument");
  HDG_CUDA_TRY(launch_face_norm2(M, coef, vals, out));
  return HDG_OK;
}

int hdg_last_error(char* buf, size_t len) {
  if (!buf || !len) return HDG_ERR_ARG;
  std::snprintf(buf, len, "%s", g_last_error.c_str());
  return HDG_OK;
}

int64_t hdg_launch_count(const hdg_mesh* M) { return M ? M->launches : -1; }

int hdg_host_table(int k, const char* name, double* out, int64_t capacity, int64_t* size) {
  if (!name || !size) return fail(HDG_ERR_ARG, "NULL argument");
  Tables T;
  std::string err;
  std::string s(name);
  int rule = 0;  // "<name>:sym": the table of the symmetric volume rule
  if (s.size() > 4 && s.compare(s.size() - 4, 4, ":sym") == 0) {
    rule = 1;
    s.resize(s.size() - 4);
  }
  if (!build_tables(k, &T, &err, rule)) return fail(HDG_ERR_UNSUPPORTED, err);
  const std::vector<double>* v = nullptr;
  if (s == "vol_pts") v = &T.vol_pts;
  else if (s == "vol_w") v = &T.vol_w;
  else if (s == "P") v = &T.P;
  else if (s == "Pd") v = &T.Pd;
  else if (s == "Chat") v = &T.Chat;
  else if (s == "face_pts") v = &T.face_pts;
  else if (s == "face_w") v = &T.face_w;
  else if (s == "Pl") v = &T.Pl;
  else if (s == "D") v = &T.D;
  else if (s == "Dmu") v = &T.Dmu;
  else if (s == "S") v = &T.S;
  else if (s == "E") v = &T.E;
  else if (s == "P1") v = &T.P1;
  else if (s == "G1") v = &T.G1;
  else if (s == "Shat1") v = &T.Shat1;
  else if (s == "sfAA") v = &T.sfAA;
  else if (s == "sfBB") v = &T.sfBB;
  else if (s == "sfCC") v = &T.sfCC;
  std::vector<double> conv;  // the int16 pair maps, returned as doubles
  if (s == "sfp2to1" || s == "sfp3to2") {
    const std::vector<int16_t>& src = (s == "sfp2to1") ? T.sfp2to1 : T.sfp3to2;
    conv.assign(src.begin(), src.end());
    v = &conv;
  }
  if (!v) return fail(HDG_ERR_ARG, "unknown table " + s);
  *size = (int64_t)v->size();
  if (out) {
    if (capacity < *size) return fail(HDG_ERR_ARG, "capacity too small");
    std::memcpy(out, v->data(), sizeof(double) * v->size());
  }
  return HDG_OK;
}

int hdg_host_expand_mesh(const double* coords, int64_t nver, const int32_t* elems, int64_t nelt,
                         const int32_t* dir, int64_t ndir, const int32_t* neu, int64_t nneu, int64_t* nfc,
                         int32_t* faces, int32_t* facebyele, int32_t* perm) {
  if (!coords || !elems || !nfc || nver < 4 || nelt < 1) return fail(HDG_ERR_ARG, "invalid mesh arrays");
  hdg_mesh M;
  M.nver = nver;
  M.nelt = nelt;
  M.ndir = ndir;
  M.nneu = nneu;
  std::vector<int32_t> own;
  int rc = build_mesh_host(&M, coords, elems, dir, neu, &own);
  if (rc) return rc;
  *nfc = M.nfc;
  if (faces) std::memcpy(faces, M.h_faces.data(), sizeof(int32_t) * M.h_faces.size());
  if (facebyele) std::memcpy(facebyele, M.h_facebyele.data(), sizeof(int32_t) * M.h_facebyele.size());
  if (perm) std::memcpy(perm, M.h_perm.data(), sizeof(int32_t) * M.h_perm.size());
  return HDG_OK;
}

}  // extern "C"
