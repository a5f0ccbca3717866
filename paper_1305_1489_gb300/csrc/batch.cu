// Batched solves of many independent HDG problems of mixed degree (C ABI hdg_batch_*).
//
// Problems of the same degree k are merged into one disjoint-union mesh (vertex numbers
// offset, faces of different problems never coincide), so that every phase of a degree
// group -- K1 assembly + condensation, boundary data and right-hand side, block-Jacobi, the
// PCG iterations, recovery -- is one kernel launch over all elements or faces of the group.
// The whole batch is recorded once as a single CUDA graph: each degree group is an
// independent branch (assembly/setup child graph -> conditional WHILE node running the PCG
// iterations until the device-side convergence flag is set -> residual/recovery child graph),
// and one cudaGraphLaunch runs everything.
//
// Per-problem accuracy: CG on the union is CG on a block-diagonal SPD system, and
// ||r_p|| <= ||r|| for every problem p, so the union is iterated to
// ||r|| <= rtol * min_p ||b_p||, which guarantees ||r_p|| <= rtol ||b_p|| for each problem;
// the per-problem relative residuals are measured after the solve and returned.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "hdg_internal.h"

struct hdg_batch {
  struct Group {
    int k = 0;
    hdg_mesh* mesh = nullptr;
    std::vector<int> probs;             // global problem ids, in union order
    std::vector<int64_t> elem_off;      // [np + 1] element ranges in the union mesh
    std::vector<int64_t> face_off;      // [np + 1] face ranges (contiguous: lexicographic faces)
    int32_t* d_face_prob = nullptr;     // [nfc] local problem index of each face
    double* d_norms = nullptr;          // [2 np] ||b_p||^2, ||r_p||^2
    double *d_uhat = nullptr, *d_q = nullptr, *d_u = nullptr;
  };
  int nprob = 0;
  std::vector<Group> groups;
  std::vector<int> prob_group, prob_local;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  int built_prec = -1, built_maxit = -1;
  int solve_prec = HDG_FP64, built_solve_prec = -1;
  std::vector<int> built_gens;  // coarse-space generation, grid and K1 shape of every group at graph build
  double built_rtol = -1.0;
};

using namespace hdg;

static void batch_release(hdg_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  for (auto& g : B->groups) {
    if (g.mesh) hdg_mesh_destroy(g.mesh);
    void* ptrs[] = {g.d_face_prob, g.d_norms, g.d_uhat, g.d_q, g.d_u};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
}

extern "C" {

int hdg_batch_create(int nprob, const double* const* coords, const int64_t* nver, const int32_t* const* elems,
                     const int64_t* nelt, const int32_t* const* dir, const int64_t* ndir, const int32_t* const* neu,
                     const int64_t* nneu, const int* k, void* stream, hdg_batch** out) {
  if (!out || nprob < 1 || !coords || !nver || !elems || !nelt || !dir || !ndir || !neu || !nneu || !k)
    return fail(HDG_ERR_ARG, "invalid batch arguments");
  *out = nullptr;
  hdg_batch* B = new (std::nothrow) hdg_batch();
  if (!B) return fail(HDG_ERR_ARG, "out of host memory");
  B->nprob = nprob;
  B->stream = (cudaStream_t)stream;
  B->prob_group.assign(nprob, -1);
  B->prob_local.assign(nprob, -1);
  int rc = HDG_OK;
  for (int kk = 1; kk <= 4 && rc == HDG_OK; ++kk) {
    std::vector<int> ids;
    for (int p = 0; p < nprob; ++p) {
      if (k[p] < 1 || k[p] > 4) {
        rc = fail(HDG_ERR_UNSUPPORTED, "batched degrees must be in 1..4");
        break;
      }
      if (k[p] == kk) ids.push_back(p);
    }
    if (rc || ids.empty()) continue;
    hdg_batch::Group g;
    g.k = kk;
    g.probs = ids;
    std::vector<double> C;
    std::vector<int32_t> E, Dl, Nl;
    std::vector<int64_t> voff(ids.size() + 1, 0);
    g.elem_off.assign(ids.size() + 1, 0);
    for (size_t i = 0; i < ids.size(); ++i) {
      const int p = ids[i];
      const int32_t vo = (int32_t)voff[i];
      C.insert(C.end(), coords[p], coords[p] + 3 * nver[p]);
      for (int64_t t = 0; t < 4 * nelt[p]; ++t) E.push_back(elems[p][t] + vo);
      for (int64_t t = 0; t < 3 * ndir[p]; ++t) Dl.push_back(dir[p][t] + vo);
      for (int64_t t = 0; t < 3 * nneu[p]; ++t) Nl.push_back(neu[p][t] + vo);
      voff[i + 1] = voff[i] + nver[p];
      g.elem_off[i + 1] = g.elem_off[i] + nelt[p];
      if (voff[i + 1] > (int64_t)1 << 30) {
        rc = fail(HDG_ERR_ARG, "batch group too large");
        break;
      }
      B->prob_group[p] = (int)B->groups.size();
      B->prob_local[p] = (int)i;
    }
    if (rc) break;
    rc = hdg_mesh_create(C.data(), (int64_t)C.size() / 3, E.data(), (int64_t)E.size() / 4, Dl.empty() ? nullptr : Dl.data(),
                         (int64_t)Dl.size() / 3, Nl.empty() ? nullptr : Nl.data(), (int64_t)Nl.size() / 3, kk, stream,
                         &g.mesh);
    if (rc) break;
    // faces are numbered lexicographically by sorted vertex triple: a problem's faces form a
    // contiguous range, identified by the problem owning the smallest vertex
    const hdg_mesh* M = g.mesh;
    std::vector<int32_t> fp(M->nfc);
    g.face_off.assign(ids.size() + 1, 0);
    for (int64_t e = 0; e < M->nfc; ++e) {
      const int64_t v0 = M->h_faces[4 * e];
      const int i = (int)(std::upper_bound(voff.begin(), voff.end(), v0) - voff.begin()) - 1;
      fp[e] = i;
      g.face_off[i + 1] = e + 1;
    }
    for (size_t i = 1; i <= ids.size(); ++i) g.face_off[i] = std::max(g.face_off[i], g.face_off[i - 1]);
    const int d2 = M->tab.d2, n = M->tab.n;
    cudaError_t ce = cudaMalloc(&g.d_face_prob, sizeof(int32_t) * M->nfc);
    if (ce == cudaSuccess) ce = cudaMemcpy(g.d_face_prob, fp.data(), sizeof(int32_t) * M->nfc, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMalloc(&g.d_norms, sizeof(double) * 2 * ids.size());
    if (ce == cudaSuccess) ce = cudaMalloc(&g.d_uhat, sizeof(double) * M->nfc * d2);
    if (ce == cudaSuccess) ce = cudaMalloc(&g.d_q, sizeof(double) * M->nelt * 3 * n);
    if (ce == cudaSuccess) ce = cudaMalloc(&g.d_u, sizeof(double) * M->nelt * n);
    B->groups.push_back(g);
    if (ce != cudaSuccess) rc = fail(HDG_ERR_CUDA, std::string("batch allocation: ") + cudaGetErrorString(ce));
  }
  if (rc) {
    batch_release(B);
    delete B;
    return rc;
  }
  *out = B;
  return HDG_OK;
}

int hdg_batch_destroy(hdg_batch* B) {
  if (!B) return HDG_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  batch_release(B);
  delete B;
  return HDG_OK;
}

int hdg_batch_num_groups(const hdg_batch* B, int* ngroups) {
  if (!B || !ngroups) return fail(HDG_ERR_ARG, "NULL argument");
  *ngroups = (int)B->groups.size();
  return HDG_OK;
}

int hdg_batch_group(const hdg_batch* B, int g, hdg_mesh** mesh, int* k, int* np, int32_t* prob_ids,
                    int64_t* elem_off, int64_t* face_off) {
  if (!B || g < 0 || g >= (int)B->groups.size()) return fail(HDG_ERR_ARG, "bad group index");
  const auto& G = B->groups[g];
  if (mesh) *mesh = G.mesh;
  if (k) *k = G.k;
  if (np) *np = (int)G.probs.size();
  if (prob_ids)
    for (size_t i = 0; i < G.probs.size(); ++i) prob_ids[i] = G.probs[i];
  if (elem_off) std::memcpy(elem_off, G.elem_off.data(), sizeof(int64_t) * G.elem_off.size());
  if (face_off) std::memcpy(face_off, G.face_off.data(), sizeof(int64_t) * G.face_off.size());
  return HDG_OK;
}

int hdg_batch_run(hdg_batch* B, int precision, double rtol, int maxit, double* relres, int* iters) {
  if (!B || !(rtol > 0) || maxit < 1) return fail(HDG_ERR_ARG, "bad batch run arguments");
  if (precision != HDG_FP64 && precision != HDG_DF32) return fail(HDG_ERR_ARG, "assembly precision must be FP64 or DF32");
  for (auto& G : B->groups) {
    if (!G.mesh->kappa) return fail(HDG_ERR_STATE, "coefficients not set on every batch group");
    if (G.mesh->beta_q) return fail(HDG_ERR_UNSUPPORTED, "batched solves are for reaction-diffusion (beta = 0)");
  }
  std::vector<int> gens;  // what the recorded graph depends on besides the arguments
  for (auto& G : B->groups) {
    gens.push_back(G.mesh->coarse_gen);
    gens.push_back(G.mesh->face_blocks);
    gens.push_back(G.mesh->k1_variant);
  }
  if (!B->exec || B->built_prec != precision || B->built_rtol != rtol || B->built_maxit != maxit ||
      B->built_gens != gens || B->built_solve_prec != B->solve_prec) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
    // one direct assembly per group first: validates the coefficients and sets the kernels'
    // launch attributes outside the capture
    for (auto& G : B->groups) {
      const int rc = hdg_assemble_condense(G.mesh, precision);
      if (rc) return rc;
    }
    cudaGraph_t graph;
    HDG_CUDA_TRY(cudaGraphCreate(&graph, 0));
    for (auto& G : B->groups) {
      cudaGraphNode_t last;
      int rc = batch_record_group(G.mesh, graph, precision, B->solve_prec, G.d_face_prob, (int)G.probs.size(),
                                  G.d_norms, rtol,
                                  maxit, G.d_q, G.d_u, G.d_uhat, &last);
      if (rc) {
        cudaGraphDestroy(graph);
        return rc;
      }
    }
    cudaError_t e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(HDG_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    B->built_prec = precision;
    B->built_rtol = rtol;
    B->built_maxit = maxit;
    B->built_gens = gens;
    B->built_solve_prec = B->solve_prec;
  }
  HDG_CUDA_TRY(cudaGraphLaunch(B->exec, B->stream));
  HDG_CUDA_TRY(cudaStreamSynchronize(B->stream));
  bool bad = false, notconv = false;
  for (size_t gi = 0; gi < B->groups.size(); ++gi) {
    auto& G = B->groups[gi];
    int it, st;
    int rc = batch_group_iterations(G.mesh, &it, &st);
    if (rc) return rc;
    G.mesh->launches += 1;
    G.mesh->assembled = true;
    G.mesh->c32_ready = false;
    G.mesh->bj64_ready = G.mesh->bj32_ready = false;
    if (G.mesh->coarse) coarse_invalidate(G.mesh);
    if (iters) iters[gi] = it;
    if (st) bad = true;
    std::vector<double> nrm(2 * G.probs.size());
    HDG_CUDA_TRY(cudaMemcpy(nrm.data(), G.d_norms, sizeof(double) * nrm.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < G.probs.size(); ++i) {
      const double bb = nrm[i], rr = nrm[G.probs.size() + i];
      const double rel = bb > 0 ? std::sqrt(rr / bb) : 0.0;
      if (relres) relres[G.probs[i]] = rel;
      if (!(rel <= rtol * 1.0000001)) notconv = true;
    }
  }
  if (bad) return fail(HDG_ERR_LOCAL_SINGULAR, "batch: a local factorisation or the PCG broke down");
  if (notconv) return fail(HDG_ERR_NOT_CONVERGED, "batch: some problem did not reach the tolerance within maxit");
  return HDG_OK;
}

int hdg_batch_set_solve_precision(hdg_batch* B, int precision) {
  if (!B) return fail(HDG_ERR_ARG, "NULL batch");
  if (precision != HDG_FP64 && precision != HDG_MIXED_FP32)
    return fail(HDG_ERR_ARG, "batch solve precision must be HDG_FP64 or HDG_MIXED_FP32");
  B->solve_prec = precision;
  return HDG_OK;
}

int hdg_batch_solution(const hdg_batch* B, int g, double** uhat, double** q, double** u) {
  if (!B || g < 0 || g >= (int)B->groups.size()) return fail(HDG_ERR_ARG, "bad group index");
  const auto& G = B->groups[g];
  if (uhat) *uhat = G.d_uhat;
  if (q) *q = G.d_q;
  if (u) *u = G.d_u;
  return HDG_OK;
}

}  // extern "C"
