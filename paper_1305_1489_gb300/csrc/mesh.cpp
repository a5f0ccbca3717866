// Expanded tetrahedral data structure (Section 2 of the paper), built on the host.
//
// From the basic mesh T (coordinates, elements, dirichlet, neumann) this computes
// T.faces (sorted vertex triples, numbered lexicographically, with their type),
// T.facebyele (local faces in the order of eq. 2.1), T.perm (eq. 2.3), and the face -> element
// adjacency used by the face-owner trace operator.  Geometry (volumes, normals, areas,
// Piola cofactors) is recomputed on the device from vertex coordinates.
#include <algorithm>
#include <array>
#include <cmath>

#include "hdg_internal.h"

namespace hdg {

namespace {
// eq. 2.1: local faces as positions in (v1, v2, v3, v4)
const int kLocal[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {3, 1, 2}};
// eq. 2.2: images of (w1, w2, w3) under F_mu (1-based vertex indices), mu = 1..6
const int kFmu[6][3] = {{1, 2, 3}, {1, 3, 2}, {3, 1, 2}, {3, 2, 1}, {2, 3, 1}, {2, 1, 3}};

typedef std::array<int32_t, 3> Tri;
Tri sorted(int32_t a, int32_t b, int32_t c) {
  Tri t = {a, b, c};
  std::sort(t.begin(), t.end());
  return t;
}
}  // namespace

int build_mesh_host(hdg_mesh* M, const double* coords, const int32_t* elems, const int32_t* dir,
                    const int32_t* neu, std::vector<int32_t>* owner_out) {
  const int64_t nelt = M->nelt, nver = M->nver;
  // orientation (Section 2: det B_K > 0)
  for (int64_t K = 0; K < nelt; ++K) {
    const int32_t* e = elems + 4 * K;
    for (int i = 0; i < 4; ++i)
      if (e[i] < 0 || e[i] >= nver) return fail(HDG_ERR_ARG, "element vertex index out of range");
    double b[3][3];
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) b[j][d] = coords[3 * e[j + 1] + d] - coords[3 * e[0] + d];
    double det = b[0][0] * (b[1][1] * b[2][2] - b[1][2] * b[2][1]) -
                 b[0][1] * (b[1][0] * b[2][2] - b[1][2] * b[2][0]) +
                 b[0][2] * (b[1][0] * b[2][1] - b[1][1] * b[2][0]);
    if (!(det > 0))
      return fail(HDG_ERR_ORIENTATION, "element " + std::to_string(K) + " has det B_K <= 0");
  }
  // all element faces, sorted by key then by (K, l)
  std::vector<std::pair<Tri, int64_t>> all(4 * nelt);
  for (int64_t K = 0; K < nelt; ++K)
    for (int l = 0; l < 4; ++l) {
      const int32_t* e = elems + 4 * K;
      all[4 * K + l] = {sorted(e[kLocal[l][0]], e[kLocal[l][1]], e[kLocal[l][2]]), 4 * K + l};
    }
  std::sort(all.begin(), all.end());
  std::vector<Tri> faces;
  std::vector<std::array<int32_t, 2>> owner;
  M->h_facebyele.assign(4 * nelt, -1);
  for (size_t i = 0; i < all.size();) {
    size_t j = i;
    while (j < all.size() && all[j].first == all[i].first) ++j;
    if (j - i > 2) return fail(HDG_ERR_NONCONFORMING, "a face is shared by more than two elements");
    int32_t id = (int32_t)faces.size();
    faces.push_back(all[i].first);
    std::array<int32_t, 2> ow = {(int32_t)all[i].second, j - i == 2 ? (int32_t)all[i + 1].second : -1};
    owner.push_back(ow);
    for (size_t t = i; t < j; ++t) M->h_facebyele[all[t].second] = id;
    i = j;
  }
  const int64_t nfc = (int64_t)faces.size();
  M->nfc = nfc;
  std::vector<int32_t> ftype(nfc, 0);
  auto find = [&](const int32_t* t) -> int64_t {
    Tri key = sorted(t[0], t[1], t[2]);
    auto it = std::lower_bound(faces.begin(), faces.end(), key);
    if (it == faces.end() || *it != key) return -1;
    return it - faces.begin();
  };
  for (int64_t i = 0; i < M->ndir; ++i) {
    int64_t e = find(dir + 3 * i);
    if (e < 0 || owner[e][1] >= 0)
      return fail(HDG_ERR_NONCONFORMING, "Dirichlet face " + std::to_string(i) + " is not a boundary face");
    ftype[e] = 1;
  }
  for (int64_t i = 0; i < M->nneu; ++i) {
    int64_t e = find(neu + 3 * i);
    if (e < 0 || owner[e][1] >= 0)
      return fail(HDG_ERR_NONCONFORMING, "Neumann face " + std::to_string(i) + " is not a boundary face");
    ftype[e] = 2;
  }
  for (int64_t e = 0; e < nfc; ++e)
    if (owner[e][1] < 0 && ftype[e] == 0)
      return fail(HDG_ERR_NONCONFORMING, "boundary face " + std::to_string(e) + " is neither Dirichlet nor Neumann");

  // perm(K,l), eq. 2.3: F_mu sends w_hat_i to the position of local vertex i in the face
  M->h_perm.assign(4 * nelt, 0);
  for (int64_t K = 0; K < nelt; ++K)
    for (int l = 0; l < 4; ++l) {
      const Tri& f = faces[M->h_facebyele[4 * K + l]];
      int pos[3];
      for (int i = 0; i < 3; ++i) {
        int32_t v = elems[4 * K + kLocal[l][i]];
        pos[i] = (f[0] == v) ? 1 : (f[1] == v) ? 2 : 3;
      }
      int mu = 0;
      for (int c = 0; c < 6; ++c)
        if (kFmu[c][0] == pos[0] && kFmu[c][1] == pos[1] && kFmu[c][2] == pos[2]) mu = c + 1;
      if (!mu) return fail(HDG_ERR_ARG, "degenerate face (repeated vertex)");
      M->h_perm[4 * K + l] = mu;
    }

  M->h_faces.resize(4 * nfc);
  for (int64_t e = 0; e < nfc; ++e) {
    for (int i = 0; i < 3; ++i) M->h_faces[4 * e + i] = faces[e][i];
    M->h_faces[4 * e + 3] = ftype[e];
  }
  owner_out->resize(2 * nfc);
  for (int64_t e = 0; e < nfc; ++e) {
    (*owner_out)[2 * e] = owner[e][0];
    (*owner_out)[2 * e + 1] = owner[e][1];
  }
  return HDG_OK;
}

int build_mesh(hdg_mesh* M, const double* coords, const int32_t* elems, const int32_t* dir,
               const int32_t* neu) {
  std::vector<int32_t> own;
  int rc = build_mesh_host(M, coords, elems, dir, neu, &own);
  if (rc) return rc;
  const int64_t nelt = M->nelt, nfc = M->nfc;
  std::vector<int32_t> ftype(nfc);
  for (int64_t e = 0; e < nfc; ++e) ftype[e] = M->h_faces[4 * e + 3];
  // device copies
  std::vector<double> vx(12 * nelt), fvx(9 * nfc);
  for (int64_t K = 0; K < nelt; ++K)
    for (int i = 0; i < 4; ++i)
      for (int d = 0; d < 3; ++d) vx[(d * 4 + i) * nelt + K] = coords[3 * elems[4 * K + i] + d];
  for (int64_t e = 0; e < nfc; ++e)
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) fvx[(d * 3 + i) * nfc + e] = coords[3 * M->h_faces[4 * e + i] + d];
  HDG_CUDA_TRY(cudaMalloc(&M->d_vx, sizeof(double) * vx.size()));
  HDG_CUDA_TRY(cudaMalloc(&M->d_fvx, sizeof(double) * fvx.size()));
  HDG_CUDA_TRY(cudaMalloc(&M->d_facebyele, sizeof(int32_t) * 4 * nelt));
  HDG_CUDA_TRY(cudaMalloc(&M->d_perm, sizeof(int32_t) * 4 * nelt));
  HDG_CUDA_TRY(cudaMalloc(&M->d_owner, sizeof(int32_t) * 2 * nfc));
  HDG_CUDA_TRY(cudaMalloc(&M->d_ftype, sizeof(int32_t) * nfc));
  HDG_CUDA_TRY(cudaMemcpy(M->d_vx, vx.data(), sizeof(double) * vx.size(), cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMemcpy(M->d_fvx, fvx.data(), sizeof(double) * fvx.size(), cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMemcpy(M->d_facebyele, M->h_facebyele.data(), sizeof(int32_t) * 4 * nelt, cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMemcpy(M->d_perm, M->h_perm.data(), sizeof(int32_t) * 4 * nelt, cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMemcpy(M->d_owner, own.data(), sizeof(int32_t) * 2 * nfc, cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMemcpy(M->d_ftype, ftype.data(), sizeof(int32_t) * nfc, cudaMemcpyHostToDevice));
  // fslot[4 K + l] = 2 f + side: face f of element K and which of its owners K is (the
  // element pass of the trace operator writes its rows to that side of the face); -(2 f +
  // side) - 1 on Dirichlet faces, whose rows the trace system does not have
  std::vector<int32_t> fslot(4 * nelt);
  for (int64_t K = 0; K < nelt; ++K)
    for (int l = 0; l < 4; ++l) {
      const int32_t f = M->h_facebyele[4 * K + l];
      const int32_t v = 2 * f + (own[2 * f] == (int32_t)(4 * K + l) ? 0 : 1);
      fslot[4 * K + l] = ftype[f] == 1 ? -v - 1 : v;
    }
  HDG_CUDA_TRY(cudaMalloc(&M->d_fslot, sizeof(int32_t) * 4 * nelt));
  HDG_CUDA_TRY(cudaMemcpy(M->d_fslot, fslot.data(), sizeof(int32_t) * 4 * nelt, cudaMemcpyHostToDevice));
  return HDG_OK;
}

}  // namespace hdg
