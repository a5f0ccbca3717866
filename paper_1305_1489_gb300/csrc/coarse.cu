// Set-up of the two-level trace preconditioner: the structure of the nested P1 hierarchy on
// the host (once per hdg_set_coarse_space) and its Galerkin values on the device (after every
// assembly).  The per-iteration kernels are in coarse.cuh.
//
// Structure (host): every element's level-0 nodes (those of its vertices), the CSR pattern of
// A_0 = Pi^T H Pi (two nodes couple when they share an element) with each element's slots in
// it, and for every level the CSR pattern of A_{l+1} = P_l^T A_l P_l with the triples
// (source entry, destination entry, w_iI w_jJ) of the product.
//
// Values (device): one warp per element forms R_K (the element's face unknowns as functions of
// its level-0 nodes), Y = C^K R_K and R_K^T Y, and adds it into A_0 (FP64 atomics); one thread
// per triple forms the coarser levels; the l1-Jacobi diagonals, FP32 copies and the dense
// inverse of the coarsest level (Gauss-Jordan, one CTA) complete it.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <numeric>
#include <vector>

#include "hdg_internal.h"
#include "coarse.cuh"

namespace hdg {

constexpr int kElemNodes = 8;  // level-0 nodes per element (4 for nested P1 spaces)
constexpr int kGalWarps = 4;

// T: arithmetic of the product and type of C^K (FP32 when the FP32 copy of the mixed solve
// exists: the coarse operator only serves the preconditioner)
template <int D2, typename T>
__global__ void __launch_bounds__(32 * kGalWarps) galerkin0_kernel(
    int64_t nelt, const T* __restrict__ C, const int32_t* __restrict__ fbe, const int32_t* __restrict__ ftype,
    const int32_t* __restrict__ fverts, const double* __restrict__ Tp, const int32_t* __restrict__ vnodes,
    const double* __restrict__ vwd, const int32_t* __restrict__ elist, const int32_t* __restrict__ eslot,
    double* __restrict__ A0) {
  constexpr int m = 4 * D2;
  __shared__ T Rs[kGalWarps][m][kElemNodes], Ys[kGalWarps][m][kElemNodes];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t K = (int64_t)blockIdx.x * kGalWarps + w; K < nelt; K += (int64_t)gridDim.x * kGalWarps) {
    int nd[kElemNodes], cnt = 0;
#pragma unroll
    for (int u = 0; u < kElemNodes; ++u) {
      nd[u] = elist[K * kElemNodes + u];
      cnt += nd[u] >= 0;
    }
    if (cnt == 0) continue;  // warp-uniform
    for (int s = lane; s < m; s += 32) {
      const int fl = s / D2, b = s - fl * D2;
      const int64_t f = fbe[4 * K + fl];
      T R[kElemNodes];
#pragma unroll
      for (int u = 0; u < kElemNodes; ++u) R[u] = (T)0;
      if (ftype[f] != 1) {
        for (int i = 0; i < 3; ++i) {
          const int64_t v = fverts[3 * f + i];
          const double tb = Tp[b * 3 + i];
          for (int j = 0; j < 4; ++j) {
            const int node = vnodes[4 * v + j];
            if (node < 0) continue;
            const T wt = (T)(tb * vwd[4 * v + j]);
#pragma unroll
            for (int u = 0; u < kElemNodes; ++u)
              if (nd[u] == node) R[u] += wt;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kElemNodes; ++u) Rs[w][s][u] = R[u];
    }
    __syncwarp();
    const T* CK = C + K * (int64_t)(m * m);
    for (int s = lane; s < m; s += 32) {
      const T* row = CK + (int64_t)s * m;  // C^K[s][t], row-major
      T y[kElemNodes];
#pragma unroll
      for (int u = 0; u < kElemNodes; ++u) y[u] = (T)0;
      for (int t = 0; t < m; ++t) {
        const T c = row[t];
#pragma unroll
        for (int u = 0; u < kElemNodes; ++u)
          if (u < cnt) y[u] = fma(c, Rs[w][t][u], y[u]);
      }
#pragma unroll
      for (int u = 0; u < kElemNodes; ++u) Ys[w][s][u] = y[u];
    }
    __syncwarp();
    for (int p = lane; p < kElemNodes * kElemNodes; p += 32) {
      const int u = p / kElemNodes, v = p - u * kElemNodes;
      if (u < cnt && v < cnt) {
        T acc = (T)0;
        for (int s = 0; s < m; ++s) acc = fma(Rs[w][s][u], Ys[w][s][v], acc);
        const int32_t slot = eslot[K * kElemNodes * kElemNodes + p];
        if (slot >= 0) atomicAdd(A0 + slot, (double)acc);
      }
    }
    __syncwarp();
  }
}

__global__ void rap_kernel(int64_t n, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                           const double* __restrict__ w, const double* __restrict__ Af, double* __restrict__ Ac) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(Ac + dst[i], w[i] * Af[src[i]]);
}

// l1-Jacobi diagonal and FP32 copy of one level; counts rows with a non-positive diagonal
__global__ void level_finish_kernel(CoarseLevel L, int32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, d = 0.0;
    for (int k = L.rowptr[i]; k < L.rowptr[i + 1]; ++k) {
      const double a = L.val[k];
      s += fabs(a);
      if (L.col[k] == i) d = a;
      L.valf[k] = (float)a;
    }
    if (!(d > 0.0)) atomicAdd(status, 1);
    L.dinv[i] = s > 0.0 ? (float)(1.0 / s) : 0.f;
  }
}

// dense inverse of the coarsest level (SPD: Gauss-Jordan in place, no pivoting), one CTA
__global__ void coarsest_inverse_kernel(CoarseLevel L, double* __restrict__ A, float* __restrict__ Ainv,
                                        int32_t* status) {
  const int64_t n = L.n;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int64_t i = tid; i < n * n; i += nt) A[i] = 0.0;
  __syncthreads();
  for (int64_t i = tid; i < n; i += nt)
    for (int k = L.rowptr[i]; k < L.rowptr[i + 1]; ++k) A[i * n + L.col[k]] = L.val[k];
  __syncthreads();
  for (int64_t p = 0; p < n; ++p) {
    double piv = A[p * n + p];
    if (!(piv > 0.0)) {
      if (tid == 0) atomicAdd(status, 1);
      piv = 1.0;
    }
    __syncthreads();
    for (int64_t j = tid; j < n; j += nt)
      if (j != p) A[p * n + j] /= piv;
    __syncthreads();
    for (int64_t q = tid; q < n * n; q += nt) {
      const int64_t i = q / n, j = q - i * n;
      if (i != p && j != p) A[q] -= A[i * n + p] * A[p * n + j];
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += nt) A[i * n + p] = (i == p) ? 1.0 / piv : -A[i * n + p] / piv;
    __syncthreads();
  }
  for (int64_t i = tid; i < n * n; i += nt) Ainv[i] = (float)A[i];
}

// ------------------------------------------------------------------ host helpers
template <typename V>
static int upload(V** dst, const std::vector<V>& src) {
  HDG_CUDA_TRY(cudaMalloc(dst, sizeof(V) * std::max<size_t>(src.size(), 1)));
  if (!src.empty()) HDG_CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

template <typename V>
static int alloc(V** dst, int64_t n) {
  HDG_CUDA_TRY(cudaMalloc(dst, sizeof(V) * std::max<int64_t>(n, 1)));
  return HDG_OK;
}

// sorted unique keys (row * ncol + col) -> CSR
static void keys_to_csr(std::vector<int64_t>& keys, int64_t nrow, int64_t ncol, std::vector<int32_t>& rowptr,
                        std::vector<int32_t>& col) {
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  rowptr.assign(nrow + 1, 0);
  col.resize(keys.size());
  for (size_t q = 0; q < keys.size(); ++q) {
    rowptr[keys[q] / ncol + 1]++;
    col[q] = (int32_t)(keys[q] % ncol);
  }
  for (int64_t i = 0; i < nrow; ++i) rowptr[i + 1] += rowptr[i];
}

static int32_t csr_find(const std::vector<int32_t>& rowptr, const std::vector<int32_t>& col, int64_t i, int64_t j) {
  auto b = col.begin() + rowptr[i], e = col.begin() + rowptr[i + 1];
  auto it = std::lower_bound(b, e, (int32_t)j);
  return (it != e && *it == j) ? (int32_t)(it - col.begin()) : -1;
}

void coarse_free(hdg_mesh* M) {
  Coarse* c = M->coarse;
  if (!c) return;
  for (CoarseLevel& L : c->lv) {
    void* ptrs[] = {L.rowptr, L.col, L.val, L.valf, L.dinv, L.pn, L.pw, L.tptr, L.tidx, L.tw, L.b, L.x, L.t};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  for (size_t l = 0; l < c->rap_src.size(); ++l) {
    cudaFree(c->rap_src[l]);
    cudaFree(c->rap_dst[l]);
    cudaFree(c->rap_w[l]);
  }
  void* ptrs[] = {c->d_lv, c->vnodes, c->vw, c->vwd, c->gptr, c->gfi, c->gw, c->fnode, c->fwt, c->elist, c->eslot,
                  c->rc, c->Tf, c->e0, c->Adense, c->Ainv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
  M->coarse = nullptr;
}

void coarse_invalidate(hdg_mesh* M) {
  if (M->coarse) M->coarse->ready = false;
}

static int set_coarse(hdg_mesh* M, int nlev, const int64_t* sizes, const int32_t* nodes, const double* weights) {
  if (nlev < 2 || !sizes || !nodes || !weights) return fail(HDG_ERR_ARG, "need nlev >= 2 levels and their arrays");
  if (nlev > kMaxTailLevels + 1) return fail(HDG_ERR_UNSUPPORTED, "at most 17 levels");
  for (int l = 0; l < nlev; ++l)
    if (sizes[l] < 1 || sizes[l] > (int64_t)1 << 30) return fail(HDG_ERR_ARG, "every level needs 1 .. 2^30 nodes");
  if (sizes[nlev - 1] > kMaxCoarsest)
    return fail(HDG_ERR_ARG, "the coarsest level may hold at most " + std::to_string(kMaxCoarsest) + " nodes");
  const int64_t nver = M->nver;
  int64_t rows = nver;
  for (int l = 0; l + 1 < nlev; ++l) rows += sizes[l];
  // validation of every interpolation row: target level sizes[l] (level 0 for mesh vertices)
  {
    int64_t off = 0;
    for (int l = -1; l + 1 < nlev; ++l) {
      const int64_t nr = (l < 0) ? nver : sizes[l], ncol = sizes[l + 1];
      for (int64_t i = off; i < off + nr; ++i)
        for (int j = 0; j < 4; ++j) {
          const int32_t nd = nodes[4 * i + j];
          const double wt = weights[4 * i + j];
          if (nd < -1 || nd >= ncol || !std::isfinite(wt))
            return fail(HDG_ERR_ARG, "interpolation row " + std::to_string(i) + " has an invalid node or weight");
        }
      off += nr;
    }
  }
  int rc = ensure_face_verts(M);
  if (rc) return rc;
  Coarse* c = new Coarse();
  M->coarse = c;
  c->nlev = nlev;
  // HDG_COARSE_TAIL_MAX: largest level handled by the single-CTA part of the V-cycle (the
  // finer levels run as grid-wide kernels); a tuning knob, default kTailMax
  if (const char* tm = std::getenv("HDG_COARSE_TAIL_MAX")) {
    const long v = std::strtol(tm, nullptr, 10);
    if (v >= 1) c->tail_max = v;
  }
  c->lv.resize(nlev);
  for (int l = 0; l < nlev; ++l) c->lv[l].n = sizes[l];

  // level-0 rows of the mesh vertices
  std::vector<int32_t> vn(nodes, nodes + 4 * nver);
  std::vector<double> vwd(weights, weights + 4 * nver);
  for (int64_t q = 0; q < 4 * nver; ++q)
    if (vn[q] < 0 || vwd[q] == 0.0) {
      vn[q] = -1;
      vwd[q] = 0.0;
    }
  std::vector<float> vw(vwd.begin(), vwd.end());

  // element node lists and the pattern of A_0
  const int64_t n0 = sizes[0];
  std::vector<int32_t> elist((size_t)M->nelt * kElemNodes, -1);
  std::vector<int64_t> keys;
  keys.reserve((size_t)M->nelt * 16);
  for (int64_t K = 0; K < M->nelt; ++K) {
    int32_t list[kElemNodes * 4];
    int cnt = 0;
    for (int fl = 0; fl < 4; ++fl) {
      const int64_t f = M->h_facebyele[4 * K + fl];
      for (int i = 0; i < 3; ++i) {
        const int64_t v = M->h_faces[4 * f + i];
        for (int j = 0; j < 4; ++j) {
          const int32_t nd = vn[4 * v + j];
          if (nd < 0) continue;
          bool seen = false;
          for (int u = 0; u < cnt; ++u) seen |= list[u] == nd;
          if (!seen) {
            if (cnt == kElemNodes) {
              coarse_free(M);
              return fail(HDG_ERR_UNSUPPORTED, "an element touches more than 8 level-0 nodes");
            }
            list[cnt++] = nd;
          }
        }
      }
    }
    std::sort(list, list + cnt);
    for (int u = 0; u < cnt; ++u) {
      elist[K * kElemNodes + u] = list[u];
      for (int v = 0; v < cnt; ++v) keys.push_back((int64_t)list[u] * n0 + list[v]);
    }
  }
  std::vector<std::vector<int32_t>> rowptr(nlev), col(nlev);
  keys_to_csr(keys, n0, n0, rowptr[0], col[0]);
  // restriction gather: for every level-0 node, the (free face, vertex slot, weight) entries
  if (M->nfc >= ((int64_t)1 << 29)) {
    coarse_free(M);
    return fail(HDG_ERR_UNSUPPORTED, "too many faces for the restriction gather");
  }
  std::vector<int32_t> gptr(n0 + 1, 0), gfi;
  std::vector<float> gw;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int32_t> fill;
    if (pass == 1) {
      for (int64_t i = 0; i < n0; ++i) gptr[i + 1] += gptr[i];
      gfi.resize(gptr[n0]);
      gw.resize(gptr[n0]);
      fill.assign(gptr.begin(), gptr.end() - 1);
    }
    for (int64_t f = 0; f < M->nfc; ++f) {
      if (M->h_faces[4 * f + 3] == 1) continue;  // Dirichlet
      for (int i = 0; i < 3; ++i) {
        const int64_t v = M->h_faces[4 * f + i];
        for (int j = 0; j < 4; ++j) {
          const int32_t nd = vn[4 * v + j];
          if (nd < 0) continue;
          if (pass == 0) {
            gptr[nd + 1]++;
          } else {
            gfi[fill[nd]] = (int32_t)(4 * f + i);
            gw[fill[nd]++] = (float)vwd[4 * v + j];
          }
        }
      }
    }
  }
  // per-face vertex nodes, when every vertex carries at most one level-0 node
  bool single = true;
  for (int64_t v = 0; v < nver && single; ++v)
    for (int j = 1; j < 4; ++j) single = single && vn[4 * v + j] < 0;
  std::vector<int32_t> fnode;
  std::vector<float> fwt;
  if (single) {
    fnode.assign(3 * M->nfc, -1);
    fwt.assign(3 * M->nfc, 0.f);
    for (int64_t f = 0; f < M->nfc; ++f) {
      if (M->h_faces[4 * f + 3] == 1) continue;  // Dirichlet: no prolongation
      for (int i = 0; i < 3; ++i) {
        const int64_t v = M->h_faces[4 * f + i];
        fnode[3 * f + i] = vn[4 * v];
        fwt[3 * f + i] = (float)vwd[4 * v];
      }
    }
  }
  std::vector<int32_t> eslot((size_t)M->nelt * kElemNodes * kElemNodes, 0);
  for (int64_t K = 0; K < M->nelt; ++K)
    for (int u = 0; u < kElemNodes; ++u)
      for (int v = 0; v < kElemNodes; ++v) {
        const int32_t a = elist[K * kElemNodes + u], b = elist[K * kElemNodes + v];
        if (a >= 0 && b >= 0) eslot[(K * kElemNodes + u) * kElemNodes + v] = csr_find(rowptr[0], col[0], a, b);
      }

  // coarser levels: interpolation, its transpose, the Galerkin pattern and triples
  int64_t off = nver;
  std::vector<std::vector<int32_t>> pn(nlev), tptr(nlev), tidx(nlev);
  std::vector<std::vector<float>> pw(nlev), tw(nlev);
  c->rap_n.assign(nlev - 1, 0);
  c->rap_src.assign(nlev - 1, nullptr);
  c->rap_dst.assign(nlev - 1, nullptr);
  c->rap_w.assign(nlev - 1, nullptr);
  for (int l = 0; l + 1 < nlev; ++l) {
    const int64_t nf = sizes[l], nc = sizes[l + 1];
    pn[l].assign(nodes + 4 * off, nodes + 4 * (off + nf));
    std::vector<double> pwd(weights + 4 * off, weights + 4 * (off + nf));
    for (int64_t q = 0; q < 4 * nf; ++q)
      if (pn[l][q] < 0 || pwd[q] == 0.0) {
        pn[l][q] = -1;
        pwd[q] = 0.0;
      }
    pw[l].assign(pwd.begin(), pwd.end());
    // transpose
    tptr[l].assign(nc + 1, 0);
    for (int64_t q = 0; q < 4 * nf; ++q)
      if (pn[l][q] >= 0) tptr[l][pn[l][q] + 1]++;
    for (int64_t J = 0; J < nc; ++J) tptr[l][J + 1] += tptr[l][J];
    tidx[l].resize(tptr[l][nc]);
    tw[l].resize(tptr[l][nc]);
    {
      std::vector<int32_t> fill(tptr[l].begin(), tptr[l].end() - 1);
      for (int64_t i = 0; i < nf; ++i)
        for (int j = 0; j < 4; ++j) {
          const int32_t J = pn[l][4 * i + j];
          if (J < 0) continue;
          tidx[l][fill[J]] = (int32_t)i;
          tw[l][fill[J]++] = (float)pwd[4 * i + j];
        }
    }
    // Galerkin triples
    std::vector<int64_t> tk;
    std::vector<int32_t> tsrc;
    std::vector<double> tws;
    for (int64_t i = 0; i < nf; ++i)
      for (int k = rowptr[l][i]; k < rowptr[l][i + 1]; ++k) {
        const int64_t j = col[l][k];
        for (int a = 0; a < 4; ++a) {
          const int32_t I = pn[l][4 * i + a];
          if (I < 0) continue;
          for (int b = 0; b < 4; ++b) {
            const int32_t J = pn[l][4 * j + b];
            if (J < 0) continue;
            tk.push_back((int64_t)I * nc + J);
            tsrc.push_back(k);
            tws.push_back(pwd[4 * i + a] * pwd[4 * j + b]);
          }
        }
      }
    std::vector<int64_t> ukeys = tk;
    keys_to_csr(ukeys, nc, nc, rowptr[l + 1], col[l + 1]);
    std::vector<int32_t> tdst(tk.size());
    for (size_t q = 0; q < tk.size(); ++q) tdst[q] = csr_find(rowptr[l + 1], col[l + 1], tk[q] / nc, tk[q] % nc);
    c->rap_n[l] = (int64_t)tk.size();
    if ((rc = upload(&c->rap_src[l], tsrc)) || (rc = upload(&c->rap_dst[l], tdst)) || (rc = upload(&c->rap_w[l], tws))) {
      coarse_free(M);
      return rc;
    }
    off += nf;
  }

  // device arrays
  for (int l = 0; l < nlev && !rc; ++l) {
    CoarseLevel& L = c->lv[l];
    L.nnz = (int64_t)col[l].size();
    rc = upload(&L.rowptr, rowptr[l]);
    if (!rc) rc = upload(&L.col, col[l]);
    if (!rc) rc = alloc(&L.val, L.nnz);
    if (!rc) rc = alloc(&L.valf, L.nnz);
    if (!rc) rc = alloc(&L.dinv, L.n);
    if (!rc) rc = alloc(&L.b, L.n);
    if (!rc) rc = alloc(&L.x, L.n);
    if (!rc) rc = alloc(&L.t, L.n);
    if (!rc && l + 1 < nlev) {
      L.nnext = sizes[l + 1];
      L.ntr = (int64_t)tidx[l].size();
      rc = upload(&L.pn, pn[l]);
      if (!rc) rc = upload(&L.pw, pw[l]);
      if (!rc) rc = upload(&L.tptr, tptr[l]);
      if (!rc) rc = upload(&L.tidx, tidx[l]);
      if (!rc) rc = upload(&L.tw, tw[l]);
    }
  }
  c->nL = sizes[nlev - 1];
  if (!rc) rc = upload(&c->vnodes, vn);
  if (!rc) rc = upload(&c->vw, vw);
  if (!rc) rc = upload(&c->vwd, vwd);
  if (!rc) rc = upload(&c->gptr, gptr);
  if (!rc) rc = upload(&c->gfi, gfi);
  if (!rc) rc = upload(&c->gw, gw);
  if (!rc && !fnode.empty()) rc = upload(&c->fnode, fnode);
  if (!rc && !fwt.empty()) rc = upload(&c->fwt, fwt);
  if (!rc) rc = upload(&c->elist, elist);
  if (!rc) rc = upload(&c->eslot, eslot);
  if (!rc) rc = alloc(&c->rc, n0);
  if (!rc) {  // FP32 copy of (varpi . D)^T Xi for the per-iteration kernels
    std::vector<double> Td(3 * M->tab.d2);
    rc = cudaMemcpy(Td.data(), M->d_Tproj, sizeof(double) * Td.size(), cudaMemcpyDeviceToHost) == cudaSuccess
             ? HDG_OK
             : fail(HDG_ERR_CUDA, "copy of the face projection table");
    if (!rc) rc = upload(&c->Tf, std::vector<float>(Td.begin(), Td.end()));
  }
  if (!rc) rc = alloc(&c->e0, n0);
  if (!rc) rc = alloc(&c->Adense, c->nL * c->nL);
  if (!rc) rc = alloc(&c->Ainv, c->nL * c->nL);
  if (!rc) rc = upload(&c->d_lv, c->lv);
  if (rc) {
    coarse_free(M);
    return rc;
  }
  c->ready = false;
  return HDG_OK;
}

// Galerkin values of the whole hierarchy on M->stream, no host synchronisation (also used
// inside the batch graph); rows with a non-positive diagonal or pivot count in d_status[3].
int coarse_launch_build(hdg_mesh* M) {
  Coarse* c = M->coarse;
  cudaStream_t st = M->stream;
  for (const CoarseLevel& L : c->lv) HDG_CUDA_TRY(cudaMemsetAsync(L.val, 0, sizeof(double) * L.nnz, st));
  const unsigned gb = (unsigned)std::min<int64_t>((M->nelt + kGalWarps - 1) / kGalWarps, 152 * 16);
#define HDG_GAL(D)                                                                                             \
  if (M->c32_ready && M->d_C32)                                                                               \
    galerkin0_kernel<D, float><<<gb, 32 * kGalWarps, 0, st>>>(M->nelt, M->d_C32, M->d_facebyele, M->d_ftype,   \
                                                              M->d_fverts, M->d_Tproj, c->vnodes, c->vwd,      \
                                                              c->elist, c->eslot, c->lv[0].val);               \
  else                                                                                                        \
    galerkin0_kernel<D, double><<<gb, 32 * kGalWarps, 0, st>>>(M->nelt, M->d_C, M->d_facebyele, M->d_ftype,   \
                                                               M->d_fverts, M->d_Tproj, c->vnodes, c->vwd,     \
                                                               c->elist, c->eslot, c->lv[0].val)
  switch (M->tab.d2) {
    case 1: HDG_GAL(1); break;
    case 3: HDG_GAL(3); break;
    case 6: HDG_GAL(6); break;
    case 10: HDG_GAL(10); break;
    case 15: HDG_GAL(15); break;
    default: return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
  }
#undef HDG_GAL
  for (int l = 0; l + 1 < c->nlev; ++l) {
    const unsigned g = (unsigned)std::min<int64_t>((c->rap_n[l] + 255) / 256, 1216);
    rap_kernel<<<std::max(g, 1u), 256, 0, st>>>(c->rap_n[l], c->rap_src[l], c->rap_dst[l], c->rap_w[l],
                                                c->lv[l].val, c->lv[l + 1].val);
  }
  for (const CoarseLevel& L : c->lv) {
    const unsigned g = (unsigned)std::min<int64_t>((L.n + 255) / 256, 1216);
    level_finish_kernel<<<g, 256, 0, st>>>(L, M->d_status + 3);
  }
  coarsest_inverse_kernel<<<1, 1024, 0, st>>>(c->lv[c->nlev - 1], c->Adense, c->Ainv, M->d_status + 3);
  M->launches += 2 + 2 * c->nlev;
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int coarse_build(hdg_mesh* M) {
  Coarse* c = M->coarse;
  if (!c) return fail(HDG_ERR_STATE, "no coarse space");
  if (!M->assembled) return fail(HDG_ERR_STATE, "coarse space before hdg_assemble_condense");
  cudaStream_t st = M->stream;
  HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 3, 0, sizeof(int32_t), st));
  int rc = coarse_launch_build(M);
  if (rc) return rc;
  int32_t st4[4];
  HDG_CUDA_TRY(cudaMemcpyAsync(st4, M->d_status, sizeof(st4), cudaMemcpyDeviceToHost, st));
  HDG_CUDA_TRY(cudaStreamSynchronize(st));
  if (st4[3]) return fail(HDG_ERR_LOCAL_SINGULAR, "coarse Galerkin matrix with a non-positive diagonal or pivot");
  c->ready = true;
  return HDG_OK;
}

}  // namespace hdg

using namespace hdg;

extern "C" {

int hdg_set_coarse_space(hdg_mesh* M, int nlev, const int64_t* sizes, const int32_t* nodes, const double* weights) {
  if (!M) return fail(HDG_ERR_ARG, "NULL mesh");
  if (M->stream) cudaStreamSynchronize(M->stream);
  // the cached PCG graphs hold pointers into the old coarse space: rebuild them at the next solve
  cudaGraphExec_t* gs[] = {&M->graph64, &M->graph32, &M->wgraph64, &M->wgraph32, &M->graph_bicg, &M->graph_bicg32,
                           &M->wgraph_bicg, &M->wgraph_bicg32};
  for (cudaGraphExec_t* g : gs)
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  M->graphs_tl = false;
  M->coarse_gen++;
  coarse_free(M);
  if (nlev == 0) return HDG_OK;
  return set_coarse(M, nlev, sizes, nodes, weights);
}

int hdg_coarse_precond_apply(hdg_mesh* M, const double* r, double* z) {
  if (!M || !r || !z) return fail(HDG_ERR_ARG, "NULL argument");
  return coarse_precond_apply(M, r, z);
}

}  // extern "C"
