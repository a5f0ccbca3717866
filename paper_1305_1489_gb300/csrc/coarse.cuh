// Two-level additive preconditioner of the trace PCG (not in the paper, which solves eq. 6.5
// directly):
//     M^-1 r = B^-1 r + Pi V(Pi^T r)
// B = block-Jacobi part of H (the d2 x d2 face blocks), Pi = trace of a continuous
// piecewise-linear field (vertex values -> face coefficients, exact for k >= 1: the trace of a
// linear function on a face is linear, so T = (varpi . D)^T Xi gives its eq. 6.3 coefficients),
// V = one symmetric V-cycle for the Galerkin matrix A_0 = Pi^T H Pi over nested P1 levels,
// A_{l+1} = P_l^T A_l P_l, with one l1-Jacobi sweep before and after each coarse correction and
// an exact dense solve on the coarsest level.  B^-1 and V are symmetric positive definite, so
// M^-1 is, and PCG stays the textbook method.
//
// The kernels below return at once when *done != 0 (the solve converged earlier in the
// captured batch of iterations).
//
// Per PCG iteration (after q = H p and alpha):
//   update_tl   x += alpha p, r -= alpha q, r.r
//   restrict    rc = Pi^T r: one warp per level-0 node gathers its (face, vertex slot, weight)
//               list (built on the host), FP32 sums, no atomics
//   down        level 0 and every level above kTailMax nodes (grid kernels, 16 lanes per
//               row): x = D^-1 b, t = b - A x; coarser grid levels first gather b = P^T t
//   vcycle      one CTA: the remaining small levels (restrict, smooth, exact coarsest,
//               prolong, smooth)
//   up          grid levels, coarse to fine: x' = x + P x_coarse, out = x' + D^-1 (b - A x');
//               level 0 writes e0
//   zc          z = B^-1 r + Pi e0, r.z, beta
// The coarse correction runs in FP32 (a preconditioner only has to be fixed, symmetric and
// positive; GB300's FP64 pipe is 1/63 of its FP32 rate); every scalar of the Krylov method and
// the FP64 solve itself are unchanged.
#pragma once

#include <cstdint>
#include <vector>

namespace hdg {

constexpr int kVcThreads = 1024;  // threads of the single-CTA V-cycle kernel
constexpr int kMaxCoarsest = 128;  // largest coarsest level (dense inverse)
constexpr int kTailMax = 1024;     // levels up to this size run inside the single-CTA kernel

// One level of the hierarchy on the device.  Level l holds A_l (CSR), the l1-Jacobi inverse
// diagonal, its interpolation from level l+1 (ELL [n][4]) and the transpose of that
// interpolation (CSR over level-(l+1) rows), and three FP32 work vectors.
struct CoarseLevel {
  int64_t n = 0, nnz = 0;
  int32_t *rowptr = nullptr, *col = nullptr;
  double* val = nullptr;   // Galerkin values (FP64, built after every assembly)
  float* valf = nullptr;   // FP32 copy used by the V-cycle
  float* dinv = nullptr;   // 1 / sum_j |a_ij|
  int32_t* pn = nullptr;   // [n][4] level-(l+1) nodes interpolating node i (-1 unused)
  float* pw = nullptr;     // [n][4] their weights
  int32_t *tptr = nullptr, *tidx = nullptr;  // transpose of (pn, pw): rows = level-(l+1) nodes
  float* tw = nullptr;
  int64_t ntr = 0;         // entries of the transpose
  int64_t nnext = 0;       // nodes of level l+1 (0 on the coarsest level)
  float *b = nullptr, *x = nullptr, *t = nullptr;
};

constexpr int kMaxTailLevels = 16;         // tail levels of the single-CTA kernel (nlev <= 17)
constexpr int64_t kTailSmemMax = 200 << 10;  // largest shared-memory copy of the tail

// bytes of the shared-memory copy of one tail level (16-byte aligned arrays)
__host__ __device__ inline int64_t tail_align(int64_t b) { return (b + 15) & ~int64_t(15); }
__host__ __device__ inline int64_t tail_level_bytes(const CoarseLevel& L) {
  int64_t b = tail_align(4 * (L.n + 1)) + 2 * tail_align(4 * L.nnz) + 4 * tail_align(4 * L.n);
  if (L.nnext > 0) b += 2 * tail_align(16 * L.n) + tail_align(4 * (L.nnext + 1)) + 2 * tail_align(4 * L.ntr);
  return b;
}

// Level-0 arguments of the face kernels.
struct CoarseArgs {
  const int32_t* fverts;  // [nfc][3] sorted face vertices
  const float* Tf;        // [d2][3]  (varpi . D)^T Xi, FP32
  const int32_t* vnodes;  // [nver][4] level-0 nodes of each mesh vertex
  const float* vw;        // [nver][4] weights
  float* rc;              // [n0] Pi^T r
  const float* e0;        // [n0] V-cycle output on level 0
  int64_t n0;
  const int32_t* gptr;    // [n0+1] CSR of the restriction gather
  const int32_t* gfi;     // 4 f + i: free face f whose vertex slot i carries the node
  const float* gw;        // weight of the node at that vertex
  const int32_t* fnode;   // [nfc][3] level-0 node of each face vertex (-1: none), or NULL when
  const float* fwt;       //   a vertex may carry several nodes; [nfc][3] their weights
};

struct Coarse {
  int nlev = 0;
  std::vector<CoarseLevel> lv;
  CoarseLevel* d_lv = nullptr;  // device copy of lv (for the V-cycle kernel)
  int32_t* vnodes = nullptr;
  float* vw = nullptr;
  double* vwd = nullptr;     // FP64 weights for the Galerkin set-up
  int32_t *gptr = nullptr, *gfi = nullptr;  // restriction gather (CoarseArgs)
  float* gw = nullptr;
  int32_t* fnode = nullptr;  // per-face vertex nodes when every vertex carries at most one node
  float* fwt = nullptr;
  int32_t* elist = nullptr;  // [nelt][8] level-0 nodes touched by the element (-1 unused)
  int32_t* eslot = nullptr;  // [nelt][64] CSR positions in A_0 of the pairs of elist
  std::vector<int64_t> rap_n;             // Galerkin triple counts per level
  std::vector<int32_t*> rap_src, rap_dst; // A_{l+1}[dst] += w A_l[src]
  std::vector<double*> rap_w;
  float* rc = nullptr;
  float* Tf = nullptr;       // FP32 copy of (varpi . D)^T Xi
  float* e0 = nullptr;
  double* Adense = nullptr;  // [nL][nL] FP64 scratch of the coarsest inverse
  float* Ainv = nullptr;     // [nL][nL]
  int64_t nL = 0;
  int64_t tail_max = kTailMax;  // levels up to this size run in the single-CTA kernel
  int64_t tail_smem = 0;        // bytes of the tail's shared-memory copy (0: the tail reads global)
  bool ready = false;        // Galerkin hierarchy built for the current assembly
};

// ------------------------------------------------------------------ per-iteration kernels
// rc = Pi^T r: one warp per level-0 node sums sum_a T[a][i] r[f][a] weighted over its list
template <typename T, int D2>
__global__ void restrict_gather_kernel(CoarseArgs CA, const T* __restrict__ r, const double* done) {
  if (*done != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; n < CA.n0; n += nwarps) {
    float s = 0.f;
    for (int k = CA.gptr[n] + lane; k < CA.gptr[n + 1]; k += 32) {
      const int32_t fi = CA.gfi[k];
      const int64_t f = fi >> 2;
      const int i = fi & 3;
      float t = 0.f;
      if constexpr (sizeof(T) == 4 && D2 % 2 == 0) {  // the face's entries start on 8 bytes: pairs
        const float2* rf = reinterpret_cast<const float2*>(r + f * D2);
#pragma unroll
        for (int a = 0; a < D2; a += 2) {
          const float2 v = rf[a / 2];
          t = fmaf(CA.Tf[a * 3 + i], v.x, t);
          t = fmaf(CA.Tf[(a + 1) * 3 + i], v.y, t);
        }
      } else {
#pragma unroll
        for (int a = 0; a < D2; ++a) t = fmaf(CA.Tf[a * 3 + i], (float)r[f * D2 + a], t);
      }
      s = fmaf(CA.gw[k], t, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) CA.rc[n] = s;
  }
}

// (Pi e0) entry a of face e
template <int D2>
__device__ __forceinline__ float prolong_face(const CoarseArgs& CA, int64_t e, int a) {
  float s = 0.f;
  if (CA.fnode) {  // one node per vertex (the P1 space of the mesh itself)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int nd = CA.fnode[3 * e + i];
      if (nd >= 0) s = fmaf(CA.Tf[a * 3 + i] * CA.fwt[3 * e + i], CA.e0[nd], s);
    }
    return s;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int64_t v = CA.fverts[3 * e + i];
    float val = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nd = CA.vnodes[4 * v + j];
      if (nd >= 0) val = fmaf(CA.vw[4 * v + j], CA.e0[nd], val);
    }
    s = fmaf(CA.Tf[a * 3 + i], val, s);
  }
  return s;
}

// Grid-wide level kernels (levels with more than the tail size, and always level 0): a group
// of 16 lanes per row shares the row's entries and sums them with shuffles.  The right-hand
// side of level 0 is rc; of a coarser level, its b.
constexpr int kRowLanes = 16;

__device__ __forceinline__ float group_sum16(float v) {
#pragma unroll
  for (int o = kRowLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// down: x = D^-1 b, t = b - A x (the x of the neighbours formed on the fly from b)
template <bool L0>
__global__ void level_down_kernel(CoarseLevel L, const float* __restrict__ rc, const double* done) {
  if (*done != 0.0) return;
  const int g = threadIdx.x & (kRowLanes - 1);
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / kRowLanes;
  // every lane of a warp runs the same number of trips (the shuffles need full warps)
  const int64_t trips = (L.n + ngroups - 1) / ngroups;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowLanes;
  for (int64_t trip = 0; trip < trips; ++trip) {
    const int64_t i = i0 + trip * ngroups;
    float ax = 0.f;
    if (i < L.n)
      for (int k = L.rowptr[i] + g; k < L.rowptr[i + 1]; k += kRowLanes) {
        const int j = L.col[k];
        ax = fmaf(L.valf[k], L.dinv[j] * (L0 ? rc[j] : L.b[j]), ax);
      }
    ax = group_sum16(ax);
    if (i < L.n && g == 0) {
      const float bi = L0 ? rc[i] : L.b[i];
      L.x[i] = L.dinv[i] * bi;
      L.t[i] = bi - ax;
    }
  }
}

// restriction to a grid level: C.b = P^T t of the finer level P
static __global__ void level_restrict_kernel(CoarseLevel P, CoarseLevel C, const double* done) {
  if (*done != 0.0) return;
  for (int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; J < C.n; J += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = P.tptr[J]; k < P.tptr[J + 1]; ++k) s = fmaf(P.tw[k], P.t[P.tidx[k]], s);
    C.b[J] = s;
  }
}

// x' = x + P x_next (the coarse correction interpolated)
__device__ __forceinline__ float level_corrected(const CoarseLevel& L, const float* __restrict__ xn, int64_t j) {
  float v = L.x[j];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int nd = L.pn[4 * j + q];
    if (nd >= 0) v = fmaf(L.pw[4 * j + q], xn[nd], v);
  }
  return v;
}

// up: out = x' + D^-1 (b - A x')
template <bool L0>
__global__ void level_up_kernel(CoarseLevel L, const float* __restrict__ xn, const float* __restrict__ rc,
                                float* __restrict__ out, const double* done) {
  if (*done != 0.0) return;
  const int g = threadIdx.x & (kRowLanes - 1);
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) / kRowLanes;
  const int64_t trips = (L.n + ngroups - 1) / ngroups;
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowLanes;
  for (int64_t trip = 0; trip < trips; ++trip) {
    const int64_t i = i0 + trip * ngroups;
    float ax = 0.f;
    if (i < L.n)
      for (int k = L.rowptr[i] + g; k < L.rowptr[i + 1]; k += kRowLanes)
        ax = fmaf(L.valf[k], level_corrected(L, xn, L.col[k]), ax);
    ax = group_sum16(ax);
    if (i < L.n && g == 0) {
      const float bi = L0 ? rc[i] : L.b[i];
      out[i] = level_corrected(L, xn, i) + L.dinv[i] * (bi - ax);
    }
  }
}

// Levels first .. nlev-1 of the V-cycle in one CTA (the tail of small levels, at most the tail
// size each).  Input: lv[first-1].t (residual of the finer level); output: lv[first].x.  With
// use_smem the tail's matrices, interpolations and vectors are first copied into dynamic
// shared memory (tail_level_bytes each), so that the dozen barrier-separated phases below
// read shared memory instead of L2.
template <typename V>
__device__ __forceinline__ V* tail_take(unsigned char*& p, int64_t count) {
  V* q = reinterpret_cast<V*>(p);
  p += tail_align(sizeof(V) * count);
  return q;
}

// Copy of the tail's arrays into shared memory in one flattened pass, so that every thread
// issues all its loads before its first store (one memory latency for the whole copy).
// Segments are 4-byte arrays: whole 16-byte chunks first, then the remaining words.
constexpr int kMaxTailSegs = kMaxTailLevels * 9;

struct TailSegs {
  const int32_t* src[kMaxTailSegs];
  int32_t* dst[kMaxTailSegs];
  int32_t start16[kMaxTailSegs + 1];  // prefix of 16-byte chunks
  int32_t startw[kMaxTailSegs + 1];   // prefix of remaining words
  int nseg;
};

__device__ __forceinline__ int tail_find(const int32_t* start, int nseg, int c) {
  int lo = 0, hi = nseg - 1;  // last segment with start[s] <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void tail_copy_all(const TailSegs& S) {
  constexpr int U = 8;
  const int bs = blockDim.x, tid = threadIdx.x;
  const int total16 = S.start16[S.nseg];
  for (int base = tid; base < total16; base += U * bs) {
    int4 v[U];
    int4* d[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = base + u * bs;
      d[u] = nullptr;
      if (c < total16) {
        const int sg = tail_find(S.start16, S.nseg, c);
        const int off = c - S.start16[sg];
        v[u] = __ldg(reinterpret_cast<const int4*>(S.src[sg]) + off);
        d[u] = reinterpret_cast<int4*>(S.dst[sg]) + off;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (d[u]) *d[u] = v[u];
  }
  const int totalw = S.startw[S.nseg];
  for (int c = tid; c < totalw; c += bs) {
    const int sg = tail_find(S.startw, S.nseg, c);
    const int full = (S.start16[sg + 1] - S.start16[sg]) * 4;
    const int w = full + (c - S.startw[sg]);
    S.dst[sg][w] = __ldg(S.src[sg] + w);
  }
}

static __global__ void __launch_bounds__(kVcThreads) vcycle_kernel(const CoarseLevel* __restrict__ lv, int first,
                                                            int nlev, const float* __restrict__ Ainv,
                                                            const double* done, int use_smem) {
  if (*done != 0.0) return;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ CoarseLevel sl[kMaxTailLevels];
  const int tid = threadIdx.x;
  const int nt = nlev - first;
  if (use_smem) {
    __shared__ TailSegs segs;
    if (tid == 0) {
      unsigned char* p = tail_smem;
      int ns = 0;
      auto add = [&](const void* src, void* dst, int64_t words) {
        segs.src[ns] = reinterpret_cast<const int32_t*>(src);
        segs.dst[ns] = reinterpret_cast<int32_t*>(dst);
        segs.start16[ns + 1] = segs.start16[ns] + (int32_t)(words / 4);
        segs.startw[ns + 1] = segs.startw[ns] + (int32_t)(words % 4);
        ++ns;
      };
      segs.start16[0] = 0;
      segs.startw[0] = 0;
      for (int t = 0; t < nt; ++t) {
        const CoarseLevel& G = lv[first + t];
        CoarseLevel S = G;
        S.rowptr = tail_take<int32_t>(p, S.n + 1);
        S.col = tail_take<int32_t>(p, S.nnz);
        S.valf = tail_take<float>(p, S.nnz);
        S.dinv = tail_take<float>(p, S.n);
        S.b = tail_take<float>(p, S.n);
        S.x = tail_take<float>(p, S.n);
        S.t = tail_take<float>(p, S.n);
        add(G.rowptr, S.rowptr, S.n + 1);
        add(G.col, S.col, S.nnz);
        add(G.valf, S.valf, S.nnz);
        add(G.dinv, S.dinv, S.n);
        if (S.nnext > 0) {
          S.pn = tail_take<int32_t>(p, 4 * S.n);
          S.pw = tail_take<float>(p, 4 * S.n);
          S.tptr = tail_take<int32_t>(p, S.nnext + 1);
          S.tidx = tail_take<int32_t>(p, S.ntr);
          S.tw = tail_take<float>(p, S.ntr);
          add(G.pn, S.pn, 4 * S.n);
          add(G.pw, S.pw, 4 * S.n);
          add(G.tptr, S.tptr, S.nnext + 1);
          add(G.tidx, S.tidx, S.ntr);
          add(G.tw, S.tw, S.ntr);
        }
        sl[t] = S;
      }
      segs.nseg = ns;
    }
    __syncthreads();
    tail_copy_all(segs);
  } else if (tid < nt) {
    sl[tid] = lv[first + tid];
  }
  __syncthreads();
  // level l of the cycle: the grid level first-1 stays in global memory
  auto lev = [&](int l) -> const CoarseLevel& { return l < first ? lv[l] : sl[l - first]; };
  int l = first;
  for (; l < nlev; ++l) {
    const CoarseLevel& P = lev(l - 1);  // interpolation l -> l-1 is stored on level l-1
    const CoarseLevel& C = lev(l);
    for (int64_t J = tid; J < C.n; J += kVcThreads) {
      float s = 0.f;
      for (int k = P.tptr[J]; k < P.tptr[J + 1]; ++k) s = fmaf(P.tw[k], P.t[P.tidx[k]], s);
      C.b[J] = s;
    }
    __syncthreads();
    if (l == nlev - 1) break;
    for (int64_t i = tid; i < C.n; i += kVcThreads) C.x[i] = C.dinv[i] * C.b[i];
    __syncthreads();
    for (int64_t i = tid; i < C.n; i += kVcThreads) {
      float ax = 0.f;
      for (int k = C.rowptr[i]; k < C.rowptr[i + 1]; ++k) ax = fmaf(C.valf[k], C.x[C.col[k]], ax);
      C.t[i] = C.b[i] - ax;
    }
    __syncthreads();
  }
  {  // coarsest: x = A^-1 b (dense)
    const CoarseLevel& C = lev(nlev - 1);
    for (int64_t i = tid; i < C.n; i += kVcThreads) {
      float s = 0.f;
      for (int64_t j = 0; j < C.n; ++j) s = fmaf(Ainv[i * C.n + j], C.b[j], s);
      C.x[i] = s;
    }
    __syncthreads();
  }
  for (l = nlev - 2; l >= first; --l) {
    const CoarseLevel& C = lev(l);
    const float* xc = lev(l + 1).x;
    for (int64_t i = tid; i < C.n; i += kVcThreads) {
      float v = C.x[i];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int nd = C.pn[4 * i + q];
        if (nd >= 0) v = fmaf(C.pw[4 * i + q], xc[nd], v);
      }
      C.x[i] = v;
    }
    __syncthreads();
    for (int64_t i = tid; i < C.n; i += kVcThreads) {
      float ax = 0.f;
      for (int k = C.rowptr[i]; k < C.rowptr[i + 1]; ++k) ax = fmaf(C.valf[k], C.x[C.col[k]], ax);
      C.t[i] = C.dinv[i] * (C.b[i] - ax);
    }
    __syncthreads();
    for (int64_t i = tid; i < C.n; i += kVcThreads) C.x[i] += C.t[i];
    __syncthreads();
  }
  if (use_smem) {  // the result of the first tail level goes back to global memory
    const CoarseLevel& C = sl[0];
    float* out = lv[first].x;
    for (int64_t i = tid; i < C.n; i += kVcThreads) out[i] = C.x[i];
  }
}

}  // namespace hdg
