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
//               list (built on the host), FP64 sums, no atomics
//   down        level 0 and every level above kTailMax nodes (grid kernels): x = D^-1 b,
//               t = b - A x; coarser grid levels first gather b = P^T t
//   vcycle      one CTA: the remaining small levels (restrict, smooth, exact coarsest,
//               prolong, smooth)
//   up          grid levels, coarse to fine: x' = x + P x_coarse, out = x' + D^-1 (b - A x');
//               level 0 writes e0
//   zc          z = B^-1 r + Pi e0, r.z, beta
// The V-cycle runs in FP32 (a preconditioner only has to be fixed, symmetric and positive);
// every scalar of the Krylov method and the FP64 solve itself are unchanged.
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
  float *b = nullptr, *x = nullptr, *t = nullptr;
};

// Level-0 arguments of the face kernels.
struct CoarseArgs {
  const int32_t* fverts;  // [nfc][3] sorted face vertices
  const double* T;        // [d2][3]  (varpi . D)^T Xi
  const int32_t* vnodes;  // [nver][4] level-0 nodes of each mesh vertex
  const float* vw;        // [nver][4] weights
  double* rc;             // [n0] Pi^T r
  const float* e0;        // [n0] V-cycle output on level 0
  int64_t n0;
  const int32_t* gptr;    // [n0+1] CSR of the restriction gather
  const int32_t* gfi;     // 4 f + i: free face f whose vertex slot i carries the node
  const float* gw;        // weight of the node at that vertex
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
  int32_t* elist = nullptr;  // [nelt][8] level-0 nodes touched by the element (-1 unused)
  int32_t* eslot = nullptr;  // [nelt][64] CSR positions in A_0 of the pairs of elist
  std::vector<int64_t> rap_n;             // Galerkin triple counts per level
  std::vector<int32_t*> rap_src, rap_dst; // A_{l+1}[dst] += w A_l[src]
  std::vector<double*> rap_w;
  double* rc = nullptr;
  float* e0 = nullptr;
  double* Adense = nullptr;  // [nL][nL] FP64 scratch of the coarsest inverse
  float* Ainv = nullptr;     // [nL][nL]
  int64_t nL = 0;
  int64_t tail_max = kTailMax;  // levels up to this size run in the single-CTA kernel
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
    double s = 0.0;
    for (int k = CA.gptr[n] + lane; k < CA.gptr[n + 1]; k += 32) {
      const int32_t fi = CA.gfi[k];
      const int64_t f = fi >> 2;
      const int i = fi & 3;
      double t = 0.0;
#pragma unroll
      for (int a = 0; a < D2; ++a) t = fma(CA.T[a * 3 + i], (double)r[f * D2 + a], t);
      s = fma((double)CA.gw[k], t, s);
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
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int64_t v = CA.fverts[3 * e + i];
    float val = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nd = CA.vnodes[4 * v + j];
      if (nd >= 0) val = fmaf(CA.vw[4 * v + j], CA.e0[nd], val);
    }
    s = fmaf((float)CA.T[a * 3 + i], val, s);
  }
  return s;
}

// Grid-wide level kernels (levels with more than kTailMax nodes, and always level 0).  The
// right-hand side of level 0 is rc (FP64); of a coarser level, its b.
// down: x = D^-1 b, t = b - A x (the x of the neighbours formed on the fly from b)
template <bool L0>
__global__ void level_down_kernel(CoarseLevel L, const double* __restrict__ rc, const double* done) {
  if (*done != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float bi = L0 ? (float)rc[i] : L.b[i];
    float ax = 0.f;
    for (int k = L.rowptr[i]; k < L.rowptr[i + 1]; ++k) {
      const int j = L.col[k];
      ax = fmaf(L.valf[k], L.dinv[j] * (L0 ? (float)rc[j] : L.b[j]), ax);
    }
    L.x[i] = L.dinv[i] * bi;
    L.t[i] = bi - ax;
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
__global__ void level_up_kernel(CoarseLevel L, const float* __restrict__ xn, const double* __restrict__ rc,
                                float* __restrict__ out, const double* done) {
  if (*done != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    float ax = 0.f;
    for (int k = L.rowptr[i]; k < L.rowptr[i + 1]; ++k) ax = fmaf(L.valf[k], level_corrected(L, xn, L.col[k]), ax);
    const float bi = L0 ? (float)rc[i] : L.b[i];
    out[i] = level_corrected(L, xn, i) + L.dinv[i] * (bi - ax);
  }
}

// Levels first .. nlev-1 of the V-cycle in one CTA (the tail of small levels, at most
// kTailMax nodes each).  Input: lv[first-1].t (residual of the finer level); output: lv[first].x.
static __global__ void __launch_bounds__(kVcThreads) vcycle_kernel(const CoarseLevel* __restrict__ lv, int first,
                                                            int nlev, const float* __restrict__ Ainv,
                                                            const double* done) {
  if (*done != 0.0) return;
  const int tid = threadIdx.x;
  int l = first;
  for (; l < nlev; ++l) {
    const CoarseLevel& P = lv[l - 1];  // interpolation l -> l-1 is stored on level l-1
    const CoarseLevel& C = lv[l];
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
    const CoarseLevel& C = lv[nlev - 1];
    for (int64_t i = tid; i < C.n; i += kVcThreads) {
      float s = 0.f;
      for (int64_t j = 0; j < C.n; ++j) s = fmaf(Ainv[i * C.n + j], C.b[j], s);
      C.x[i] = s;
    }
    __syncthreads();
  }
  for (l = nlev - 2; l >= first; --l) {
    const CoarseLevel& C = lv[l];
    const float* xc = lv[l + 1].x;
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
}

}  // namespace hdg
