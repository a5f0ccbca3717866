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
//   update_tl   x += alpha p, r -= alpha q, r.r, and rc = Pi^T r (face -> vertex -> level-0
//               node, FP64 atomics; one thread per free face)
//   l0_down     level 0 (grid): x0 = D0^-1 b0, t0 = b0 - A0 x0         (b0 = rc, FP32)
//   vcycle      one CTA: levels 1 .. L-1 (restrict t0, smooth, exact coarsest, prolong, smooth)
//   l0_up       level 0 (grid): x0' = x0 + P0 x1, e0 = x0' + D0^-1 (b0 - A0 x0')
//   zc          z = B^-1 r + Pi e0, r.z, beta; clears rc for the next restriction
// The V-cycle runs in FP32 (a preconditioner only has to be fixed, symmetric and positive);
// every scalar of the Krylov method and the FP64 solve itself are unchanged.
#pragma once

#include <cstdint>
#include <vector>

namespace hdg {

constexpr int kVcThreads = 1024;  // threads of the single-CTA V-cycle kernel
constexpr int kMaxCoarsest = 128;  // largest coarsest level (dense inverse)

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
  double* rc;             // [n0] Pi^T r (FP64 accumulation)
  const float* e0;        // [n0] V-cycle output on level 0
  int64_t n0;
};

struct Coarse {
  int nlev = 0;
  std::vector<CoarseLevel> lv;
  CoarseLevel* d_lv = nullptr;  // device copy of lv (for the V-cycle kernel)
  int32_t* vnodes = nullptr;
  float* vw = nullptr;
  double* vwd = nullptr;     // FP64 weights for the Galerkin set-up
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
  bool ready = false;        // Galerkin hierarchy built for the current assembly
};

// ------------------------------------------------------------------ per-iteration kernels
// rc += Pi^T r for the free faces of a tile (called by one thread per face, a == 0)
template <typename T, int D2>
__device__ __forceinline__ void restrict_face(const CoarseArgs& CA, const T* __restrict__ r, int64_t e) {
  double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < D2; ++a) {
    const double ra = (double)r[e * D2 + a];
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = fma(CA.T[a * 3 + i], ra, s[i]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int64_t v = CA.fverts[3 * e + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nd = CA.vnodes[4 * v + j];
      if (nd >= 0) atomicAdd(CA.rc + nd, (double)CA.vw[4 * v + j] * s[i]);
    }
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

// level 0, down: x0 = D^-1 b, t0 = b - A x0 with b = rc (x0 of the neighbours computed on the fly)
static __global__ void l0_down_kernel(CoarseLevel L0, const double* __restrict__ rc, const double* done) {
  if (*done != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L0.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float bi = (float)rc[i];
    float ax = 0.f;
    for (int k = L0.rowptr[i]; k < L0.rowptr[i + 1]; ++k) {
      const int j = L0.col[k];
      ax = fmaf(L0.valf[k], L0.dinv[j] * (float)rc[j], ax);
    }
    L0.x[i] = L0.dinv[i] * bi;
    L0.t[i] = bi - ax;
  }
}

// level 0, up: x0' = x0 + P0 x1, e0 = x0' + D^-1 (b - A x0')
__device__ __forceinline__ float l0_corrected(const CoarseLevel& L0, const float* __restrict__ x1, int64_t j) {
  float v = L0.x[j];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int nd = L0.pn[4 * j + q];
    if (nd >= 0) v = fmaf(L0.pw[4 * j + q], x1[nd], v);
  }
  return v;
}

static __global__ void l0_up_kernel(CoarseLevel L0, const float* __restrict__ x1, const double* __restrict__ rc,
                             float* __restrict__ e0, const double* done) {
  if (*done != 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L0.n; i += (int64_t)gridDim.x * blockDim.x) {
    float ax = 0.f;
    for (int k = L0.rowptr[i]; k < L0.rowptr[i + 1]; ++k) ax = fmaf(L0.valf[k], l0_corrected(L0, x1, L0.col[k]), ax);
    e0[i] = l0_corrected(L0, x1, i) + L0.dinv[i] * ((float)rc[i] - ax);
  }
}

// Levels 1 .. nlev-1 of the V-cycle in one CTA (the coarse levels are small: 1/8 of the
// previous one each).  Input: lv[0].t (level-0 residual); output: lv[1].x.
static __global__ void __launch_bounds__(kVcThreads) vcycle_kernel(const CoarseLevel* __restrict__ lv, int nlev,
                                                            const float* __restrict__ Ainv, const double* done) {
  if (*done != 0.0) return;
  const int tid = threadIdx.x;
  int l = 1;
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
  for (l = nlev - 2; l >= 1; --l) {
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
