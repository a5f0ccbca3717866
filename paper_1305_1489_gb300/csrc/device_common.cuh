// Device helpers shared by the libhdg kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hdg {

template <int K>
struct Dims {
  static constexpr int n = (K + 1) * (K + 2) * (K + 3) / 6;  // dim P_k(K)
  static constexpr int d2 = (K + 1) * (K + 2) / 2;           // dim P_k(e)
  static constexpr int m = 4 * d2;                           // dim R_k(dK)
  static constexpr int nq = (K + 2) * (K + 2) * (K + 2);     // volume nodes
  static constexpr int nf = (K + 2) * (K + 2);               // face nodes
  static constexpr int n1 = (K + 2) * (K + 3) * (K + 4) / 6; // dim P_{k+1}(K)
  // per-element recovery record (eq. 5.3 through the factors of K1), column-major blocks:
  // [H|h]^T [m+1][n] | V^T [m][n] | W_*^T [3][n][n] | U_s [n(n+1)/2] | U_M [n(n+1)/2] | normals [12]
  // (U packed by columns, column i holding U_0i .. U_(i-1)i and then 1/U_ii)
  static constexpr int tri = n * (n + 1) / 2;
  static constexpr int rec = n * (m + 1) + n * m + 3 * n * n + 2 * tri + 12;
};

// Launch shape of K1 (one element per CTA): threads per CTA and the number of CTAs each SM
// should hold (register budget 65536 / (NT * MINB) per thread); shared memory per CTA is
// 3.7 / 17 / 58 / 156 KB for k = 1..4.
template <int K>
struct K1Occupancy {
  static constexpr int NT = (K >= 3) ? 256 : 128;
  static constexpr int MINB = (K == 1) ? 8 : (K == 2) ? 4 : (K == 3) ? 3 : 1;
};

// Element geometry from the SoA vertex array vx [12][nelt] (x1..x4, y1..y4, z1..z4).
//  a[*][#] = (det B_K B_K^-T)_{*#}, the Piola cofactors of eq. 3.8;
//  nrm[l] = outward normal of local face l (eq. 2.1 order) with |nrm[l]| = |e_l| (Section 2).
struct Geo {
  double a[3][3];
  double det, vol;
  double nrm[4][3];
  double area[4];
};

__device__ __forceinline__ void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}

__device__ __forceinline__ void element_geometry(const double* __restrict__ vx, int64_t nelt,
                                                 int64_t K, Geo& g) {
  double v[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int d = 0; d < 3; ++d) v[i][d] = vx[(d * 4 + i) * nelt + K];
  double e1[3], e2[3], e3[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    e1[d] = v[1][d] - v[0][d];
    e2[d] = v[2][d] - v[0][d];
    e3[d] = v[3][d] - v[0][d];
  }
  // B_K = [e1 e2 e3]; det B B^-T has columns e2 x e3, e3 x e1, e1 x e2
  double c1[3], c2[3], c3[3];
  cross3(e2, e3, c1);
  cross3(e3, e1, c2);
  cross3(e1, e2, c3);
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    g.a[s][0] = c1[s];
    g.a[s][1] = c2[s];
    g.a[s][2] = c3[s];
  }
  g.det = e1[0] * c1[0] + e1[1] * c1[1] + e1[2] * c1[2];
  g.vol = g.det / 6.0;
  // faces 1 and 3 of eq. 2.1 are inward with their vertex order, faces 2 and 4 outward
  double f4a[3], f4b[3], t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g.nrm[0][d] = -0.5 * c3[d];   // -(1/2) e1 x e2
    g.nrm[2][d] = -0.5 * c1[d];   // -(1/2) e2 x e3
    f4a[d] = v[1][d] - v[3][d];
    f4b[d] = v[2][d] - v[3][d];
  }
  cross3(e1, e3, t);
#pragma unroll
  for (int d = 0; d < 3; ++d) g.nrm[1][d] = 0.5 * t[d];
  cross3(f4a, f4b, t);
#pragma unroll
  for (int d = 0; d < 3; ++d) g.nrm[3][d] = 0.5 * t[d];
#pragma unroll
  for (int l = 0; l < 4; ++l)
    g.area[l] = sqrt(g.nrm[l][0] * g.nrm[l][0] + g.nrm[l][1] * g.nrm[l][1] + g.nrm[l][2] * g.nrm[l][2]);
}

// In-place Cholesky (lower) of an N x N symmetric positive definite matrix in shared memory,
// row-major, by one warp (left-looking by columns).  invd receives 1/L_jj.  Returns, on
// every lane, whether all pivots were positive.
template <int N>
__device__ __forceinline__ bool warp_cholesky(double* A, double* invd, int lane) {
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    // L_jj = sqrt(A_jj - sum_{l<j} L_jl^2)
    double s = 0.0;
    for (int l = lane; l < j; l += 32) s = fma(A[j * N + l], A[j * N + l], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    double d = A[j * N + j] - s;
    ok = ok && (d > 0.0);
    d = sqrt(d);
    double id = 1.0 / d;
    __syncwarp();
    if (lane == 0) {
      A[j * N + j] = d;
      invd[j] = id;
    }
    // L_ij = (A_ij - sum_{l<j} L_il L_jl) / L_jj for i > j
    for (int i = j + 1 + lane; i < N; i += 32) {
      double t = A[i * N + j];
      for (int l = 0; l < j; ++l) t = fma(-A[i * N + l], A[j * N + l], t);
      A[i * N + j] = t * id;
    }
    __syncwarp();
  }
  return ok;
}

// In-place LU without pivoting (Doolittle: unit-lower L below the diagonal, U on and above)
// of an N x N matrix in shared memory, by one warp.  Used for matrices whose symmetric part
// is positive definite (then every leading minor is non-zero).  invd receives 1/U_jj.
template <int N>
__device__ __forceinline__ bool warp_lu(double* A, double* invd, int lane) {
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    const double piv = A[j * N + j];
    ok = ok && (piv != 0.0) && isfinite(piv);
    const double ip = 1.0 / piv;
    if (lane == 0) invd[j] = ip;
    for (int i = j + 1 + lane; i < N; i += 32) A[i * N + j] *= ip;
    __syncwarp();
    const int w = N - j - 1;
    for (int t = lane; t < w * w; t += 32) {
      const int i = j + 1 + t / w, l = j + 1 + t % w;
      A[i * N + l] = fma(-A[i * N + j], A[j * N + l], A[i * N + l]);
    }
    __syncwarp();
  }
  return ok;
}

// Forward substitution L x = b for one right-hand-side column held in registers.
template <int N>
__device__ __forceinline__ void fwd_subst(const double* __restrict__ L, const double* invd, double* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    double s = x[l];
#pragma unroll
    for (int i = 0; i < l; ++i) s = fma(-L[l * N + i], x[i], s);
    x[l] = s * invd[l];
  }
}

// Forward substitution with the unit-lower factor of warp_lu.
template <int N>
__device__ __forceinline__ void fwd_subst_unit(const double* __restrict__ LU, double* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    double s = x[l];
#pragma unroll
    for (int i = 0; i < l; ++i) s = fma(-LU[l * N + i], x[i], s);
    x[l] = s;
  }
}

// Forward substitution U^T x = b (U^T is lower triangular) with the factor of warp_lu.
template <int N>
__device__ __forceinline__ void fwd_subst_Ut(const double* __restrict__ LU, const double* invd, double* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    double s = x[l];
#pragma unroll
    for (int i = 0; i < l; ++i) s = fma(-LU[i * N + l], x[i], s);
    x[l] = s * invd[l];
  }
}



// Deterministic grid reduction: every block contributes one value per slot (nslots <= 4);
// the last block to arrive sums the per-block partials in block order and calls fin(sums).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;  // valid on thread 0
}

}  // namespace hdg
