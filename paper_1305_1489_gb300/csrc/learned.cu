// Learned initial guess for the trace solve: coarse prolongation / restriction, the coarse
// Galerkin solve that produces the training targets, and the FP32 kernels of the small
// network (linear layers, tanh, mean-squared loss, Adam) trained on the GPU.
//
// Coarse space: a continuous piecewise-linear field given by its values c at nc coarse nodes.
// The caller supplies, for every mesh vertex v, up to four (coarse node, weight) pairs so that
// the field's value at v is sum_j w_vj c_{node_vj} (for nested meshes the field is linear on
// every element).  Its trace on a face e is linear, hence in P_k(e) for k >= 1, and its
// coefficients in the face basis are exact:
//     u_hat_e = T [V(w1), V(w2), V(w3)],   T = (varpi . D)^T Xi    (eq. 6.3 with the face rule)
// with w1 < w2 < w3 the face's vertices.  Pi maps c to the free trace entries (Dirichlet faces
// get 0); Pi^T is its adjoint.  The coarse Galerkin problem (Pi^T H Pi) c = Pi^T b gives the
// trace of range(Pi) closest to the solution in the energy norm of H.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {

// prolongation: one thread per (face, entry)
__global__ void prolong_kernel(const int32_t* __restrict__ fverts, const int32_t* __restrict__ ftype, int64_t nfc,
                               int d2, const double* __restrict__ T, const int32_t* __restrict__ nodes,
                               const double* __restrict__ w, const double* __restrict__ c, double* __restrict__ uhat) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfc * d2) return;
  const int64_t e = t / d2;
  const int a = (int)(t - e * d2);
  double s = 0.0;
  if (ftype[e] != 1) {
    for (int i = 0; i < 3; ++i) {
      const int64_t v = fverts[3 * e + i];
      double val = 0.0;
      for (int j = 0; j < 4; ++j) {
        const int nd = nodes[4 * v + j];
        if (nd >= 0) val = fma(w[4 * v + j], c[nd], val);
      }
      s = fma(T[a * 3 + i], val, s);
    }
  }
  uhat[t] = s;
}

// restriction (adjoint of prolong_kernel): one thread per face, atomics into the coarse vector
__global__ void restrict_kernel(const int32_t* __restrict__ fverts, const int32_t* __restrict__ ftype, int64_t nfc,
                                int d2, const double* __restrict__ T, const int32_t* __restrict__ nodes,
                                const double* __restrict__ w, const double* __restrict__ y, double* __restrict__ c) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nfc || ftype[e] == 1) return;
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int a = 0; a < d2; ++a) s = fma(T[a * 3 + i], y[e * d2 + a], s);
    const int64_t v = fverts[3 * e + i];
    for (int j = 0; j < 4; ++j) {
      const int nd = nodes[4 * v + j];
      if (nd >= 0) atomicAdd(c + nd, w[4 * v + j] * s);
    }
  }
}

// random Fourier field: out[i] = g(x_i) (or exp(g)) with
//   g(x) = sigma M^-1/2 sum_m (xi_m cos(omega_m.x) + eta_m sin(omega_m.x)),  amps = [xi; eta]
constexpr int kMaxModes = 1024;
__global__ void fourier_field_kernel(int64_t n, const double* __restrict__ X, const double* __restrict__ Y,
                                     const double* __restrict__ Z, int M, const double* __restrict__ omega,
                                     const double* __restrict__ amps, double scale, int exponentiate,
                                     double* __restrict__ out) {
  __shared__ double om[3 * kMaxModes], am[2 * kMaxModes];
  for (int t = threadIdx.x; t < 3 * M; t += blockDim.x) om[t] = omega[t];
  for (int t = threadIdx.x; t < 2 * M; t += blockDim.x) am[t] = amps[t];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[i], y = Y[i], z = Z[i];
    double g = 0.0;
    for (int m = 0; m < M; ++m) {
      double sn, cs;
      sincos(fma(om[3 * m], x, fma(om[3 * m + 1], y, om[3 * m + 2] * z)), &sn, &cs);
      g = fma(am[m], cs, fma(am[M + m], sn, g));
    }
    g *= scale;
    out[i] = exponentiate ? exp(g) : g;
  }
}

// ---------------------------------------------------------------- small vector kernels
__global__ void vec_axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void vec_dot_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ y, double* out) {
  __shared__ double ws[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ws[i];
    out[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- network kernels (FP32)
// C[M][N] = act(alpha * sum_k A(m,k) B(k,n) + beta * C + bias[n]); A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  32x32 output tiles, 8x8 threads each computing 4x4.
constexpr int TG = 32;
__global__ void nn_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int sam, int sak,
                               const float* __restrict__ B, int sbk, int sbn, float* __restrict__ Cm, int ldc,
                               float beta, const float* __restrict__ bias, int act) {
  __shared__ float As[TG][TG + 1], Bs[TG][TG + 1];
  const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;
  const int m0 = blockIdx.y * TG, n0 = blockIdx.x * TG;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TG) {
    for (int t = threadIdx.x; t < TG * TG; t += 64) {
      const int r = t / TG, cc = t % TG;
      const int m = m0 + r, k = k0 + cc;
      As[r][cc] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : 0.f;
      const int kk = k0 + r, n = n0 + cc;
      Bs[r][cc] = (kk < K && n < N) ? B[(int64_t)kk * sbk + (int64_t)n * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TG; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) {
        float v = acc[i][j];
        if (beta != 0.f) v += beta * Cm[(int64_t)m * ldc + n];
        if (bias) v += bias[n];
        if (act == 1) v = tanhf(v);
        Cm[(int64_t)m * ldc + n] = v;
      }
    }
}

__global__ void nn_to_f64_kernel(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void nn_to_f32_kernel(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// dZ = dY * (1 - Y^2) (tanh) in place
__global__ void nn_tanh_bwd_kernel(int64_t n, const float* __restrict__ Y, float* __restrict__ dY) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dY[i] *= (1.f - Y[i] * Y[i]);
}

// db[n] = sum_m dZ[m][n]
__global__ void nn_colsum_kernel(int M, int N, const float* __restrict__ dZ, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dZ[(int64_t)m * N + n];
  db[n] = s;
}

// loss = mean((p - t)^2) over n entries; grad = 2 (p - t) / n
__global__ void nn_mse_kernel(int64_t n, const float* __restrict__ p, const float* __restrict__ t,
                              float* __restrict__ grad, float* loss_partial) {
  __shared__ float ws[8];
  float s = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = p[i] - t[i];
    grad[i] = 2.f * d / (float)n;
    s = fmaf(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tt = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tt += ws[i];
    loss_partial[blockIdx.x] = tt / (float)n;
  }
}

// Adam (Kingma and Ba 2015) with bias correction
__global__ void nn_adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace hdg

using namespace hdg;

int hdg::ensure_face_verts(hdg_mesh* M) {
  if (M->d_fverts) return HDG_OK;
  std::vector<int32_t> fv(3 * M->nfc);
  for (int64_t e = 0; e < M->nfc; ++e)
    for (int i = 0; i < 3; ++i) fv[3 * e + i] = M->h_faces[4 * e + i];
  // T = (varpi . D)^T Xi, d2 x 3
  const Tables& T = M->tab;
  std::vector<double> Tm(T.d2 * 3, 0.0);
  for (int a = 0; a < T.d2; ++a)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int r = 0; r < T.nf; ++r) s += T.face_w[r] * T.D[r * T.d2 + a] * T.xi[3 * r + i];
      Tm[a * 3 + i] = s;
    }
  HDG_CUDA_TRY(cudaMalloc(&M->d_fverts, sizeof(int32_t) * fv.size()));
  HDG_CUDA_TRY(cudaMemcpy(M->d_fverts, fv.data(), sizeof(int32_t) * fv.size(), cudaMemcpyHostToDevice));
  HDG_CUDA_TRY(cudaMalloc(&M->d_Tproj, sizeof(double) * Tm.size()));
  HDG_CUDA_TRY(cudaMemcpy(M->d_Tproj, Tm.data(), sizeof(double) * Tm.size(), cudaMemcpyHostToDevice));
  return HDG_OK;
}

static int launch_prolong(hdg_mesh* M, const int32_t* nodes, const double* w, const double* c, double* uhat) {
  const int64_t tot = M->nfc * M->tab.d2;
  prolong_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(M->d_fverts, M->d_ftype, M->nfc, M->tab.d2,
                                                                       M->d_Tproj, nodes, w, c, uhat);
  M->launches++;
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

static int launch_restrict(hdg_mesh* M, const int32_t* nodes, const double* w, const double* y, double* c, int64_t nc) {
  HDG_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(double) * nc, M->stream));
  restrict_kernel<<<(unsigned)((M->nfc + 255) / 256), 256, 0, M->stream>>>(M->d_fverts, M->d_ftype, M->nfc,
                                                                           M->tab.d2, M->d_Tproj, nodes, w, y, c);
  M->launches++;
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

static double host_dot(hdg_mesh* M, const double* x, const double* y, int64_t n, double* part) {
  vec_dot_kernel<<<64, 256, 0, M->stream>>>(n, x, y, part);
  M->launches++;
  double h[64];
  cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, M->stream);
  cudaStreamSynchronize(M->stream);
  double s = 0.0;
  for (int i = 0; i < 64; ++i) s += h[i];
  return s;
}

// Target normalisation of the network's training (column statistics of the target matrix),
// and its fold into the last layer after training.  A column with zero spread keeps the scale
// 1, so its standardised values are 0 and the fold returns its mean.
__global__ void nn_colstats_kernel(int64_t M, int N, const double* __restrict__ T, double* mean, double* scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int64_t i = 0; i < M; ++i) s += T[i * N + j];
  const double mu = s / (double)M;
  double v = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    const double d = T[i * N + j] - mu;
    v = fma(d, d, v);
  }
  const double sd = sqrt(v / (double)M);
  mean[j] = mu;
  scale[j] = sd > 0.0 ? sd : 1.0;
}

__global__ void nn_standardize_kernel(int64_t M, int N, const double* __restrict__ T, const double* __restrict__ mean,
                                      const double* __restrict__ scale, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * N) return;
  const int j = (int)(t % N);
  out[t] = (float)((T[t] - mean[j]) / scale[j]);
}

// last layer y = W x + b on standardised targets -> y' = diag(scale) y + mean
__global__ void nn_fold_affine_kernel(int Nout, int Nin, float* W, float* b, const double* __restrict__ mean,
                                      const double* __restrict__ scale) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)Nout * Nin) {
    const int i = (int)(t / Nin);
    W[t] = (float)((double)W[t] * scale[i]);
  }
  if (t < Nout) b[t] = (float)fma((double)b[t], scale[t], mean[t]);
}

extern "C" {

int hdg_nn_colstats(int64_t M, int N, const double* T, double* mean, double* scale, void* stream) {
  if (M < 1 || N < 1 || !T || !mean || !scale) return fail(HDG_ERR_ARG, "bad nn_colstats arguments");
  nn_colstats_kernel<<<(N + 127) / 128, 128, 0, (cudaStream_t)stream>>>(M, N, T, mean, scale);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_standardize(int64_t M, int N, const double* T, const double* mean, const double* scale, float* out,
                       void* stream) {
  if (M < 1 || N < 1 || !T || !mean || !scale || !out) return fail(HDG_ERR_ARG, "bad nn_standardize arguments");
  const int64_t tot = M * N;
  nn_standardize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(M, N, T, mean, scale, out);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_fold_affine(int Nout, int Nin, float* W, float* b, const double* mean, const double* scale,
                       void* stream) {
  if (Nout < 1 || Nin < 1 || !W || !b || !mean || !scale) return fail(HDG_ERR_ARG, "bad nn_fold_affine arguments");
  const int64_t tot = (int64_t)Nout * Nin;
  nn_fold_affine_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(Nout, Nin, W, b, mean, scale);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_prolong(hdg_mesh* M, const int32_t* nodes, const double* weights, const double* coarse, double* uhat) {
  if (!M || !nodes || !weights || !coarse || !uhat) return fail(HDG_ERR_ARG, "NULL argument");
  int rc = ensure_face_verts(M);
  if (rc) return rc;
  return launch_prolong(M, nodes, weights, coarse, uhat);
}

int hdg_restrict(hdg_mesh* M, const int32_t* nodes, const double* weights, int64_t nc, const double* y, double* coarse) {
  if (!M || !nodes || !weights || !coarse || !y || nc < 1) return fail(HDG_ERR_ARG, "bad argument");
  int rc = ensure_face_verts(M);
  if (rc) return rc;
  return launch_restrict(M, nodes, weights, y, coarse, nc);
}

// Coarse Galerkin solve (Pi^T H Pi) c = Pi^T b by CG (matrix-free, FP64), b = the assembled
// right-hand side.  c: device [nc] output.
int hdg_coarse_solve(hdg_mesh* M, const int32_t* nodes, const double* weights, int64_t nc, double* c, double rtol,
                     int maxit, int* iters, double* relres) {
  if (!M || !nodes || !weights || !c || nc < 1 || !(rtol > 0) || maxit < 1) return fail(HDG_ERR_ARG, "bad argument");
  if (!M->assembled) return fail(HDG_ERR_STATE, "coarse solve before hdg_assemble_condense");
  int rc = ensure_face_verts(M);
  if (rc) return rc;
  const int64_t nv = M->nfc * M->tab.d2;
  double *r, *p, *q, *tr, *ty, *part;
  HDG_CUDA_TRY(cudaMalloc(&r, sizeof(double) * nc));
  HDG_CUDA_TRY(cudaMalloc(&p, sizeof(double) * nc));
  HDG_CUDA_TRY(cudaMalloc(&q, sizeof(double) * nc));
  HDG_CUDA_TRY(cudaMalloc(&tr, sizeof(double) * nv));
  HDG_CUDA_TRY(cudaMalloc(&ty, sizeof(double) * nv));
  HDG_CUDA_TRY(cudaMalloc(&part, sizeof(double) * 64));
  double rn, bn;
  // b (free entries) = residual of x = 0
  HDG_CUDA_TRY(cudaMemsetAsync(tr, 0, sizeof(double) * nv, M->stream));
  rc = hdg_trace_residual(M, tr, ty, &rn, &bn);
  int it = 0;
  double rr = 0.0, rr0 = 0.0;
  if (!rc) rc = launch_restrict(M, nodes, weights, ty, r, nc);  // r = Pi^T b (c = 0)
  if (!rc) {
    HDG_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(double) * nc, M->stream));
    HDG_CUDA_TRY(cudaMemcpyAsync(p, r, sizeof(double) * nc, cudaMemcpyDeviceToDevice, M->stream));
    rr = rr0 = host_dot(M, r, r, nc, part);
    while (it < maxit && rr > rtol * rtol * rr0) {
      // q = Pi^T H Pi p
      rc = launch_prolong(M, nodes, weights, p, tr);
      if (rc) break;
      rc = hdg_trace_apply(M, tr, ty);
      if (rc) break;
      rc = launch_restrict(M, nodes, weights, ty, q, nc);
      if (rc) break;
      const double pq = host_dot(M, p, q, nc, part);
      if (!(pq > 0.0)) break;
      const double alpha = rr / pq;
      vec_axpby_kernel<<<64, 256, 0, M->stream>>>(nc, alpha, p, 1.0, c);
      vec_axpby_kernel<<<64, 256, 0, M->stream>>>(nc, -alpha, q, 1.0, r);
      M->launches += 2;
      const double rr_new = host_dot(M, r, r, nc, part);
      vec_axpby_kernel<<<64, 256, 0, M->stream>>>(nc, 1.0, r, rr_new / rr, p);
      M->launches++;
      rr = rr_new;
      ++it;
    }
  }
  cudaFree(r);
  cudaFree(p);
  cudaFree(q);
  cudaFree(tr);
  cudaFree(ty);
  cudaFree(part);
  if (rc) return rc;
  if (iters) *iters = it;
  if (relres) *relres = rr0 > 0 ? std::sqrt(rr / rr0) : 0.0;
  return HDG_OK;
}

// x0 = alpha Pi c with alpha = (w.b)/(w.H w), w = Pi c: the energy-optimal multiple of the
// prolonged coarse field (a one-vector coarse correction of the zero initial guess).
int hdg_coarse_guess(hdg_mesh* M, const int32_t* nodes, const double* weights, const double* c, double* x0,
                     double* alpha) {
  if (!M || !nodes || !weights || !c || !x0) return fail(HDG_ERR_ARG, "NULL argument");
  if (!M->assembled) return fail(HDG_ERR_STATE, "coarse guess before hdg_assemble_condense");
  int rc = ensure_face_verts(M);
  if (rc) return rc;
  const int64_t nv = M->nfc * M->tab.d2;
  double *hw, *b, *part;
  HDG_CUDA_TRY(cudaMalloc(&hw, sizeof(double) * nv));
  HDG_CUDA_TRY(cudaMalloc(&b, sizeof(double) * nv));
  HDG_CUDA_TRY(cudaMalloc(&part, sizeof(double) * 64));
  double rn, bn, a = 0.0;
  HDG_CUDA_TRY(cudaMemsetAsync(hw, 0, sizeof(double) * nv, M->stream));
  rc = hdg_trace_residual(M, hw, b, &rn, &bn);  // b (free entries)
  if (!rc) rc = launch_prolong(M, nodes, weights, c, x0);
  if (!rc) rc = hdg_trace_apply(M, x0, hw);
  if (!rc) {
    const double wb = host_dot(M, x0, b, nv, part), whw = host_dot(M, x0, hw, nv, part);
    a = whw > 0.0 ? wb / whw : 0.0;
    vec_axpby_kernel<<<304, 256, 0, M->stream>>>(nv, 0.0, x0, a, x0);
    M->launches++;
    cudaStreamSynchronize(M->stream);
  }
  cudaFree(hw);
  cudaFree(b);
  cudaFree(part);
  if (alpha) *alpha = a;
  return rc;
}

int hdg_fourier_field(int64_t n, const double* X, const double* Y, const double* Z, int M, const double* omega,
                      const double* amps, double sigma, int exponentiate, double* out, void* stream) {
  if (n < 0 || !X || !Y || !Z || !omega || !amps || !out) return fail(HDG_ERR_ARG, "bad argument");
  if (M < 1 || M > kMaxModes) return fail(HDG_ERR_ARG, "number of modes must be in [1, 1024]");
  if (n == 0) return HDG_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  fourier_field_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, X, Y, Z, M, omega, amps,
                                                                           sigma / std::sqrt((double)M),
                                                                           exponentiate, out);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

// ------------------------------------------------------------------ network kernels
int hdg_nn_gemm(int M, int N, int K, const float* A, int sam, int sak, const float* B, int sbk, int sbn, float* C,
                int ldc, float beta, const float* bias, int act, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(HDG_ERR_ARG, "bad gemm arguments");
  dim3 grid((N + TG - 1) / TG, (M + TG - 1) / TG);
  nn_gemm_kernel<<<grid, 64, 0, (cudaStream_t)stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, beta, bias, act);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_to_f64(int64_t n, const float* x, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(HDG_ERR_ARG, "bad argument");
  if (n == 0) return HDG_OK;
  nn_to_f64_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, (cudaStream_t)stream>>>(n, x, y);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_to_f32(int64_t n, const double* x, float* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(HDG_ERR_ARG, "bad argument");
  if (n == 0) return HDG_OK;
  nn_to_f32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1216), 256, 0, (cudaStream_t)stream>>>(n, x, y);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_tanh_bwd(int64_t n, const float* Y, float* dY, void* stream) {
  nn_tanh_bwd_kernel<<<304, 256, 0, (cudaStream_t)stream>>>(n, Y, dY);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_colsum(int M, int N, const float* dZ, float* db, void* stream) {
  nn_colsum_kernel<<<(N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(M, N, dZ, db);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_mse(int64_t n, const float* pred, const float* target, float* grad, float* loss_partial /*[64]*/,
               void* stream) {
  nn_mse_kernel<<<64, 256, 0, (cudaStream_t)stream>>>(n, pred, target, grad, loss_partial);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int hdg_nn_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                int step, void* stream) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  nn_adam_kernel<<<304, 256, 0, (cudaStream_t)stream>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

}  // extern "C"
