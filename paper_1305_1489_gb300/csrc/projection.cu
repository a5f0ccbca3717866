// HDG projection (eq. 9.13), face L2 projection (eq. 9.12) and the norms of the error
// functions (Section 9, eq. 10.1-10.2).  FP64; diagnostics, outside the solve.
//
// Projection, per element (one CTA): with the orthonormal hierarchical basis
// (sum_q omega_q P_i P_j = delta_ij) the rows of eq. 9.13 tested against P_{k-1} give the first
// n - d2 coefficients of each of q_x, q_y, q_z, u directly, (v, P_i)_K / |K| =
// sum_q omega_q v(x_q) P_i(x_q).  The face rows then fix the top d2 coefficients of the four
// components: for local face l and trace function a,
//   sum_* N_l* E_l[a][top] Q_*top + T_l E_l[a][top] U_top
//     = sum_r varpi_r (q.N_l + T_l u)(x_r^l) D^mu_a(q_hat_r) - (the same with the low part),
// with E_l = (varpi . D^mu)^T P^l the face table of eq. 4.10 (mu = perm(K, l)), N_l the
// area-scaled normal and T_l = tau_l |e_l| (eq. 4.22): an m x m system, solved by Gaussian
// elimination with partial pivoting in shared memory.
#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {

template <int K, int NT>
__global__ void __launch_bounds__(NT) projection_kernel(const double* __restrict__ geo, const int32_t* __restrict__ perm,
                                                        const double* __restrict__ tau, const double* __restrict__ P,
                                                        const double* __restrict__ w, const double* __restrict__ E,
                                                        const double* __restrict__ Dmu, const double* __restrict__ wf,
                                                        const double* __restrict__ q_vol, const double* __restrict__ u_vol,
                                                        const double* __restrict__ q_face,
                                                        const double* __restrict__ u_face, int64_t nelt, int nq,
                                                        double* __restrict__ Pq, double* __restrict__ Pu,
                                                        int32_t* status) {
  using D = Dims<K>;  // nq: nodes of the volume rule in use
  constexpr int n = D::n, d2 = D::d2, m = D::m, nf = D::nf, nlow = n - d2;
  constexpr int LD = m + 1;  // augmented row: [B | rhs]
  __shared__ double B[m * LD];
  __shared__ double low[4][nlow > 0 ? nlow : 1];
  __shared__ double g[4][nf];
  __shared__ double Nl[4][3], Tl[4];
  __shared__ int mu[4], s_piv, s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t Ke = blockIdx.x;
  const double* ge = geo + Ke * kGeoStride;
  if (tid < 4) {
    for (int d = 0; d < 3; ++d) Nl[tid][d] = ge[9 + 3 * tid + d];
    Tl[tid] = (tau ? tau[Ke * 4 + tid] : 1.0) * ge[21 + tid];
    mu[tid] = perm[Ke * 4 + tid] - 1;
  }
  if (tid == 0) s_bad = 0;
  // low coefficients: (v, P_i)_K / |K| for i < n - d2 (none at k = 0: those rows are void)
  if constexpr (nlow > 0)
    for (int t = tid; t < 4 * nlow; t += NT) {
      const int c = t / nlow, i = t - c * nlow;
      const double* v = (c < 3 ? q_vol + ((int64_t)c * nelt + Ke) * nq : u_vol + Ke * nq);
      double s = 0.0;
      for (int qn = 0; qn < nq; ++qn) s = fma(w[qn] * v[qn], P[qn * n + i], s);
      low[c][i] = s;
      if (c < 3) Pq[(Ke * 3 + c) * n + i] = s;
      else Pu[Ke * n + i] = s;
    }
  __syncthreads();
  // (q.N_l + T_l u) at the element-local face nodes
  for (int t = tid; t < 4 * nf; t += NT) {
    const int l = t / nf, r = t - l * nf;
    double s = Tl[l] * u_face[(Ke * 4 + l) * nf + r];
    for (int c = 0; c < 3; ++c) s = fma(Nl[l][c], q_face[(((int64_t)c * nelt + Ke) * 4 + l) * nf + r], s);
    g[l][r] = s;
  }
  __syncthreads();
  // the face rows: B (top columns) and the right-hand side
  for (int t = tid; t < m * m; t += NT) {
    const int row = t / m, col = t - row * m;
    const int l = row / d2, a = row - l * d2, cc = col / d2, j = nlow + (col - cc * d2);
    const double e = E[((l * 6 + mu[l]) * d2 + a) * n + j];
    B[row * LD + col] = (cc < 3 ? Nl[l][cc] : Tl[l]) * e;
  }
  for (int row = tid; row < m; row += NT) {
    const int l = row / d2, a = row - l * d2;
    const double* Dm = Dmu + (int64_t)mu[l] * nf * d2;
    double s = 0.0;
    for (int r = 0; r < nf; ++r) s = fma(wf[r] * g[l][r], Dm[r * d2 + a], s);
    const double* El = E + ((l * 6 + mu[l]) * d2 + a) * n;
    for (int j = 0; j < nlow; ++j)
      s -= El[j] * (Nl[l][0] * low[0][j] + Nl[l][1] * low[1][j] + Nl[l][2] * low[2][j] + Tl[l] * low[3][j]);
    B[row * LD + m] = s;
  }
  __syncthreads();
  // Gaussian elimination with partial pivoting
  for (int j = 0; j < m; ++j) {
    if (warp == 0) {
      double best = -1.0;
      int bi = j;
      for (int i = j + lane; i < m; i += 32) {
        const double v = fabs(B[i * LD + j]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        s_piv = bi;
        if (!(best > 0.0)) s_bad = 1;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != j)
      for (int c = j + tid; c < LD; c += NT) {
        const double t0 = B[j * LD + c];
        B[j * LD + c] = B[pr * LD + c];
        B[pr * LD + c] = t0;
      }
    __syncthreads();
    const double piv = B[j * LD + j];
    const double ip = piv != 0.0 ? 1.0 / piv : 0.0;
    const int rows = m - j - 1, cols = LD - j - 1;
    for (int t = tid; t < rows * cols; t += NT) {
      const int i = j + 1 + t / cols, c = j + 1 + t % cols;
      B[i * LD + c] = fma(-B[i * LD + j] * ip, B[j * LD + c], B[i * LD + c]);
    }
    __syncthreads();
  }
  // back substitution by one warp, column-oriented; x overwrites the rhs column
  if (warp == 0) {
    for (int i = m - 1; i >= 0; --i) {
      const double xi = B[i * LD + m] / B[i * LD + i];
      __syncwarp();
      if (lane == 0) B[i * LD + m] = xi;
      for (int r = lane; r < i; r += 32) B[r * LD + m] = fma(-B[r * LD + i], xi, B[r * LD + m]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int t = tid; t < m; t += NT) {
    const int cc = t / d2, j = nlow + (t - cc * d2);
    const double x = s_bad ? __longlong_as_double(0x7ff8000000000000LL) : B[t * LD + m];
    if (cc < 3) Pq[(Ke * 3 + cc) * n + j] = x;
    else Pu[Ke * n + j] = x;
  }
  if (tid == 0 && s_bad) atomicAdd(status + 5, 1);
}

cudaError_t launch_projection(hdg_mesh* M, const double* q_vol, const double* u_vol, const double* q_face,
                              const double* u_face, double* Pq, double* Pu) {
  const unsigned g = (unsigned)M->nelt;
#define HDG_PJ(KK, NTT)                                                                                     \
  projection_kernel<KK, NTT><<<g, NTT, 0, M->stream>>>(M->d_geo, M->d_perm, M->tau, M->dt.P, M->dt.vol_w,  \
                                                       M->dt.E, M->dt.Dmu, M->dt.face_w, q_vol, u_vol, q_face, \
                                                       u_face, M->nelt, M->tab.nq, Pq, Pu, M->d_status)
  switch (M->k) {
    case 0: HDG_PJ(0, 64); break;
    case 1: HDG_PJ(1, 64); break;
    case 2: HDG_PJ(2, 64); break;
    case 3: HDG_PJ(3, 128); break;
    case 4: HDG_PJ(4, 128); break;
    default: return cudaErrorInvalidValue;
  }
#undef HDG_PJ
  M->launches++;
  return cudaGetLastError();
}

// eq. 9.12 on every face (D orthonormal: sum_r varpi_r D_a D_b = delta_ab)
__global__ void face_projection_kernel(const double* __restrict__ D, const double* __restrict__ wf, int nf, int d2,
                                       const double* __restrict__ vals, int64_t nfc, double* __restrict__ Pu) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfc * d2) return;
  const int64_t e = t / d2;
  const int a = (int)(t - e * d2);
  double s = 0.0;
  for (int r = 0; r < nf; ++r) s = fma(wf[r] * D[r * d2 + a], vals[e * nf + r], s);
  Pu[t] = s;
}

cudaError_t launch_face_projection(hdg_mesh* M, const double* vals, double* Pu) {
  const int64_t tot = M->nfc * M->tab.d2;
  face_projection_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(M->dt.D, M->dt.face_w, M->tab.nf,
                                                                               M->tab.d2, vals, M->nfc, Pu);
  M->launches++;
  return cudaGetLastError();
}

// Norms by quadrature with deterministic two-level sums: each block reduces its part in a
// fixed order into part[2 * block]; norm_finish_kernel adds the kNormBlocks partials in order.
constexpr int kNormBlocks = 608;  // 4 per SM
constexpr int kNormThreads = 256;

__device__ __forceinline__ void block_sum2(double a, double b, double* part) {
  __shared__ double sa[kNormThreads / 32], sb[kNormThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < kNormThreads / 32; ++i) {
      x += sa[i];
      y += sb[i];
    }
    part[2 * blockIdx.x] = x;
    part[2 * blockIdx.x + 1] = y;
  }
}

// sum_K |K| sum_q omega_q (vals - sum_j coef_j P_j)^2 and sum_K |K| sum_q omega_q vals^2
__global__ void __launch_bounds__(kNormThreads) volume_norm_kernel(const double* __restrict__ geo,
                                                                   const double* __restrict__ Pt, int dim,
                                                                   const double* __restrict__ w, int nq,
                                                                   const double* __restrict__ coef,
                                                                   const double* __restrict__ vals, int64_t nelt,
                                                                   double* part) {
  double se = 0.0, sr = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nelt * nq; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Ke = t / nq;
    const int qn = (int)(t - Ke * nq);
    const double v = vals ? vals[t] : 0.0;
    double f = v;
    if (coef)
      for (int j = 0; j < dim; ++j) f = fma(-coef[Ke * dim + j], Pt[qn * dim + j], f);
    const double wk = geo[Ke * kGeoStride + 25] * w[qn];
    se = fma(wk * f, f, se);
    sr = fma(wk * v, v, sr);
  }
  block_sum2(se, sr, part);
}

// ||vals - sum_a coef_a D_a||_h^2 and ||vals||_h^2 with ||v||_h^2 = sum_e |e|^2 sum_r varpi_r v_r^2
__global__ void __launch_bounds__(kNormThreads) face_norm_kernel(const double* __restrict__ fvx,
                                                                 const double* __restrict__ D, int d2,
                                                                 const double* __restrict__ wf, int nf,
                                                                 const double* __restrict__ coef,
                                                                 const double* __restrict__ vals, int64_t nfc,
                                                                 double* part) {
  double se = 0.0, sr = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nfc * nf; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / nf;
    const int r = (int)(t - e * nf);
    const double v = vals ? vals[t] : 0.0;
    double f = v;
    if (coef)
      for (int a = 0; a < d2; ++a) f = fma(-coef[e * d2 + a], D[r * d2 + a], f);
    double u1[3], u2[3], c[3];
    for (int d = 0; d < 3; ++d) {
      const double x0 = fvx[(d * 3 + 0) * nfc + e];
      u1[d] = fvx[(d * 3 + 1) * nfc + e] - x0;
      u2[d] = fvx[(d * 3 + 2) * nfc + e] - x0;
    }
    cross3(u1, u2, c);
    const double a2 = 0.25 * (c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);  // |e|^2
    se = fma(a2 * wf[r] * f, f, se);
    sr = fma(a2 * wf[r] * v, v, sr);
  }
  block_sum2(se, sr, part);
}

__global__ void norm_finish_kernel(const double* __restrict__ part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < kNormBlocks; ++i) {
      x += part[2 * i];
      y += part[2 * i + 1];
    }
    out[0] = x;
    out[1] = y;
  }
}

static cudaError_t norm_buffer(hdg_mesh* M) {
  if (M->d_norm) return cudaSuccess;
  return cudaMalloc(&M->d_norm, sizeof(double) * (2 * kNormBlocks + 2));
}

cudaError_t launch_volume_norm2(hdg_mesh* M, int degree, const double* coef, const double* vals, double* out_host) {
  cudaError_t e = norm_buffer(M);
  if (e != cudaSuccess) return e;
  const bool hi = degree == M->k + 1;
  volume_norm_kernel<<<kNormBlocks, kNormThreads, 0, M->stream>>>(
      M->d_geo, hi ? M->dt.P1 : M->dt.P, hi ? M->tab.n1 : M->tab.n, M->dt.vol_w, M->tab.nq, coef, vals, M->nelt,
      M->d_norm);
  norm_finish_kernel<<<1, 32, 0, M->stream>>>(M->d_norm, M->d_norm + 2 * kNormBlocks);
  M->launches += 2;
  e = cudaMemcpyAsync(out_host, M->d_norm + 2 * kNormBlocks, 2 * sizeof(double), cudaMemcpyDeviceToHost, M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  return e;
}

cudaError_t launch_face_norm2(hdg_mesh* M, const double* coef, const double* vals, double* out_host) {
  cudaError_t e = norm_buffer(M);
  if (e != cudaSuccess) return e;
  face_norm_kernel<<<kNormBlocks, kNormThreads, 0, M->stream>>>(M->d_fvx, M->dt.D, M->tab.d2, M->dt.face_w,
                                                                 M->tab.nf, coef, vals, M->nfc, M->d_norm);
  norm_finish_kernel<<<1, 32, 0, M->stream>>>(M->d_norm, M->d_norm + 2 * kNormBlocks);
  M->launches += 2;
  e = cudaMemcpyAsync(out_host, M->d_norm + 2 * kNormBlocks, 2 * sizeof(double), cudaMemcpyDeviceToHost, M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  return e;
}

}  // namespace hdg
