// K2 local recovery (eq. 5.3), K5 superconvergent postprocess (eq. 9.11), and the
// quadrature-node helper (eq. 3.4, 6.2).  FP64.
#include "device_async.cuh"
#include "device_common.cuh"
#include "device_df.cuh"
#include "hdg_internal.h"

namespace hdg {

// ----------------------------------------------------------------------- nodes
__global__ void qnodes_kernel(const double* __restrict__ vx, const double* __restrict__ lam,
                              int64_t nelt, int nq, double* X, double* Y, double* Z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nelt * nq) return;
  const int64_t K = t / nq;
  const int q = (int)(t - K * nq);
  double out[3];
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s = fma(lam[q * 4 + i], vx[(d * 4 + i) * nelt + K], s);
    out[d] = s;
  }
  X[t] = out[0];
  Y[t] = out[1];
  Z[t] = out[2];
}

__global__ void fnodes_kernel(const double* __restrict__ fvx, const double* __restrict__ xi,
                              int64_t nfc, int nf, double* X, double* Y, double* Z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfc * nf) return;
  const int64_t e = t / nf;
  const int r = (int)(t - e * nf);
  double out[3];
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) s = fma(xi[r * 3 + i], fvx[(d * 3 + i) * nfc + e], s);
    out[d] = s;
  }
  X[t] = out[0];
  Y[t] = out[1];
  Z[t] = out[2];
}

cudaError_t launch_qnodes(hdg_mesh* M, double* X, double* Y, double* Z, double* FX, double* FY,
                          double* FZ) {
  const int nq = M->tab.nq, nf = M->tab.nf;
  if (X) {
    int64_t tot = M->nelt * nq;
    qnodes_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(M->d_vx, M->dt.lam, M->nelt, nq, X, Y, Z);
    M->launches++;
  }
  if (FX) {
    int64_t tot = M->nfc * nf;
    fnodes_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(M->d_fvx, M->dt.xi, M->nfc, nf, FX, FY, FZ);
    M->launches++;
  }
  return cudaGetLastError();
}

// F_K(q_hat_r^l) for every element, local face l (eq. 2.5 / 4.1) and face node r
__global__ void efnodes_kernel(const double* __restrict__ vx, const double* __restrict__ qf, int64_t nelt, int nf,
                               double* X, double* Y, double* Z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nelt * 4 * nf) return;
  const int64_t K = t / (4 * nf);
  const int rem = (int)(t - K * 4 * nf), l = rem / nf, r = rem - l * nf;
  const double s = qf[2 * r], u = qf[2 * r + 1];
  double ref[3];
  switch (l) {  // q_hat^l of Section 4
    case 0: ref[0] = s; ref[1] = u; ref[2] = 0.0; break;
    case 1: ref[0] = s; ref[1] = 0.0; ref[2] = u; break;
    case 2: ref[0] = 0.0; ref[1] = s; ref[2] = u; break;
    default: ref[0] = s; ref[1] = u; ref[2] = 1.0 - s - u; break;
  }
  double out[3];
  for (int d = 0; d < 3; ++d) {
    const double v1 = vx[(d * 4 + 0) * nelt + K];
    double acc = v1;
    for (int j = 0; j < 3; ++j) acc = fma(vx[(d * 4 + j + 1) * nelt + K] - v1, ref[j], acc);
    out[d] = acc;
  }
  X[t] = out[0];
  Y[t] = out[1];
  Z[t] = out[2];
}

cudaError_t launch_element_face_nodes(hdg_mesh* M, double* X, double* Y, double* Z) {
  const int64_t tot = M->nelt * 4 * M->tab.nf;
  efnodes_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(M->d_vx, M->dt.face_pts, M->nelt, M->tab.nf,
                                                                       X, Y, Z);
  M->launches++;
  return cudaGetLastError();
}

// ----------------------------------------------------------------------- recovery
// u = U_s^-1 (H u_dK + h);  q_* = U_M^-1 (W_* u - V (n_* o u_dK))   (eq. 5.3 through the
// factors of K1: S_u = U_s^T U_s, or L U_s with convection, and M_{kappa^-1} = U_M^T U_M; H, h,
// V, W_* are the forward-substituted blocks).  One warp per element; the record is
// column-major so that every column read is unit-stride across the lanes, and the two
// upper-triangular solves run by columns from the last unknown (lane l owns rows l, l + 32).
constexpr int kRecWarps = 4;

// U x = b in place for NV right-hand sides; x[a][v] is row lane + 32 a of right-hand side v.
// U packed by columns with the inverse diagonal last in each column.
template <int N, int NV>
__device__ __forceinline__ void upper_solve(const double* __restrict__ U, double (&x)[(N + 31) / 32][NV], int lane) {
  constexpr int NA = (N + 31) / 32;
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const double* col = U + i * (i + 1) / 2;
    const double inv = __ldg(col + i);
    double xi[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) xi[v] = __shfl_sync(0xffffffffu, x[i >> 5][v], i & 31) * inv;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int l = lane + 32 * a;
      if (l < i) {
        const double uli = __ldg(col + l);
#pragma unroll
        for (int v = 0; v < NV; ++v) x[a][v] = fma(-uli, xi[v], x[a][v]);
      } else if (l == i) {
#pragma unroll
        for (int v = 0; v < NV; ++v) x[a][v] = xi[v];
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(32 * kRecWarps) recover_kernel(const double* __restrict__ rec,
                                                                const int32_t* __restrict__ fbe,
                                                                const double* __restrict__ uhat, int64_t nelt,
                                                                double* __restrict__ q, double* __restrict__ u) {
  using D = Dims<K>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, NA = (n + 31) / 32;
  __shared__ double suh[kRecWarps][m], su[kRecWarps][n];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t Ke = (int64_t)blockIdx.x * kRecWarps + warp;
  if (Ke >= nelt) return;  // a whole warp leaves together
  const double* HT = rec + Ke * (int64_t)D::rec;
  const double* VT = HT + n * (m + 1);
  const double* WT = VT + n * m;
  const double* Us = WT + 3 * n * n;
  const double* UM = Us + D::tri;
  const double* nrm = UM + D::tri;
  for (int t = lane; t < m; t += 32) suh[warp][t] = __ldg(uhat + (int64_t)__ldg(fbe + Ke * 4 + t / d2) * d2 + (t % d2));
  __syncwarp();
  double x[NA][1];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int i = lane + 32 * a;
    double s0 = 0.0, s1 = 0.0;
    if (i < n) {
      s0 = __ldg(HT + m * n + i);
#pragma unroll 8
      for (int r = 0; r < m; r += 2) {
        s0 = fma(__ldg(HT + r * n + i), suh[warp][r], s0);
        if (r + 1 < m) s1 = fma(__ldg(HT + (r + 1) * n + i), suh[warp][r + 1], s1);
      }
    }
    x[a][0] = s0 + s1;
  }
  upper_solve<n, 1>(Us, x, lane);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int i = lane + 32 * a;
    if (i < n) {
      su[warp][i] = x[a][0];
      u[Ke * n + i] = x[a][0];
    }
  }
  __syncwarp();
  double nv[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) nv[t] = __ldg(nrm + t);
  double z[NA][3];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int l = lane + 32 * a;
    double s[3] = {0.0, 0.0, 0.0};
    if (l < n) {
#pragma unroll 4
      for (int c = 0; c < n; ++c) {
        const double uc = su[warp][c];
        s[0] = fma(__ldg(WT + (0 * n + c) * n + l), uc, s[0]);
        s[1] = fma(__ldg(WT + (1 * n + c) * n + l), uc, s[1]);
        s[2] = fma(__ldg(WT + (2 * n + c) * n + l), uc, s[2]);
      }
      // V (n_* o u_dK) = sum_l n_{l*} V_l u_dK,l: one product per face, then the normals
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        double w0 = 0.0, w1 = 0.0;
#pragma unroll
        for (int a2 = 0; a2 < d2; a2 += 2) {
          const int r = fl * d2 + a2;
          w0 = fma(__ldg(VT + r * n + l), suh[warp][r], w0);
          if (a2 + 1 < d2) w1 = fma(__ldg(VT + (r + 1) * n + l), suh[warp][r + 1], w1);
        }
        const double w = w0 + w1;
        s[0] = fma(-w, nv[3 * fl + 0], s[0]);
        s[1] = fma(-w, nv[3 * fl + 1], s[1]);
        s[2] = fma(-w, nv[3 * fl + 2], s[2]);
      }
    }
    z[a][0] = s[0];
    z[a][1] = s[1];
    z[a][2] = s[2];
  }
  upper_solve<n, 3>(UM, z, lane);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int l = lane + 32 * a;
    if (l < n) {
      q[(Ke * 3 + 0) * n + l] = z[a][0];
      q[(Ke * 3 + 1) * n + l] = z[a][1];
      q[(Ke * 3 + 2) * n + l] = z[a][2];
    }
  }
}

// The same recovery in double-float on the FP32 pipe, for the record of the double-float
// K1 (entries stored as (hi, lo) float pairs).  One warp (one CTA) per element: the element's
// record, one contiguous block, is brought into shared memory by a single bulk asynchronous
// copy while the lanes gather u_dK, so the kernel streams the records at the copy engine's
// rate.  The accumulations are compensated (dacc), the triangular solves keep every pending
// right-hand side as an unnormalised accumulator, and u_dK and the results cross to and
// from FP64 once.  A copy that does not complete within the wait limit (it cannot, short of
// a hardware fault) leaves NaN in the element's q and u and counts in status[4].
constexpr int kRecWaitPolls = 1 << 16;

__device__ __forceinline__ df shfl_df(df x, int src) {
  return df_make(__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src));
}

template <int N, int NV>
__device__ __forceinline__ void upper_solve_df(const df* U, dacc (&x)[(N + 31) / 32][NV], int lane) {
  constexpr int NA = (N + 31) / 32;
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    const df* col = U + i * (i + 1) / 2;
    const df inv = col[i];
    df xi[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) xi[v] = df_mul(shfl_df(dacc_result(x[i >> 5][v]), i & 31), inv);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int l = lane + 32 * a;
      if (l < i) {
        const df uli = col[l];
#pragma unroll
        for (int v = 0; v < NV; ++v) dacc_msub(x[a][v], uli, xi[v]);
      } else if (l == i) {
#pragma unroll
        for (int v = 0; v < NV; ++v) x[a][v] = dacc_from(xi[v]);
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(32) recover_df_kernel(const double* __restrict__ rec, const int32_t* __restrict__ fbe,
                                                       const double* __restrict__ uhat, int64_t nelt,
                                                       double* __restrict__ q, double* __restrict__ u,
                                                       int32_t* status) {
  using D = Dims<K>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, NA = (n + 31) / 32;
  constexpr uint32_t kBytes = sizeof(df) * D::rec;
  static_assert(kBytes % 16 == 0, "the record must be a whole number of 16-byte units");
  extern __shared__ __align__(128) unsigned char rec_smem[];
  __shared__ df suh[m], su[n];
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x;
  const int64_t Ke = blockIdx.x;
  const df* HT = reinterpret_cast<const df*>(rec_smem);
  if (lane == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, kBytes);
    bulk_g2s(rec_smem, reinterpret_cast<const df*>(rec) + Ke * (int64_t)D::rec, kBytes, &bar);
  }
  for (int t = lane; t < m; t += 32)
    suh[t] = df_from_double(__ldg(uhat + (int64_t)__ldg(fbe + Ke * 4 + t / d2) * d2 + (t % d2)));
  __syncwarp();
  if (!mbar_wait(&bar, 0, kRecWaitPolls)) {
    mbar_wait(&bar, 0, kRecWaitPolls);  // give the copy in flight a second chance to land
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int l = lane; l < n; l += 32) {
      u[Ke * n + l] = nan;
      for (int st = 0; st < 3; ++st) q[(Ke * 3 + st) * n + l] = nan;
    }
    if (lane == 0) atomicAdd(status + 4, 1);
    return;
  }
  const df* VT = HT + n * (m + 1);
  const df* WT = VT + n * m;
  const df* Us = WT + 3 * n * n;
  const df* UM = Us + D::tri;
  const df* nrm = UM + D::tri;
  dacc x[NA][1];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int i = lane + 32 * a;
    dacc s = dacc_zero();
    if (i < n) {
      s = dacc_from(HT[m * n + i]);
#pragma unroll 8
      for (int r = 0; r < m; ++r) dacc_mac(s, HT[r * n + i], suh[r]);
    }
    x[a][0] = s;
  }
  upper_solve_df<n, 1>(Us, x, lane);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int i = lane + 32 * a;
    if (i < n) {
      const df ui = dacc_result(x[a][0]);
      su[i] = ui;
      u[Ke * n + i] = df_to_double(ui);
    }
  }
  __syncwarp();
  df nv[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) nv[t] = nrm[t];
  dacc z[NA][3];
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int l = lane + 32 * a;
    z[a][0] = z[a][1] = z[a][2] = dacc_zero();
    if (l < n) {
#pragma unroll 4
      for (int c = 0; c < n; ++c) {
        const df uc = su[c];
        dacc_mac(z[a][0], WT[(0 * n + c) * n + l], uc);
        dacc_mac(z[a][1], WT[(1 * n + c) * n + l], uc);
        dacc_mac(z[a][2], WT[(2 * n + c) * n + l], uc);
      }
      // V (n_* o u_dK) = sum_l n_{l*} V_l u_dK,l: one product per face, then the normals
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        dacc w = dacc_zero();
#pragma unroll
        for (int a2 = 0; a2 < d2; ++a2) dacc_mac(w, VT[(fl * d2 + a2) * n + l], suh[fl * d2 + a2]);
        const df wv = dacc_result(w);
        dacc_msub(z[a][0], nv[3 * fl + 0], wv);
        dacc_msub(z[a][1], nv[3 * fl + 1], wv);
        dacc_msub(z[a][2], nv[3 * fl + 2], wv);
      }
    }
  }
  upper_solve_df<n, 3>(UM, z, lane);
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int l = lane + 32 * a;
    if (l < n) {
      q[(Ke * 3 + 0) * n + l] = df_to_double(dacc_result(z[a][0]));
      q[(Ke * 3 + 1) * n + l] = df_to_double(dacc_result(z[a][1]));
      q[(Ke * 3 + 2) * n + l] = df_to_double(dacc_result(z[a][2]));
    }
  }
}

// The same recovery for small elements (k <= 2, n <= 10): E = 32 / n elements per warp, lane
// group g (lanes g n .. g n + n - 1) working on element g exactly as one warp does above (row l
// of its element on lane g n + l, shuffles within the group), so that the lanes are not left
// idle by the short columns.  The E records arrive by E bulk copies on one mbarrier.
template <int K>
__global__ void __launch_bounds__(32) recover_df_multi_kernel(const double* __restrict__ rec,
                                                             const int32_t* __restrict__ fbe,
                                                             const double* __restrict__ uhat, int64_t nelt,
                                                             double* __restrict__ q, double* __restrict__ u,
                                                             int32_t* status) {
  using D = Dims<K>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, E = 32 / n;
  static_assert(n <= 16, "one lane group of n lanes per element");
  constexpr uint32_t kBytes = sizeof(df) * D::rec;
  static_assert(kBytes % 16 == 0, "the record must be a whole number of 16-byte units");
  extern __shared__ __align__(128) unsigned char rec_smem[];
  __shared__ df suh[E][m], su[E][n];
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x;
  const int g = lane / n < E ? lane / n : E - 1;  // the lanes past E n shadow the last group
  const int l = lane - (lane / n) * n;
  const int64_t K0 = (int64_t)blockIdx.x * E;
  const int ne = (int)((nelt - K0) < E ? (nelt - K0) : E);  // elements of this block
  const bool act = lane / n < ne;
  const int64_t Ke = K0 + g;
  const int base = g * n;  // first lane of the group
  if (lane == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, kBytes * (uint32_t)ne);
    for (int e = 0; e < ne; ++e)
      bulk_g2s(rec_smem + e * kBytes, reinterpret_cast<const df*>(rec) + (K0 + e) * (int64_t)D::rec, kBytes, &bar);
  }
  for (int t = lane; t < ne * m; t += 32) {
    const int e = t / m, r = t - e * m;
    suh[e][r] = df_from_double(__ldg(uhat + (int64_t)__ldg(fbe + (K0 + e) * 4 + r / d2) * d2 + (r % d2)));
  }
  __syncwarp();
  if (!mbar_wait(&bar, 0, kRecWaitPolls)) {
    mbar_wait(&bar, 0, kRecWaitPolls);  // give the copies in flight a second chance to land
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (act) {
      u[Ke * n + l] = nan;
      for (int st = 0; st < 3; ++st) q[(Ke * 3 + st) * n + l] = nan;
    }
    if (lane == 0) atomicAdd(status + 4, 1);
    return;
  }
  const df* HT = reinterpret_cast<const df*>(rec_smem + g * kBytes);
  const df* VT = HT + n * (m + 1);
  const df* WT = VT + n * m;
  const df* Us = WT + 3 * n * n;
  const df* UM = Us + D::tri;
  const df* nrm = UM + D::tri;
  // u = U_s^-1 (H u_dK + h)
  dacc x = dacc_from(HT[m * n + l]);
#pragma unroll 8
  for (int r = 0; r < m; ++r) dacc_mac(x, HT[r * n + l], suh[g][r]);
#pragma unroll
  for (int i = n - 1; i >= 0; --i) {
    const df* col = Us + i * (i + 1) / 2;
    const df xi = df_mul(shfl_df(dacc_result(x), base + i), col[i]);
    if (l < i) dacc_msub(x, col[l], xi);
    else if (l == i) x = dacc_from(xi);
  }
  const df ui = dacc_result(x);
  su[g][l] = ui;
  if (act) u[Ke * n + l] = df_to_double(ui);
  __syncwarp();
  // q_* = U_M^-1 (W_* u - V (n_* o u_dK))
  dacc z[3] = {dacc_zero(), dacc_zero(), dacc_zero()};
#pragma unroll
  for (int c = 0; c < n; ++c) {
    const df uc = su[g][c];
    dacc_mac(z[0], WT[(0 * n + c) * n + l], uc);
    dacc_mac(z[1], WT[(1 * n + c) * n + l], uc);
    dacc_mac(z[2], WT[(2 * n + c) * n + l], uc);
  }
#pragma unroll
  for (int fl = 0; fl < 4; ++fl) {
    dacc w = dacc_zero();
#pragma unroll
    for (int a2 = 0; a2 < d2; ++a2) dacc_mac(w, VT[(fl * d2 + a2) * n + l], suh[g][fl * d2 + a2]);
    const df wv = dacc_result(w);
    dacc_msub(z[0], nrm[3 * fl + 0], wv);
    dacc_msub(z[1], nrm[3 * fl + 1], wv);
    dacc_msub(z[2], nrm[3 * fl + 2], wv);
  }
#pragma unroll
  for (int i = n - 1; i >= 0; --i) {
    const df* col = UM + i * (i + 1) / 2;
    const df inv = col[i];
    df xi[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) xi[v] = df_mul(shfl_df(dacc_result(z[v]), base + i), inv);
    if (l < i) {
      const df uli = col[l];
#pragma unroll
      for (int v = 0; v < 3; ++v) dacc_msub(z[v], uli, xi[v]);
    } else if (l == i) {
#pragma unroll
      for (int v = 0; v < 3; ++v) z[v] = dacc_from(xi[v]);
    }
  }
  if (act) {
#pragma unroll
    for (int v = 0; v < 3; ++v) q[(Ke * 3 + v) * n + l] = df_to_double(dacc_result(z[v]));
  }
}

// The same recovery for small elements without staging the records: every record entry is read
// once, by the lane of its row (the lanes of a group read consecutive entries) or by the whole
// group (a pivot, the normals), so each lane loads its entries straight from global memory
// (read-only, streaming) and no shared memory holds them.  Blocks of kRdWarps warps, each warp
// on E = 32 / n elements as in recover_df_multi_kernel; without the 22 KB of staged records per
// warp, the SM holds several times more warps to hide the memory and shuffle latencies of the
// triangular solves.
constexpr int kRdWarps = 4;

__device__ __forceinline__ df ldcs_df(const df* p) {
  const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
  return df_make(v.x, v.y);
}

template <int K>
__global__ void __launch_bounds__(32 * kRdWarps) recover_df_direct_kernel(const double* __restrict__ rec,
                                                                        const int32_t* __restrict__ fbe,
                                                                        const double* __restrict__ uhat, int64_t nelt,
                                                                        double* __restrict__ q, double* __restrict__ u) {
  using D = Dims<K>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, E = 32 / n;
  static_assert(n <= 16, "one lane group of n lanes per element");
  __shared__ df suh_[kRdWarps][E][m], su_[kRdWarps][E][n];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  df(*suh)[m] = suh_[w];
  df(*su)[n] = su_[w];
  const int g = lane / n < E ? lane / n : E - 1;  // the lanes past E n shadow the last group
  const int l = lane - (lane / n) * n;
  const int64_t K0 = ((int64_t)blockIdx.x * kRdWarps + w) * E;
  if (K0 >= nelt) return;  // whole warps only: no block-wide barrier below
  const int ne = (int)((nelt - K0) < E ? (nelt - K0) : E);  // elements of this warp
  const bool act = lane / n < ne;
  const int64_t Ke = K0 + (g < ne ? g : ne - 1);  // a shadow or idle group repeats a valid element
  const int base = g * n;  // first lane of the group
  for (int t = lane; t < ne * m; t += 32) {
    const int e = t / m, r = t - e * m;
    suh[e][r] = df_from_double(__ldg(uhat + (int64_t)__ldg(fbe + (K0 + e) * 4 + r / d2) * d2 + (r % d2)));
  }
  __syncwarp();
  const df* HT = reinterpret_cast<const df*>(rec) + Ke * (int64_t)D::rec;
  const df* VT = HT + n * (m + 1);
  const df* WT = VT + n * m;
  const df* Us = WT + 3 * n * n;
  const df* UM = Us + D::tri;
  const df* nrm = UM + D::tri;
  const int ge = g < ne ? g : ne - 1;
  // u = U_s^-1 (H u_dK + h)
  dacc x = dacc_from(ldcs_df(HT + m * n + l));
#pragma unroll 8
  for (int r = 0; r < m; ++r) dacc_mac(x, ldcs_df(HT + r * n + l), suh[ge][r]);
#pragma unroll
  for (int i = n - 1; i >= 0; --i) {
    const df* col = Us + i * (i + 1) / 2;
    const df ci = ldcs_df(col + i);
    const df cl = l < i ? ldcs_df(col + l) : df_make(0.f, 0.f);
    const df xi = df_mul(shfl_df(dacc_result(x), base + i), ci);
    if (l < i) dacc_msub(x, cl, xi);
    else if (l == i) x = dacc_from(xi);
  }
  const df ui = dacc_result(x);
  su[ge][l] = ui;
  if (act) u[Ke * n + l] = df_to_double(ui);
  __syncwarp();
  // q_* = U_M^-1 (W_* u - V (n_* o u_dK))
  dacc z[3] = {dacc_zero(), dacc_zero(), dacc_zero()};
#pragma unroll
  for (int c = 0; c < n; ++c) {
    const df uc = su[ge][c];
    dacc_mac(z[0], ldcs_df(WT + (0 * n + c) * n + l), uc);
    dacc_mac(z[1], ldcs_df(WT + (1 * n + c) * n + l), uc);
    dacc_mac(z[2], ldcs_df(WT + (2 * n + c) * n + l), uc);
  }
#pragma unroll
  for (int fl = 0; fl < 4; ++fl) {
    dacc wv = dacc_zero();
#pragma unroll
    for (int a2 = 0; a2 < d2; ++a2) dacc_mac(wv, ldcs_df(VT + (fl * d2 + a2) * n + l), suh[ge][fl * d2 + a2]);
    const df wr = dacc_result(wv);
    dacc_msub(z[0], ldcs_df(nrm + 3 * fl + 0), wr);
    dacc_msub(z[1], ldcs_df(nrm + 3 * fl + 1), wr);
    dacc_msub(z[2], ldcs_df(nrm + 3 * fl + 2), wr);
  }
#pragma unroll
  for (int i = n - 1; i >= 0; --i) {
    const df* col = UM + i * (i + 1) / 2;
    const df inv = ldcs_df(col + i);
    const df uli = l < i ? ldcs_df(col + l) : df_make(0.f, 0.f);
    df xi[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) xi[v] = df_mul(shfl_df(dacc_result(z[v]), base + i), inv);
    if (l < i) {
#pragma unroll
      for (int v = 0; v < 3; ++v) dacc_msub(z[v], uli, xi[v]);
    } else if (l == i) {
#pragma unroll
      for (int v = 0; v < 3; ++v) z[v] = dacc_from(xi[v]);
    }
  }
  if (act) {
#pragma unroll
    for (int v = 0; v < 3; ++v) q[(Ke * 3 + v) * n + l] = df_to_double(dacc_result(z[v]));
  }
}

// elements e0 .. e0 + count - 1 (q, u and the record offset to their first element; the
// kernels see a mesh of count elements)
template <int K>
static cudaError_t launch_recover_df(hdg_mesh* M, const double* uhat, double* q, double* u, int64_t e0, int64_t count) {
  using D = Dims<K>;
  const double* rec = M->d_rec + e0 * (int64_t)D::rec;
  const int32_t* fbe = M->d_facebyele + 4 * e0;
  q += e0 * 3 * D::n;
  u += e0 * D::n;
  if constexpr (D::n <= 10) {
    constexpr int E = 32 / D::n, PER = E * kRdWarps;
    recover_df_direct_kernel<K><<<(unsigned)((count + PER - 1) / PER), 32 * kRdWarps, 0, M->stream>>>(rec, fbe, uhat,
                                                                                                     count, q, u);
    return cudaSuccess;
  } else {
    const int smem = (int)(sizeof(df) * D::rec);
    cudaError_t e = cudaFuncSetAttribute(recover_df_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    recover_df_kernel<K><<<(unsigned)count, 32, smem, M->stream>>>(rec, fbe, uhat, count, q, u, M->d_status);
    return cudaSuccess;
  }
}

template <int K>
static void launch_recover_fp64(hdg_mesh* M, const double* uhat, double* q, double* u, int64_t e0, int64_t count) {
  using D = Dims<K>;
  const unsigned g = (unsigned)((count + kRecWarps - 1) / kRecWarps);
  recover_kernel<K><<<g, 32 * kRecWarps, 0, M->stream>>>(M->d_rec + e0 * (int64_t)D::rec, M->d_facebyele + 4 * e0,
                                                          uhat, count, q + e0 * 3 * D::n, u + e0 * D::n);
}

cudaError_t launch_recover_range(hdg_mesh* M, const double* uhat, double* q, double* u, int64_t e0, int64_t count) {
  if (count <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
#define HDG_REC(KK)                                                  \
  if (M->rec_df) e = launch_recover_df<KK>(M, uhat, q, u, e0, count); \
  else launch_recover_fp64<KK>(M, uhat, q, u, e0, count)
  switch (M->k) {
    case 0: HDG_REC(0); break;
    case 1: HDG_REC(1); break;
    case 2: HDG_REC(2); break;
    case 3: HDG_REC(3); break;
    case 4: HDG_REC(4); break;
    default: return cudaErrorInvalidValue;
  }
#undef HDG_REC
  if (e != cudaSuccess) return e;
  M->launches++;
  return cudaGetLastError();
}

cudaError_t launch_recover(hdg_mesh* M, const double* uhat, double* q, double* u) {
  return launch_recover_range(M, uhat, q, u, 0, M->nelt);
}

// ----------------------------------------------------------------------- postprocess
// (grad u*, grad w)_K = -(kappa^-1 q_h, grad w)_K for w in P_{k+1}(K), (u*, 1)_K = (u_h, 1)_K.
// With the orthonormal hierarchical basis P'_1 = 1 and P'_i (i > 1) has zero mean, so
// u*_1 = u_{h,1} and the coefficients 2..n1 solve the (n1-1) x (n1-1) SPD stiffness system.
template <int K, int NT, int NQ>
__global__ void __launch_bounds__(NT) postprocess_kernel(
    const double* __restrict__ vx, const double* __restrict__ kappa, const double* __restrict__ P,
    const double* __restrict__ G1, const double* __restrict__ Shat1, const double* __restrict__ w,
    const int16_t* __restrict__ pairs1, const double* __restrict__ q, const double* __restrict__ u,
    int64_t nelt, double* __restrict__ ustar, int32_t* status) {
  using D = Dims<K>;
  constexpr int n = D::n, nq = NQ, n1 = D::n1, nr = n1 - 1;  // NQ: nodes of the volume rule in use
  constexpr int NP = nr * (nr + 1) / 2;
  __shared__ double Ks[nr * nr], rhs[nr], invd[nr], rpart[6 * nr];
  __shared__ double qs[3 * n], Qs[3 * nq];
  __shared__ double s_a[3][3], s_det, s_g[6];
  __shared__ int s_bad;
  const int64_t Ke = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    Geo g;
    element_geometry(vx, nelt, Ke, g);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s_a[i][j] = g.a[i][j];
    s_det = g.det;
    const int pr[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    const double idet = 1.0 / g.det;
    for (int c = 0; c < 6; ++c) {
      double s = 0.0;
      for (int st = 0; st < 3; ++st) s += g.a[st][pr[c][0]] * g.a[st][pr[c][1]];
      s_g[c] = s * idet;
    }
    s_bad = 0;
  }
  for (int t = tid; t < 3 * n; t += NT) qs[t] = q[Ke * 3 * n + t];
  __syncthreads();
  // Q_#(p) = omega kappa^-1 sum_* a_{*#} q_*(p) at each node
  for (int p = tid; p < nq; p += NT) {
    double qh[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
      const double pv = __ldg(P + p * n + i);
      qh[0] = fma(qs[i], pv, qh[0]);
      qh[1] = fma(qs[n + i], pv, qh[1]);
      qh[2] = fma(qs[2 * n + i], pv, qh[2]);
    }
    const double wk = w[p] / kappa[Ke * nq + p];
    for (int h = 0; h < 3; ++h)
      Qs[h * nq + p] = wk * (s_a[0][h] * qh[0] + s_a[1][h] * qh[1] + s_a[2][h] * qh[2]);
  }
  // reduced stiffness (indices 1..n1-1)
  for (int t = tid; t < NP; t += NT) {
    const int i = pairs1[2 * t], j = pairs1[2 * t + 1];  // 0-based into 1..n1-1
    const int I = i + 1, J = j + 1;
    double s = 0.0;
    for (int c = 0; c < 6; ++c) {
      const double sij = __ldg(Shat1 + (c * n1 + I) * n1 + J);
      const double sji = __ldg(Shat1 + (c * n1 + J) * n1 + I);
      const bool diag = (c == 0 || c == 3 || c == 5);
      s = fma(s_g[c], diag ? sij : sij + sji, s);
    }
    Ks[i * nr + j] = s;
    Ks[j * nr + i] = s;
  }
  __syncthreads();
  // right-hand side: the (h, i) sums split in two halves of the nodes so that whole warps
  // share the work (GB300's FP64 pipe charges a warp instruction whatever its active lanes)
  constexpr int NPART = 6 * nr;
  constexpr int half = (nq + 1) / 2;
  for (int t = tid; t < NPART; t += NT) {
    const int hh = t / (2 * nr), rem = t - hh * 2 * nr, part = rem / nr, i = rem - part * nr;
    const int p0 = part * half, p1 = part ? nq : half;
    double s = 0.0;
    for (int p = p0; p < p1; ++p) s = fma(Qs[hh * nq + p], __ldg(G1 + (hh * nq + p) * n1 + i + 1), s);
    rpart[t] = s;
  }
  __syncthreads();
  for (int i = tid; i < nr; i += NT) {
    double s = 0.0;
    for (int hh = 0; hh < 3; ++hh) s += rpart[hh * 2 * nr + i] + rpart[hh * 2 * nr + nr + i];
    rhs[i] = s * (-1.0 / 6.0);
  }
  // Cholesky of the reduced stiffness, right-looking, the trailing updates spread over the CTA
  for (int j = 0; j < nr; ++j) {
    if (tid == 0) {
      // only 1 / L_jj is used below: one reciprocal square root instead of a root and a divide
      // (both run on the FP64 pipe, serially, once per column)
      const double dj = Ks[j * nr + j];
      if (!(dj > 0.0)) s_bad = 1;
      invd[j] = rsqrt(dj > 0.0 ? dj : 1.0);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nr; i += NT) Ks[i * nr + j] *= invd[j];
    __syncthreads();
    const int mt = nr - j - 1;  // trailing block (lower triangle incl. diagonal): mt (mt + 1) / 2
    for (int t = tid; t < mt * (mt + 1) / 2; t += NT) {
      int a = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > t) --a;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int b = t - a * (a + 1) / 2;  // b <= a
      const int i = j + 1 + a, k = j + 1 + b;
      Ks[i * nr + k] = fma(-Ks[i * nr + j], Ks[k * nr + j], Ks[i * nr + k]);
    }
    __syncthreads();
  }
  // L y = rhs and L^T x = y by one warp, column-oriented so that every lane has work
  if (warp == 0) {
    for (int i = 0; i < nr; ++i) {
      const double yi = rhs[i] * invd[i];
      __syncwarp();
      if (lane == 0) rhs[i] = yi;
      for (int l = i + 1 + lane; l < nr; l += 32) rhs[l] = fma(-Ks[l * nr + i], yi, rhs[l]);
      __syncwarp();
    }
    for (int i = nr - 1; i >= 0; --i) {
      const double xi = rhs[i] * invd[i];
      __syncwarp();
      if (lane == 0) rhs[i] = xi;
      for (int l = lane; l < i; l += 32) rhs[l] = fma(-Ks[i * nr + l], xi, rhs[l]);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int t = tid; t < n1; t += NT) ustar[Ke * n1 + t] = (t == 0) ? u[Ke * n] : rhs[t - 1];
  if (tid == 0 && s_bad) atomicAdd(status + 2, 1);
}

// The same postprocess in double-float on the FP32 pipe (after a double-float assembly):
// geometry from the per-mesh table, the stiffness and right-hand side by compensated sums,
// the Cholesky factorisation block-wide (group_cholesky_df: reciprocal square roots by
// Newton-Raphson, no FP64), the two triangular solves by one warp with every pending entry an
// unnormalised accumulator; inputs and results cross to and from FP64 once.
template <int K, int NT>
__global__ void __launch_bounds__(NT) postprocess_df_kernel(
    const double* __restrict__ geo, const double* __restrict__ kappa, const df* __restrict__ P,
    const df* __restrict__ G1, const df* __restrict__ Shat1, const double* __restrict__ w,
    const int16_t* __restrict__ pairs1, const double* __restrict__ q, const double* __restrict__ u,
    int64_t nelt, double* __restrict__ ustar, int32_t* status) {
  using D = Dims<K>;
  constexpr int n = D::n, nq = D::nq, n1 = D::n1, nr = n1 - 1, NA = (nr + 31) / 32;
  constexpr int NP = nr * (nr + 1) / 2;
  __shared__ df Ks[nr * nr], rhs[nr], invd[nr], rpart[6 * nr];
  __shared__ df qs[3 * n], Qs[3 * nq];
  __shared__ df s_a[3][3], s_g[6];
  __shared__ int s_bad;
  const int64_t Ke = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* ge = geo + Ke * kGeoStride;
  if (tid < 9) s_a[tid / 3][tid % 3] = df_from_double(ge[tid]);
  if (tid >= 32 && tid < 38) {  // g_c = sum_* a_{*#} a_{*%} / det for (#, %) = xx, xy, xz, yy, yz, zz
    const int c = tid - 32;
    const int p0 = c < 3 ? 0 : c < 5 ? 1 : 2, p1 = c < 3 ? c : c < 5 ? c - 2 : 2;
    double s = 0.0;
    for (int st = 0; st < 3; ++st) s += ge[3 * st + p0] * ge[3 * st + p1];
    s_g[c] = df_from_double(s / ge[26]);
  }
  if (tid == 0) s_bad = 0;
  for (int t = tid; t < 3 * n; t += NT) qs[t] = df_from_double(q[Ke * 3 * n + t]);
  __syncthreads();
  // Q_#(p) = omega kappa^-1 sum_* a_{*#} q_*(p) at each node
  for (int p = tid; p < nq; p += NT) {
    dacc qh[3] = {dacc_zero(), dacc_zero(), dacc_zero()};
    for (int i = 0; i < n; ++i) {
      const df pv = P[p * n + i];
      dacc_mac(qh[0], qs[i], pv);
      dacc_mac(qh[1], qs[n + i], pv);
      dacc_mac(qh[2], qs[2 * n + i], pv);
    }
    const df q0 = dacc_result(qh[0]), q1 = dacc_result(qh[1]), q2 = dacc_result(qh[2]);
    const df wk = df_from_double(w[p] / kappa[Ke * nq + p]);
    for (int h = 0; h < 3; ++h) {
      dacc s = dacc_zero();
      dacc_mac(s, s_a[0][h], q0);
      dacc_mac(s, s_a[1][h], q1);
      dacc_mac(s, s_a[2][h], q2);
      Qs[h * nq + p] = df_mul(wk, dacc_result(s));
    }
  }
  // reduced stiffness (indices 1..n1-1)
  for (int t = tid; t < NP; t += NT) {
    const int i = pairs1[2 * t], j = pairs1[2 * t + 1];  // 0-based into 1..n1-1
    const int I = i + 1, J = j + 1;
    dacc s = dacc_zero();
    for (int c = 0; c < 6; ++c) {
      const df sij = Shat1[(c * n1 + I) * n1 + J];
      const bool diag = (c == 0 || c == 3 || c == 5);
      dacc_mac(s, s_g[c], diag ? sij : df_add(sij, Shat1[(c * n1 + J) * n1 + I]));
    }
    const df v = dacc_result(s);
    Ks[i * nr + j] = v;
    Ks[j * nr + i] = v;
  }
  __syncthreads();
  constexpr int half = (nq + 1) / 2;
  for (int t = tid; t < 6 * nr; t += NT) {
    const int hh = t / (2 * nr), rem = t - hh * 2 * nr, part = rem / nr, i = rem - part * nr;
    const int p0 = part * half, p1 = part ? nq : half;
    dacc s = dacc_zero();
    for (int p = p0; p < p1; ++p) dacc_mac(s, Qs[hh * nq + p], G1[(hh * nq + p) * n1 + i + 1]);
    rpart[t] = dacc_result(s);
  }
  __syncthreads();
  for (int i = tid; i < nr; i += NT) {
    dacc s = dacc_zero();
    for (int hh = 0; hh < 3; ++hh) {
      dacc_add(s, rpart[hh * 2 * nr + i]);
      dacc_add(s, rpart[hh * 2 * nr + nr + i]);
    }
    rhs[i] = df_mul(dacc_result(s), df_from_double(-1.0 / 6.0));
  }
  __syncthreads();
  const bool ok = group_cholesky_df<nr, NT>(Ks, invd, pairs1, tid);
  if (!ok && tid == 0) s_bad = 1;
  __syncthreads();
  // L y = rhs, L^T x = y by one warp, column-oriented; lane l owns rows l and l + 32
  if (warp == 0) {
    dacc x[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int l = lane + 32 * a;
      x[a] = l < nr ? dacc_from(rhs[l]) : dacc_zero();
    }
    for (int i = 0; i < nr; ++i) {
      df xi = df_make(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < NA; ++a)
        if ((i >> 5) == a) xi = shfl_df(dacc_result(x[a]), i & 31);
      xi = df_mul(xi, invd[i]);
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const int l = lane + 32 * a;
        if (l > i && l < nr) dacc_msub(x[a], Ks[l * nr + i], xi);
        else if (l == i) x[a] = dacc_from(xi);
      }
    }
    for (int i = nr - 1; i >= 0; --i) {
      df xi = df_make(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < NA; ++a)
        if ((i >> 5) == a) xi = shfl_df(dacc_result(x[a]), i & 31);
      xi = df_mul(xi, invd[i]);
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        const int l = lane + 32 * a;
        if (l < i) dacc_msub(x[a], Ks[i * nr + l], xi);
        else if (l == i) x[a] = dacc_from(xi);
      }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const int l = lane + 32 * a;
      if (l < nr) ustar[Ke * n1 + 1 + l] = df_to_double(dacc_result(x[a]));
    }
    if (lane == 0) ustar[Ke * n1] = u[Ke * n];
  }
  if (tid == 0 && s_bad) atomicAdd(status + 2, 1);
}

cudaError_t launch_postprocess(hdg_mesh* M, const double* q, const double* u, double* ustar) {
  const unsigned g = (unsigned)M->nelt;
#define HDG_PPQ(KK, NTT, NQQ)                                                                          \
  postprocess_kernel<KK, NTT, NQQ><<<g, NTT, 0, M->stream>>>(M->d_vx, M->kappa, M->dt.P, M->dt.G1,      \
                                                            M->dt.Shat1, M->dt.vol_w, M->dt.pairs_n1, q, \
                                                            u, M->nelt, ustar, M->d_status)
  // the conical rule's (k+2)^3 nodes, or the symmetric rule's C(k+5, 4)
#define HDG_PP(KK, NTT)                                                           \
  if (M->tab.nq == (KK + 2) * (KK + 3) * (KK + 4) * (KK + 5) / 24)               \
    HDG_PPQ(KK, NTT, (KK + 2) * (KK + 3) * (KK + 4) * (KK + 5) / 24);            \
  else                                                                            \
    HDG_PPQ(KK, NTT, Dims<KK>::nq)
#define HDG_PPDF(KK, NTT)                                                                              \
  postprocess_df_kernel<KK, NTT><<<g, NTT, 0, M->stream>>>(                                             \
      M->d_geo, M->kappa, reinterpret_cast<const df*>(M->dt.P_df), reinterpret_cast<const df*>(M->dt.G1_df), \
      reinterpret_cast<const df*>(M->dt.Shat1_df), M->dt.vol_w, M->dt.pairs_n1, q, u, M->nelt, ustar, M->d_status)
  if (M->rec_df) {  // after a double-float assembly: the double-float postprocess
    switch (M->k) {
      case 1: HDG_PPDF(1, 64); break;
      case 2: HDG_PPDF(2, 64); break;
      case 3: HDG_PPDF(3, 128); break;
      case 4: HDG_PPDF(4, 128); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (M->k) {
      case 0: HDG_PP(0, 64); break;
      case 1: HDG_PP(1, 64); break;
      case 2: HDG_PP(2, 64); break;
      case 3: HDG_PP(3, 128); break;
      case 4: HDG_PP(4, 128); break;
      default: return cudaErrorInvalidValue;
    }
  }
#undef HDG_PPDF
#undef HDG_PP
#undef HDG_PPQ
  M->launches++;
  return cudaGetLastError();
}

}  // namespace hdg
