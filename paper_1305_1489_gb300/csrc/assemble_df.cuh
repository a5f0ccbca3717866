#pragma once
// K1 in double-float arithmetic (precision HDG_DF32): the same per-element assembly and static
// condensation as assemble.cu (reaction-diffusion path), with every operation carried out as
// double-float on the FP32 pipe (device_df.cuh) instead of native FP64.  On GB300 the FP64
// pipe runs at 1/63 of the FP32 rate, so the FP64-accurate condensation is faster this way.
// Inputs (kappa, c, f in FP64) are split into double-float once per node; outputs (C^K, C_f^K,
// the recovery record) are written back as FP64 in the same layouts as the FP64 kernel, so
// the trace solve, recovery and postprocess are unchanged.  Algorithm (see assemble.cu):
//   L L^T = M_{kappa^-1};  W_* = L^-1 C_*^T;  V = L^-1 E^T;  S_u = M_c + tauPP + sum W^T W;
//   G = diag(T) E + sum_* diag(n_*) V^T W_*;  L_s L_s^T = S_u;  [H | h] = L_s^-1 [G^T | f];
//   C^K = (n_l . n_l') o (V^T V) - H^T H + tauDD;  C_f^K = H^T h;
//   recovery record: [H | h], V, W_* and the factors L_s, L (K2 does the back substitutions).
// Convection (CONV = true, the reading of Section 9 in assemble.cu): B_c = -(beta P_j, grad P_i)
// joins S_u, which is then factored by LU without pivoting; alphaDP = <(beta.nu) D_i, P_j> and
// alphaDD = <(beta.nu) D_i, D_j> per face; G_col = G - alphaDP;  H_col = L^-1 G_col^T,
// H_row = U^-T G^T, h = L^-1 f;  C^K = (n_l . n_l') o V^T V - H_row^T H_col + tauDD - alphaDD,
// C_f = H_row^T h.  B_c is formed as P^T Gq with Gq[q][i] = sum_# bw_#(q) dhat_# P_i(q) and
// bw_#(q) = -(omega_q / 6) sum_* a_{*#} beta_*(p_q), so its n^2 entries cost nq n products
// each instead of 3 nq n.
#include <cstdlib>

#include "device_common.cuh"
#include "device_df.cuh"
#include "hdg_internal.h"

namespace hdg {

struct AsmDfArgs {
  const double* geo;
  const int32_t* perm;
  const double *kappa, *c, *f, *tau;
  const df *P, *Chat, *S, *E;  // double-float copies of the reference tables
  const df *AA, *BB, *CC;      // sum-factorisation tables of the volume masses
  const double *beta_q, *beta_f;  // convection: [3][nelt][nq], [3][nelt][4][nf] (FP64)
  const df *Pd, *Pl, *Dmu;        // convection: reference gradients, face traces, face bases
  const double* wf;               // face weights varpi_r
  const df *w_df, *wf_df;         // volume and face weights as double-float pairs
  const int16_t *p2to1, *p3to2;
  const double* w;
  const int16_t *pairs_n, *pairs_m;
  double *C, *Cf, *rec;
  int32_t* status;
  int64_t nelt;
  int nu;  // u unknowns kept: n (HDG), n - d2 (hybridised BDM: u in P_{k-1}, tau = 0)
  // HDG_MIXED_BF16 (MASSIN): per element [M_{kappa^-1} pairs | M_c pairs | f^K] in FP32 from the
  // tensor-core contraction (tc_mass.cu), stride m3stride floats; NULL otherwise
  const float* mass3;
  int m3stride;
  int64_t e0, count;  // this launch's elements: e0 .. e0 + count - 1 (one CTA each)
};

// Shared-memory plan.  C is formed in one pass near the end (C = (n_l . n_l') o V^T V
// + tauDD - H^T H), so its space first holds the weighted coefficients kw, cw, fw (read only
// by the first phase) and then the face-weighted sums Wt_l = sum_* n_{l*} W_* (read only by
// the phase that forms G): WTF faces at a time, all four when they fit.
template <int K, bool CONV = false>
struct AsmDfSmem {
  using D = Dims<K>;
  static constexpr int n = D::n, m = D::m, nq = D::nq, nf = D::nf, d2 = D::d2;
  static constexpr int o_M = 0;
  static constexpr int o_S = o_M + n * n;
  static constexpr int o_W = o_S + n * n;
  static constexpr int o_V = o_W + 3 * n * n;
  static constexpr int o_G = o_V + n * m;
  static constexpr int o_C = o_G + n * (m + 1);
  static constexpr int o_kw = o_C, o_cw = o_kw + nq, o_fw = o_cw + nq;
  static constexpr int o_Wt = o_C;
  static constexpr int WTF = (4 * n * n <= m * m) ? 4 : 2;  // faces of Wt held at once
  static_assert(3 * nq <= m * m, "kw, cw, fw must fit in the space of C");
  // sum factorisation of the masses: T1 [(kw, cw) np1 + fw (k+1)][nn^2] over W and V, T2
  // [(kw, cw) np2 + fw d2][nn] in C after kw, cw, fw
  static constexpr int nn = K + 2, np1 = (K + 1) * (K + 2) / 2, np2 = D::d2 * (D::d2 + 1) / 2;
  static constexpr int o_T1 = o_W, o_T2 = o_C + 3 * nq;
  static_assert((2 * np1 + K + 1) * nn * nn <= 3 * n * n + n * m, "T1 must fit in the space of W and V");
  static_assert(3 * nq + (2 * np2 + D::d2) * nn <= m * m, "T2 must fit in the space of C");
  static_assert(WTF * n * n <= m * m, "Wt must fit in the space of C");
  // convection: H_row^T [n][m] (alphaDP^T, then G^T, then H_row), the volume weights bw
  // [3][nq], Gq [nq][n], the face weights varpi_r beta.n_l [4][nf] and alphaDD [4][d2][d2]
  static constexpr int o_Hr = o_C + m * m;
  static constexpr int o_bw = o_Hr + (CONV ? n * m : 0);
  static constexpr int o_Gq = o_bw + (CONV ? 3 * nq : 0);
  static constexpr int o_bn = o_Gq + (CONV ? nq * n : 0);
  static constexpr int o_aDD = o_bn + (CONV ? 4 * nf : 0);
  static constexpr int total = o_aDD + (CONV ? 4 * d2 * d2 : 0);
  static constexpr size_t bytes = sizeof(df) * total;
};

// Launch shapes of K1 per degree: variant 0 is the default; the others trade threads per
// element for resident elements per SM (hdg_autotune times them all).
template <int K, int V>
struct K1Shape {
  static constexpr int NT = K1Occupancy<K>::NT, MINB = K1Occupancy<K>::MINB;
};
template <> struct K1Shape<1, 1> { static constexpr int NT = 64, MINB = 16; };
template <> struct K1Shape<2, 1> { static constexpr int NT = 128, MINB = 6; };
template <> struct K1Shape<2, 2> { static constexpr int NT = 128, MINB = 9; };  // 56 registers
template <> struct K1Shape<3, 1> { static constexpr int NT = 192, MINB = 4; };
template <> struct K1Shape<3, 2> { static constexpr int NT = 128, MINB = 5; };
template <> struct K1Shape<4, 1> { static constexpr int NT = 128, MINB = 2; };
template <> struct K1Shape<4, 2> { static constexpr int NT = 192, MINB = 2; };

// barrier among the warps 1 .. NT/32 - 1 (warp 0 is busy with a factorisation meanwhile)
template <int NT>
__device__ __forceinline__ void sync_workers() {
  asm volatile("bar.sync 1, %0;" ::"r"(NT - 32) : "memory");
}

__device__ __forceinline__ df shfl_xor_df(df x, int o) {
  return df_make(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
}

template <int N>
__device__ __forceinline__ void fwd_subst_df(const df* __restrict__ L, const df* invd, df* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    dacc s = dacc_from(x[l]);
#pragma unroll
    for (int i = 0; i < l; ++i) dacc_msub(s, L[l * N + i], x[i]);
    x[l] = df_mul(dacc_result(s), invd[l]);
  }
}

__device__ __forceinline__ df ldg_df(const df* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df_make(v.x, v.y);
}

// L x = b with the unit-lower factor of warp_lu_df
template <int N>
__device__ __forceinline__ void fwd_subst_unit_df(const df* __restrict__ LU, df* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    dacc s = dacc_from(x[l]);
#pragma unroll
    for (int i = 0; i < l; ++i) dacc_msub(s, LU[l * N + i], x[i]);
    x[l] = dacc_result(s);
  }
}

// U^T x = b (U^T lower triangular) with the factor of warp_lu_df
template <int N>
__device__ __forceinline__ void fwd_subst_Ut_df(const df* __restrict__ LU, const df* invd, df* x) {
#pragma unroll
  for (int l = 0; l < N; ++l) {
    dacc s = dacc_from(x[l]);
#pragma unroll
    for (int i = 0; i < l; ++i) dacc_msub(s, LU[i * N + l], x[i]);
    x[l] = df_mul(dacc_result(s), invd[l]);
  }
}

// LU without pivoting (unit-lower L below the diagonal, U on and above) of the N x N
// double-float matrix A by one warp, right-looking: at step j column j is scaled by 1/U_jj
// and the trailing block updated, A_il -= L_ij U_jl.  invd receives 1/U_jj (formed in FP64,
// N per element).  For S_u with convection, whose symmetric part is positive definite, every
// leading minor is non-zero.  Returns, on every lane, whether all pivots were non-zero.
template <int N>
__device__ __forceinline__ bool warp_lu_df(df* A, df* invd, int lane) {
  bool ok = true;
  for (int j = 0; j < N; ++j) {
    const df piv = A[j * N + j];
    ok = ok && (piv.hi != 0.f) && isfinite(piv.hi);
    const df ip = df_recip(piv.hi != 0.f ? piv : df_make(1.f, 0.f));
    if (lane == 0) invd[j] = ip;
    for (int i = j + 1 + lane; i < N; i += 32) A[i * N + j] = df_mul(A[i * N + j], ip);
    __syncwarp();
    const int w = N - j - 1;
    for (int t = lane; t < w * w; t += 32) {
      const int i = j + 1 + t / w, l = j + 1 + t % w;
      dacc s = dacc_from(A[i * N + l]);
      dacc_msub(s, A[i * N + j], A[j * N + l]);
      A[i * N + l] = dacc_result(s);
    }
    __syncwarp();
  }
  return ok;
}

template <int K, int NT, int MINB, bool CONV, bool MASSIN = false>
__global__ void __launch_bounds__(NT, MINB) assemble_df_kernel(AsmDfArgs A) {
  using D = Dims<K>;
  using SM = AsmDfSmem<K, CONV>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, nq = D::nq, nf = D::nf;
  constexpr int NP = n * (n + 1) / 2, MP = m * (m + 1) / 2;
  extern __shared__ df smd[];
  df* kw = smd + SM::o_kw;
  df* cw = smd + SM::o_cw;
  df* fw = smd + SM::o_fw;
  df* Ms = smd + SM::o_M;
  df* Ss = smd + SM::o_S;
  df* W = smd + SM::o_W;
  df* V = smd + SM::o_V;
  df* Wt = smd + SM::o_Wt;
  df* Gt = smd + SM::o_G;
  df* Cs = smd + SM::o_C;
  df* Hr = smd + SM::o_Hr;    // convection only
  df* bw = smd + SM::o_bw;
  df* Gq = smd + SM::o_Gq;
  df* bn = smd + SM::o_bn;
  df* aDD = smd + SM::o_aDD;
  __shared__ df s_a[3][3], s_nrm[4][3], s_T[4], s_nn[4][4], s_vol;
  __shared__ df invdM[n], invdS[n];
  __shared__ int s_perm[4];
  __shared__ int s_bad, s_coef;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t Ke = A.e0 + blockIdx.x;

  // this thread's coefficient loads of the next phase, issued before the first barrier so that
  // they overlap the geometry loads (tasks t = tid, tid + NT: kappa, c, f at node t; with
  // convection beta at volume node t - nq, then beta at face node t - 2 nq)
  constexpr int NTASK = CONV ? 2 * nq + 4 * nf : nq;
  constexpr int NPRE = (NTASK + NT - 1) / NT;
  double pre[NPRE][3];
#pragma unroll
  for (int i = 0; i < NPRE; ++i) {
    const int t = tid + i * NT;
    pre[i][0] = pre[i][1] = pre[i][2] = 0.0;
    if (t < nq) {
      if constexpr (!MASSIN) {  // with MASSIN the masses and f^K arrive formed
        pre[i][0] = __ldg(A.kappa + Ke * nq + t);
        pre[i][1] = __ldg(A.c + Ke * nq + t);
        pre[i][2] = __ldg(A.f + Ke * nq + t);
      }
    } else if (CONV && t < 2 * nq) {
#pragma unroll
      for (int st = 0; st < 3; ++st) pre[i][st] = __ldg(A.beta_q + ((int64_t)st * A.nelt + Ke) * nq + (t - nq));
    } else if (CONV && t < NTASK) {
#pragma unroll
      for (int st = 0; st < 3; ++st) pre[i][st] = __ldg(A.beta_f + ((int64_t)st * A.nelt + Ke) * 4 * nf + (t - 2 * nq));
    }
  }

  // the element's geometry (formed once per mesh by geometry_kernel) in double-float, one
  // value per thread: cofactors a (9), normals (12), T_l = tau_l |e_l| (4), the volume
  if (tid < 21) {
    const df v = df_from_double(__ldg(A.geo + Ke * kGeoStride + tid));
    if (tid < 9) s_a[tid / 3][tid % 3] = v;
    else s_nrm[(tid - 9) / 3][(tid - 9) % 3] = v;
  } else if (tid < 25) {
    const int l = tid - 21;
    const double tau = A.nu < n ? 0.0 : A.tau ? A.tau[Ke * 4 + l] : 1.0;
    s_T[l] = df_from_double(tau * __ldg(A.geo + Ke * kGeoStride + tid));  // eq. 4.22 (0 for BDM)
  } else if (tid == 25) {
    s_vol = df_from_double(__ldg(A.geo + Ke * kGeoStride + 25));
  } else if (tid < 30) {
    s_perm[tid - 26] = A.perm[Ke * 4 + tid - 26] - 1;
  } else if (tid == 30) {
    s_bad = 0;
    s_coef = 0;
  }
  __syncthreads();
  if (tid < 16) {  // n_l . n_l'
    const int a = tid / 4, b = tid % 4;
    dacc s = dacc_zero();
#pragma unroll
    for (int d = 0; d < 3; ++d) dacc_mac(s, s_nrm[a][d], s_nrm[b][d]);
    s_nn[a][b] = dacc_result(s);
  }

  // coefficients weighted by |K| omega_q; with convection also the volume weights bw and the
  // face weights bn, each task on its own thread, in double-float arithmetic (the FP64 values
  // are only converted; the reciprocal of kappa is a Newton step on the FP32 pipe).
#pragma unroll
  for (int ip = 0; ip < NPRE; ++ip) {
    const int t = tid + ip * NT;
    if (t >= NTASK) break;
    if (t < nq) {
      if constexpr (MASSIN) continue;
      const int q = t;
      const double kap = pre[ip][0], cc = pre[ip][1], ff = pre[ip][2];
      if (!(kap > 0.0) || !(cc >= 0.0) || !isfinite(kap) || !isfinite(cc) || !isfinite(ff)) s_coef = 1;
      const df vw = df_mul(s_vol, ldg_df(A.w_df + q));
      kw[q] = df_mul(vw, df_recip(kap > 0.0 ? df_from_double(kap) : df_make(1.f, 0.f)));
      cw[q] = df_mul(vw, df_from_double(cc));
      fw[q] = df_mul(vw, df_from_double(ff));
    } else if (t < 2 * nq) {
      // bw_#(q) = -(omega_q / 6) sum_* a_{*#} beta_*(p_q)  (B_c = sum_q sum_# bw P_qj dhat_# P_qi)
      const int q = t - nq;
      const df b0 = df_from_double(pre[ip][0]), b1 = df_from_double(pre[ip][1]), b2 = df_from_double(pre[ip][2]);
      const df sc = df_mul(ldg_df(A.w_df + q), df_from_double(-1.0 / 6.0));
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        dacc a = dacc_zero();
        dacc_mac(a, s_a[0][h], b0);
        dacc_mac(a, s_a[1][h], b1);
        dacc_mac(a, s_a[2][h], b2);
        bw[h * nq + q] = df_mul(sc, dacc_result(a));
      }
    } else {
      // varpi_r beta(x_{r,l}^K) . n_l at the element's face nodes
      const int u = t - 2 * nq, fl = u / nf, r = u - fl * nf;
      dacc acc = dacc_zero();
#pragma unroll
      for (int st = 0; st < 3; ++st) dacc_mac(acc, s_nrm[fl][st], df_from_double(pre[ip][st]));
      bn[u] = df_mul(ldg_df(A.wf_df + r), dacc_result(acc));
    }
  }
  __syncthreads();

  // M_{kappa^-1}, M_c and the f^K column by sum factorisation over the conical nodes
  // (i, j, l): sum_q g_q P_a P_b = sum_i CC_ab(i) sum_j BB(j) sum_l g AA(l).  f_a is the
  // (0, a) entry of the same sum with g = fw, since P_0 = 1: its pairs are the first k + 1
  // 1-D pairs, the first d2 2-D pairs and the first n 3-D pairs.
  constexpr int nn = SM::nn, nn2 = nn * nn, np1 = SM::np1, np2 = SM::np2;
  df* T1 = smd + SM::o_T1;  // [kw: np1 | cw: np1 | fw: k+1][nn2]
  df* T2 = smd + SM::o_T2;  // [kw: np2 | cw: np2 | fw: d2][nn]
  for (int t = tid; t < (MASSIN ? 0 : np1 * nn2); t += NT) {  // T1 = sum_l g A_pa A_pb
    const int p1 = t / nn2, ij = t - p1 * nn2;
    const bool wf = p1 <= K;
    dacc s1 = dacc_zero(), s2 = dacc_zero(), s3 = dacc_zero();
#pragma unroll
    for (int l = 0; l < nn; ++l) {
      const df a = ldg_df(A.AA + p1 * nn + l);
      dacc_mac(s1, kw[ij * nn + l], a);
      dacc_mac(s2, cw[ij * nn + l], a);
      if (wf) dacc_mac(s3, fw[ij * nn + l], a);
    }
    T1[t] = dacc_result(s1);
    T1[np1 * nn2 + t] = dacc_result(s2);
    if (wf) T1[2 * np1 * nn2 + t] = dacc_result(s3);
  }
  if constexpr (CONV) {  // Gq[q][i] = sum_# bw_#(q) dhat_# P_i(p_hat_q)
    for (int t = tid; t < nq * n; t += NT) {
      const int q = t / n, i = t - q * n;
      dacc g = dacc_zero();
#pragma unroll
      for (int h = 0; h < 3; ++h) dacc_mac(g, bw[h * nq + q], ldg_df(A.Pd + (h * nq + q) * n + i));
      Gq[t] = dacc_result(g);
    }
  }
  __syncthreads();
  for (int t = tid; t < (MASSIN ? 0 : np2 * nn); t += NT) {  // T2 = sum_j B_a2 B_b2 T1
    const int p2 = t / nn, i = t - p2 * nn;
    const bool wf = p2 < d2;
    const df* t1 = T1 + A.p2to1[p2] * nn2 + i * nn;
    dacc s1 = dacc_zero(), s2 = dacc_zero(), s3 = dacc_zero();
#pragma unroll
    for (int j = 0; j < nn; ++j) {
      const df b = ldg_df(A.BB + p2 * nn + j);
      dacc_mac(s1, t1[j], b);
      dacc_mac(s2, t1[np1 * nn2 + j], b);
      if (wf) dacc_mac(s3, t1[2 * np1 * nn2 + j], b);
    }
    T2[t] = dacc_result(s1);
    T2[np2 * nn + t] = dacc_result(s2);
    if (wf) T2[2 * np2 * nn + t] = dacc_result(s3);
  }
  __syncthreads();
  if constexpr (MASSIN) {  // M_ab, S_ab (+ tauPP), f_b from the tensor-core contraction
    const float* mr = A.mass3 + Ke * (int64_t)A.m3stride;
    for (int t = tid; t < NP; t += NT) {
      const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
      const df v1 = df_make(__ldg(mr + t), 0.f);
      dacc s2 = dacc_from(df_make(__ldg(mr + NP + t), 0.f));
#pragma unroll
      for (int l = 0; l < 4; ++l) dacc_mac(s2, s_T[l], ldg_df(A.S + (l * n + i) * n + j));
      const df v2 = dacc_result(s2);
      Ms[i * n + j] = v1;
      Ms[j * n + i] = v1;
      Ss[i * n + j] = v2;
      Ss[j * n + i] = v2;
      if (t < n) Gt[j * (m + 1) + m] = j < A.nu ? df_make(__ldg(mr + 2 * NP + j), 0.f) : df_make(0.f, 0.f);
    }
  }
  for (int t = tid; t < (MASSIN ? 0 : NP); t += NT) {  // M_ab, S_ab = sum_i C_a C_b T2 (+ tauPP), f_b
    const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
    const df* t2 = T2 + A.p3to2[t] * nn;
    const bool wf = t < n;
    dacc s1 = dacc_zero(), s2 = dacc_zero(), s3 = dacc_zero();
#pragma unroll
    for (int ii = 0; ii < nn; ++ii) {
      const df c = ldg_df(A.CC + t * nn + ii);
      dacc_mac(s1, t2[ii], c);
      dacc_mac(s2, t2[np2 * nn + ii], c);
      if (wf) dacc_mac(s3, t2[2 * np2 * nn + ii], c);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) dacc_mac(s2, s_T[l], ldg_df(A.S + (l * n + i) * n + j));
    const df v1 = dacc_result(s1), v2 = dacc_result(s2);
    Ms[i * n + j] = v1;
    Ms[j * n + i] = v1;
    Ss[i * n + j] = v2;
    Ss[j * n + i] = v2;
    if (wf) Gt[j * (m + 1) + m] = j < A.nu ? dacc_result(s3) : df_make(0.f, 0.f);  // pair (0, j)
  }
  // C_*^T from C_hat and the cofactors, V = E^T (both where T1 was)
  for (int t = tid; t < 3 * n * n; t += NT) {
    const int st = t / (n * n), rem = t - st * n * n, l = rem / n, cidx = rem - l * n;
    dacc s = dacc_zero();
#pragma unroll
    for (int h = 0; h < 3; ++h) dacc_mac(s, s_a[st][h], ldg_df(A.Chat + (h * n + cidx) * n + l));
    W[t] = dacc_result(s);
  }
  for (int t = tid; t < n * m; t += NT) {
    const int l = t / m, r = t - l * m, fl = r / d2, a = r - fl * d2;
    V[t] = ldg_df(A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n + l);
  }
  __syncthreads();

  if constexpr (!CONV) {  // every thread of the block factors M (nothing else can proceed meanwhile)
    const bool ok = group_cholesky_df<n, NT>(Ms, invdM, A.pairs_n, tid);
    if (!ok && tid == 0) s_bad = 1;
  } else if (warp == 0) {  // convection: warp 0 factors M while the other warps form the
    const bool ok = group_cholesky_df<n, 32>(Ms, invdM, A.pairs_n, lane);  // convection blocks
    if (!ok && lane == 0) s_bad = 1;
  } else {
    // B_c[i][j] = sum_q P_qj Gq[q][i] and B_c[j][i] = sum_q P_qi Gq[q][j], into S_u
    for (int t = tid - 32; t < NP; t += NT - 32) {
      const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
      dacc bij = dacc_from(Ss[i * n + j]), bji = dacc_from(Ss[j * n + i]);
#pragma unroll 4
      for (int q = 0; q < nq; ++q) {
        dacc_mac(bij, ldg_df(A.P + q * n + j), Gq[q * n + i]);
        dacc_mac(bji, ldg_df(A.P + q * n + i), Gq[q * n + j]);
      }
      Ss[i * n + j] = dacc_result(bij);
      if (i != j) Ss[j * n + i] = dacc_result(bji);
    }
    // bD[l][r'][a] = varpi (beta.n) D^mu_{r'a} into Gq's space (Gq is read by B_c above, so
    // the workers meet at a barrier first), then alphaDP^T[l][r] = sum_r' bD P^l_{r'l} and
    // alphaDD[l][a][b] = sum_r' bD[l][r'][a] D^mu_{r'b}
    sync_workers<NT>();
    df* bD = Gq;
    static_assert(4 * nf * d2 <= nq * n, "bD must fit in the space of Gq");
    for (int t = tid - 32; t < 4 * nf * d2; t += NT - 32) {
      const int fl = t / (nf * d2), ra = t - fl * nf * d2, rr = ra / d2, a = ra - rr * d2;
      bD[t] = df_mul(bn[fl * nf + rr], ldg_df(A.Dmu + (s_perm[fl] * nf + rr) * d2 + a));
    }
    sync_workers<NT>();
    for (int t = tid - 32; t < n * m; t += NT - 32) {
      const int l = t / m, r = t - l * m, fl = r / d2, a = r - fl * d2;
      const df* Pl = A.Pl + fl * nf * n;
      const df* bd = bD + fl * nf * d2;
      dacc acc = dacc_zero();
#pragma unroll 4
      for (int rr = 0; rr < nf; ++rr) dacc_mac(acc, bd[rr * d2 + a], ldg_df(Pl + rr * n + l));
      Hr[t] = dacc_result(acc);
    }
    for (int t = tid - 32; t < 4 * d2 * d2; t += NT - 32) {
      const int fl = t / (d2 * d2), ab = t - fl * d2 * d2, a = ab / d2, b = ab - a * d2;
      const df* Dm = A.Dmu + s_perm[fl] * nf * d2;
      const df* bd = bD + fl * nf * d2;
      dacc acc = dacc_zero();
#pragma unroll 4
      for (int rr = 0; rr < nf; ++rr) dacc_mac(acc, bd[rr * d2 + a], ldg_df(Dm + rr * d2 + b));
      aDD[t] = dacc_result(acc);
    }
  }
  __syncthreads();

  for (int t = tid; t < 3 * n + m; t += NT) {
    df* base;
    int col, stride;
    if (t < 3 * n) {
      base = W + (t / n) * n * n;
      col = t % n;
      stride = n;
    } else {
      base = V;
      col = t - 3 * n;
      stride = m;
    }
    df x[n];
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = base[l * stride + col];
    fwd_subst_df<n>(Ms, invdM, x);
#pragma unroll
    for (int l = 0; l < n; ++l) base[l * stride + col] = x[l];
  }
  __syncthreads();

  for (int t = tid; t < NP; t += NT) {
    const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
    if constexpr (CONV) {  // S_u is not symmetric: the same W^T W term joins both entries
      dacc s = dacc_zero();
#pragma unroll
      for (int st = 0; st < 3; ++st)
#pragma unroll 4
        for (int l = 0; l < n; ++l) dacc_mac(s, W[st * n * n + l * n + i], W[st * n * n + l * n + j]);
      const df w = dacc_result(s);
      Ss[i * n + j] = df_add(Ss[i * n + j], w);
      if (i != j) Ss[j * n + i] = df_add(Ss[j * n + i], w);
    } else {
      dacc s = dacc_from(Ss[i * n + j]);
#pragma unroll
      for (int st = 0; st < 3; ++st)
#pragma unroll 4
        for (int l = 0; l < n; ++l) dacc_mac(s, W[st * n * n + l * n + i], W[st * n * n + l * n + j]);
      // BDM: the degree-k u unknowns are decoupled (identity rows and columns), which erases
      // them from the elimination exactly as the paper erases their rows and columns of A_1
      const df v = (i < A.nu && j < A.nu) ? dacc_result(s) : df_make(i == j ? 1.f : 0.f, 0.f);
      Ss[i * n + j] = v;
      Ss[j * n + i] = v;
    }
  }
  constexpr int WTF = SM::WTF;
  for (int t = tid; t < WTF * n * n; t += NT) {
    const int fl = t / (n * n), rem = t - fl * n * n;
    dacc s = dacc_zero();
#pragma unroll
    for (int st = 0; st < 3; ++st) dacc_mac(s, s_nrm[fl][st], W[st * n * n + rem]);
    Wt[t] = dacc_result(s);
  }
  __syncthreads();

  if (warp == 0) {
    const bool ok = CONV ? warp_lu_df<n>(Ss, invdS, lane) : group_cholesky_df<n, 32>(Ss, invdS, A.pairs_n, lane);
    if (!ok && lane == 0) s_bad = 1;
  } else {
    // G^T[j][r] = T_l E[r][j] + (V^T Wt_l)[r][j] for the columns r of face l, WTF faces per pass
#pragma unroll 1
    for (int f0 = 0; f0 < 4; f0 += WTF) {
      if (f0 > 0) {
        sync_workers<NT>();  // every column of the previous faces is done with Wt
        for (int t = tid - 32; t < WTF * n * n; t += NT - 32) {
          const int fl = f0 + t / (n * n), rem = t % (n * n);
          dacc s = dacc_zero();
#pragma unroll
          for (int st = 0; st < 3; ++st) dacc_mac(s, s_nrm[fl][st], W[st * n * n + rem]);
          Wt[t] = dacc_result(s);
        }
        sync_workers<NT>();
      }
      for (int t = tid - 32; t < n * WTF * d2; t += NT - 32) {
        const int j = t / (WTF * d2), r = f0 * d2 + (t - j * (WTF * d2)), fl = r / d2, a = r - fl * d2;
        dacc g = dacc_zero();
        dacc_mac(g, s_T[fl], ldg_df(A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n + j));
        const df* wt = Wt + (fl - f0) * n * n;
#pragma unroll 4
        for (int l = 0; l < n; ++l) dacc_mac(g, V[l * m + r], wt[l * n + j]);
        if constexpr (CONV) {
          const df gv = dacc_result(g);
          Gt[j * (m + 1) + r] = df_sub(gv, Hr[j * m + r]);  // G_col^T = (G - alphaDP)^T
          Hr[j * m + r] = gv;                              // G^T
        } else {
          Gt[j * (m + 1) + r] = j < A.nu ? dacc_result(g) : df_make(0.f, 0.f);
        }
      }
    }
  }
  __syncthreads();

  // [H | h] = L_s^-1 [G^T | f] by the first m + 1 threads (the back substitutions of the
  // recovery are left to K2); meanwhile the others write the parts of the recovery record
  // that are already final: V^T, W_*^T, U_s and U_M packed by columns (column i: U_0i ..
  // U_(i-1)i, then 1/U_ii, with U = L^T), the normals.  Column-major blocks, so that the
  // recovery kernel reads them with unit stride; every entry a double-float pair (8 bytes,
  // the layout of the FP64 record), read by the double-float recovery kernel.
  // (convection: [H_col | h] = L^-1 [G_col^T | f] by the first m + 1 threads and H_row =
  // U^-T G^T by the next m; U_s is the U of the LU)
  df* R = reinterpret_cast<df*>(A.rec) + Ke * (int64_t)D::rec;
  constexpr int NTRI = (m + 1) + (CONV ? m : 0);
  static_assert(NT > NTRI, "K1 needs more threads than triangular solves");
  if (tid < m + 1) {
    df x[n];
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = Gt[l * (m + 1) + tid];
    if constexpr (CONV) fwd_subst_unit_df<n>(Ss, x); else fwd_subst_df<n>(Ss, invdS, x);
#pragma unroll
    for (int l = 0; l < n; ++l) Gt[l * (m + 1) + tid] = x[l];
  } else if (tid < NTRI) {
    const int col = tid - (m + 1);
    df x[n];
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = Hr[l * m + col];
    fwd_subst_Ut_df<n>(Ss, invdS, x);
#pragma unroll
    for (int l = 0; l < n; ++l) Hr[l * m + col] = x[l];
  } else {
    constexpr int o_V = n * (m + 1), o_W = o_V + n * m, o_U = o_W + 3 * n * n;
    for (int t = tid - NTRI; t < n * m; t += NT - NTRI) {
      const int r = t / n, l = t - r * n;
      R[o_V + t] = V[l * m + r];
    }
    for (int t = tid - NTRI; t < 3 * n * n; t += NT - NTRI) {
      const int st = t / (n * n), rem = t - st * n * n, c = rem / n, l = rem - c * n;
      R[o_W + t] = W[st * n * n + l * n + c];
    }
    for (int t = tid - NTRI; t < n * n; t += NT - NTRI) {
      const int i = t / n, l = t - i * n;
      if (l <= i) {
        R[o_U + i * (i + 1) / 2 + l] = (l == i) ? invdS[i] : (CONV ? Ss[l * n + i] : Ss[t]);
        R[o_U + D::tri + i * (i + 1) / 2 + l] = (l == i) ? invdM[i] : Ms[t];
      }
    }
    for (int t = tid - NTRI; t < 12; t += NT - NTRI)
      R[o_U + 2 * D::tri + t] = s_nrm[t / 3][t % 3];
  }
  __syncthreads();

  // C = (n_l . n_l') o V^T V + tauDD - H^T H  (V = L^-1 E^T; H = rows of G^T);
  // convection: C = (n_l . n_l') o V^T V + tauDD - alphaDD - H_row^T H_col, C_f = H_row^T h
  if constexpr (CONV) {  // the symmetric V^T V part once per pair (r <= s), both entries after
    for (int t = tid; t < MP; t += NT) {
      const int r = A.pairs_m[2 * t], s = A.pairs_m[2 * t + 1];
      const int fr = r / d2, fs = s / d2;
      dacc b = dacc_zero();
#pragma unroll 4
      for (int l = 0; l < n; ++l) dacc_mac(b, V[l * m + r], V[l * m + s]);
      df cv = df_mul(s_nn[fr][fs], dacc_result(b));
      if (r == s) cv = df_add(cv, s_T[fr]);
      df crs = cv, csr = cv;
      if (fr == fs) {
        crs = df_sub(cv, aDD[fr * d2 * d2 + (r - fr * d2) * d2 + (s - fs * d2)]);
        csr = df_sub(cv, aDD[fr * d2 * d2 + (s - fs * d2) * d2 + (r - fr * d2)]);
      }
      dacc h1 = dacc_from(crs), h2 = dacc_from(csr);
#pragma unroll 4
      for (int j = 0; j < n; ++j) {
        dacc_msub(h1, Hr[j * m + r], Gt[j * (m + 1) + s]);
        dacc_msub(h2, Hr[j * m + s], Gt[j * (m + 1) + r]);
      }
      Cs[r * m + s] = dacc_result(h1);
      if (r != s) Cs[s * m + r] = dacc_result(h2);
    }
  }
  for (int t = tid; t < (CONV ? 0 : MP); t += NT) {
    const int r = A.pairs_m[2 * t], s = A.pairs_m[2 * t + 1];
    const int fr = r / d2, fs = s / d2;
    dacc b = dacc_zero();
#pragma unroll 4
    for (int l = 0; l < n; ++l) dacc_mac(b, V[l * m + r], V[l * m + s]);
    df cv = df_mul(s_nn[fr][fs], dacc_result(b));
    if (r == s) cv = df_add(cv, s_T[fr]);
    dacc hh = dacc_from(cv);
#pragma unroll 4
    for (int j = 0; j < n; ++j) dacc_msub(hh, Gt[j * (m + 1) + r], Gt[j * (m + 1) + s]);
    const df v = dacc_result(hh);
    Cs[r * m + s] = v;
    Cs[s * m + r] = v;
  }
  for (int r = tid; r < m; r += NT) {
    dacc s = dacc_zero();
    const df* hrow = CONV ? Hr : Gt;
    const int ld = CONV ? m : (m + 1);
#pragma unroll 4
    for (int j = 0; j < n; ++j) dacc_mac(s, hrow[j * ld + r], Gt[j * (m + 1) + m]);
    A.Cf[Ke * m + r] = df_to_double(dacc_result(s));
  }
  for (int t = tid; t < n * (m + 1); t += NT) {  // [H | h]^T
    const int r = t / n, i = t - r * n;
    R[t] = Gt[i * (m + 1) + r];
  }
  __syncthreads();

  double* Cout = A.C + Ke * (int64_t)(m * m);  // row-major, as in assemble.cu
  for (int t = tid; t < m * m; t += NT) Cout[t] = df_to_double(Cs[t]);
  if (tid == 0) {
    if (s_bad) atomicAdd(A.status + 0, 1);
    if (s_coef) atomicAdd(A.status + 1, 1);
  }
}

template <int K, int V, bool CONV, bool MASSIN = false>
static cudaError_t launch_df_shape(hdg_mesh* M, const AsmDfArgs& a) {
  constexpr int NT = K1Shape<K, V>::NT, MINB = K1Shape<K, V>::MINB;
  const size_t smem = AsmDfSmem<K, CONV>::bytes;
  static bool attrs_set = false;  // once per instantiation (the element-range launches repeat)
  if (!attrs_set) {
    cudaError_t e = cudaFuncSetAttribute(assemble_df_kernel<K, NT, MINB, CONV, MASSIN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(assemble_df_kernel<K, NT, MINB, CONV, MASSIN>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attrs_set = true;
  }
  assemble_df_kernel<K, NT, MINB, CONV, MASSIN><<<(unsigned)a.count, NT, smem, M->stream>>>(a);
  M->launches += 1;
  return cudaGetLastError();
}

// argument block of a K1 launch over the mesh (assemble_df.cu)
AsmDfArgs df_args(hdg_mesh* M);

}  // namespace hdg
