// K1 in double-float arithmetic with W_* streamed one direction at a time (reaction-diffusion,
// k = 4), and the dispatch of the double-float K1 over all of its launch shapes.
//
// The kernel of assemble_df.cuh keeps W_* = L^-1 C_*^T for the three directions in shared
// memory at once, so that S_u = M_c + tauPP + sum_* W_*^T W_* and the face-weighted sums
// Wt_l = sum_* n_{l*} W_* that form G are each built in one pass; at k = 4 that holds 109 KB per
// element and an SM keeps two elements resident (eight warps at 128 threads).  Here one
// direction is held at a time: each pass solves L W_* = C_*^T column by column (the columns read
// straight from the reference tables), adds W_*^T W_* to S_u, writes W_*^T to the recovery
// record and adds diag(n_*) V^T W_* into G^T, so G costs three products with V instead of one
// (27 % more arithmetic at k = 4) but the element needs 63 KB and three are resident per
// SM.  C^K is formed where M, S_u and W_* were once they are dead.  Measured on GB300 at
// 24,576 elements: 14.5 ms against 12.8 ms for the best shape of assemble_df.cuh (the extra
// products and the three rounds of triangular solves outweigh the third resident element), so
// the autotuner keeps it as a candidate that does not win there.  Same algorithm as
// assemble_df.cuh otherwise (the elimination of eq. 5.1-5.2 with the blocks of eq. 3.55-3.56
// and 4.5-4.10; C^K and C_f^K as eq. 5.5-5.6, the record of eq. 5.3):
//   L L^T = M_{kappa^-1};  V = L^-1 E^T;  for * = 1..3: W_* = L^-1 C_*^T, S_u += W_*^T W_*,
//   G += diag(n_*) V^T W_*  (G starts at diag(T) E);  L_s L_s^T = S_u;
//   [H | h] = L_s^-1 [G^T | f];  C^K = (n_l . n_l') o V^T V - H^T H + tauDD;  C_f^K = H^T h;
// with the same recovery record as the other double-float kernel.
#include <cstdlib>

#include "assemble_df.cuh"

namespace hdg {

// Shared-memory plan (df units): M | S | Wb (one direction of W) | V | G^T [n][m+1].  Before
// the factorisations the weighted coefficients kw, cw, fw and then T2 of the sum factorisation
// sit in G's space, T1 in S and Wb; f^K waits in a static array until G is final.
template <int K>
struct LeanSmem {
  using D = Dims<K>;
  static constexpr int n = D::n, m = D::m, nq = D::nq, d2 = D::d2;
  static constexpr int o_M = 0, o_S = n * n, o_Wb = 2 * n * n, o_V = 3 * n * n, o_G = o_V + n * m;
  static constexpr int total = o_G + n * (m + 1);
  static constexpr int nn = K + 2, np1 = (K + 1) * (K + 2) / 2, np2 = d2 * (d2 + 1) / 2;
  static constexpr int o_kw = o_G, o_cw = o_kw + nq, o_fw = o_cw + nq;
  static constexpr int o_T1 = o_S, o_T2 = o_G;
  static_assert(3 * nq <= n * (m + 1), "kw, cw, fw must fit in the space of G");
  static_assert((2 * np1 + K + 1) * nn * nn <= 2 * n * n, "T1 must fit in the space of S and Wb");
  static_assert((2 * np2 + d2) * nn <= n * (m + 1), "T2 must fit in the space of G");
  static_assert(m * m <= 3 * n * n, "C^K must fit in the space of M, S and Wb (dead by then)");
  static constexpr size_t bytes = sizeof(df) * total;
};

// launch shapes (threads, resident elements per SM) of the streamed kernel
template <int K, int V>
struct LeanShape;
template <> struct LeanShape<4, 0> { static constexpr int NT = 128, MINB = 3; };
template <> struct LeanShape<4, 1> { static constexpr int NT = 192, MINB = 3; };
constexpr int kLeanShapes = 2;

template <int K, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) assemble_df_lean_kernel(AsmDfArgs A) {
  using D = Dims<K>;
  using SM = LeanSmem<K>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, nq = D::nq;
  constexpr int NP = n * (n + 1) / 2, MP = m * (m + 1) / 2;
  static_assert(NT > m + 1, "the triangular solves of [G^T | f] need m + 1 threads");
  extern __shared__ df smd[];
  df* kw = smd + SM::o_kw;
  df* cw = smd + SM::o_cw;
  df* fw = smd + SM::o_fw;
  df* Ms = smd + SM::o_M;
  df* Ss = smd + SM::o_S;
  df* Wb = smd + SM::o_Wb;
  df* V = smd + SM::o_V;
  df* Gt = smd + SM::o_G;
  __shared__ df s_a[3][3], s_nrm[4][3], s_T[4], s_nn[4][4], s_vol;
  __shared__ df invdM[n], invdS[n], s_f[n];
  __shared__ int s_perm[4];
  __shared__ int s_bad, s_coef;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t Ke = A.e0 + blockIdx.x;

  // coefficient loads issued before the first barrier (they overlap the geometry loads)
  constexpr int NPRE = (nq + NT - 1) / NT;
  double pre[NPRE][3];
#pragma unroll
  for (int i = 0; i < NPRE; ++i) {
    const int t = tid + i * NT;
    pre[i][0] = pre[i][1] = pre[i][2] = 0.0;
    if (t < nq) {
      pre[i][0] = __ldg(A.kappa + Ke * nq + t);
      pre[i][1] = __ldg(A.c + Ke * nq + t);
      pre[i][2] = __ldg(A.f + Ke * nq + t);
    }
  }
  // geometry: cofactors a (9), normals (12), T_l = tau_l |e_l| (4), the volume
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
  // coefficients weighted by |K| omega_q (the reciprocal of kappa a Newton step on the FP32 pipe)
#pragma unroll
  for (int ip = 0; ip < NPRE; ++ip) {
    const int q = tid + ip * NT;
    if (q >= nq) break;
    const double kap = pre[ip][0], cc = pre[ip][1], ff = pre[ip][2];
    if (!(kap > 0.0) || !(cc >= 0.0) || !isfinite(kap) || !isfinite(cc) || !isfinite(ff)) s_coef = 1;
    const df vw = df_mul(s_vol, ldg_df(A.w_df + q));
    kw[q] = df_mul(vw, df_recip(kap > 0.0 ? df_from_double(kap) : df_make(1.f, 0.f)));
    cw[q] = df_mul(vw, df_from_double(cc));
    fw[q] = df_mul(vw, df_from_double(ff));
  }
  __syncthreads();

  // M_{kappa^-1}, M_c and f^K by sum factorisation over the conical nodes (as assemble_df.cuh)
  constexpr int nn = SM::nn, nn2 = nn * nn, np1 = SM::np1, np2 = SM::np2;
  df* T1 = smd + SM::o_T1;
  df* T2 = smd + SM::o_T2;
  for (int t = tid; t < np1 * nn2; t += NT) {  // T1 = sum_l g A_pa A_pb
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
  __syncthreads();
  for (int t = tid; t < np2 * nn; t += NT) {  // T2 = sum_j B_a2 B_b2 T1
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
  for (int t = tid; t < NP; t += NT) {  // M_ab, S_ab = sum_i C_a C_b T2 (+ tauPP), f_b
    const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
    const df* t2 = T2 + A.p3to2[t] * nn;
    const bool wf = t < n;  // the first n pairs are (0, j): P_0 = 1 gives f_j
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
    if (wf) s_f[j] = j < A.nu ? dacc_result(s3) : df_make(0.f, 0.f);
  }
  __syncthreads();
  {
    const bool ok = group_cholesky_df<n, NT>(Ms, invdM, A.pairs_n, tid);
    if (!ok && tid == 0) s_bad = 1;
  }
  __syncthreads();

  constexpr int o_V = n * (m + 1), o_W = o_V + n * m, o_U = o_W + 3 * n * n;
  df* R = reinterpret_cast<df*>(A.rec) + Ke * (int64_t)D::rec;
#pragma unroll 1
  for (int st = 0; st < 3; ++st) {
    // W_st = L^-1 C_st^T column by column (C_st^T[l][c] = sum_h a_{st h} Chat_h[c][l]); with the
    // first direction also V = L^-1 E^T (column r of face l: E[r][.] of the face's permutation)
    for (int t = tid; t < n + (st == 0 ? m : 0); t += NT) {
      df x[n];
      if (t < n) {
        const df a0 = s_a[st][0], a1 = s_a[st][1], a2 = s_a[st][2];
#pragma unroll
        for (int l = 0; l < n; ++l) {
          dacc s = dacc_zero();
          dacc_mac(s, a0, ldg_df(A.Chat + t * n + l));
          dacc_mac(s, a1, ldg_df(A.Chat + (n + t) * n + l));
          dacc_mac(s, a2, ldg_df(A.Chat + (2 * n + t) * n + l));
          x[l] = dacc_result(s);
        }
      } else {
        const int r = t - n, fl = r / d2, a = r - fl * d2;
        const df* e = A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n;
#pragma unroll
        for (int l = 0; l < n; ++l) x[l] = ldg_df(e + l);
      }
      fwd_subst_df<n>(Ms, invdM, x);
      if (t < n) {
#pragma unroll
        for (int l = 0; l < n; ++l) Wb[l * n + t] = x[l];
      } else {
#pragma unroll
        for (int l = 0; l < n; ++l) V[l * m + t - n] = x[l];
      }
    }
    __syncthreads();
    // S_u += W_st^T W_st (BDM: the decoupled degree-k u unknowns become identity rows and
    // columns after the last direction), W_st^T into the record
    for (int t = tid; t < NP; t += NT) {
      const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
      dacc s = dacc_from(Ss[i * n + j]);
#pragma unroll 5
      for (int l = 0; l < n; ++l) dacc_mac(s, Wb[l * n + i], Wb[l * n + j]);
      df v = dacc_result(s);
      if (st == 2 && !(i < A.nu && j < A.nu)) v = df_make(i == j ? 1.f : 0.f, 0.f);
      Ss[i * n + j] = v;
      Ss[j * n + i] = v;
    }
    for (int t = tid; t < n * n; t += NT) {
      const int c = t / n, l = t - c * n;
      R[o_W + st * n * n + t] = Wb[l * n + c];
    }
    if (st < 2) {
      // G^T[j][r] (+)= n_{l st} (V^T W_st)[r][j] for the columns r of face l, from diag(T) E
      for (int t = tid; t < n * m; t += NT) {
        const int j = t / m, r = t - j * m, fl = r / d2, a = r - fl * d2;
        dacc y = dacc_zero();
#pragma unroll 5
        for (int l = 0; l < n; ++l) dacc_mac(y, V[l * m + r], Wb[l * n + j]);
        dacc g = dacc_zero();
        if (st == 0) dacc_mac(g, s_T[fl], ldg_df(A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n + j));
        else g = dacc_from(Gt[j * (m + 1) + r]);
        dacc_mac(g, s_nrm[fl][st], dacc_result(y));
        Gt[j * (m + 1) + r] = dacc_result(g);
      }
    }
    __syncthreads();
  }

  // warp 0 factors S_u while the others finish G^T with the last direction, append f^K and
  // write the parts of the record that are final: V^T, U_M (column-packed, 1/U_ii last), normals
  if (warp == 0) {
    const bool ok = group_cholesky_df<n, 32>(Ss, invdS, A.pairs_n, lane);
    if (!ok && lane == 0) s_bad = 1;
  } else {
    for (int t = tid - 32; t < n * m; t += NT - 32) {
      const int j = t / m, r = t - j * m, fl = r / d2;
      dacc y = dacc_zero();
#pragma unroll 5
      for (int l = 0; l < n; ++l) dacc_mac(y, V[l * m + r], Wb[l * n + j]);
      dacc g = dacc_from(Gt[j * (m + 1) + r]);
      dacc_mac(g, s_nrm[fl][2], dacc_result(y));
      Gt[j * (m + 1) + r] = j < A.nu ? dacc_result(g) : df_make(0.f, 0.f);
    }
    for (int j = tid - 32; j < n; j += NT - 32) Gt[j * (m + 1) + m] = s_f[j];
    for (int t = tid - 32; t < n * m; t += NT - 32) {
      const int r = t / n, l = t - r * n;
      R[o_V + t] = V[l * m + r];
    }
    for (int t = tid - 32; t < n * n; t += NT - 32) {
      const int i = t / n, l = t - i * n;
      if (l <= i) R[o_U + D::tri + i * (i + 1) / 2 + l] = (l == i) ? invdM[i] : Ms[t];
    }
    for (int t = tid - 32; t < 12; t += NT - 32) R[o_U + 2 * D::tri + t] = s_nrm[t / 3][t % 3];
  }
  __syncthreads();

  // [H | h] = L_s^-1 [G^T | f] by the first m + 1 threads; the others write U_s
  if (tid < m + 1) {
    df x[n];
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = Gt[l * (m + 1) + tid];
    fwd_subst_df<n>(Ss, invdS, x);
#pragma unroll
    for (int l = 0; l < n; ++l) Gt[l * (m + 1) + tid] = x[l];
  } else {
    for (int t = tid - (m + 1); t < n * n; t += NT - (m + 1)) {
      const int i = t / n, l = t - i * n;
      if (l <= i) R[o_U + i * (i + 1) / 2 + l] = (l == i) ? invdS[i] : Ss[t];
    }
  }
  __syncthreads();

  // C = (n_l . n_l') o V^T V + tauDD - H^T H, C_f = H^T h, [H | h]^T into the record
  double* Cout = A.C + Ke * (int64_t)(m * m);  // row-major, as in assemble.cu
  df* Cs = smd;                                // M, S_u and Wb are dead
  for (int t = tid; t < MP; t += NT) {
    const int r = A.pairs_m[2 * t], s = A.pairs_m[2 * t + 1];
    const int fr = r / d2, fs = s / d2;
    dacc b = dacc_zero();
#pragma unroll 5
    for (int l = 0; l < n; ++l) dacc_mac(b, V[l * m + r], V[l * m + s]);
    df cv = df_mul(s_nn[fr][fs], dacc_result(b));
    if (r == s) cv = df_add(cv, s_T[fr]);
    dacc hh = dacc_from(cv);
#pragma unroll 5
    for (int j = 0; j < n; ++j) dacc_msub(hh, Gt[j * (m + 1) + r], Gt[j * (m + 1) + s]);
    const df v = dacc_result(hh);
    Cs[r * m + s] = v;
    Cs[s * m + r] = v;
  }
  for (int r = tid; r < m; r += NT) {
    dacc s = dacc_zero();
#pragma unroll 5
    for (int j = 0; j < n; ++j) dacc_mac(s, Gt[j * (m + 1) + r], Gt[j * (m + 1) + m]);
    A.Cf[Ke * m + r] = df_to_double(dacc_result(s));
  }
  for (int t = tid; t < n * (m + 1); t += NT) {
    const int r = t / n, i = t - r * n;
    R[t] = Gt[i * (m + 1) + r];
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += NT) Cout[t] = df_to_double(Cs[t]);
  if (tid == 0) {
    if (s_bad) atomicAdd(A.status + 0, 1);
    if (s_coef) atomicAdd(A.status + 1, 1);
  }
}

template <int K, int V>
static cudaError_t launch_lean_shape(hdg_mesh* M, const AsmDfArgs& a) {
  constexpr int NT = LeanShape<K, V>::NT, MINB = LeanShape<K, V>::MINB;
  const size_t smem = LeanSmem<K>::bytes;
  static bool attrs_set = false;  // once per instantiation (the element-range launches repeat)
  if (!attrs_set) {
    cudaError_t e = cudaFuncSetAttribute(assemble_df_lean_kernel<K, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(assemble_df_lean_kernel<K, NT, MINB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
    if (e != cudaSuccess) return e;
    attrs_set = true;
  }
  assemble_df_lean_kernel<K, NT, MINB><<<(unsigned)a.count, NT, smem, M->stream>>>(a);
  M->launches += 1;
  return cudaGetLastError();
}

// the streamed kernel applies to reaction-diffusion at k = 4
static bool lean_applies(const hdg_mesh* M) { return M->k == 4 && M->beta_q == nullptr; }

int k1_shape_count(const hdg_mesh* M) { return k1_variants(M->k) + (lean_applies(M) ? kLeanShapes : 0); }

int k1_shape_threads(const hdg_mesh* M, int v) {
  const int nb = k1_variants(M->k);
  if (v < nb || !lean_applies(M)) return k1_threads(M->k, v < nb ? v : 0);
  return v - nb ? LeanShape<4, 1>::NT : LeanShape<4, 0>::NT;
}

// the shape the launch takes: HDG_K1_VARIANT overrides the tuned one (tests of every shape)
static int k1_shape_of(const hdg_mesh* M) {
  int v = M->k1_variant;
  if (const char* ev = std::getenv("HDG_K1_VARIANT")) v = std::atoi(ev);
  return v;
}

static cudaError_t launch_lean(hdg_mesh* M, const AsmDfArgs& a, int lv) {
  M->rec_df = true;
  return lv ? launch_lean_shape<4, 1>(M, a) : launch_lean_shape<4, 0>(M, a);
}

cudaError_t launch_k1(hdg_mesh* M) {
  const int v = k1_shape_of(M), nb = k1_variants(M->k);
  if (v >= nb && v < nb + kLeanShapes && lean_applies(M)) return launch_lean(M, df_args(M), v - nb);
  return launch_assemble_df(M);
}

cudaError_t launch_k1_range(hdg_mesh* M, int64_t e0, int64_t count) {
  const int v = k1_shape_of(M), nb = k1_variants(M->k);
  if (v >= nb && v < nb + kLeanShapes && lean_applies(M)) {
    if (count <= 0) return cudaErrorInvalidValue;
    AsmDfArgs a = df_args(M);
    a.e0 = e0;
    a.count = count;
    return launch_lean(M, a, v - nb);
  }
  return launch_assemble_df_range(M, e0, count);
}

}  // namespace hdg
