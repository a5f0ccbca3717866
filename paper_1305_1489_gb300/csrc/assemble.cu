// K1: per-element quadrature assembly of the local blocks and static condensation, FP64.
//
// For each element K (one CTA per element) this forms, from kappa, c, f at the volume nodes:
//   M = M_{kappa^-1}, M_c (eq. 3.55), C_* (eq. 3.56), tauPP (eq. 4.5), tauDD (eq. 4.8),
//   n_*DP = diag(n_*) E and tauDP = diag(T) E with E the perm-selected face tables (eq. 4.10),
//   f^K (Section 3 "Source terms"),
// and eliminates (q, u) from the local system of eq. 5.1-5.2 by two Cholesky factorisations
// instead of an LU of the 4n x 4n matrix A_1 (same C^K and C_f^K to rounding):
//   L L^T = M;  W_* = L^-1 C_*^T;  V = L^-1 E^T
//   S_u = M_c + tauPP + sum_* W_*^T W_*          (Schur complement of the q block)
//   G = diag(T) E + sum_* diag(n_*) V^T W_*      (face block l: V_l^T (sum_* n_{l*} W_*))
//   L_s L_s^T = S_u;  H = L_s^-1 G^T;  h = L_s^-1 f
//   C^K = (n_l . n_l') o (V^T V) - H^T H + tauDD   (eq. 5.5)
//   C_f^K = H^T h                                 (eq. 5.6)
// and stores the factored recovery operators of eq. 5.3, which K2 applies with two
// triangular solves per element (one right-hand side each instead of m + 1 + m + 3n here):
//   u = L_s^-T (H u_dK + h);  q_* = L^-T (W_* u - V (n_* o u_dK))
//   (= M^-1 (C_*^T u - E^T (n_* o u_dK))).
//
// Convection (CONV = true; reading of Section 9: div(q + beta u) + c u = f, flux
// q.nu + (beta.nu) u_hat + tau (u - u_hat)) adds to the same elimination
//   B_c = -(beta P_j, grad P_i)_K (eq. 9.1 matrices) to S_u, which is then non-symmetric and
//   factored by LU without pivoting (its symmetric part is positive definite when
//   c + div(beta)/2 >= 0 and tau - beta.nu/2 > 0);
//   alphaDP = <(beta.nu) D_i, P_j> and alphaDD = <(beta.nu) D_i, D_j> per face (element
//   parametrisation of eq. 4.1, beta given at the element's face nodes);
//   G_col = G - alphaDP;  S_u = L U;  H_col = L^-1 G_col^T,  H_row = U^-T G^T;
//   C^K = (n_l . n_l') o (V^T V) - H_row^T H_col + tauDD - alphaDD,  C_f = H_row^T L^-1 f;
//   u = U^-1 (H_col u_dK + L^-1 f).
#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {

struct AsmArgs {
  const double* vx;
  const int32_t* perm;
  const double *kappa, *c, *f, *tau;
  const double *beta_q, *beta_f;  // [3][nelt][nq], [3][nelt][4][nf] (convection only)
  const double *P, *Chat, *S, *E, *w;
  const double *Pd, *Pl, *Dmu, *wf;  // convection only
  const int16_t *pairs_n, *pairs_m;
  double *C, *Cf, *rec;
  int32_t* status;
  int64_t nelt;
  int nu;  // u unknowns kept: n (HDG), n - d2 (hybridised BDM: u in P_{k-1}, tau = 0)
};

// NQ: volume nodes of the rule in use ((k+2)^3 conical, or the symmetric rule's count)
template <int K, bool CONV, int NQ>
struct AsmSmem {
  using D = Dims<K>;
  static constexpr int n = D::n, m = D::m, nq = NQ, nf = D::nf, d2 = D::d2;
  static constexpr int o_kw = 0, o_cw = o_kw + nq, o_fw = o_cw + nq;
  static constexpr int o_M = o_fw + nq;          // n*n   M -> L
  static constexpr int o_S = o_M + n * n;        // n*n   S_u -> L_s
  static constexpr int o_W = o_S + n * n;        // 3 n n W_*[l][c]
  static constexpr int o_V = o_W + 3 * n * n;    // n*m   V[l][r]
  static constexpr int o_Wt = o_V + n * m;       // 4 n n (sum_* n_{l*} W_*)[l'][j]
  static constexpr int o_G = o_Wt + 4 * n * n;   // n*(m+1) G^T | f -> H | h
  static constexpr int o_C = o_G + n * (m + 1);  // m*m
  // convection: H_row^T [n][m] (first alphaDP^T, then G^T, then H_row), 3 x nq reference
  // convection weights, 4 x nf face weights varpi (beta . n_l), alphaDD [4][d2][d2]
  static constexpr int o_Hr = o_C + m * m;
  static constexpr int o_bw = o_Hr + (CONV ? n * m : 0);
  static constexpr int o_bn = o_bw + (CONV ? 3 * nq : 0);
  static constexpr int o_aDD = o_bn + (CONV ? 4 * nf : 0);
  static constexpr int total = o_aDD + (CONV ? 4 * d2 * d2 : 0);
  static constexpr size_t bytes = sizeof(double) * total;
};

template <int K, int NT, bool CONV, int NQ>
__global__ void __launch_bounds__(NT, K1Occupancy<K>::MINB) assemble_kernel(AsmArgs A) {
  using D = Dims<K>;
  using SM = AsmSmem<K, CONV, NQ>;
  constexpr int n = D::n, m = D::m, d2 = D::d2, nq = NQ, nf = D::nf;
  constexpr int NP = n * (n + 1) / 2, MP = m * (m + 1) / 2;
  extern __shared__ double sm[];
  double* kw = sm + SM::o_kw;
  double* cw = sm + SM::o_cw;
  double* fw = sm + SM::o_fw;
  double* Ms = sm + SM::o_M;
  double* Ss = sm + SM::o_S;
  double* W = sm + SM::o_W;
  double* V = sm + SM::o_V;
  double* Wt = sm + SM::o_Wt;
  double* Gt = sm + SM::o_G;
  double* Cs = sm + SM::o_C;
  double* Hr = sm + SM::o_Hr;
  double* bw = sm + SM::o_bw;
  double* bn = sm + SM::o_bn;
  double* aDD = sm + SM::o_aDD;
  __shared__ double s_a[3][3], s_nrm[4][3], s_T[4], s_vol;
  __shared__ double invdM[n], invdS[n];
  __shared__ int s_perm[4];
  __shared__ int s_bad, s_coef;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int64_t Ke = blockIdx.x;

  if (tid == 0) {
    Geo g;
    element_geometry(A.vx, A.nelt, Ke, g);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s_a[i][j] = g.a[i][j];
    for (int l = 0; l < 4; ++l) {
      for (int d = 0; d < 3; ++d) s_nrm[l][d] = g.nrm[l][d];
      double tau = A.nu < n ? 0.0 : A.tau ? A.tau[Ke * 4 + l] : 1.0;
      s_T[l] = tau * g.area[l];  // T_l = tau_l |e_l|, eq. 4.22 (0 for BDM)
      s_perm[l] = A.perm[Ke * 4 + l] - 1;
    }
    s_vol = g.vol;
    s_bad = 0;
    s_coef = 0;
  }
  __syncthreads();

  // coefficients weighted by |K| omega_q (eq. 3.2, 3.55)
  for (int q = tid; q < nq; q += NT) {
    double kap = A.kappa[Ke * nq + q], cc = A.c[Ke * nq + q], ff = A.f[Ke * nq + q];
    if (!(kap > 0.0) || !(cc >= 0.0) || !isfinite(kap) || !isfinite(cc) || !isfinite(ff)) s_coef = 1;
    double vw = s_vol * A.w[q];
    kw[q] = vw / kap;
    cw[q] = vw * cc;
    fw[q] = vw * ff;
    if constexpr (CONV) {
      // -(1/6) omega_q sum_* a_{*#} beta_*(p_q): B_c = sum_q sum_# bw[#][q] P_qj dhat_# P_qi
      const double b0 = A.beta_q[(0 * A.nelt + Ke) * nq + q], b1 = A.beta_q[(1 * A.nelt + Ke) * nq + q],
                   b2 = A.beta_q[(2 * A.nelt + Ke) * nq + q];
      const double sc = -A.w[q] / 6.0;
#pragma unroll
      for (int h = 0; h < 3; ++h) bw[h * nq + q] = sc * (s_a[0][h] * b0 + s_a[1][h] * b1 + s_a[2][h] * b2);
    }
  }
  if constexpr (CONV) {
    // varpi_r beta(x_{r,l}^K) . n_l at the element's face nodes
    for (int t = tid; t < 4 * nf; t += NT) {
      const int fl = t / nf, r = t - fl * nf;
      double acc = 0.0;
#pragma unroll
      for (int st = 0; st < 3; ++st) acc = fma(A.beta_f[((int64_t)st * A.nelt + Ke) * 4 * nf + t], s_nrm[fl][st], acc);
      bn[t] = A.wf[r] * acc;
    }
  }
  __syncthreads();

  // masses M_{kappa^-1}, M_c + tauPP (lower+upper), f^K, C_*^T, E^T
  for (int t = tid; t < NP; t += NT) {
    const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
    double s1 = 0.0, s2 = 0.0;
#pragma unroll 5
    for (int q = 0; q < nq; ++q) {
      double pp = __ldg(A.P + q * n + i) * __ldg(A.P + q * n + j);
      s1 = fma(kw[q], pp, s1);
      s2 = fma(cw[q], pp, s2);
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) s2 = fma(s_T[l], __ldg(A.S + (l * n + i) * n + j), s2);
    Ms[i * n + j] = s1;
    Ms[j * n + i] = s1;
    if constexpr (CONV) {
      double bij = 0.0, bji = 0.0;  // B_c[i][j] = sum bw P_qj d P_qi,  B_c[j][i] = sum bw P_qi d P_qj
      for (int q = 0; q < nq; ++q) {
        const double pi = __ldg(A.P + q * n + i), pj = __ldg(A.P + q * n + j);
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const double wq = bw[h * nq + q];
          bij = fma(wq * pj, __ldg(A.Pd + (h * nq + q) * n + i), bij);
          bji = fma(wq * pi, __ldg(A.Pd + (h * nq + q) * n + j), bji);
        }
      }
      Ss[i * n + j] = s2 + bij;
      Ss[j * n + i] = s2 + bji;
    } else {
      Ss[i * n + j] = s2;
      Ss[j * n + i] = s2;
    }
  }
  for (int i = tid; i < n; i += NT) {
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s = fma(fw[q], __ldg(A.P + q * n + i), s);
    Gt[i * (m + 1) + m] = i < A.nu ? s : 0.0;  // BDM: no degree-k u test functions
  }
  for (int t = tid; t < 3 * n * n; t += NT) {
    const int st = t / (n * n), rem = t - st * n * n, l = rem / n, cidx = rem - l * n;
    // (C_*^T)[l][c] = C_*[c][l] = sum_# a_{*#} C_hat^#[c][l]
    double s = 0.0;
#pragma unroll
    for (int h = 0; h < 3; ++h) s = fma(s_a[st][h], __ldg(A.Chat + (h * n + cidx) * n + l), s);
    W[t] = s;
  }
  for (int t = tid; t < n * m; t += NT) {
    const int l = t / m, r = t - l * m, fl = r / d2, a = r - fl * d2;
    V[t] = __ldg(A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n + l);  // E^T
    if constexpr (CONV) {
      // alphaDP^T[l][r] = sum_r' varpi (beta.n) D^mu_{r'a} P^l_{r'l}
      const double* Dm = A.Dmu + (int64_t)s_perm[fl] * nf * d2;
      const double* Pl = A.Pl + (int64_t)fl * nf * n;
      double acc = 0.0;
      for (int rr = 0; rr < nf; ++rr) acc = fma(bn[fl * nf + rr] * __ldg(Dm + rr * d2 + a), __ldg(Pl + rr * n + l), acc);
      Hr[t] = acc;
    }
  }
  if constexpr (CONV) {
    for (int t = tid; t < 4 * d2 * d2; t += NT) {
      const int fl = t / (d2 * d2), ab = t - fl * d2 * d2, a = ab / d2, b = ab - a * d2;
      const double* Dm = A.Dmu + (int64_t)s_perm[fl] * nf * d2;
      double acc = 0.0;
      for (int rr = 0; rr < nf; ++rr) acc = fma(bn[fl * nf + rr] * __ldg(Dm + rr * d2 + a), __ldg(Dm + rr * d2 + b), acc);
      aDD[t] = acc;
    }
  }
  __syncthreads();

  // L L^T = M (one warp)
  if (warp == 0) {
    bool ok = warp_cholesky<n>(Ms, invdM, lane);
    if (!ok && lane == 0) s_bad = 1;
  }
  __syncthreads();

  // W_* = L^-1 C_*^T (3n columns), V = L^-1 E^T (m columns)
  for (int t = tid; t < 3 * n + m; t += NT) {
    double* base;
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
    double x[n];
#pragma unroll
    for (int l = 0; l < n; ++l) x[l] = base[l * stride + col];
    fwd_subst<n>(Ms, invdM, x);
#pragma unroll
    for (int l = 0; l < n; ++l) base[l * stride + col] = x[l];
  }
  __syncthreads();

  // S_u += sum_* W_*^T W_*;  Wt_l = sum_* n_{l*} W_*;  C = (n_l . n_l') (V^T V) + tauDD
  for (int t = tid; t < NP; t += NT) {
    const int i = A.pairs_n[2 * t], j = A.pairs_n[2 * t + 1];
    double s = 0.0;
#pragma unroll
    for (int st = 0; st < 3; ++st)
#pragma unroll 4
      for (int l = 0; l < n; ++l) s = fma(W[st * n * n + l * n + i], W[st * n * n + l * n + j], s);
    if (i < A.nu && j < A.nu) {  // (S_u is not symmetric with convection: update both entries)
      Ss[i * n + j] += s;
      if (i != j) Ss[j * n + i] += s;
    } else {  // BDM: the degree-k u unknowns are decoupled (identity rows and columns), which
              // erases them from the elimination as the paper erases their rows and columns of A_1
      Ss[i * n + j] = (i == j) ? 1.0 : 0.0;
      if (i != j) Ss[j * n + i] = 0.0;
    }
  }
  for (int t = tid; t < 4 * n * n; t += NT) {
    const int fl = t / (n * n), rem = t - fl * n * n;
    Wt[t] = s_nrm[fl][0] * W[rem] + s_nrm[fl][1] * W[n * n + rem] + s_nrm[fl][2] * W[2 * n * n + rem];
  }
  for (int t = tid; t < MP; t += NT) {
    const int r = A.pairs_m[2 * t], s = A.pairs_m[2 * t + 1];
    const int fr = r / d2, fs = s / d2;
    double b = 0.0;
#pragma unroll 4
    for (int l = 0; l < n; ++l) b = fma(V[l * m + r], V[l * m + s], b);
    const double nn = s_nrm[fr][0] * s_nrm[fs][0] + s_nrm[fr][1] * s_nrm[fs][1] + s_nrm[fr][2] * s_nrm[fs][2];
    double cv = nn * b + (r == s ? s_T[fr] : 0.0);
    if constexpr (CONV) {
      if (fr == fs) cv -= aDD[fr * d2 * d2 + (r - fr * d2) * d2 + (s - fs * d2)];
    }
    Cs[r * m + s] = cv;
    Cs[s * m + r] = cv;
  }
  __syncthreads();

  // warp 0: L_s L_s^T = S_u;  other warps: G^T[j][r] = T_l E[r][j] + sum_l' V[l'][r] Wt_l[l'][j]
  if (warp == 0) {
    bool ok = CONV ? warp_lu<n>(Ss, invdS, lane) : warp_cholesky<n>(Ss, invdS, lane);
    if (!ok && lane == 0) s_bad = 1;
  } else {
    for (int t = tid - 32; t < n * m; t += NT - 32) {
      const int j = t / m, r = t - j * m, fl = r / d2, a = r - fl * d2;
      double g = s_T[fl] * __ldg(A.E + ((fl * 6 + s_perm[fl]) * d2 + a) * n + j);
      const double* wt = Wt + fl * n * n;
#pragma unroll 4
      for (int l = 0; l < n; ++l) g = fma(V[l * m + r], wt[l * n + j], g);
      if constexpr (CONV) {
        Gt[j * (m + 1) + r] = g - Hr[j * m + r];  // G_col^T = (G - alphaDP)^T
        Hr[j * m + r] = g;                       // G^T
      } else {
        Gt[j * (m + 1) + r] = j < A.nu ? g : 0.0;
      }
    }
  }
  __syncthreads();

  // [H | h] = L_s^-1 [G^T | f]  (convection: [H_col | h] = L^-1 [G_col^T | f] and H_row = U^-T G^T);
  // the back substitutions of the recovery are left to K2
  constexpr int NTRI = (m + 1) + (CONV ? m : 0);
  for (int t = tid; t < NTRI; t += NT) {
    double x[n];
    if (t < m + 1) {
#pragma unroll
      for (int l = 0; l < n; ++l) x[l] = Gt[l * (m + 1) + t];
      if constexpr (CONV) fwd_subst_unit<n>(Ss, x); else fwd_subst<n>(Ss, invdS, x);
#pragma unroll
      for (int l = 0; l < n; ++l) Gt[l * (m + 1) + t] = x[l];
    } else {
      const int col = t - (m + 1);
#pragma unroll
      for (int l = 0; l < n; ++l) x[l] = Hr[l * m + col];
      fwd_subst_Ut<n>(Ss, invdS, x);
#pragma unroll
      for (int l = 0; l < n; ++l) Hr[l * m + col] = x[l];
    }
  }
  __syncthreads();

  // C -= H^T H;  C_f = H^T h   (convection: C -= H_row^T H_col;  C_f = H_row^T h)
  if constexpr (CONV) {
    for (int t = tid; t < m * m; t += NT) {
      const int r = t / m, s = t - r * m;
      double hh = 0.0;
#pragma unroll 4
      for (int j = 0; j < n; ++j) hh = fma(Hr[j * m + r], Gt[j * (m + 1) + s], hh);
      Cs[t] -= hh;
    }
  } else {
    for (int t = tid; t < MP; t += NT) {
      const int r = A.pairs_m[2 * t], s = A.pairs_m[2 * t + 1];
      double hh = 0.0;
#pragma unroll 4
      for (int j = 0; j < n; ++j) hh = fma(Gt[j * (m + 1) + r], Gt[j * (m + 1) + s], hh);
      Cs[r * m + s] -= hh;
      if (r != s) Cs[s * m + r] -= hh;
    }
  }
  for (int r = tid; r < m; r += NT) {
    const double* hrow = CONV ? Hr : Gt;
    const int ld = CONV ? m : (m + 1);
    double s = 0.0;
#pragma unroll 4
    for (int j = 0; j < n; ++j) s = fma(hrow[j * ld + r], Gt[j * (m + 1) + m], s);
    A.Cf[Ke * m + r] = s;
  }
  __syncthreads();

  // C^K row-major, [K][r][s] with r = l d2 + a: the row block of local face l is contiguous
  // and each row is one unit-stride array, read by the trace operator with 16-byte loads
  double* Cout = A.C + Ke * (int64_t)(m * m);
  for (int t = tid; t < m * m; t += NT) Cout[t] = Cs[t];
  __syncthreads();

  // recovery record, column-major so that the recovery kernel reads it with unit stride:
  // [H | h]^T [m+1][n], V^T [m][n], W_*^T [3][n][n], U_s and U_M packed by columns (column i:
  // U_0i .. U_(i-1)i, then 1/U_ii; U_s = L_s^T, or the U of the LU with convection; U_M = L^T),
  // normals [4][3]
  double* R = A.rec + Ke * (int64_t)D::rec;
  for (int t = tid; t < n * (m + 1); t += NT) {
    const int r = t / n, i = t - r * n;
    R[t] = Gt[i * (m + 1) + r];
  }
  R += n * (m + 1);
  for (int t = tid; t < n * m; t += NT) {
    const int r = t / n, l = t - r * n;
    R[t] = V[l * m + r];
  }
  R += n * m;
  for (int t = tid; t < 3 * n * n; t += NT) {
    const int st = t / (n * n), rem = t - st * n * n, c = rem / n, l = rem - c * n;
    R[t] = W[st * n * n + l * n + c];
  }
  R += 3 * n * n;
  for (int t = tid; t < n * n; t += NT) {
    const int i = t / n, l = t - i * n;  // U_li, l <= i
    if (l <= i) {
      const double us = (l == i) ? invdS[i] : (CONV ? Ss[l * n + i] : Ss[i * n + l]);
      R[i * (i + 1) / 2 + l] = us;
      R[D::tri + i * (i + 1) / 2 + l] = (l == i) ? invdM[i] : Ms[i * n + l];
    }
  }
  R += 2 * D::tri;
  if (tid < 12) R[tid] = s_nrm[tid / 3][tid % 3];
  if (tid == 0) {
    if (s_bad) atomicAdd(A.status + 0, 1);
    if (s_coef) atomicAdd(A.status + 1, 1);
  }
}

template <int K, bool CONV, int NQ>
static cudaError_t launch_kq(hdg_mesh* M, const AsmArgs& a) {
  constexpr int NT = K1Occupancy<K>::NT;
  const size_t smem = AsmSmem<K, CONV, NQ>::bytes;
  cudaError_t e =
      cudaFuncSetAttribute(assemble_kernel<K, NT, CONV, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(assemble_kernel<K, NT, CONV, NQ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  assemble_kernel<K, NT, CONV, NQ><<<(unsigned)M->nelt, NT, smem, M->stream>>>(a);
  M->launches += 1;
  return cudaGetLastError();
}

// the conical rule's (k+2)^3 nodes, or the symmetric rule's C(k+5, 4)
template <int K, bool CONV>
static cudaError_t launch_k(hdg_mesh* M, const AsmArgs& a) {
  constexpr int NQS = (K + 2) * (K + 3) * (K + 4) * (K + 5) / 24;
  if (M->tab.nq == NQS) return launch_kq<K, CONV, NQS>(M, a);
  if (M->tab.nq == Dims<K>::nq) return launch_kq<K, CONV, Dims<K>::nq>(M, a);
  return cudaErrorInvalidValue;
}

cudaError_t launch_assemble(hdg_mesh* M) {
  M->rec_df = false;
  AsmArgs a;
  a.vx = M->d_vx;
  a.perm = M->d_perm;
  a.kappa = M->kappa;
  a.c = M->c;
  a.f = M->f;
  a.tau = M->tau;
  a.beta_q = M->beta_q;
  a.beta_f = M->beta_f;
  a.Pd = M->dt.Pd;
  a.Pl = M->dt.Pl;
  a.Dmu = M->dt.Dmu;
  a.wf = M->dt.face_w;
  a.P = M->dt.P;
  a.Chat = M->dt.Chat;
  a.S = M->dt.S;
  a.E = M->dt.E;
  a.w = M->dt.vol_w;
  a.pairs_n = M->dt.pairs_n;
  a.pairs_m = M->dt.pairs_m;
  a.C = M->d_C;
  a.Cf = M->d_Cf;
  a.rec = M->d_rec;
  a.nu = M->method == HDG_METHOD_BDM ? M->tab.n - M->tab.d2 : M->tab.n;
  a.status = M->d_status;
  a.nelt = M->nelt;
  const bool conv = M->beta_q != nullptr;
  switch (M->k) {
    case 0: return conv ? cudaErrorInvalidValue : launch_k<0, false>(M, a);
    case 1: return conv ? launch_k<1, true>(M, a) : launch_k<1, false>(M, a);
    case 2: return conv ? launch_k<2, true>(M, a) : launch_k<2, false>(M, a);
    case 3: return conv ? launch_k<3, true>(M, a) : launch_k<3, false>(M, a);
    case 4: return conv ? launch_k<4, true>(M, a) : launch_k<4, false>(M, a);
  }
  return cudaErrorInvalidValue;
}

int64_t rec_stride_of(int k) {
  switch (k) {
    case 0: return Dims<0>::rec;
    case 1: return Dims<1>::rec;
    case 2: return Dims<2>::rec;
    case 3: return Dims<3>::rec;
    case 4: return Dims<4>::rec;
  }
  return 0;
}

}  // namespace hdg
