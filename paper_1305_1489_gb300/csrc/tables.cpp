// Reference-element tables of the HDG method (host, built once per degree k).
//
// Quadrature (eq. 3.1 and Section 4 "Integrals on faces"; the paper leaves the rule open):
// conical-product Gauss-Jacobi rules with n = k+2 points per collapsed direction, exact to
// total degree 2k+3.  The 1-D Gauss-Jacobi rules come from the symmetric tridiagonal Jacobi
// matrix of the monic recurrence (Golub-Welsch): its eigenvalues, found by Sturm-sequence
// bisection in long double, are the nodes; the weights are mu_0 / sum_j p_j(x)^2 with p_j
// the orthonormal polynomials (Christoffel numbers).
//
// The smaller symmetric volume rule (rule 1, the paper's remark that such rules can be found in
// the literature): Grundmann-Moller of index s = k + 1 (SIAM J. Numer. Anal. 15, 1978), exact to
// the same degree 2s + 1 = 2k + 3 with C(s + 4, 4) nodes: level i = 0..s has the nodes with
// barycentric coordinates (2 b_j + 1) / (d + 3 - 2i), b in N^4, |b| = s - i, d = 2s + 1, all of
// weight (-1)^i 2^-2s (d + 3 - 2i)^d / (i! (d + 3 - i)!) on the simplex of volume 1/6 (times 6
// here, so that the weights sum to one).  Some weights are negative.  Formed in long double.
//
// Bases (eq. 3.3 and Section 4 "Bases, faces, and boundaries"): Dubiner bases in collapsed
// coordinates, orthonormal (int_{K_hat} P_i P_j = delta_ij / 6, int_{K_hat_2} D_i D_j =
// delta_ij / 2), ordered by degree then (p, q[, r]).  Gradients are taken analytically
// through the collapsed coordinates using d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1).
#include <cmath>
#include <cstring>
#include <utility>

#include "hdg_internal.h"

namespace hdg {

int d3_of(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }
int d2_of(int k) { return (k + 1) * (k + 2) / 2; }

namespace {

typedef long double LD;

// Monic Jacobi recurrence on [-1,1] for the weight (1-x)^a (1+x)^b.
void jacobi_recurrence(int N, LD a, LD b, std::vector<LD>* alpha, std::vector<LD>* beta) {
  alpha->assign(N, 0);
  beta->assign(N, 0);
  for (int j = 0; j < N; ++j) {
    LD s = 2 * j + a + b;
    (*alpha)[j] = (j == 0) ? (b - a) / (a + b + 2) : (b * b - a * a) / (s * (s + 2));
    if (j >= 1)
      (*beta)[j] = 4 * j * (j + a) * (j + b) * (j + a + b) / (s * s * (s + 1) * (s - 1));
  }
}

// Number of eigenvalues of the Jacobi matrix smaller than x (Sturm sequence).
int sturm_count(const std::vector<LD>& al, const std::vector<LD>& be, LD x) {
  int cnt = 0;
  LD d = 1;
  for (size_t i = 0; i < al.size(); ++i) {
    d = (al[i] - x) - (i ? be[i] / d : 0);
    if (d == 0) d = 1e-300L;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// n-point Gauss rule on [0,1] for the weight (1-t)^a.
void gauss_jacobi01(int n, double a, std::vector<double>* t, std::vector<double>* w) {
  std::vector<LD> al, be;
  jacobi_recurrence(n, a, 0, &al, &be);
  LD mu0 = std::pow((LD)2, (LD)(a + 1)) / (a + 1);
  t->resize(n);
  w->resize(n);
  for (int i = 0; i < n; ++i) {
    LD lo = -1, hi = 1;  // the i-th smallest eigenvalue
    for (int it = 0; it < 200; ++it) {
      LD mid = (lo + hi) / 2;
      if (sturm_count(al, be, mid) > i) hi = mid; else lo = mid;
    }
    LD x = (lo + hi) / 2;
    LD p0 = 1, p1 = 0, s = 1;  // orthonormal (up to p_0 = 1) polynomials at x
    LD pm = 0;
    for (int j = 0; j + 1 < n; ++j) {
      p1 = ((x - al[j]) * p0 - (j ? std::sqrt(be[j]) * pm : 0)) / std::sqrt(be[j + 1]);
      pm = p0;
      p0 = p1;
      s += p1 * p1;
    }
    LD wi = mu0 / s;
    (*t)[i] = (double)((x + 1) / 2);
    (*w)[i] = (double)(wi / std::pow((LD)2, (LD)(a + 1)));
  }
}

// Jacobi polynomial P_n^(a,b)(x) by the three-term recurrence.
double jacobi(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2) * x + (a - b));
  for (int j = 2; j <= n; ++j) {
    double s = 2 * j + a + b;
    double c1 = 2 * j * (j + a + b) * (s - 2);
    double c2 = (s - 1) * (s * (s - 2) * x + a * a - b * b);
    double c3 = 2 * (j + a - 1) * (j + b - 1) * s;
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

double djacobi(int n, double a, double b, double x) {
  return n == 0 ? 0.0 : 0.5 * (n + a + b + 1) * jacobi(n - 1, a + 1, b + 1, x);
}

struct Idx3 { int p, q, r; };
std::vector<Idx3> index3(int k) {
  std::vector<Idx3> v;
  for (int d = 0; d <= k; ++d)
    for (int p = 0; p <= d; ++p)
      for (int q = 0; q <= d - p; ++q) v.push_back({p, q, d - p - q});
  return v;
}

// 3-D Dubiner function (p,q,r) and its gradient at (x,y,z) in K_hat (interior points).
void dubiner3(int p, int q, int r, double x, double y, double z, double* val, double* g) {
  double w = 1 - y - z, v = 1 - z;
  double a = 2 * x / w - 1, b = 2 * y / v - 1, c = 2 * z - 1;
  double nrm = std::sqrt((2 * p + 1) * (p + q + 1) * (2.0 * p + 2 * q + 2 * r + 3) / 3.0);
  double Pa = jacobi(p, 0, 0, a), dPa = djacobi(p, 0, 0, a);
  double Pb = jacobi(q, 2 * p + 1, 0, b), dPb = djacobi(q, 2 * p + 1, 0, b);
  double Pc = jacobi(r, 2 * p + 2 * q + 2, 0, c), dPc = djacobi(r, 2 * p + 2 * q + 2, 0, c);
  double wp = std::pow(w, p), vq = std::pow(v, q);
  double A = wp * Pa, Bq = vq * Pb, Cr = Pc;
  // dA/dx = 2 w^(p-1) P'(a);  dA/dy = dA/dz = w^(p-1) (-p P(a) + (a+1) P'(a))
  double wpm = p ? std::pow(w, p - 1) : 0.0;
  double Ax = 2 * wpm * dPa, Ay = p ? wpm * (-p * Pa + (a + 1) * dPa) : 0.0;
  double vqm = q ? std::pow(v, q - 1) : 0.0;
  double By = 2 * vqm * dPb, Bz = q ? vqm * (-q * Pb + (b + 1) * dPb) : 0.0;
  double Cz = 2 * dPc;
  *val = nrm * A * Bq * Cr;
  if (g) {
    g[0] = nrm * Ax * Bq * Cr;
    g[1] = nrm * (Ay * Bq * Cr + A * By * Cr);
    g[2] = nrm * (Ay * Bq * Cr + A * Bz * Cr + A * Bq * Cz);
  }
}

// 2-D Dubiner function (p,q) at (s,t) in K_hat_2.
double dubiner2(int p, int q, double s, double t) {
  double v = 1 - t;
  double a = 2 * s / v - 1, b = 2 * t - 1;
  double nrm = std::sqrt((2.0 * p + 1) * (p + q + 1));
  return nrm * jacobi(p, 0, 0, a) * std::pow(v, p) * jacobi(q, 2 * p + 1, 0, b);
}

// F_mu of eq. 2.2
void F_mu(int mu, double s, double t, double* so, double* to) {
  double r = 1 - s - t;
  switch (mu) {
    case 1: *so = s; *to = t; break;
    case 2: *so = t; *to = s; break;
    case 3: *so = t; *to = r; break;
    case 4: *so = s; *to = r; break;
    case 5: *so = r; *to = s; break;
    default: *so = r; *to = t; break;
  }
}

}  // namespace

int symmetric_rule_nodes(int k) {
  const int s = k + 1;
  return (s + 1) * (s + 2) * (s + 3) * (s + 4) / 24;  // C(s + 4, 4)
}

namespace {
// Grundmann-Moller nodes (x, y, z) = barycentrics 1..3 and weights (sum one), see the header
void symmetric_volume_rule(int k, std::vector<double>* pts, std::vector<double>* w) {
  const int s = k + 1, d = 2 * s + 1;
  pts->clear();
  w->clear();
  for (int i = 0; i <= s; ++i) {
    LD fi = 1, fdi = 1;
    for (int j = 2; j <= i; ++j) fi *= j;
    for (int j = 2; j <= d + 3 - i; ++j) fdi *= j;
    const LD den = (LD)(d + 3 - 2 * i);
    LD wt = std::pow(den, (LD)d) / (fi * fdi) / std::pow((LD)2, (LD)(2 * s));
    if (i & 1) wt = -wt;
    const int mlev = s - i;
    for (int b0 = 0; b0 <= mlev; ++b0)
      for (int b1 = 0; b1 <= mlev - b0; ++b1)
        for (int b2 = 0; b2 <= mlev - b0 - b1; ++b2) {
          const int b3 = mlev - b0 - b1 - b2;
          pts->push_back((double)((2 * b1 + 1) / den));
          pts->push_back((double)((2 * b2 + 1) / den));
          pts->push_back((double)((2 * b3 + 1) / den));
          w->push_back((double)(6 * wt));
        }
  }
}
}  // namespace

bool build_tables(int k, Tables* T, std::string* err, int rule) {
  if (k < 0 || k > 4) {
    *err = "degree k must be in 0..4";
    return false;
  }
  if (rule != 0 && rule != 1) {
    *err = "unknown volume rule";
    return false;
  }
  const int nn = k + 2;
  T->k = k;
  T->rule = rule;
  T->n = d3_of(k);
  T->d2 = d2_of(k);
  T->m = 4 * T->d2;
  T->nq = rule == 1 ? symmetric_rule_nodes(k) : nn * nn * nn;
  T->nf = nn * nn;
  T->n1 = d3_of(k + 1);
  const int n = T->n, d2 = T->d2, nq = T->nq, nf = T->nf, n1 = T->n1;

  // volume rule: z = t1 (weight (1-t)^2), y = t2 (1-t1) (weight (1-t)), x = t3 (1-t1)(1-t2)
  std::vector<double> t1, w1, t2, w2, t3, w3;
  gauss_jacobi01(nn, 2.0, &t1, &w1);
  gauss_jacobi01(nn, 1.0, &t2, &w2);
  gauss_jacobi01(nn, 0.0, &t3, &w3);
  T->vol_pts.resize(nq * 3);
  T->vol_w.resize(nq);
  T->lam.resize(nq * 4);
  double wsum = 0;
  if (rule == 1) {
    std::vector<double> sp, sw;
    symmetric_volume_rule(k, &sp, &sw);
    for (int q = 0; q < nq; ++q) {
      const double x = sp[3 * q], y = sp[3 * q + 1], z = sp[3 * q + 2];
      T->vol_pts[3 * q] = x;
      T->vol_pts[3 * q + 1] = y;
      T->vol_pts[3 * q + 2] = z;
      T->vol_w[q] = sw[q];
      wsum += sw[q];
      T->lam[4 * q] = 1 - x - y - z;
      T->lam[4 * q + 1] = x;
      T->lam[4 * q + 2] = y;
      T->lam[4 * q + 3] = z;
    }
  }
  for (int i = 0; i < (rule == 1 ? 0 : nn); ++i)
    for (int j = 0; j < nn; ++j)
      for (int l = 0; l < nn; ++l) {
        int q = (i * nn + j) * nn + l;
        double z = t1[i], y = t2[j] * (1 - t1[i]), x = t3[l] * (1 - t1[i]) * (1 - t2[j]);
        T->vol_pts[3 * q] = x;
        T->vol_pts[3 * q + 1] = y;
        T->vol_pts[3 * q + 2] = z;
        T->vol_w[q] = 6.0 * w1[i] * w2[j] * w3[l];
        wsum += T->vol_w[q];
        T->lam[4 * q] = 1 - x - y - z;
        T->lam[4 * q + 1] = x;
        T->lam[4 * q + 2] = y;
        T->lam[4 * q + 3] = z;
      }
  if (std::fabs(wsum - 1.0) > 1e-13) {
    *err = "volume quadrature weights do not sum to one";
    return false;
  }

  // face rule: t = u1 (weight (1-u)), s = u2 (1 - u1)
  std::vector<double> u1, v1, u2, v2;
  gauss_jacobi01(nn, 1.0, &u1, &v1);
  gauss_jacobi01(nn, 0.0, &u2, &v2);
  T->face_pts.resize(nf * 2);
  T->face_w.resize(nf);
  T->xi.resize(nf * 3);
  for (int i = 0; i < nn; ++i)
    for (int j = 0; j < nn; ++j) {
      int r = i * nn + j;
      double t = u1[i], s = u2[j] * (1 - u1[i]);
      T->face_pts[2 * r] = s;
      T->face_pts[2 * r + 1] = t;
      T->face_w[r] = 2.0 * v1[i] * v2[j];
      T->xi[3 * r] = 1 - s - t;
      T->xi[3 * r + 1] = s;
      T->xi[3 * r + 2] = t;
    }

  // volume basis tables
  auto idx = index3(k);
  auto idx1 = index3(k + 1);
  T->P.assign(nq * n, 0);
  T->Pd.assign(3 * nq * n, 0);
  T->P1.assign(nq * n1, 0);
  T->G1.assign(3 * nq * n1, 0);
  for (int q = 0; q < nq; ++q) {
    const double* p = &T->vol_pts[3 * q];
    for (int j = 0; j < n1; ++j) {
      double v, g[3];
      dubiner3(idx1[j].p, idx1[j].q, idx1[j].r, p[0], p[1], p[2], &v, g);
      T->P1[q * n1 + j] = v;
      for (int d = 0; d < 3; ++d) T->G1[(d * nq + q) * n1 + j] = g[d];
      if (j < n) {
        T->P[q * n + j] = v;
        for (int d = 0; d < 3; ++d) T->Pd[(d * nq + q) * n + j] = g[d];
      }
    }
  }
  // eq. 3.7: C_hat^* = (1/6) (omega . P)^T P^*
  T->Chat.assign(3 * n * n, 0);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int q = 0; q < nq; ++q) s += T->vol_w[q] * T->P[q * n + i] * T->Pd[(d * nq + q) * n + j];
        T->Chat[(d * n + i) * n + j] = s / 6.0;
      }
  // stiffness pieces of the degree-(k+1) basis
  const int pr[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  T->Shat1.assign(6 * n1 * n1, 0);
  for (int c = 0; c < 6; ++c)
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) {
        double s = 0;
        for (int q = 0; q < nq; ++q)
          s += T->vol_w[q] * T->G1[(pr[c][0] * nq + q) * n1 + i] * T->G1[(pr[c][1] * nq + q) * n1 + j];
        T->Shat1[(c * n1 + i) * n1 + j] = s / 6.0;
      }

  // face tables: P^l (eq. 4.4), D (eq. 4.7), D^mu
  T->Pl.assign(4 * nf * n, 0);
  T->D.assign(nf * d2, 0);
  T->Dmu.assign(6 * nf * d2, 0);
  for (int r = 0; r < nf; ++r) {
    double s = T->face_pts[2 * r], t = T->face_pts[2 * r + 1];
    double pts[4][3] = {{s, t, 0}, {s, 0, t}, {0, s, t}, {s, t, 1 - s - t}};
    for (int l = 0; l < 4; ++l)
      for (int j = 0; j < n; ++j) {
        double v;
        dubiner3(idx[j].p, idx[j].q, idx[j].r, pts[l][0], pts[l][1], pts[l][2], &v, nullptr);
        T->Pl[(l * nf + r) * n + j] = v;
      }
    int col = 0;
    for (int d = 0; d <= k; ++d)
      for (int p = 0; p <= d; ++p, ++col) {
        int qq = d - p;
        T->D[r * d2 + col] = dubiner2(p, qq, s, t);
        for (int mu = 1; mu <= 6; ++mu) {
          double so, to;
          F_mu(mu, s, t, &so, &to);
          T->Dmu[((mu - 1) * nf + r) * d2 + col] = dubiner2(p, qq, so, to);
        }
      }
  }
  // eq. 4.5 pieces and eq. 4.10 pieces
  T->S.assign(4 * n * n, 0);
  T->E.assign(4 * 6 * d2 * n, 0);
  for (int l = 0; l < 4; ++l) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int r = 0; r < nf; ++r)
          s += T->face_w[r] * T->Pl[(l * nf + r) * n + i] * T->Pl[(l * nf + r) * n + j];
        T->S[(l * n + i) * n + j] = s;
      }
    for (int mu = 0; mu < 6; ++mu)
      for (int a = 0; a < d2; ++a)
        for (int j = 0; j < n; ++j) {
          double s = 0;
          for (int r = 0; r < nf; ++r)
            s += T->face_w[r] * T->Dmu[(mu * nf + r) * d2 + a] * T->Pl[(l * nf + r) * n + j];
          T->E[((l * 6 + mu) * d2 + a) * n + j] = s;
        }
  }

  // Sum-factorisation tables.  At the node z = t1_i, y = t2_j (1 - t1_i),
  // x = t3_l (1 - t1_i)(1 - t2_j) the collapsed coordinates are a = 2 t3_l - 1, b = 2 t2_j - 1,
  // c = 2 t1_i - 1, and the Dubiner function (p, q, r) is nrm A_p(l) B_pq(j) C'_pqr(i) with
  //   A_p = P_p^(0,0)(a),  B_pq = (1 - t2)^p P_q^(2p+1,0)(b),  C'_pqr = (1 - t1)^(p+q) P_r^(2p+2q+2,0)(c)
  // (the normalisation nrm goes into C).  The conical rule only: the symmetric rule has no
  // tensor structure (the assembly that needs these tables refuses it).
  if (rule == 0) {
    std::vector<double> A((k + 1) * nn), B, C(n * nn);
    std::vector<std::pair<int, int>> idx2;
    for (int p = 0; p <= k; ++p)
      for (int q = 0; q + p <= k; ++q) idx2.push_back({p, q});
    B.resize(idx2.size() * nn);
    for (int p = 0; p <= k; ++p)
      for (int l = 0; l < nn; ++l) A[p * nn + l] = jacobi(p, 0, 0, 2 * t3[l] - 1);
    for (size_t a2 = 0; a2 < idx2.size(); ++a2) {
      const int p = idx2[a2].first, q = idx2[a2].second;
      for (int j = 0; j < nn; ++j) B[a2 * nn + j] = std::pow(1 - t2[j], p) * jacobi(q, 2 * p + 1, 0, 2 * t2[j] - 1);
    }
    std::vector<int> id2(n);
    for (int a = 0; a < n; ++a) {
      const int p = idx[a].p, q = idx[a].q, r = idx[a].r;
      for (size_t a2 = 0; a2 < idx2.size(); ++a2)
        if (idx2[a2].first == p && idx2[a2].second == q) id2[a] = (int)a2;
      const double nrm = std::sqrt((2 * p + 1) * (p + q + 1) * (2.0 * p + 2 * q + 2 * r + 3) / 3.0);
      for (int i = 0; i < nn; ++i)
        C[a * nn + i] = nrm * std::pow(1 - t1[i], p + q) * jacobi(r, 2 * p + 2 * q + 2, 0, 2 * t1[i] - 1);
    }
    // the factors must reproduce the basis table
    for (int i = 0; i < nn; ++i)
      for (int j = 0; j < nn; ++j)
        for (int l = 0; l < nn; ++l)
          for (int a = 0; a < n; ++a) {
            const double v = A[idx[a].p * nn + l] * B[id2[a] * nn + j] * C[a * nn + i];
            const double ref = T->P[((i * nn + j) * nn + l) * n + a];
            if (std::fabs(v - ref) > 1e-11 * (1.0 + std::fabs(ref))) {
              *err = "sum-factorisation tables do not reproduce the volume basis";
              return false;
            }
          }
    std::vector<int> p1of(( k + 1) * (k + 1));
    T->sfAA.clear();
    int np1 = 0;
    for (int pa = 0; pa <= k; ++pa)
      for (int pb = pa; pb <= k; ++pb) {
        p1of[pa * (k + 1) + pb] = p1of[pb * (k + 1) + pa] = np1++;
        for (int l = 0; l < nn; ++l) T->sfAA.push_back(A[pa * nn + l] * A[pb * nn + l]);
      }
    const int nd2 = (int)idx2.size();
    std::vector<int> p2of(nd2 * nd2);
    T->sfBB.clear();
    T->sfp2to1.clear();
    int np2 = 0;
    for (int a2 = 0; a2 < nd2; ++a2)
      for (int b2 = a2; b2 < nd2; ++b2) {
        p2of[a2 * nd2 + b2] = p2of[b2 * nd2 + a2] = np2++;
        T->sfp2to1.push_back((int16_t)p1of[idx2[a2].first * (k + 1) + idx2[b2].first]);
        for (int j = 0; j < nn; ++j) T->sfBB.push_back(B[a2 * nn + j] * B[b2 * nn + j]);
      }
    T->sfCC.clear();
    T->sfp3to2.clear();
    for (int a = 0; a < n; ++a)
      for (int b = a; b < n; ++b) {
        T->sfp3to2.push_back((int16_t)p2of[id2[a] * nd2 + id2[b]]);
        for (int i = 0; i < nn; ++i) T->sfCC.push_back(C[a * nn + i] * C[b * nn + i]);
      }
    T->np1 = np1;
    T->np2 = np2;
  }
  return true;
}

}  // namespace hdg
