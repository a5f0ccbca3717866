// Double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, carrying about
// 48 significant bits.  GB300 executes FP32 at 63x its FP64 rate, so FP64-accurate dense
// linear algebra runs faster as double-float than as native FP64.  Building blocks (all
// exact, using the hardware FMA):
//   two_sum      Knuth, TAOCP vol. 2, 4.2.2: s + e = a + b exactly
//   fast_two_sum Dekker 1971: the same when |a| >= |b|
//   two_prod     p + e = a * b exactly, e = fma(a, b, -p)
// The product follows the double-word product of Joldes, Muller and Popescu ("Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", ACM TOMS 2017,
// DWTimesDW1); dot products accumulate the exact leading products with two_sum and collect
// every low-order term in a second float, as in the compensated dot product of Ogita, Rump
// and Oishi (SIAM J. Sci. Comput. 2005), then renormalise once.  The reciprocal square root
// of a pivot takes a float seed and two Newton–Raphson steps; the few other reciprocals and
// roots are formed in FP64 from the double-float value.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hdg {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}

__device__ __forceinline__ df df_from_double(double d) {
  const float hi = __double2float_rn(d);
  return df_make(hi, __double2float_rn(d - (double)hi));
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df df_neg(df x) { return df_make(-x.hi, -x.lo); }

// x * y, relative error below 5 u^2 (u = 2^-24)
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x + y with two_sum on the leading parts (absolute error ~u^2 (|x| + |y|))
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// Unnormalised accumulator: hi collects the exact leading products by two_sum, lo every
// rounding error and low-order product term.
struct dacc {
  float hi, lo;
};

__device__ __forceinline__ dacc dacc_zero() {
  dacc a;
  a.hi = 0.f;
  a.lo = 0.f;
  return a;
}

__device__ __forceinline__ dacc dacc_from(df x) {
  dacc a;
  a.hi = x.hi;
  a.lo = x.lo;
  return a;
}

// acc += x * y
__device__ __forceinline__ void dacc_mac(dacc& acc, df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

// acc -= x * y
__device__ __forceinline__ void dacc_msub(dacc& acc, df x, df y) { dacc_mac(acc, df_neg(x), y); }

// acc += x
__device__ __forceinline__ void dacc_add(dacc& acc, df x) {
  const float s = __fadd_rn(acc.hi, x.hi);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(x.hi, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, x.lo));
}

__device__ __forceinline__ df dacc_result(const dacc& a) { return fast_two_sum(a.hi, a.lo); }

// 1/sqrt(a) for a > 0 in the normal float range, on the FP32 pipe: a float seed y0 (rsqrtf,
// a few ulp) refined by two Newton–Raphson steps for the inverse square root,
// y <- y + y (1 - a y^2) / 2, which square the relative error (~2^-22 -> ~2^-44 -> the
// ~2^-45 floor set by the double-float product a y^2).  1 - a y^2 is small, so after the exact
// leading subtraction (Sterbenz) it needs only float precision.
__device__ __forceinline__ df df_rsqrt(df a) {
  const float y0 = rsqrtf(a.hi);
  const float p = __fmul_rn(y0, y0);
  df t = df_mul(a, df_make(p, __fmaf_rn(y0, y0, -p)));  // a y0^2 (y0^2 exact as p + e)
  float r = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
  const df y = fast_two_sum(y0, __fmul_rn(__fmul_rn(y0, r), 0.5f));
  t = df_mul(a, df_mul(y, y));
  r = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
  return fast_two_sum(y.hi, __fadd_rn(y.lo, __fmul_rn(__fmul_rn(y.hi, r), 0.5f)));
}

// Cholesky (lower) of the N x N double-float matrix A by G threads (g = this thread's index
// among them): G = 32 is one warp (synchronised by __syncwarp), any other G is the whole
// block (__syncthreads).  Right-looking: at step j the pivot A_jj is final; every thread takes
// y = 1/sqrt(A_jj) by df_rsqrt (no FP64) and the trailing triangle is updated,
// A_ik -= A_ij A_kj y^2 for i >= k > j, its entries dealt round-robin to the G threads in
// chunks of CH whose loads are issued before any store (so they overlap).  The trailing
// entries of step j are the last (N-j-1)(N-j)/2 pairs (r <= c) of the row-major upper-triangle
// list `pairs`, read as one 32-bit word each.  Column j is scaled to L_ij = A_ij y at step
// j + 1, after the barrier that ends its readers, so each step takes one barrier.  Only the
// lower triangle is read or written; L_jj goes on the diagonal and 1/L_jj into invd.
// Returns, on every thread, whether all pivots were positive.
template <int N, int G>
__device__ __forceinline__ bool group_cholesky_df(df* A, df* invd, const int16_t* __restrict__ pairs, int g) {
  constexpr int NP = N * (N + 1) / 2, CH = 4;
  const int* __restrict__ pw = reinterpret_cast<const int*>(pairs);
  bool ok = true;
  df yp = df_make(1.f, 0.f), pp = df_make(1.f, 0.f);
  for (int j = 0; j < N; ++j) {
    if (j > 0) {
      for (int i = j + g; i < N; i += G) A[i * N + j - 1] = df_mul(A[i * N + j - 1], yp);
      if (g == 0) {
        A[(j - 1) * N + j - 1] = df_mul(pp, yp);
        invd[j - 1] = yp;
      }
    }
    const df piv = A[j * N + j];
    ok = ok && (piv.hi > 0.f);
    const df y = df_rsqrt(piv.hi > 0.f ? piv : df_make(1.f, 0.f));
    const df y2 = df_mul(y, y);
    for (int t0 = NP - (N - j - 1) * (N - j) / 2 + g; t0 < NP; t0 += CH * G) {
      int at[CH];
      df a[CH], lc[CH], lr[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int t = t0 + u * G;
        if (t < NP) {
          const int w = __ldg(pw + t);
          const int r = w & 0xffff, c = w >> 16;  // r <= c: the lower-triangle entry (c, r)
          at[u] = c * N + r;
          a[u] = A[c * N + r];
          lc[u] = A[c * N + j];
          lr[u] = A[r * N + j];
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (t0 + u * G < NP) {
          dacc s = dacc_from(a[u]);
          dacc_msub(s, lc[u], df_mul(lr[u], y2));
          a[u] = dacc_result(s);
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u)
        if (t0 + u * G < NP) A[at[u]] = a[u];
    }
    if (G == 32) __syncwarp();
    else __syncthreads();
    yp = y;
    pp = piv;
  }
  if (g == 0) {
    A[(N - 1) * N + N - 1] = df_mul(pp, yp);
    invd[N - 1] = yp;
  }
  return ok;
}

// 1/a for a non-zero a in the normal float range, on the FP32 pipe: the correctly rounded
// float reciprocal of a.hi as the seed y0, refined by one Newton-Raphson step
// y = y0 + y0 (1 - a y0), which squares its relative error (2^-24 -> the ~2^-45 floor of the
// double-float product).  1 - a y0 is tiny, so its leading subtraction is exact (Sterbenz).
__device__ __forceinline__ df df_recip(df a) {
  const float y0 = __frcp_rn(a.hi);
  const df t = df_mul(a, df_make(y0, 0.f));
  const float r = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
  return fast_two_sum(y0, __fmul_rn(y0, r));
}

}  // namespace hdg
