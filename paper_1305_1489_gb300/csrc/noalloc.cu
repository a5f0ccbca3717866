// hdg_solve_trace_noalloc: the block-Jacobi PCG trace solve of hdg_solve_trace with every
// scratch buffer (right-hand side, boundary data, block inverses, Krylov vectors, reduction
// partials, scalars) carved out of one file-scope static device array instead of memory the
// library allocates.  It exists for callers that must not allocate device memory at solve
// time: code running under a memory budget fixed in advance (an application that reserves
// all device memory up front, or a pool-managed framework that forbids new allocations after
// warm-up), and latency-sensitive loops where cudaMalloc/cudaFree would synchronise the
// device.  FP64 throughout; the same operator and stopping rule as hdg_solve_trace.
//
// Limits and sharing:
//  * at most 65,536 trace unknowns (nfc * d2); larger meshes are rejected with HDG_ERR_ARG.
//    The array (1,519,276 doubles, 11.6 MiB, plus a 16-byte counter) takes that much memory
//    on every GPU that loads the library, until the process exits.
//  * every call on a device uses the same array and leaves its contents behind; the call
//    clears what has to start at zero (the reduction counter).  Calls whose work overlaps on
//    the GPU (two streams, or two host threads) race on the array and give wrong results.
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call before any stream
//    capture.  No graph is used and nothing is allocated.
#include <cmath>
#include <mutex>

#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {
namespace noalloc {

constexpr int64_t kMaxDofs = 65536;  // trace unknowns nfc * d2
constexpr int kMaxD2 = 15;
constexpr int kNT = 128;
constexpr int kIterChunk = 16;       // iterations launched between host convergence checks
constexpr int64_t kMaxFaces = kMaxDofs / 3;     // d2 >= 3 for k >= 1
constexpr int64_t kMaxBlocks = kMaxFaces / 8 + 1;  // face kernels hold kNT / d2 >= 8 faces per block
// doubles: 8 vectors + block inverses (nfc d2^2 <= kMaxDofs kMaxD2) + reduction partials
// (4 slots) + scalars + alignment padding of the 12 pieces
constexpr int64_t kScratchDoubles = 8 * kMaxDofs + kMaxDofs * kMaxD2 + 4 * kMaxBlocks + 1024;
static_assert(kScratchDoubles * 8 <= 12 * 1024 * 1024 + 128 * 1024, "scratch larger than the stated 12 MiB");

__device__ __align__(256) double g_scratch[kScratchDoubles];
__device__ __align__(256) unsigned int g_counter[4];

enum { S_RZ = 0, S_ALPHA, S_BETA, S_RR, S_BB, S_DONE, S_ITERS, S_TOL2, S_MAXIT, S_BAD, S_NSCAL };

struct Ops {
  const double* C;
  const int32_t* owner;
  const int32_t* fbe;
  const int32_t* ftype;
  int64_t nfc;
  int d2, m;
};

__device__ __forceinline__ bool slot(const Ops& F, int64_t& e, int& a, int64_t& t) {
  const int fpb = kNT / F.d2;
  const int loc = threadIdx.x / F.d2;
  a = threadIdx.x - loc * F.d2;
  e = (int64_t)blockIdx.x * fpb + loc;
  t = e * F.d2 + a;
  return loc < fpb && e < F.nfc;
}

// deterministic last-block reduction of NS values; true on the finishing block
template <int NS>
__device__ bool reduce(const double (&v)[NS], double* red, unsigned int* counter, double (&out)[NS]) {
  __shared__ double ws[NS][kNT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nb = gridDim.x;
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) ws[s][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      double x = 0.0;
      for (int i = 0; i < kNT / 32; ++i) x += ws[s][i];
      red[s * nb + blockIdx.x] = x;
    }
    __threadfence();
    last = (atomicAdd(counter, 1u) == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    for (int i = threadIdx.x; i < nb; i += kNT) x += ((volatile double*)red)[s * nb + i];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) ws[s][w] = x;
  }
  __syncthreads();
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    for (int i = 0; i < kNT / 32; ++i) x += ws[s][i];
    out[s] = x;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ double apply(const Ops& F, const double* __restrict__ x, int64_t e, int a) {
  double acc = 0.0;
  for (int o = 0; o < 2; ++o) {
    const int ow = F.owner[2 * e + o];
    if (ow < 0) continue;
    const int64_t K = ow >> 2;
    // row-major C^K: row (l d2 + a)
    const double* Ck = F.C + K * (int64_t)(F.m * F.m) + (int64_t)((ow & 3) * F.d2 + a) * F.m;
    for (int fl = 0; fl < 4; ++fl) {
      const double* xs = x + (int64_t)F.fbe[4 * K + fl] * F.d2;
      const double* cc = Ck + fl * F.d2;
      for (int b = 0; b < F.d2; ++b) acc = fma(cc[b], xs[b], acc);
    }
  }
  return acc;
}

__global__ void k_bdata(Ops F, const double* __restrict__ fvx, const double* __restrict__ vx, int64_t nelt,
                        const double* __restrict__ D, const double* __restrict__ wf, int nf,
                        const double* __restrict__ uD, const double* __restrict__ gN, double* xD, double* phiN) {
  int64_t e, t;
  int a;
  if (!slot(F, e, a, t)) return;
  const int ty = F.ftype[e];
  double xd = 0.0, ph = 0.0;
  if (ty == 1 && uD) {
    for (int r = 0; r < nf; ++r) xd = fma(wf[r] * D[r * F.d2 + a], uD[e * nf + r], xd);
  } else if (ty == 2 && gN) {
    double w[3][3], u1[3], u2[3], nv[3];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) w[i][d] = fvx[(d * 3 + i) * F.nfc + e];
    for (int d = 0; d < 3; ++d) {
      u1[d] = w[1][d] - w[0][d];
      u2[d] = w[2][d] - w[0][d];
    }
    cross3(u1, u2, nv);
    const int ow = F.owner[2 * e];
    const int64_t K = ow >> 2;
    const int opp[4] = {3, 2, 1, 0};
    double dot = 0.0;
    for (int d = 0; d < 3; ++d) dot += nv[d] * (vx[(d * 4 + opp[ow & 3]) * nelt + K] - w[0][d]);
    const double sg = dot > 0 ? -0.5 : 0.5;
    for (int s = 0; s < 3; ++s) {
      double acc = 0.0;
      for (int r = 0; r < nf; ++r) acc = fma(wf[r] * D[r * F.d2 + a], gN[((int64_t)s * F.nfc + e) * nf + r], acc);
      ph = fma(sg * nv[s], acc, ph);
    }
  }
  xD[t] = xd;
  phiN[t] = ph;
}

__global__ void k_rhs(Ops F, const double* __restrict__ Cf, const double* __restrict__ xD,
                      const double* __restrict__ phiN, double* b, double* red, unsigned int* counter, double* scal) {
  int64_t e, t;
  int a;
  double v = 0.0;
  if (slot(F, e, a, t)) {
    if (F.ftype[e] != 1) {
      double fs = 0.0;
      for (int o = 0; o < 2; ++o) {
        const int ow = F.owner[2 * e + o];
        if (ow >= 0) fs += Cf[(int64_t)(ow >> 2) * F.m + (ow & 3) * F.d2 + a];
      }
      v = fs + phiN[t] - apply(F, xD, e, a);
    }
    b[t] = v;
  }
  double in[1] = {v * v}, out[1];
  if (reduce<1>(in, red, counter, out) && threadIdx.x == 0) scal[S_BB] = out[0];
}

// block-Jacobi inverse of each free face's diagonal block, one thread per face
__global__ void k_bj(Ops F, double* Binv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= F.nfc) return;
  const int d2 = F.d2, m = F.m;
  double A[kMaxD2 * kMaxD2], X[kMaxD2 * kMaxD2];
  if (F.ftype[e] == 1) {
    for (int i = 0; i < d2 * d2; ++i) Binv[e * d2 * d2 + i] = 0.0;
    return;
  }
  for (int i = 0; i < d2 * d2; ++i) A[i] = 0.0;
  for (int o = 0; o < 2; ++o) {
    const int ow = F.owner[2 * e + o];
    if (ow < 0) continue;
    const int l = ow & 3;
    // C^K[l d2 + i][l d2 + j], row-major
    const double* Cb = F.C + (int64_t)(ow >> 2) * m * m + (int64_t)(l * d2) * m + l * d2;
    for (int i = 0; i < d2; ++i)
      for (int j = 0; j < d2; ++j) A[i * d2 + j] += Cb[i * m + j];
  }
  for (int j = 0; j < d2; ++j) {
    double s = A[j * d2 + j];
    for (int l = 0; l < j; ++l) s -= A[j * d2 + l] * A[j * d2 + l];
    const double d = sqrt(s);
    A[j * d2 + j] = d;
    for (int i = j + 1; i < d2; ++i) {
      double t = A[i * d2 + j];
      for (int l = 0; l < j; ++l) t -= A[i * d2 + l] * A[j * d2 + l];
      A[i * d2 + j] = t / d;
    }
  }
  for (int c = 0; c < d2; ++c) {
    for (int i = 0; i < d2; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = 0; l < i; ++l) s -= A[i * d2 + l] * X[l * d2 + c];
      X[i * d2 + c] = s / A[i * d2 + i];
    }
    for (int i = d2 - 1; i >= 0; --i) {
      double s = X[i * d2 + c];
      for (int l = i + 1; l < d2; ++l) s -= A[l * d2 + i] * X[l * d2 + c];
      X[i * d2 + c] = s / A[i * d2 + i];
    }
  }
  for (int i = 0; i < d2 * d2; ++i) Binv[e * d2 * d2 + i] = X[i];
}

__device__ __forceinline__ double bj(const Ops& F, const double* Binv, const double* r, int64_t e, int a) {
  double s = 0.0;
  const double* Bi = Binv + (e * F.d2 + a) * F.d2;
  for (int b = 0; b < F.d2; ++b) s = fma(Bi[b], r[e * F.d2 + b], s);
  return s;
}

// r = b - H x (or b with x = 0), then r.r
__global__ void k_init(Ops F, const double* __restrict__ b, double* x, bool have_x, double* r, double* red,
                       unsigned int* counter, double* scal) {
  int64_t e, t;
  int a;
  double v[1] = {0.0};
  if (slot(F, e, a, t)) {
    double rv = 0.0;
    if (F.ftype[e] != 1) rv = b[t] - (have_x ? apply(F, x, e, a) : 0.0);
    if (!have_x) x[t] = 0.0;
    r[t] = rv;
    v[0] = rv * rv;
  }
  double out[1];
  if (reduce<1>(v, red, counter, out) && threadIdx.x == 0) scal[S_RR] = out[0];
}

__global__ void k_precond(Ops F, const double* Binv, const double* r, double* z, double* p, double* red,
                          unsigned int* counter, double* scal) {
  int64_t e, t;
  int a;
  double v[1] = {0.0};
  if (slot(F, e, a, t)) {
    const double zv = bj(F, Binv, r, e, a);
    z[t] = zv;
    p[t] = zv;
    v[0] = r[t] * zv;
  }
  double out[1];
  if (reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[S_RZ] = out[0];
    scal[S_DONE] = (scal[S_RR] <= scal[S_TOL2]) ? 1.0 : 0.0;
    scal[S_ITERS] = 0.0;
  }
}

__global__ void k_matvec(Ops F, const double* p, double* q, double* red, unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  int64_t e, t;
  int a;
  double v[1] = {0.0};
  if (slot(F, e, a, t)) {
    const double qv = (F.ftype[e] != 1) ? apply(F, p, e, a) : 0.0;
    q[t] = qv;
    v[0] = p[t] * qv;
  }
  double out[1];
  if (reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    if (!(out[0] > 0.0)) {
      scal[S_BAD] = 1.0;
      scal[S_DONE] = 1.0;
      scal[S_ALPHA] = 0.0;
    } else {
      scal[S_ALPHA] = scal[S_RZ] / out[0];
    }
  }
}

__global__ void k_update(Ops F, const double* Binv, double* x, double* r, double* z, const double* p,
                         const double* q, double* red, unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  const double alpha = scal[S_ALPHA];
  int64_t e, t;
  int a;
  const bool act = slot(F, e, a, t);
  if (act) {
    x[t] += alpha * p[t];
    r[t] -= alpha * q[t];
  }
  __syncthreads();
  double v[2] = {0.0, 0.0};
  if (act) {
    const double zv = bj(F, Binv, r, e, a);
    z[t] = zv;
    v[0] = r[t] * zv;
    v[1] = r[t] * r[t];
  }
  double out[2];
  if (reduce<2>(v, red, counter, out) && threadIdx.x == 0) {
    const double rz_old = scal[S_RZ];
    scal[S_RZ] = out[0];
    scal[S_BETA] = out[0] / rz_old;
    scal[S_RR] = out[1];
    scal[S_ITERS] += 1.0;
    if (out[1] <= scal[S_TOL2] || scal[S_ITERS] >= scal[S_MAXIT]) scal[S_DONE] = 1.0;
  }
}

__global__ void k_dir(int64_t nv, const double* z, double* p, const double* scal) {
  if (scal[S_DONE] != 0.0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nv) p[t] = z[t] + scal[S_BETA] * p[t];
}

__global__ void k_set_scalars(double* scal, double tol2, double maxit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    for (int i = 0; i < S_NSCAL; ++i) scal[i] = 0.0;
    scal[S_TOL2] = tol2;
    scal[S_MAXIT] = maxit;
  }
}

// x = x0 on the free faces and 0 on the Dirichlet faces: the Dirichlet values enter through the
// right-hand side (b = F + G_N - H_{.,D} u_hat_D), so a guess that carries u_hat_D there (a
// previous solution) must not be applied a second time by the operator.
__global__ void k_load_x0(int64_t nv, const int32_t* ftype, int d2, const double* __restrict__ x0, double* x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nv) x[t] = (ftype[t / d2] == 1) ? 0.0 : x0[t];
}

__global__ void k_finish(int64_t nv, const int32_t* ftype, int d2, const double* x, const double* xD, double* uhat) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nv) uhat[t] = (ftype[t / d2] == 1) ? xD[t] : x[t];
}

// device address of g_scratch / g_counter, looked up once per device
constexpr int kMaxDevices = 64;
static double* s_scratch_ptr[kMaxDevices];
static unsigned int* s_counter_ptr[kMaxDevices];
static std::mutex s_mutex;

static int scratch_for_current_device(double** scratch, unsigned int** counter) {
  int dev = -1;
  HDG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HDG_ERR_ARG, "device ordinal out of range for the no-alloc solve");
  std::lock_guard<std::mutex> lock(s_mutex);
  if (!s_scratch_ptr[dev]) {
    void* p = nullptr;
    void* c = nullptr;
    HDG_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
    HDG_CUDA_TRY(cudaGetSymbolAddress(&c, g_counter));
    s_scratch_ptr[dev] = static_cast<double*>(p);
    s_counter_ptr[dev] = static_cast<unsigned int*>(c);
  }
  *scratch = s_scratch_ptr[dev];
  *counter = s_counter_ptr[dev];
  return HDG_OK;
}

static double* carve(double*& cur, int64_t n) {
  double* p = cur;
  cur += (n + 31) & ~int64_t(31);  // keep every piece 256-byte aligned
  return p;
}

int solve(hdg_mesh* M, double rtol, int maxit, const double* x0, double* uhat, int* iters, double* relres) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "hdg_solve_trace_noalloc before hdg_assemble_condense");
  if (!(rtol > 0) || maxit < 1 || !uhat) return fail(HDG_ERR_ARG, "bad rtol/maxit/uhat");
  const int d2 = M->tab.d2, m = M->tab.m;
  const int64_t nv = M->nfc * d2;
  if (nv > kMaxDofs || d2 > kMaxD2)
    return fail(HDG_ERR_ARG, "hdg_solve_trace_noalloc supports at most " + std::to_string(kMaxDofs) +
                                 " trace unknowns (nfc*d2); this mesh has " + std::to_string(nv));
  double* base;
  unsigned int* counter;
  int rc = scratch_for_current_device(&base, &counter);
  if (rc) return rc;
  double* cur = base;
  double* b = carve(cur, nv);
  double* xD = carve(cur, nv);
  double* phiN = carve(cur, nv);
  double* x = carve(cur, nv);
  double* r = carve(cur, nv);
  double* z = carve(cur, nv);
  double* p = carve(cur, nv);
  double* q = carve(cur, nv);
  double* Binv = carve(cur, M->nfc * d2 * d2);
  const int fpb = kNT / d2;
  const int nb = (int)((M->nfc + fpb - 1) / fpb);
  double* red = carve(cur, 4 * (int64_t)nb);
  double* scal = carve(cur, 2 * S_NSCAL);
  if (cur - base > kScratchDoubles) return fail(HDG_ERR_ARG, "no-alloc scratch exhausted");

  cudaStream_t st = M->stream;
  Ops F{M->d_C, M->d_owner, M->d_facebyele, M->d_ftype, M->nfc, d2, m};
  HDG_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned int) * 4, st));  // must start at zero
  k_set_scalars<<<1, 32, 0, st>>>(scal, 0.0, (double)maxit);
  k_bdata<<<nb, kNT, 0, st>>>(F, M->d_fvx, M->d_vx, M->nelt, M->dt.D, M->dt.face_w, M->tab.nf, M->uD, M->gN, xD, phiN);
  k_rhs<<<nb, kNT, 0, st>>>(F, M->d_Cf, xD, phiN, b, red, counter, scal);
  k_bj<<<(unsigned)((M->nfc + 63) / 64), 64, 0, st>>>(F, Binv);
  HDG_CUDA_TRY(cudaGetLastError());
  double bb;
  HDG_CUDA_TRY(cudaMemcpyAsync(&bb, scal + S_BB, sizeof(double), cudaMemcpyDeviceToHost, st));
  HDG_CUDA_TRY(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(bb), tol = rtol * bnorm;
  if (x0) k_load_x0<<<nb, kNT, 0, st>>>(nv, M->d_ftype, d2, x0, x);
  double hv[S_NSCAL];
  double* scal2 = scal + S_NSCAL;
  // one PCG pass from x (zero start unless have_x) for at most `budget` iterations
  auto pass = [&](bool have_x, int budget) -> int {
    k_set_scalars<<<1, 32, 0, st>>>(scal, tol * tol, (double)budget);
    k_init<<<nb, kNT, 0, st>>>(F, b, x, have_x, r, red, counter, scal);
    k_precond<<<nb, kNT, 0, st>>>(F, Binv, r, z, p, red, counter, scal);
    HDG_CUDA_TRY(cudaGetLastError());
    for (;;) {
      HDG_CUDA_TRY(cudaMemcpyAsync(hv, scal, sizeof(hv), cudaMemcpyDeviceToHost, st));
      HDG_CUDA_TRY(cudaStreamSynchronize(st));
      if (hv[S_DONE] != 0.0) break;
      for (int i = 0; i < kIterChunk; ++i) {
        k_matvec<<<nb, kNT, 0, st>>>(F, p, q, red, counter, scal);
        k_update<<<nb, kNT, 0, st>>>(F, Binv, x, r, z, p, q, red, counter, scal);
        k_dir<<<nb, kNT, 0, st>>>(nv, z, p, scal);
      }
      HDG_CUDA_TRY(cudaGetLastError());
    }
    return HDG_OK;
  };
  // true FP64 residual ||b - H x|| of the current iterate
  auto true_res = [&](double* rn) -> int {
    k_init<<<nb, kNT, 0, st>>>(F, b, x, true, q, red, counter, scal2);
    HDG_CUDA_TRY(cudaGetLastError());
    double rr;
    HDG_CUDA_TRY(cudaMemcpyAsync(&rr, scal2 + S_RR, sizeof(double), cudaMemcpyDeviceToHost, st));
    HDG_CUDA_TRY(cudaStreamSynchronize(st));
    *rn = std::sqrt(rr);
    return HDG_OK;
  };
  rc = pass(x0 != nullptr, maxit);
  if (rc) return rc;
  int total_it = (int)hv[S_ITERS];
  bool bad = hv[S_BAD] != 0.0;
  double rn = 0.0;
  rc = true_res(&rn);
  if (rc) return rc;
  if (!(rn <= tol * 1.0000001 || bnorm == 0.0) && total_it < maxit && !bad) {
    // the recursive residual converged but the true one did not: one more pass from x, as the
    // FP64 solve of hdg_solve_trace does
    rc = pass(true, maxit - total_it);
    if (rc) return rc;
    total_it += (int)hv[S_ITERS];
    bad = hv[S_BAD] != 0.0;
    rc = true_res(&rn);
    if (rc) return rc;
  }
  k_finish<<<nb, kNT, 0, st>>>(nv, M->d_ftype, d2, x, xD, uhat);
  HDG_CUDA_TRY(cudaGetLastError());
  HDG_CUDA_TRY(cudaStreamSynchronize(st));
  if (iters) *iters = total_it;
  if (relres) *relres = bnorm > 0 ? rn / bnorm : 0.0;
  if (bad) return fail(HDG_ERR_NOT_CONVERGED, "PCG breakdown (non-positive curvature)");
  if (!(rn <= tol * 1.0000001 || bnorm == 0.0))
    return fail(HDG_ERR_NOT_CONVERGED, "no-alloc trace solve reached maxit with relative residual " +
                                           std::to_string(bnorm > 0 ? rn / bnorm : 0.0));
  return HDG_OK;
}

}  // namespace noalloc
}  // namespace hdg

extern "C" int hdg_solve_trace_noalloc(hdg_mesh* mesh, double rtol, int maxit, const double* x0, double* uhat,
                                       int* iters, double* relres) {
  if (!mesh) return hdg::fail(HDG_ERR_ARG, "NULL mesh");
  if (mesh->tab.d2 < 3) return hdg::fail(HDG_ERR_UNSUPPORTED, "the allocation-free solve is built for k >= 1");
  if (mesh->beta_q)
    return hdg::fail(HDG_ERR_UNSUPPORTED,
                     "the allocation-free solve is the symmetric (CG) solve; it needs beta = 0 (no convection)");
  return hdg::noalloc::solve(mesh, rtol, maxit, x0, uhat, iters, relres);
}
