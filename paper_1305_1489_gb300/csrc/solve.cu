// Trace system of Section 6: boundary data (eq. 6.3, 6.4), right-hand side F + G_N - H_{.,D} u_D
// (eq. 6.5 with Dirichlet elimination), block-Jacobi preconditioned CG on the free faces (BiCGStab
// when convection makes H non-symmetric), and the FP32-inner / FP64-outer mixed-precision variant.
//
// Operator: matrix-free, element by element, "face owner" form.  Each face e gathers the row
// blocks of C^K that belong to it from its (at most two) elements:
//     (H x)_e = sum_{K owns e as local face l} (C^K x_dK)_{l-block}
// which is the sparse assembly of Section 6 applied without forming H.  Every row of every C^K
// is read once per product; there are no atomics and the result is deterministic.  K1 stores
// C^K row-major, so the row block of a face is one contiguous array and each of the face's d2
// threads reads its own row with 16-byte loads.
//
// Scheduling: every face kernel runs on a persistent grid (M->face_blocks blocks, at most
// kMaxBlocks, each looping over tiles of kNT / d2 whole faces), so the deterministic
// last-block reductions sum at most that many per-block partials.  hdg_autotune picks the
// grid size per mesh by timing the trace operator.  Scalars (alpha, beta, r.z, r.r) stay on the device;
// batches of iterations are captured in a CUDA graph and the host reads the convergence flag
// after each replay.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <cmath>
#include <vector>

#include "device_async.cuh"
#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {

constexpr int kNT = 128;          // threads per block in the face kernels
constexpr int kMaxBlocks = 152 * 32;  // largest persistent grid (size of the partials buffer)
constexpr int kGraphIters = 16;   // PCG iterations per graph replay

// scalar slots (double) of a solve
enum { S_RZ = 0, S_ALPHA, S_BETA, S_RR, S_BB, S_DONE, S_ITERS, S_TOL2, S_MAXIT, S_PQ, S_BAD, S_BODIES, S_MAXBODIES, S_NSCAL };

struct FaceArgs {
  const int32_t* owner;  // [nfc][2] 4K + l
  const int32_t* fbe;    // [nelt][4]
  const int32_t* ftype;  // [nfc]
  int64_t nfc;
};

// Tile t of a block holds faces [t*FPB, (t+1)*FPB); thread -> (face e, entry a).
template <int D2>
struct Tile {
  static constexpr int FPB = kNT / D2;
  int64_t e, t;
  int a;
  bool act;
  __device__ __forceinline__ Tile(const FaceArgs& F, int64_t tile) {
    const int loc = threadIdx.x / D2;
    a = threadIdx.x - loc * D2;
    e = tile * FPB + loc;
    t = e * D2 + a;
    act = loc < FPB && e < F.nfc;
  }
};

template <int D2>
__device__ __forceinline__ int64_t ntiles(const FaceArgs& F) {
  return (F.nfc + Tile<D2>::FPB - 1) / Tile<D2>::FPB;
}

}  // namespace hdg
#include "coarse.cuh"
namespace hdg {

// Last-block-done reduction of NSLOT values; returns true on the block that finishes.  The
// finishing block sums the per-block partials in block order, so the result is deterministic.
template <int NSLOT>
__device__ bool grid_reduce(const double (&v)[NSLOT], double* red, unsigned int* counter, double (&out)[NSLOT]) {
  __shared__ double wsum[NSLOT][kNT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = gridDim.x;
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    double x = v[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) wsum[s][w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      double x = 0.0;
      for (int i = 0; i < kNT / 32; ++i) x += wsum[s][i];
      red[s * nb + blockIdx.x] = x;
    }
    __threadfence();
    unsigned int ticket = atomicAdd(counter, 1u);
    last = (ticket == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    // eight independent loads per trip, so that the partials arrive in one memory latency
    double x = 0.0;
    const double* rs = red + s * nb;
    for (int i0 = threadIdx.x; i0 < nb; i0 += 8 * kNT) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (i0 + u * kNT < nb) ? __ldcg(rs + i0 + u * kNT) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) x += v[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) wsum[s][w] = x;
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NSLOT; ++s) {
    double x = 0.0;
    for (int i = 0; i < kNT / 32; ++i) x += wsum[s][i];
    out[s] = x;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// (H x)_e entry a: the face's row blocks of C^K (row-major storage) times x_dK.  Each
// owner's column (m values, unit stride across the face's d2 threads) and the gathered x_dK
// are loaded into registers before any FMA, so every thread keeps 2m loads in flight.
// C^K is stored row-major, [K][r][s] = C^K[r][s] with r = l d2 + a, so that thread a of face
// l reads its row as 16-byte loads (m/4 for the FP32 copy, m/2 in FP64).
template <int D2>
__device__ __forceinline__ float face_apply_rm(const float* __restrict__ C, const float* __restrict__ x,
                                               const FaceArgs& F, int64_t e, int a) {
  constexpr int m = 4 * D2;
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const int ow = __ldg(F.owner + 2 * e + o);
    if (ow < 0) continue;
    const int64_t K = ow >> 2;
    const float4* row = reinterpret_cast<const float4*>(C + K * (int64_t)(m * m) + (ow & 3) * (m * D2) + a * m);
    const int4 fb = __ldg(reinterpret_cast<const int4*>(F.fbe) + K);
    const int f4[4] = {fb.x, fb.y, fb.z, fb.w};
    float4 cv[m / 4];
    float xv[m];
#pragma unroll
    for (int q = 0; q < m / 4; ++q) cv[q] = __ldg(row + q);
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      const float* xs = x + (int64_t)f4[fl] * D2;
      if constexpr (D2 % 2 == 0) {  // a face's entries start on an 8-byte boundary: read in pairs
#pragma unroll
        for (int b = 0; b < D2; b += 2) {
          const float2 v = *reinterpret_cast<const float2*>(xs + b);
          xv[fl * D2 + b] = v.x;
          xv[fl * D2 + b + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int b = 0; b < D2; ++b) xv[fl * D2 + b] = xs[b];
      }
    }
    asm volatile("" ::: "memory");
#pragma unroll
    for (int q = 0; q < m / 4; ++q) {
      acc0 = fmaf(cv[q].x, xv[4 * q], acc0);
      acc1 = fmaf(cv[q].y, xv[4 * q + 1], acc1);
      acc0 = fmaf(cv[q].z, xv[4 * q + 2], acc0);
      acc1 = fmaf(cv[q].w, xv[4 * q + 3], acc1);
    }
  }
  return acc0 + acc1;
}

template <typename T, int D2>
__device__ __forceinline__ T face_apply(const T* __restrict__ C, const T* __restrict__ x, const FaceArgs& F,
                                        int64_t e, int a) {
  if constexpr (sizeof(T) == 4) {
    return face_apply_rm<D2>(C, x, F, e, a);
  } else {
    // C^K row-major [K][r][s] (r = l d2 + a): thread a reads its row as m/2 16-byte loads
    constexpr int m = 4 * D2;
    double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int ow = __ldg(F.owner + 2 * e + o);
      if (ow < 0) continue;
      const int64_t K = ow >> 2;
      const double2* row =
          reinterpret_cast<const double2*>(C + K * (int64_t)(m * m) + ((ow & 3) * D2 + a) * (int64_t)m);
      const int4 fb = __ldg(reinterpret_cast<const int4*>(F.fbe) + K);
      const int f4[4] = {fb.x, fb.y, fb.z, fb.w};
      double2 cv[m / 2];
      double xv[m];
#pragma unroll
      for (int q = 0; q < m / 2; ++q) cv[q] = __ldg(row + q);
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        const double* xs = x + (int64_t)f4[fl] * D2;
#pragma unroll
        for (int b = 0; b < D2; ++b) xv[fl * D2 + b] = xs[b];
      }
      asm volatile("" ::: "memory");  // keep every load above issued before the first FMA
#pragma unroll
      for (int q = 0; q < m / 2; ++q) {
        acc0 = fma(cv[q].x, xv[2 * q], acc0);
        acc1 = fma(cv[q].y, xv[2 * q + 1], acc1);
      }
    }
    return (T)(acc0 + acc1);
  }
}

// ------------------------------------------------------------------ element-major operator
// The same product H x in two passes (eq. 6.5 summed element by element):
//   element pass  for every element K and row r = l d2 + a of C^K, the sum_s C^K[r][s] x_dK[s]
//                 goes to Y[side][f d2 + a], f the element's face l and side which of the
//                 face's two owners K is (the per-mesh table fslot = 2 f + side, negative on
//                 Dirichlet faces, whose rows are not stored);
//   face sum      (H x) = Y[0] + Y[1], a flat 16-byte-vectorised stream fused with the dot
//                 products that consume H x (Y stays 0 where nothing is stored: Dirichlet
//                 faces, and side 1 of the boundary faces, which have one owner).
// The element pass is a persistent streaming kernel: the C^K of a group of EB consecutive
// elements is one contiguous block, which one producer thread copies into a ring of NST
// shared-memory stages with 1-D bulk copies (the tensor memory accelerator) completed on the
// stage's "full" mbarrier; one consumer thread per row of the group waits for the stage, takes
// the dot product of its row with the group's x_dK (gathered through the element's four face
// numbers one group ahead, staged in shared memory) and arrives on the stage's "empty" mbarrier,
// which the producer waits on before it reuses the stage.  Every wait is bounded: one that runs
// out counts in status[7] and the kernel runs on (its output is then garbage, which the solve
// reports as HDG_ERR_CUDA), waiting at the end, again bounded, for its own copies in flight.
template <typename T, int D2>
struct EmPass {
  static constexpr int m = 4 * D2;
  static constexpr int EB = (192 / m) > 0 ? 192 / m : 1;  // elements per group
  static constexpr int ROWS = EB * m;                      // rows of a group (consumer threads)
  static constexpr int CW = (ROWS + 31) / 32;              // consumer warps
  static constexpr int NTHR = 32 * CW + 32;                // + the producer warp
  static constexpr int GBYTES = EB * m * m * (int)sizeof(T);
  static constexpr int NSTR = (200 * 1024) / GBYTES;
  static constexpr int NST = NSTR > 4 ? 4 : (NSTR < 2 ? 2 : NSTR);  // stages of the ring
  static constexpr int XBYTES = 2 * 32 * CW * (int)sizeof(T);       // x_dK, double-buffered
  static constexpr int SMEM = NST * GBYTES + XBYTES;
  static_assert(GBYTES % 16 == 0 && (m * (int)sizeof(T)) % 16 == 0, "16-byte bulk copies and rows");
  static_assert(SMEM <= 227 * 1024, "element pass ring");
};
constexpr int kEmWaitPolls = 1 << 22;  // bounded mbarrier waits (far above a copy's latency)

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename T, int D2>
__global__ void __launch_bounds__(EmPass<T, D2>::NTHR) em_apply_kernel(const T* __restrict__ C, const T* __restrict__ x,
                                                                       const int32_t* __restrict__ fslot, int64_t nelt,
                                                                       int64_t nvp, T* __restrict__ Y,
                                                                       const double* done, int32_t* status) {
  using P = EmPass<T, D2>;
  constexpr int m = P::m, EB = P::EB, NST = P::NST;
  constexpr int VW = 16 / sizeof(T);
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  if (*done != 0.0) return;
  extern __shared__ __align__(128) unsigned char em_smem[];
  T* ring = reinterpret_cast<T*>(em_smem);                     // [NST][EB m m]
  T* xs = reinterpret_cast<T*>(em_smem + NST * P::GBYTES);     // [2][32 CW]
  __shared__ __align__(8) uint64_t full[NST], empty[NST];
  const int tid = threadIdx.x;
  const int64_t ngroups = (nelt + EB - 1) / EB;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 32 * P::CW);
    }
  }
  __syncthreads();
  int fails = 0;
  if (tid >= 32 * P::CW) {
    // producer: one thread streams the groups' C^K blocks into the ring
    if (tid == 32 * P::CW) {
      int it = 0;
      for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, ++it) {
        const int s = it % NST;
        if (it >= NST && !mbar_wait(&empty[s], (uint32_t)((it / NST) - 1) & 1u, kEmWaitPolls)) ++fails;
        const int64_t ne = min((int64_t)EB, nelt - g * EB);
        const uint32_t bytes = (uint32_t)(ne * m * m * (int64_t)sizeof(T));
        mbar_expect_tx(&full[s], bytes);
        bulk_g2s(ring + (size_t)s * EB * m * m, C + g * EB * (int64_t)(m * m), bytes, &full[s]);
      }
      // the copies still in flight land before the block exits: the last use of each stage
      for (int u = 0; u < NST && u < it; ++u) {
        const int last = it - 1 - u, s = last % NST;
        if (!mbar_wait(&full[s], (uint32_t)(last / NST) & 1u, kEmWaitPolls)) ++fails;
      }
    }
  } else {
    // consumers: thread (el, r) owns row r of the group's element el
    const int el = tid / m, r = tid - el * m;
    const bool lane_act = el < EB;
    // the gather of x_dK is pipelined over the groups: the face number two groups ahead and
    // the value one group ahead are in flight while a group is computed, so that no iteration
    // waits on more than one memory latency
    constexpr int kNone = INT32_MIN;         // no row (past the last element)
    auto face_of = [&](int64_t g) -> int {  // fslot of this thread's row of group g
      const int64_t K = g * EB + el;
      return (lane_act && g < ngroups && K < nelt) ? __ldg(fslot + 4 * K + r / D2) : kNone;
    };
    auto x_of = [&](int fs) -> T {
      if (fs == kNone) return (T)0;
      const int f2 = fs >= 0 ? fs : -fs - 1;  // 2 f + side
      return x[(int64_t)(f2 >> 1) * D2 + (r % D2)];
    };
    const int64_t G = gridDim.x;
    int fcur = face_of(blockIdx.x);
    T xn = x_of(fcur);
    int f1 = face_of(blockIdx.x + G);
    int it = 0;
    for (int64_t g = blockIdx.x; g < ngroups; g += G, ++it) {
      const int s = it % NST;
      T* xb = xs + (it & 1) * 32 * P::CW;
      xb[tid] = xn;
      const int fs = fcur;      // this group's output slot
      fcur = f1;
      xn = x_of(f1);            // the next group's x_dK
      f1 = face_of(g + 2 * G);  // the face numbers of the group after it
      asm volatile("bar.sync 1, %0;" ::"r"(32 * P::CW) : "memory");  // xb complete
      if (!mbar_wait(&full[s], (uint32_t)(it / NST) & 1u, kEmWaitPolls)) ++fails;
      const int64_t K = g * EB + el;
      if (lane_act && K < nelt && fs >= 0) {
        const V* row = reinterpret_cast<const V*>(ring + (size_t)s * EB * m * m + (size_t)(el * m + r) * m);
        const V* xr = reinterpret_cast<const V*>(xb + el * m);
        T acc0 = (T)0, acc1 = (T)0;
#pragma unroll
        for (int q = 0; q < m / VW; ++q) {
          const V cq = row[q], xq = xr[q];
          if constexpr (sizeof(T) == 4) {
            acc0 = fmaf(cq.x, xq.x, acc0);
            acc1 = fmaf(cq.y, xq.y, acc1);
            acc0 = fmaf(cq.z, xq.z, acc0);
            acc1 = fmaf(cq.w, xq.w, acc1);
          } else {
            acc0 = fma(cq.x, xq.x, acc0);
            acc1 = fma(cq.y, xq.y, acc1);
          }
        }
        Y[(fs & 1) * nvp + (int64_t)(fs >> 1) * D2 + (r % D2)] = acc0 + acc1;
      }
      mbar_arrive(&empty[s]);
    }
  }
  if (fails) atomicAdd(status + 7, 1);
}

// blocks of the element pass: every SM's resident blocks, or fewer when there are fewer groups
// (HDG_FACE_BLOCKS caps the grid in the tests, so that each block takes many groups)
template <typename T, int D2>
static int em_grid(hdg_mesh* M) {
  using P = EmPass<T, D2>;
  static int per_sm = 0, sms = 0;
  if (!per_sm) {
    cudaFuncSetAttribute(em_apply_kernel<T, D2>, cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, em_apply_kernel<T, D2>, P::NTHR, P::SMEM);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t ngroups = (M->nelt + P::EB - 1) / P::EB;
  int64_t g = std::min<int64_t>(ngroups, (int64_t)per_sm * sms);
  if (M->grid_cap > 0) g = std::min<int64_t>(g, M->grid_cap);
  return (int)std::max<int64_t>(g, 1);
}



// row a of face e's block inverse times the face's d2 residual entries
template <typename T, int D2>
__device__ __forceinline__ T bj_apply(const T* __restrict__ Binv, const T* __restrict__ r, int64_t e, int a) {
  T s0 = (T)0, s1 = (T)0;
  const T* Bi = Binv + (e * D2 + a) * D2;
  const T* re = r + e * D2;
#pragma unroll
  for (int b = 0; b < D2; ++b) {
    if (b & 1) s1 = fma(Bi[b], re[b], s1); else s0 = fma(Bi[b], re[b], s0);
  }
  return s0 + s1;
}

// ------------------------------------------------------------------ setup kernels
// u_hat_D (eq. 6.3, with (varpi . D)^T D = I for the orthonormal basis and exact rule) on
// Dirichlet faces, Phi_N (eq. 6.4) on Neumann faces.
template <int D2>
__global__ void bdata_kernel(FaceArgs F, const double* __restrict__ fvx, const double* __restrict__ vx,
                             int64_t nelt, const double* __restrict__ D, const double* __restrict__ wf,
                             int nf, const double* __restrict__ uD, const double* __restrict__ gN,
                             double* __restrict__ xD, double* __restrict__ phiN) {
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const int64_t e = T_.e, t = T_.t;
    const int a = T_.a;
    const int ty = F.ftype[e];
    double xd = 0.0, ph = 0.0;
    if (ty == 1 && uD) {
      for (int r = 0; r < nf; ++r) xd = fma(wf[r] * D[r * D2 + a], uD[e * nf + r], xd);
    } else if (ty == 2 && gN) {
      // n_e: outward normal of the owning element, |n_e| = |e|
      double w[3][3];
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) w[i][d] = fvx[(d * 3 + i) * F.nfc + e];
      double u1[3], u2[3], nv[3];
      for (int d = 0; d < 3; ++d) {
        u1[d] = w[1][d] - w[0][d];
        u2[d] = w[2][d] - w[0][d];
      }
      cross3(u1, u2, nv);
      const int ow = F.owner[2 * e];
      const int64_t K = ow >> 2;
      const int opp[4] = {3, 2, 1, 0};  // vertex of K not on local face l (eq. 2.1)
      const int vi = opp[ow & 3];
      double dot = 0.0;
      for (int d = 0; d < 3; ++d) dot += nv[d] * (vx[(d * 4 + vi) * nelt + K] - w[0][d]);
      const double sg = dot > 0 ? -0.5 : 0.5;
      for (int s = 0; s < 3; ++s) {
        double acc = 0.0;
        for (int r = 0; r < nf; ++r) acc = fma(wf[r] * D[r * D2 + a], gN[((int64_t)s * F.nfc + e) * nf + r], acc);
        ph = fma(sg * nv[s], acc, ph);
      }
    }
    xD[t] = xd;
    phiN[t] = ph;
  }
}

// b = F + G_N - H x_D on free faces (F assembled from C_f^K), 0 on Dirichlet faces.
template <int D2>
__global__ void rhs_kernel(FaceArgs F, const double* __restrict__ C, const double* __restrict__ Cf,
                           const double* __restrict__ xD, const double* __restrict__ phiN, double* __restrict__ b,
                           double* red, unsigned int* counter, double* scal) {
  constexpr int m = 4 * D2;
  double v = 0.0;
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    double bv = 0.0;
    if (F.ftype[T_.e] != 1) {
      double fsum = 0.0;
      for (int o = 0; o < 2; ++o) {
        const int ow = F.owner[2 * T_.e + o];
        if (ow < 0) continue;
        fsum += Cf[(int64_t)(ow >> 2) * m + (ow & 3) * D2 + T_.a];
      }
      bv = fsum + phiN[T_.t] - face_apply<double, D2>(C, xD, F, T_.e, T_.a);
    }
    b[T_.t] = bv;
    v = fma(bv, bv, v);
  }
  double in[1] = {v}, out[1];
  if (grid_reduce<1>(in, red, counter, out) && threadIdx.x == 0) scal[S_BB] = out[0];
}

// Inverse of each free face's diagonal block of H (block-Jacobi): Cholesky, or Gauss-Jordan
// without pivoting for convection (the block's symmetric part is positive definite).  TB is
// the arithmetic and output type: FP64 for the FP64 solves, FP32 for the inner FP32 solve.
template <int D2, typename TB>
__global__ void bj_kernel(FaceArgs F, const double* __restrict__ C, TB* __restrict__ Binv, int32_t* status,
                          bool nonsym) {
  constexpr int m = 4 * D2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= F.nfc) return;
  TB A[D2 * D2], X[D2 * D2];
  if (F.ftype[e] == 1) {
    for (int i = 0; i < D2 * D2; ++i) Binv[e * D2 * D2 + i] = (TB)0;
    return;
  }
  for (int i = 0; i < D2 * D2; ++i) A[i] = (TB)0;
  for (int o = 0; o < 2; ++o) {
    const int ow = F.owner[2 * e + o];
    if (ow < 0) continue;
    const int l = ow & 3;
    // C^K[l d2 + i][l d2 + j], row-major
    const double* Cb = C + (int64_t)(ow >> 2) * m * m + (int64_t)(l * D2) * m + l * D2;
    for (int i = 0; i < D2; ++i)
      for (int j = 0; j < D2; ++j) A[i * D2 + j] += (TB)Cb[i * m + j];
  }
  bool ok = true;
  if (nonsym) {
    for (int i = 0; i < D2 * D2; ++i) X[i] = (TB)0;
    for (int i = 0; i < D2; ++i) X[i * D2 + i] = (TB)1;
    for (int j = 0; j < D2; ++j) {
      const TB piv = A[j * D2 + j];
      ok = ok && piv != (TB)0 && isfinite(piv);
      const TB ip = (TB)1 / piv;
      for (int c = 0; c < D2; ++c) {
        A[j * D2 + c] *= ip;
        X[j * D2 + c] *= ip;
      }
      for (int i = 0; i < D2; ++i) {
        if (i == j) continue;
        const TB f = A[i * D2 + j];
        for (int c = 0; c < D2; ++c) {
          A[i * D2 + c] -= f * A[j * D2 + c];
          X[i * D2 + c] -= f * X[j * D2 + c];
        }
      }
    }
  } else {
    for (int j = 0; j < D2; ++j) {  // in-place lower Cholesky
      TB s = A[j * D2 + j];
      for (int l = 0; l < j; ++l) s -= A[j * D2 + l] * A[j * D2 + l];
      ok = ok && s > (TB)0;
      const TB d = sqrt(s);
      A[j * D2 + j] = d;
      for (int i = j + 1; i < D2; ++i) {
        TB t = A[i * D2 + j];
        for (int l = 0; l < j; ++l) t -= A[i * D2 + l] * A[j * D2 + l];
        A[i * D2 + j] = t / d;
      }
    }
    for (int c = 0; c < D2; ++c) {  // columns of A^-1 = L^-T L^-1 e_c
      for (int i = 0; i < D2; ++i) {
        TB s = (i == c) ? (TB)1 : (TB)0;
        for (int l = 0; l < i; ++l) s -= A[i * D2 + l] * X[l * D2 + c];
        X[i * D2 + c] = s / A[i * D2 + i];
      }
      for (int i = D2 - 1; i >= 0; --i) {
        TB s = X[i * D2 + c];
        for (int l = i + 1; l < D2; ++l) s -= A[l * D2 + i] * X[l * D2 + c];
        X[i * D2 + c] = s / A[i * D2 + i];
      }
    }
  }
  for (int i = 0; i < D2 * D2; ++i) Binv[e * D2 * D2 + i] = X[i];
  if (!ok) atomicAdd(status + 3, 1);
}

// FP32 copy of C^K (same row-major layout)
template <int D2>
__global__ void convert_c32_kernel(const double* __restrict__ C, float* __restrict__ C32, int64_t nelt) {
  constexpr int m = 4 * D2;
  const int64_t n = nelt * m * m;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    C32[i] = (float)C[i];
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ a, T* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

// ------------------------------------------------------------------ PCG kernels
// init: r = b - H x (x given) or r = b (x = 0);  r.r
template <typename T, int D2>
__global__ void pcg_init_kernel(FaceArgs F, const T* __restrict__ C, const T* __restrict__ b, T* __restrict__ x,
                                bool have_x, T* __restrict__ r, double* red, unsigned int* counter, double* scal) {
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    T rv = (T)0;
    if (F.ftype[T_.e] != 1) rv = b[T_.t] - (have_x ? face_apply<T, D2>(C, x, F, T_.e, T_.a) : (T)0);
    if (!have_x) x[T_.t] = (T)0;
    r[T_.t] = rv;
    v[0] = fma((double)rv, (double)rv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) scal[S_RR] = out[0];
}

// z = B^-1 r;  p = z;  r.z
template <typename T, int D2>
__global__ void pcg_precond_kernel(FaceArgs F, const T* __restrict__ Binv, const T* __restrict__ r, T* __restrict__ z,
                                   T* __restrict__ p, double* red, unsigned int* counter, double* scal) {
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const T zv = bj_apply<T, D2>(Binv, r, T_.e, T_.a);
    z[T_.t] = zv;
    p[T_.t] = zv;
    v[0] = fma((double)r[T_.t], (double)zv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[S_RZ] = out[0];
    scal[S_DONE] = (scal[S_RR] <= scal[S_TOL2]) ? 1.0 : 0.0;
    scal[S_ITERS] = 0.0;
  }
}

// q = H p (free faces), alpha = rz / (p.q)
template <typename T, int D2>
__global__ void pcg_matvec_kernel(FaceArgs F, const T* __restrict__ C, const T* __restrict__ p, T* __restrict__ q,
                                  double* red, unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const T qv = (F.ftype[T_.e] != 1) ? face_apply<T, D2>(C, p, F, T_.e, T_.a) : (T)0;
    q[T_.t] = qv;
    v[0] = fma((double)p[T_.t], (double)qv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[S_PQ] = out[0];
    if (!(out[0] > 0.0)) {  // breakdown: H not SPD on the Krylov space
      scal[S_BAD] = 1.0;
      scal[S_DONE] = 1.0;
      scal[S_ALPHA] = 0.0;
    } else {
      scal[S_ALPHA] = scal[S_RZ] / out[0];
    }
  }
}

// x += alpha p;  r -= alpha q;  z = B^-1 r;  beta = r.z_new / r.z;  convergence test on r.r
template <typename T, int D2>
__global__ void pcg_update_kernel(FaceArgs F, const T* __restrict__ Binv, T* __restrict__ x, T* __restrict__ r,
                                  T* __restrict__ z, const T* __restrict__ p, const T* __restrict__ q, double* red,
                                  unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  const T alpha = (T)scal[S_ALPHA];
  double v[2] = {0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (T_.act) {
      x[T_.t] = fma(alpha, p[T_.t], x[T_.t]);
      r[T_.t] = fma(-alpha, q[T_.t], r[T_.t]);
    }
    __syncthreads();  // the d2 entries of r of each face of the tile are updated
    if (T_.act) {
      const T zv = bj_apply<T, D2>(Binv, r, T_.e, T_.a);
      z[T_.t] = zv;
      const double rv = (double)r[T_.t];
      v[0] = fma(rv, (double)zv, v[0]);
      v[1] = fma(rv, rv, v[1]);
    }
  }
  double out[2];
  if (grid_reduce<2>(v, red, counter, out) && threadIdx.x == 0) {
    const double rz_old = scal[S_RZ];
    scal[S_RZ] = out[0];
    scal[S_BETA] = out[0] / rz_old;
    scal[S_RR] = out[1];
    scal[S_ITERS] += 1.0;
    if (out[1] <= scal[S_TOL2] || scal[S_ITERS] >= scal[S_MAXIT]) scal[S_DONE] = 1.0;
  }
}

template <typename T>
__global__ void pcg_dir_kernel(int64_t ntot, const T* __restrict__ z, T* __restrict__ p, const double* scal) {
  if (scal[S_DONE] != 0.0) return;
  const T beta = (T)scal[S_BETA];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntot; t += (int64_t)gridDim.x * blockDim.x)
    p[t] = fma(beta, p[t], z[t]);
}

// Two-level variant of the update: x += alpha p;  r -= alpha q;  r.r.  The preconditioned
// residual is formed by the restriction, the V-cycle and pcg_zc_kernel.
template <typename T, int D2>
__global__ void pcg_update_tl_kernel(FaceArgs F, T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                     const T* __restrict__ q, double* red, unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  const T alpha = (T)scal[S_ALPHA];
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (T_.act) {
      x[T_.t] = fma(alpha, p[T_.t], x[T_.t]);
      const T rv = fma(-alpha, q[T_.t], r[T_.t]);
      r[T_.t] = rv;
      v[0] = fma((double)rv, (double)rv, v[0]);
    }
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[S_RR] = out[0];
    scal[S_ITERS] += 1.0;
    if (out[0] <= scal[S_TOL2] || scal[S_ITERS] >= scal[S_MAXIT]) scal[S_DONE] = 1.0;
  }
}

// z = B^-1 r + Pi e0;  r.z;  INIT: p = z and the convergence flag, else beta.
template <typename T, int D2, bool INIT>
__global__ void pcg_zc_kernel(FaceArgs F, CoarseArgs CA, const T* __restrict__ Binv, const T* __restrict__ r,
                              T* __restrict__ z, T* __restrict__ p, double* red, unsigned int* counter, double* scal) {
  if (!INIT && scal[S_DONE] != 0.0) return;
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    T zv = bj_apply<T, D2>(Binv, r, T_.e, T_.a);
    if (F.ftype[T_.e] != 1) zv += (T)prolong_face<D2>(CA, T_.e, T_.a);
    z[T_.t] = zv;
    if (INIT) p[T_.t] = zv;
    v[0] = fma((double)r[T_.t], (double)zv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    if (INIT) {
      scal[S_RZ] = out[0];
      scal[S_DONE] = (scal[S_RR] <= scal[S_TOL2]) ? 1.0 : 0.0;
      scal[S_ITERS] = 0.0;
    } else {
      scal[S_BETA] = out[0] / scal[S_RZ];
      scal[S_RZ] = out[0];
    }
  }
}

// End of one body of the device-driven loop: keep looping while the solve is not done and
// fewer than scal[max_slot] bodies have run (the host sets that bound before every launch).
// The body counter is independent of the reductions, so the loop ends even if a reduction
// never completes.
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, double* scal, int done_slot, int bodies_slot,
                                    int max_slot) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double nb = scal[bodies_slot] + 1.0;
    scal[bodies_slot] = nb;
    const bool more = scal[done_slot] == 0.0 && nb < scal[max_slot];
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

// ------------------------------------------------------------------ BiCGStab (convection)
// Right-preconditioned BiCGStab (van der Vorst 1992) for the non-symmetric trace matrix of
// convection-diffusion, in FP64 or (inner solve of the mixed-precision path) FP32 vectors,
// with the block-Jacobi or the two-level preconditioner M^-1 = B^-1 + Pi V(Pi^T .).  Vectors:
// x, r, rhat (shadow residual), p, v, s, t, ph = M^-1 p, sh = M^-1 s.  Scalars rho, alpha,
// omega, beta (FP64) on the device.  Per iteration: p, [coarse cycle of p, ph], v = H ph, s,
// [coarse cycle of s, sh], t = H sh, x and r: five kernels with block-Jacobi, seven plus two
// coarse cycles with the two-level preconditioner.
enum { B_RHO = 0, B_ALPHA, B_OMEGA, B_BETA, B_RR, B_DONE, B_ITERS, B_TOL2, B_MAXIT, B_BAD, B_BODIES, B_MAXBODIES,
       B_NSCAL };
static_assert((int)B_NSCAL <= (int)S_NSCAL, "BiCGStab scalars share the PCG scalar block");

template <typename T>
struct BicgVecs {
  T *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
};

// r = b - H x (or b), rhat = r, p = v = 0; rho = rhat.r, beta = 0, omega = 1, rr
template <typename T, int D2>
__global__ void bicg_init_kernel(FaceArgs F, const T* __restrict__ C, const T* __restrict__ b, BicgVecs<T> V,
                                 bool have_x, double* red, unsigned int* counter, double* scal) {
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const int64_t t = T_.t;
    T rv = (T)0;
    if (F.ftype[T_.e] != 1) rv = b[t] - (have_x ? face_apply<T, D2>(C, V.x, F, T_.e, T_.a) : (T)0);
    if (!have_x) V.x[t] = (T)0;
    V.r[t] = rv;
    V.rh[t] = rv;
    V.p[t] = (T)0;
    V.v[t] = (T)0;
    v[0] = fma((double)rv, (double)rv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[B_RHO] = out[0];
    scal[B_RR] = out[0];
    scal[B_BETA] = 0.0;
    scal[B_OMEGA] = 1.0;
    scal[B_ITERS] = 0.0;
    scal[B_DONE] = (out[0] <= scal[B_TOL2]) ? 1.0 : 0.0;
  }
}

// p = r + beta (p - omega v);  ph = B^-1 p (block-Jacobi only: with the two-level
// preconditioner ph is formed after the coarse cycle of p)
template <typename T, int D2, bool TL>
__global__ void bicg_p_kernel(FaceArgs F, const T* __restrict__ Binv, BicgVecs<T> V, const double* scal) {
  if (scal[B_DONE] != 0.0) return;
  const T beta = (T)scal[B_BETA], omega = (T)scal[B_OMEGA];
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (T_.act) V.p[T_.t] = fma(beta, fma(-omega, V.v[T_.t], V.p[T_.t]), V.r[T_.t]);
    if constexpr (!TL) {
      __syncthreads();
      if (T_.act) V.ph[T_.t] = bj_apply<T, D2>(Binv, V.p, T_.e, T_.a);
    }
  }
}

// out = B^-1 in + Pi e0 (the two-level preconditioner, after the coarse cycle of `in`)
template <typename T, int D2, int DONE>
__global__ void bicg_tl_kernel(FaceArgs F, CoarseArgs CA, const T* __restrict__ Binv, const T* __restrict__ in,
                               T* __restrict__ out, const double* scal) {
  if (scal[DONE] != 0.0) return;
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    T zv = bj_apply<T, D2>(Binv, in, T_.e, T_.a);
    if (F.ftype[T_.e] != 1) zv += (T)prolong_face<D2>(CA, T_.e, T_.a);
    out[T_.t] = zv;
  }
}

// v = H ph;  alpha = rho / (rhat . v)
template <typename T, int D2>
__global__ void bicg_v_kernel(FaceArgs F, const T* __restrict__ C, BicgVecs<T> V, double* red,
                              unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  double v[1] = {0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const T vv = (F.ftype[T_.e] != 1) ? face_apply<T, D2>(C, V.ph, F, T_.e, T_.a) : (T)0;
    V.v[T_.t] = vv;
    v[0] = fma((double)V.rh[T_.t], (double)vv, v[0]);
  }
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    if (out[0] == 0.0 || !isfinite(out[0])) {
      scal[B_BAD] = 1.0;
      scal[B_DONE] = 1.0;
      scal[B_ALPHA] = 0.0;
    } else {
      scal[B_ALPHA] = scal[B_RHO] / out[0];
    }
  }
}

// s = r - alpha v;  sh = B^-1 s (block-Jacobi only)
template <typename T, int D2, bool TL>
__global__ void bicg_s_kernel(FaceArgs F, const T* __restrict__ Binv, BicgVecs<T> V, const double* scal) {
  if (scal[B_DONE] != 0.0) return;
  const T alpha = (T)scal[B_ALPHA];
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (T_.act) V.s[T_.t] = fma(-alpha, V.v[T_.t], V.r[T_.t]);
    if constexpr (!TL) {
      __syncthreads();
      if (T_.act) V.sh[T_.t] = bj_apply<T, D2>(Binv, V.s, T_.e, T_.a);
    }
  }
}

// t = H sh;  omega = (t.s) / (t.t)
template <typename T, int D2>
__global__ void bicg_t_kernel(FaceArgs F, const T* __restrict__ C, BicgVecs<T> V, double* red,
                              unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  double v[2] = {0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const T tv = (F.ftype[T_.e] != 1) ? face_apply<T, D2>(C, V.sh, F, T_.e, T_.a) : (T)0;
    V.t[T_.t] = tv;
    v[0] = fma((double)tv, (double)V.s[T_.t], v[0]);
    v[1] = fma((double)tv, (double)tv, v[1]);
  }
  double out[2];
  if (grid_reduce<2>(v, red, counter, out) && threadIdx.x == 0) scal[B_OMEGA] = (out[1] > 0.0) ? out[0] / out[1] : 0.0;
}

// x += alpha ph + omega sh;  r = s - omega t;  rho' = rhat.r;  beta = (rho'/rho)(alpha/omega)
template <typename T, int D2>
__global__ void bicg_x_kernel(FaceArgs F, BicgVecs<T> V, double* red, unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  const double alpha = scal[B_ALPHA], omega = scal[B_OMEGA];
  double v[2] = {0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    const int64_t t = T_.t;
    V.x[t] = fma((T)alpha, V.ph[t], fma((T)omega, V.sh[t], V.x[t]));
    const T rv = fma((T)(-omega), V.t[t], V.s[t]);
    V.r[t] = rv;
    v[0] = fma((double)V.rh[t], (double)rv, v[0]);
    v[1] = fma((double)rv, (double)rv, v[1]);
  }
  double out[2];
  if (grid_reduce<2>(v, red, counter, out) && threadIdx.x == 0) {
    const double rho_old = scal[B_RHO];
    scal[B_BETA] = (out[0] / rho_old) * (alpha / omega);
    scal[B_RHO] = out[0];
    scal[B_RR] = out[1];
    scal[B_ITERS] += 1.0;
    if (omega == 0.0 || out[0] == 0.0 || !isfinite(out[1])) {
      scal[B_BAD] = (out[1] <= scal[B_TOL2]) ? 0.0 : 1.0;
      scal[B_DONE] = 1.0;
    }
    if (out[1] <= scal[B_TOL2] || scal[B_ITERS] >= scal[B_MAXIT]) scal[B_DONE] = 1.0;
  }
}

// Flat vector forms of the elementwise BiCGStab steps: the vectors as plain arrays of nv
// entries, W = 16 / sizeof(T) entries per 16-byte load (the extra vectors are laid out with a
// stride rounded up to W, so every vector starts 16-byte aligned), the remainder entries one
// by one.  Dirichlet entries need no mask: r, v, t, ph, sh all vanish there.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  static constexpr int W = 4;
};
template <>
struct Vec16<double> {
  using V = double2;
  static constexpr int W = 2;
};

template <typename T, typename F>
__device__ __forceinline__ void flat_loop(int64_t nv, F&& f) {
  constexpr int W = Vec16<T>::W;
  const int64_t nvec = nv / W;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride) f(i, true);
  for (int64_t i = nvec * W + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) f(i, false);
}

#define HDG_LD(ptr) (reinterpret_cast<const VT*>(ptr)[i])
#define HDG_ST(ptr, val) (reinterpret_cast<VT*>(ptr)[i] = (val))

// p = r + beta (p - omega v)  (two-level path: ph follows the coarse cycle of p)
template <typename T>
__global__ void bicg_p_flat_kernel(int64_t nv, BicgVecs<T> V, const double* scal) {
  if (scal[B_DONE] != 0.0) return;
  using VT = typename Vec16<T>::V;
  const T beta = (T)scal[B_BETA], omega = (T)scal[B_OMEGA];
  flat_loop<T>(nv, [&](int64_t i, bool vec) {
    if (vec) {
      const VT rr = HDG_LD(V.r), pp = HDG_LD(V.p), vq = HDG_LD(V.v);
      const T* r = reinterpret_cast<const T*>(&rr);
      const T* pv = reinterpret_cast<const T*>(&pp);
      const T* vv = reinterpret_cast<const T*>(&vq);
      VT o;
      T* ov = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int w = 0; w < Vec16<T>::W; ++w) ov[w] = fma(beta, fma(-omega, vv[w], pv[w]), r[w]);
      HDG_ST(V.p, o);
    } else {
      V.p[i] = fma(beta, fma(-omega, V.v[i], V.p[i]), V.r[i]);
    }
  });
}

// s = r - alpha v  (two-level path)
template <typename T>
__global__ void bicg_s_flat_kernel(int64_t nv, BicgVecs<T> V, const double* scal) {
  if (scal[B_DONE] != 0.0) return;
  using VT = typename Vec16<T>::V;
  const T alpha = (T)scal[B_ALPHA];
  flat_loop<T>(nv, [&](int64_t i, bool vec) {
    if (vec) {
      const VT rv = HDG_LD(V.r), vv = HDG_LD(V.v);
      const T* r = reinterpret_cast<const T*>(&rv);
      const T* v = reinterpret_cast<const T*>(&vv);
      VT o;
      T* ov = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int w = 0; w < Vec16<T>::W; ++w) ov[w] = fma(-alpha, v[w], r[w]);
      HDG_ST(V.s, o);
    } else {
      V.s[i] = fma(-alpha, V.v[i], V.r[i]);
    }
  });
}

// x += alpha ph + omega sh;  r = s - omega t;  rho' = rhat.r;  beta = (rho'/rho)(alpha/omega)
template <typename T>
__global__ void bicg_x_flat_kernel(int64_t nv, BicgVecs<T> V, double* red, unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  using VT = typename Vec16<T>::V;
  const double alpha = scal[B_ALPHA], omega = scal[B_OMEGA];
  const T a = (T)alpha, o = (T)omega;
  double v[2] = {0.0, 0.0};
  flat_loop<T>(nv, [&](int64_t i, bool vec) {
    if (vec) {
      const VT xv = HDG_LD(V.x), phv = HDG_LD(V.ph), shv = HDG_LD(V.sh), sv = HDG_LD(V.s), tv = HDG_LD(V.t),
               rhv = HDG_LD(V.rh);
      const T *x = reinterpret_cast<const T*>(&xv), *ph = reinterpret_cast<const T*>(&phv),
              *sh = reinterpret_cast<const T*>(&shv), *sp = reinterpret_cast<const T*>(&sv),
              *tp = reinterpret_cast<const T*>(&tv), *rh = reinterpret_cast<const T*>(&rhv);
      VT xo, ro;
      T* xw = reinterpret_cast<T*>(&xo);
      T* rw = reinterpret_cast<T*>(&ro);
#pragma unroll
      for (int w = 0; w < Vec16<T>::W; ++w) {
        xw[w] = fma(a, ph[w], fma(o, sh[w], x[w]));
        rw[w] = fma(-o, tp[w], sp[w]);
        v[0] = fma((double)rh[w], (double)rw[w], v[0]);
        v[1] = fma((double)rw[w], (double)rw[w], v[1]);
      }
      HDG_ST(V.x, xo);
      HDG_ST(V.r, ro);
    } else {
      V.x[i] = fma(a, V.ph[i], fma(o, V.sh[i], V.x[i]));
      const T rv = fma(-o, V.t[i], V.s[i]);
      V.r[i] = rv;
      v[0] = fma((double)V.rh[i], (double)rv, v[0]);
      v[1] = fma((double)rv, (double)rv, v[1]);
    }
  });
  double out[2];
  if (grid_reduce<2>(v, red, counter, out) && threadIdx.x == 0) {
    const double rho_old = scal[B_RHO];
    scal[B_BETA] = (out[0] / rho_old) * (alpha / omega);
    scal[B_RHO] = out[0];
    scal[B_RR] = out[1];
    scal[B_ITERS] += 1.0;
    if (omega == 0.0 || out[0] == 0.0 || !isfinite(out[1])) {
      scal[B_BAD] = (out[1] <= scal[B_TOL2]) ? 0.0 : 1.0;
      scal[B_DONE] = 1.0;
    }
    if (out[1] <= scal[B_TOL2] || scal[B_ITERS] >= scal[B_MAXIT]) scal[B_DONE] = 1.0;
  }
}
// The face sums of the element pass (H x = Y[0] + Y[1], 0 on Dirichlet rows), flat and fused
// with the reductions of the kernels they replace: q = H p with p.q and alpha (PCG), v = H ph
// with rhat.v and alpha, t = H sh with t.s, t.t and omega (BiCGStab).
// out = Y[0] + Y[1];  v[0] += a.out;  with NS = 2 also v[1] += out.out
template <typename T, int NS>
__device__ __forceinline__ void em_sum_loop(int64_t nv, int64_t nvp, const T* __restrict__ Y, T* __restrict__ out,
                                            const T* __restrict__ a, double (&v)[NS]) {
  using VT = typename Vec16<T>::V;
  const T* Y1 = Y + nvp;
  flat_loop<T>(nv, [&](int64_t i, bool vec) {
    if (vec) {
      const VT y0 = HDG_LD(Y), y1 = HDG_LD(Y1), av = HDG_LD(a);
      const T *p0 = reinterpret_cast<const T*>(&y0), *p1 = reinterpret_cast<const T*>(&y1),
              *pa = reinterpret_cast<const T*>(&av);
      VT o;
      T* ow = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int w = 0; w < Vec16<T>::W; ++w) {
        ow[w] = p0[w] + p1[w];
        v[0] = fma((double)pa[w], (double)ow[w], v[0]);
        if (NS == 2) v[NS - 1] = fma((double)ow[w], (double)ow[w], v[NS - 1]);
      }
      HDG_ST(out, o);
    } else {
      const T o = Y[i] + Y1[i];
      out[i] = o;
      v[0] = fma((double)a[i], (double)o, v[0]);
      if (NS == 2) v[NS - 1] = fma((double)o, (double)o, v[NS - 1]);
    }
  });
}

// y = H x from the element pass alone (hdg_trace_apply in the element form)
template <typename T>
__global__ void em_sum_kernel(int64_t nv, int64_t nvp, const T* __restrict__ Y, T* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) y[i] = Y[i] + Y[nvp + i];
}

// q = H p from the element pass;  alpha = rz / (p.q)
template <typename T>
__global__ void pcg_matvec_em_kernel(int64_t nv, int64_t nvp, const T* __restrict__ Y, const T* __restrict__ p,
                                     T* __restrict__ q, double* red, unsigned int* counter, double* scal) {
  if (scal[S_DONE] != 0.0) return;
  double v[1] = {0.0};
  em_sum_loop<T, 1>(nv, nvp, Y, q, p, v);
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    scal[S_PQ] = out[0];
    if (!(out[0] > 0.0)) {  // breakdown: H not SPD on the Krylov space
      scal[S_BAD] = 1.0;
      scal[S_DONE] = 1.0;
      scal[S_ALPHA] = 0.0;
    } else {
      scal[S_ALPHA] = scal[S_RZ] / out[0];
    }
  }
}

// v = H ph from the element pass;  alpha = rho / (rhat . v)
template <typename T>
__global__ void bicg_v_em_kernel(int64_t nv, int64_t nvp, const T* __restrict__ Y, BicgVecs<T> V, double* red,
                                 unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  double v[1] = {0.0};
  em_sum_loop<T, 1>(nv, nvp, Y, V.v, V.rh, v);
  double out[1];
  if (grid_reduce<1>(v, red, counter, out) && threadIdx.x == 0) {
    if (out[0] == 0.0 || !isfinite(out[0])) {
      scal[B_BAD] = 1.0;
      scal[B_DONE] = 1.0;
      scal[B_ALPHA] = 0.0;
    } else {
      scal[B_ALPHA] = scal[B_RHO] / out[0];
    }
  }
}

// t = H sh from the element pass;  omega = (t.s) / (t.t)
template <typename T>
__global__ void bicg_t_em_kernel(int64_t nv, int64_t nvp, const T* __restrict__ Y, BicgVecs<T> V, double* red,
                                 unsigned int* counter, double* scal) {
  if (scal[B_DONE] != 0.0) return;
  double v[2] = {0.0, 0.0};
  em_sum_loop<T, 2>(nv, nvp, Y, V.t, V.s, v);
  double out[2];
  if (grid_reduce<2>(v, red, counter, out) && threadIdx.x == 0) scal[B_OMEGA] = (out[1] > 0.0) ? out[0] / out[1] : 0.0;
}

#undef HDG_LD
#undef HDG_ST

// y = H x on the free faces, 0 on Dirichlet faces
template <int D2>
__global__ void apply_kernel(FaceArgs F, const double* __restrict__ C, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t tile = blockIdx.x; tile < ntiles<D2>(F); tile += gridDim.x) {
    Tile<D2> T_(F, tile);
    if (!T_.act) continue;
    y[T_.t] = (F.ftype[T_.e] != 1) ? face_apply<double, D2>(C, x, F, T_.e, T_.a) : 0.0;
  }
}

// zero the Dirichlet entries of a caller's initial guess (the unknowns are the free faces)
__global__ void mask_dirichlet_kernel(int64_t ntot, const int32_t* ftype, int d2, double* x) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntot; t += (int64_t)gridDim.x * blockDim.x)
    if (ftype[t / d2] == 1) x[t] = 0.0;
}

__global__ void finish_kernel(int64_t ntot, const int32_t* ftype, int d2, const double* x, const double* xD,
                              double* uhat) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntot; t += (int64_t)gridDim.x * blockDim.x)
    uhat[t] = (ftype[t / d2] == 1) ? xD[t] : x[t];
}

__global__ void axpy_f32_kernel(int64_t n, const float* __restrict__ d, double* __restrict__ x) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    x[t] += (double)d[t];
}

// ------------------------------------------------------------------ host side
static FaceArgs face_args(hdg_mesh* M) {
  FaceArgs F;
  F.owner = M->d_owner;
  F.fbe = M->d_facebyele;
  F.ftype = M->d_ftype;
  F.nfc = M->nfc;
  return F;
}

// blocks of the face kernels: persistent grid over tiles of kNT / d2 whole faces
static int nblocks(hdg_mesh* M) {
  const int fpb = kNT / M->tab.d2;
  const int64_t tiles = (M->nfc + fpb - 1) / fpb;
  const int64_t cap = std::min<int64_t>(M->face_blocks, kMaxBlocks);
  return (int)(tiles < cap ? tiles : cap);
}

// the FP32 inner solve has its own persistent grid (hdg_autotune tunes both)
template <typename T>
static int nblocks_t(hdg_mesh* M) {
  if (sizeof(T) == 8) return nblocks(M);
  const int save = M->face_blocks;
  M->face_blocks = M->face_blocks32;
  const int nb = nblocks(M);
  M->face_blocks = save;
  return nb;
}

// shared-memory copy of the V-cycle's tail (set before any capture of the kernel)
static int grid_levels(const Coarse* c);
static void prepare_tail(hdg_mesh* M) {
  Coarse* c = M->coarse;
  const int G = grid_levels(c);
  int64_t bytes = 0;
  for (int l = G; l < c->nlev; ++l) bytes += tail_level_bytes(c->lv[l]);
  const bool fits = c->nlev - G <= kMaxTailLevels && bytes <= kTailSmemMax &&
                    cudaFuncSetAttribute(vcycle_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
                        cudaSuccess;
  cudaGetLastError();
  c->tail_smem = fits ? bytes : 0;
}

static CoarseArgs coarse_args(hdg_mesh* M) {
  prepare_tail(M);
  const Coarse* c = M->coarse;
  CoarseArgs a;
  a.fverts = M->d_fverts;
  a.Tf = c->Tf;
  a.vnodes = c->vnodes;
  a.vw = c->vw;
  a.rc = c->rc;
  a.e0 = c->e0;
  a.n0 = c->lv[0].n;
  a.gptr = c->gptr;
  a.gfi = c->gfi;
  a.gw = c->gw;
  a.fnode = c->fnode;
  a.fwt = c->fwt;
  return a;
}

// number of levels run as grid kernels: level 0 and the following levels above tail_max nodes
static int grid_levels(const Coarse* c) {
  int G = 1;
  while (G < c->nlev - 1 && c->lv[G].n > c->tail_max) ++G;
  return G;
}

// kernels of one coarse correction (restriction of r, V-cycle): 2 G + 2
static int coarse_cycle_kernels(const Coarse* c) { return 2 * grid_levels(c) + 2; }

// restriction of r and one V-cycle: grid levels down, the single-CTA tail, grid levels up
template <typename T, int D2>
static void coarse_cycle(hdg_mesh* M, const CoarseArgs& CA, const T* r, cudaStream_t st, const double* done) {
  Coarse* c = M->coarse;
  const int G = grid_levels(c);
  // the level kernels loop over their rows when the grid is capped (HDG_FACE_BLOCKS caps it
  // further in the tests, to exercise those loops on small meshes)
  const int64_t cap = M->grid_cap > 0 ? std::min<int64_t>(M->grid_cap, kMaxBlocks) : kMaxBlocks;
  auto grid = [cap](int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, cap); };
  auto rows = [cap](int64_t n) { return (int)std::min<int64_t>((n * kRowLanes + 255) / 256, cap); };
  const int gr = (int)std::min<int64_t>({(c->lv[0].n + 7) / 8, (int64_t)152 * 16, cap});  // one warp per node
  restrict_gather_kernel<T, D2><<<gr, 256, 0, st>>>(CA, r, done);
  level_down_kernel<true><<<rows(c->lv[0].n), 256, 0, st>>>(c->lv[0], c->rc, done);
  for (int l = 1; l < G; ++l) {
    level_restrict_kernel<<<grid(c->lv[l].n), 256, 0, st>>>(c->lv[l - 1], c->lv[l], done);
    level_down_kernel<false><<<rows(c->lv[l].n), 256, 0, st>>>(c->lv[l], nullptr, done);
  }
  vcycle_kernel<<<1, kVcThreads, c->tail_smem, st>>>(c->d_lv, G, c->nlev, c->Ainv, done, c->tail_smem > 0);
  for (int l = G - 1; l >= 0; --l) {
    const float* xn = (l + 1 == G) ? c->lv[G].x : c->lv[l + 1].t;
    float* out = (l == 0) ? c->e0 : c->lv[l].t;
    if (l == 0)
      level_up_kernel<true><<<rows(c->lv[0].n), 256, 0, st>>>(c->lv[0], xn, c->rc, out, done);
    else
      level_up_kernel<false><<<rows(c->lv[l].n), 256, 0, st>>>(c->lv[l], xn, nullptr, out, done);
  }
}

// graphs captured with or without the coarse correction are not interchangeable
static void match_graphs(hdg_mesh* M, bool tl) {
  const int em = (M->em64 ? 2 : 0) | (M->em32 ? 1 : 0);  // nor are those of the two operator forms
  if (M->graphs_tl == tl && M->graphs_em == em) return;
  cudaGraphExec_t* gs[] = {&M->graph64, &M->graph32, &M->wgraph64, &M->wgraph32, &M->graph_bicg, &M->graph_bicg32,
                           &M->wgraph_bicg, &M->wgraph_bicg32};
  for (cudaGraphExec_t* g : gs)
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
  M->graphs_tl = tl;
  M->graphs_em = em;
}


static int64_t bicg_stride(int64_t nv, int w) { return (nv + w - 1) / w * w; }

// the element-pass output buffer of a precision
template <typename T>
static T* em_buf(hdg_mesh* M) {
  if constexpr (sizeof(T) == 8) return reinterpret_cast<T*>(M->d_Y);
  else return reinterpret_cast<T*>(M->d_Y32);
}

static int ensure_workspace(hdg_mesh* M, bool mixed) {
  const int64_t nv = M->nfc * M->tab.d2;
  if (!M->d_b) {
    HDG_CUDA_TRY(cudaMalloc(&M->d_b, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_x, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_r, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_z, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_p, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_q, sizeof(double) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_uhatD, sizeof(double) * 2 * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_BJ, sizeof(double) * M->nfc * M->tab.d2 * M->tab.d2));
    HDG_CUDA_TRY(cudaMalloc(&M->d_red, sizeof(double) * 4 * kMaxBlocks));
    HDG_CUDA_TRY(cudaMalloc(&M->d_scal, sizeof(double) * 2 * S_NSCAL));
    HDG_CUDA_TRY(cudaMalloc(&M->d_counter, sizeof(unsigned int) * 4));
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_counter, 0, sizeof(unsigned int) * 4, M->stream));
    // element-pass outputs [2 sides][nvp], FP64 and FP32: the entries that the pass never stores
    // (Dirichlet rows, side 1 of the boundary faces) stay 0
    const int64_t nvp = bicg_stride(M->nfc * M->tab.d2, 4);
    HDG_CUDA_TRY(cudaMalloc(&M->d_Y, sizeof(double) * 2 * nvp));
    HDG_CUDA_TRY(cudaMalloc(&M->d_Y32, sizeof(float) * 2 * nvp));
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_Y, 0, sizeof(double) * 2 * nvp, M->stream));
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_Y32, 0, sizeof(float) * 2 * nvp, M->stream));
    M->red_blocks = kMaxBlocks;
  }
  if (M->beta_q && !M->d_bicg) HDG_CUDA_TRY(cudaMalloc(&M->d_bicg, sizeof(double) * 4 * bicg_stride(nv, 2)));
  if (M->beta_q && mixed && !M->d_bicg32)
    HDG_CUDA_TRY(cudaMalloc(&M->d_bicg32, sizeof(float) * 4 * bicg_stride(nv, 4)));
  if (mixed && !M->d_C32) {
    HDG_CUDA_TRY(cudaMalloc(&M->d_C32, sizeof(float) * M->nelt * M->tab.m * M->tab.m));
    HDG_CUDA_TRY(cudaMalloc(&M->d_BJ32, sizeof(float) * M->nfc * M->tab.d2 * M->tab.d2));
    HDG_CUDA_TRY(cudaMalloc(&M->d_r32, sizeof(float) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_x32, sizeof(float) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_z32, sizeof(float) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_p32, sizeof(float) * nv));
    HDG_CUDA_TRY(cudaMalloc(&M->d_q32, sizeof(float) * nv));
  }
  return HDG_OK;
}

// Build an executable graph that runs `body` (a capture callback on stream cs) inside a
// conditional WHILE node; the body must end with loop_control_kernel on the same handle.
// Returns false (and leaves *exec null) if the driver refuses conditional nodes.
template <typename BodyFn>
static bool build_while_graph(cudaStream_t cs, cudaGraphExec_t* exec, BodyFn body) {
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
  cudaGraphConditionalHandle h;
  bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraphNode_t node;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  ok = ok && cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  if (ok) {
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      body(cs, h);
      cudaGraph_t out = nullptr;
      ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
  }
  ok = ok && cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
  cudaGraphDestroy(g);
  if (!ok) {
    *exec = nullptr;
    cudaGetLastError();
  }
  return ok;
}

template <int D2>
struct Solver {
  // Boundary data, block-Jacobi inverse and right-hand side (once per assembled system).
  static int prepare_rhs(hdg_mesh* M) {
    if (M->rhs_ready) return HDG_OK;
    FaceArgs F = face_args(M);
    const int64_t nv = M->nfc * D2;
    const int nb = nblocks(M);
    double* xD = M->d_uhatD;
    double* phiN = M->d_uhatD + nv;
    bdata_kernel<D2><<<nb, kNT, 0, M->stream>>>(F, M->d_fvx, M->d_vx, M->nelt, M->dt.D, M->dt.face_w, M->tab.nf,
                                                M->uD, M->gN, xD, phiN);
    rhs_kernel<D2><<<nb, kNT, 0, M->stream>>>(F, M->d_C, M->d_Cf, xD, phiN, M->d_b, M->d_red, M->d_counter,
                                              M->d_scal);
    M->launches += 2;
    HDG_CUDA_TRY(cudaGetLastError());
    double bb;
    HDG_CUDA_TRY(cudaMemcpyAsync(&bb, M->d_scal + S_BB, sizeof(double), cudaMemcpyDeviceToHost, M->stream));
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    M->bnorm = std::sqrt(bb);
    M->rhs_ready = true;
    M->bj64_ready = M->bj32_ready = false;
    return HDG_OK;
  }

  // Block-Jacobi inverses of the current assembly, in the precision of the solve that uses
  // them (the FP32 inner solve computes its own in FP32); a non-SPD block counts in status[3].
  template <typename TB>
  static int ensure_bj(hdg_mesh* M) {
    const bool f32 = sizeof(TB) == 4;
    if (f32 ? M->bj32_ready : M->bj64_ready) return HDG_OK;
    int rc = ensure_workspace(M, f32);
    if (rc) return rc;
    TB* out = f32 ? reinterpret_cast<TB*>(M->d_BJ32) : reinterpret_cast<TB*>(M->d_BJ);
    bj_kernel<D2, TB><<<(unsigned)((M->nfc + 63) / 64), 64, 0, M->stream>>>(face_args(M), M->d_C, out, M->d_status,
                                                                           M->beta_q != nullptr);
    M->launches++;
    HDG_CUDA_TRY(cudaGetLastError());
    (f32 ? M->bj32_ready : M->bj64_ready) = true;
    return HDG_OK;
  }

  // One PCG solve of H_T x = rhs to ||r|| <= sqrt(tol2) (absolute), T in {double, float}.
  template <typename T>
  static int pcg_run(hdg_mesh* M, const T* C, const T* Binv, const T* rhs, T* x, bool have_x, T* r, T* z, T* p,
                     T* q, double* scal, double tol2, int maxit, cudaGraphExec_t* graph, int* iters, bool* bad) {
    FaceArgs F = face_args(M);
    const int nb = nblocks_t<T>(M);
    const int64_t nv = M->nfc * D2;
    double hs[S_NSCAL] = {0};
    hs[S_TOL2] = tol2;
    hs[S_MAXIT] = (double)maxit;
    hs[S_MAXBODIES] = (double)(maxit / kGraphIters + 2);  // bound of the device-driven loop
    HDG_CUDA_TRY(cudaMemcpyAsync(scal, hs, sizeof(hs), cudaMemcpyHostToDevice, M->stream));
    const bool tl = M->coarse != nullptr && M->coarse->ready;
    match_graphs(M, tl);
    const CoarseArgs CA = tl ? coarse_args(M) : CoarseArgs{};
    const bool em = sizeof(T) == 8 ? M->em64 : M->em32;
    T* Y = em_buf<T>(M);
    const int64_t nvp = bicg_stride(M->nfc * D2, 4);
    const int eg = em ? em_grid<T, D2>(M) : 0;
    const int per_it = (tl ? 4 + coarse_cycle_kernels(M->coarse) : 3) + (em ? 1 : 0);  // kernels per iteration
    pcg_init_kernel<T, D2><<<nb, kNT, 0, M->stream>>>(F, C, rhs, x, have_x, r, M->d_red, M->d_counter, scal);
    if (tl) {
      coarse_cycle<T, D2>(M, CA, r, M->stream, scal + S_DONE);
      pcg_zc_kernel<T, D2, true><<<nb, kNT, 0, M->stream>>>(F, CA, Binv, r, z, p, M->d_red, M->d_counter, scal);
      M->launches += 2 + coarse_cycle_kernels(M->coarse);
    } else {
      pcg_precond_kernel<T, D2><<<nb, kNT, 0, M->stream>>>(F, Binv, r, z, p, M->d_red, M->d_counter, scal);
      M->launches += 2;
    }
    HDG_CUDA_TRY(cudaGetLastError());
    if (!M->cap_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = M->cap_stream;
    auto iteration = [&](cudaStream_t st) {
      if (em) {
        em_apply_kernel<T, D2><<<eg, EmPass<T, D2>::NTHR, EmPass<T, D2>::SMEM, st>>>(C, p, M->d_fslot, M->nelt, nvp,
                                                                                   Y, scal + S_DONE, M->d_status);
        pcg_matvec_em_kernel<T><<<nb, kNT, 0, st>>>(nv, nvp, Y, p, q, M->d_red, M->d_counter, scal);
      } else {
        pcg_matvec_kernel<T, D2><<<nb, kNT, 0, st>>>(F, C, p, q, M->d_red, M->d_counter, scal);
      }
      if (tl) {
        pcg_update_tl_kernel<T, D2><<<nb, kNT, 0, st>>>(F, x, r, p, q, M->d_red, M->d_counter, scal);
        coarse_cycle<T, D2>(M, CA, r, st, scal + S_DONE);
        pcg_zc_kernel<T, D2, false><<<nb, kNT, 0, st>>>(F, CA, Binv, r, z, p, M->d_red, M->d_counter, scal);
      } else {
        pcg_update_kernel<T, D2><<<nb, kNT, 0, st>>>(F, Binv, x, r, z, p, q, M->d_red, M->d_counter, scal);
      }
      pcg_dir_kernel<T><<<nb, kNT, 0, st>>>(nv, z, p, scal);
    };
    auto body = [&](cudaStream_t st, cudaGraphConditionalHandle h) {
      for (int it = 0; it < kGraphIters; ++it) iteration(st);
      loop_control_kernel<<<1, 32, 0, st>>>(h, scal, S_DONE, S_BODIES, S_MAXBODIES);
    };
    cudaGraphExec_t* wg = (sizeof(T) == 8) ? &M->wgraph64 : &M->wgraph32;
    if (!*wg && !M->no_cond_graphs) {
      if (!build_while_graph(cs, wg, body)) M->no_cond_graphs = true;
    }
    double hv[S_NSCAL];
    if (*wg) {
      // device-driven loop: one graph launch runs the iterations until convergence
      HDG_CUDA_TRY(cudaGraphLaunch(*wg, M->stream));
      M->launches += 1;
      HDG_CUDA_TRY(cudaMemcpyAsync(hv, scal, sizeof(hv), cudaMemcpyDeviceToHost, M->stream));
      HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
      M->launches += (int64_t)(per_it * kGraphIters + 1) * (int64_t)hv[S_BODIES];
    } else {
      if (!*graph) {
        // capture on a private stream (the caller's may be the legacy default stream, which
        // cannot be captured); the graph is then launched on the caller's stream
        cudaGraph_t g;
        HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < kGraphIters; ++it) iteration(cs);
        HDG_CUDA_TRY(cudaStreamEndCapture(cs, &g));
        HDG_CUDA_TRY(cudaGraphInstantiate(graph, g, 0));
        cudaGraphDestroy(g);
      }
      for (;;) {
        HDG_CUDA_TRY(cudaMemcpyAsync(hv, scal, sizeof(hv), cudaMemcpyDeviceToHost, M->stream));
        HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
        if (hv[S_DONE] != 0.0) break;
        HDG_CUDA_TRY(cudaGraphLaunch(*graph, M->stream));
        M->launches += per_it * kGraphIters;
      }
    }
    *iters = (int)hv[S_ITERS];
    *bad = hv[S_BAD] != 0.0;
    return HDG_OK;
  }

  // One BiCGStab solve of H_T x = rhs to ||r|| <= sqrt(tol2) (absolute), T in {double, float},
  // block-Jacobi or two-level right preconditioning; the iterations run in a device-driven
  // conditional WHILE loop (host-driven replays when the driver refuses conditional nodes).
  template <typename T>
  static int bicg_run(hdg_mesh* M, const T* C, const T* Binv, const T* rhs, BicgVecs<T> V, bool have_x,
                      double* scal, double tol2, int maxit, cudaGraphExec_t* graph, cudaGraphExec_t* wg,
                      int* iters, bool* bad) {
    FaceArgs F = face_args(M);
    const int nb = nblocks_t<T>(M);
    double hs[B_NSCAL] = {0};
    hs[B_TOL2] = tol2;
    hs[B_MAXIT] = (double)maxit;
    hs[B_MAXBODIES] = (double)(maxit / kGraphIters + 2);  // bound of the device-driven loop
    HDG_CUDA_TRY(cudaMemcpyAsync(scal, hs, sizeof(hs), cudaMemcpyHostToDevice, M->stream));
    const bool tl = M->coarse != nullptr && M->coarse->ready;
    match_graphs(M, tl);
    const CoarseArgs CA = tl ? coarse_args(M) : CoarseArgs{};
    const bool em = sizeof(T) == 8 ? M->em64 : M->em32;
    T* Y = em_buf<T>(M);
    const int64_t nvp = bicg_stride(M->nfc * D2, 4);
    const int eg = em ? em_grid<T, D2>(M) : 0;
    const int per_it = (tl ? 7 + 2 * coarse_cycle_kernels(M->coarse) : 5) + (em ? 2 : 0);  // kernels per iteration
    bicg_init_kernel<T, D2><<<nb, kNT, 0, M->stream>>>(F, C, rhs, V, have_x, M->d_red, M->d_counter, scal);
    M->launches++;
    HDG_CUDA_TRY(cudaGetLastError());
    if (!M->cap_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = M->cap_stream;
    const int64_t nv = M->nfc * D2;
    auto iteration = [&](cudaStream_t st) {
      if (tl) {
        bicg_p_flat_kernel<T><<<nb, kNT, 0, st>>>(nv, V, scal);
        coarse_cycle<T, D2>(M, CA, V.p, st, scal + B_DONE);
        bicg_tl_kernel<T, D2, B_DONE><<<nb, kNT, 0, st>>>(F, CA, Binv, V.p, V.ph, scal);
      } else {
        bicg_p_kernel<T, D2, false><<<nb, kNT, 0, st>>>(F, Binv, V, scal);
      }
      if (em) {
        em_apply_kernel<T, D2><<<eg, EmPass<T, D2>::NTHR, EmPass<T, D2>::SMEM, st>>>(C, V.ph, M->d_fslot, M->nelt,
                                                                                   nvp, Y, scal + B_DONE, M->d_status);
        bicg_v_em_kernel<T><<<nb, kNT, 0, st>>>(nv, nvp, Y, V, M->d_red, M->d_counter, scal);
      } else {
        bicg_v_kernel<T, D2><<<nb, kNT, 0, st>>>(F, C, V, M->d_red, M->d_counter, scal);
      }
      if (tl) {
        bicg_s_flat_kernel<T><<<nb, kNT, 0, st>>>(nv, V, scal);
        coarse_cycle<T, D2>(M, CA, V.s, st, scal + B_DONE);
        bicg_tl_kernel<T, D2, B_DONE><<<nb, kNT, 0, st>>>(F, CA, Binv, V.s, V.sh, scal);
      } else {
        bicg_s_kernel<T, D2, false><<<nb, kNT, 0, st>>>(F, Binv, V, scal);
      }
      if (em) {
        em_apply_kernel<T, D2><<<eg, EmPass<T, D2>::NTHR, EmPass<T, D2>::SMEM, st>>>(C, V.sh, M->d_fslot, M->nelt,
                                                                                   nvp, Y, scal + B_DONE, M->d_status);
        bicg_t_em_kernel<T><<<nb, kNT, 0, st>>>(nv, nvp, Y, V, M->d_red, M->d_counter, scal);
      } else {
        bicg_t_kernel<T, D2><<<nb, kNT, 0, st>>>(F, C, V, M->d_red, M->d_counter, scal);
      }
      bicg_x_flat_kernel<T><<<nb, kNT, 0, st>>>(nv, V, M->d_red, M->d_counter, scal);
    };
    auto body = [&](cudaStream_t st, cudaGraphConditionalHandle h) {
      for (int it = 0; it < kGraphIters; ++it) iteration(st);
      loop_control_kernel<<<1, 32, 0, st>>>(h, scal, B_DONE, B_BODIES, B_MAXBODIES);
    };
    if (!*wg && !M->no_cond_graphs) {
      if (!build_while_graph(cs, wg, body)) M->no_cond_graphs = true;
    }
    double hv[B_NSCAL];
    if (*wg) {
      HDG_CUDA_TRY(cudaGraphLaunch(*wg, M->stream));
      M->launches += 1;
      HDG_CUDA_TRY(cudaMemcpyAsync(hv, scal, sizeof(hv), cudaMemcpyDeviceToHost, M->stream));
      HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
      M->launches += (int64_t)(per_it * kGraphIters + 1) * (int64_t)hv[B_BODIES];
    } else {
      if (!*graph) {
        cudaGraph_t g;
        HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < kGraphIters; ++it) iteration(cs);
        HDG_CUDA_TRY(cudaStreamEndCapture(cs, &g));
        HDG_CUDA_TRY(cudaGraphInstantiate(graph, g, 0));
        cudaGraphDestroy(g);
      }
      for (;;) {
        HDG_CUDA_TRY(cudaMemcpyAsync(hv, scal, sizeof(hv), cudaMemcpyDeviceToHost, M->stream));
        HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
        if (hv[B_DONE] != 0.0) break;
        HDG_CUDA_TRY(cudaGraphLaunch(*graph, M->stream));
        M->launches += per_it * kGraphIters;
      }
    }
    *iters = (int)hv[B_ITERS];
    *bad = hv[B_BAD] != 0.0;
    return HDG_OK;
  }

  // the extra vectors s, t, ph, sh at strides rounded up to whole 16-byte units
  BicgVecs<double> static bicg_vecs64(hdg_mesh* M) {
    const int64_t sv = bicg_stride(M->nfc * D2, 2);
    return BicgVecs<double>{M->d_x, M->d_r, M->d_z, M->d_p, M->d_q, M->d_bicg, M->d_bicg + sv, M->d_bicg + 2 * sv,
                            M->d_bicg + 3 * sv};
  }
  BicgVecs<float> static bicg_vecs32(hdg_mesh* M) {
    const int64_t sv = bicg_stride(M->nfc * D2, 4);
    return BicgVecs<float>{M->d_x32, M->d_q32, M->d_z32, M->d_p32, reinterpret_cast<float*>(M->d_q), M->d_bicg32,
                           M->d_bicg32 + sv, M->d_bicg32 + 2 * sv, M->d_bicg32 + 3 * sv};
  }

  // ||b - H x||_2 over the free dofs in FP64, r written to `r`.
  // (have_x false: x is zero, so r = b without the product)
  static int true_residual(hdg_mesh* M, const double* x, double* r, double* rnorm, bool have_x = true) {
    FaceArgs F = face_args(M);
    const int nb = nblocks(M);
    double* scal = M->d_scal + S_NSCAL;
    pcg_init_kernel<double, D2><<<nb, kNT, 0, M->stream>>>(F, M->d_C, M->d_b, const_cast<double*>(x), have_x, r,
                                                           M->d_red, M->d_counter, scal);
    M->launches++;
    HDG_CUDA_TRY(cudaGetLastError());
    double rr;
    HDG_CUDA_TRY(cudaMemcpyAsync(&rr, scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, M->stream));
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    *rnorm = std::sqrt(rr);
    return HDG_OK;
  }

  // The FP64 solve from x (zero start unless have_x): BiCGStab with up to three restarted
  // passes when convection makes H non-symmetric, else PCG with one restarted pass when the
  // recursive residual converged but the true one did not.
  static int fp64_solve(hdg_mesh* M, bool have_x, double tol, int maxit, int* total_it, bool* converged, bool* bad,
                        double* rnorm) {
    const double bnorm = M->bnorm;
    int rc;
    *total_it = 0;
    *converged = false;
    *bad = false;
    if (M->beta_q) {
      for (int pass = 0; pass < 3 && !*converged && *total_it < maxit; ++pass) {
        int it;
        rc = bicg_run<double>(M, M->d_C, M->d_BJ, M->d_b, bicg_vecs64(M), have_x, M->d_scal, tol * tol,
                              maxit - *total_it, &M->graph_bicg, &M->wgraph_bicg, &it, bad);
        if (rc) return rc;
        *total_it += it;
        rc = true_residual(M, M->d_x, M->d_q, rnorm);
        if (rc) return rc;
        *converged = *rnorm <= tol * 1.0000001 || bnorm == 0.0;
        have_x = true;  // restart from the current iterate if the recursive residual drifted
        if (*bad && !*converged) *bad = false;
      }
      return HDG_OK;
    }
    int it;
    rc = pcg_run<double>(M, M->d_C, M->d_BJ, M->d_b, M->d_x, have_x, M->d_r, M->d_z, M->d_p, M->d_q, M->d_scal,
                         tol * tol, maxit, &M->graph64, &it, bad);
    if (rc) return rc;
    *total_it = it;
    rc = true_residual(M, M->d_x, M->d_q, rnorm);
    if (rc) return rc;
    *converged = *rnorm <= tol * 1.0000001 || bnorm == 0.0;
    if (!*converged && it < maxit && !*bad) {
      rc = pcg_run<double>(M, M->d_C, M->d_BJ, M->d_b, M->d_x, true, M->d_r, M->d_z, M->d_p, M->d_q, M->d_scal,
                           tol * tol, maxit - it, &M->graph64, &it, bad);
      if (rc) return rc;
      *total_it += it;
      rc = true_residual(M, M->d_x, M->d_q, rnorm);
      if (rc) return rc;
      *converged = *rnorm <= tol * 1.0000001;
    }
    return HDG_OK;
  }

  static int solve(hdg_mesh* M, int precision, double rtol, int maxit, const double* x0, double* uhat, int* iters,
                   double* relres) {
    const bool mixed = precision == HDG_MIXED_FP32;
    int rc = ensure_workspace(M, mixed);
    if (rc) return rc;
    rc = prepare_rhs(M);
    if (rc) return rc;
    const int64_t nv = M->nfc * D2;
    const int nb = nblocks(M);
    const double bnorm = M->bnorm;
    const double tol = rtol * bnorm;
    int total_it = 0;
    bool converged = false, bad = false;
    double rnorm = 0.0;
    if (mixed && !M->c32_ready) {  // FP32 copy of C^K (also read by the coarse set-up below)
      convert_c32_kernel<D2><<<1216, 256, 0, M->stream>>>(M->d_C, M->d_C32, M->nelt);
      M->launches++;
      M->c32_ready = true;
    }
    if (M->coarse && !M->coarse->ready) {
      rc = coarse_build(M);
      if (rc) return rc;
    }
    rc = mixed ? ensure_bj<float>(M) : ensure_bj<double>(M);
    if (rc) return rc;
    if (x0) {
      HDG_CUDA_TRY(cudaMemcpyAsync(M->d_x, x0, sizeof(double) * nv, cudaMemcpyDeviceToDevice, M->stream));
      mask_dirichlet_kernel<<<nb, kNT, 0, M->stream>>>(nv, M->d_ftype, D2, M->d_x);
      M->launches++;
    }
    if (!mixed) {
      rc = fp64_solve(M, x0 != nullptr, tol, maxit, &total_it, &converged, &bad, &rnorm);
      if (rc) return rc;
    } else {
      // mixed: FP32 copies of C^K and the block inverses, FP64 outer residual and update
      if (!x0) HDG_CUDA_TRY(cudaMemsetAsync(M->d_x, 0, sizeof(double) * nv, M->stream));
      double prev = INFINITY;
      bool fallback = false;
      for (int outer = 0; outer < 30; ++outer) {
        rc = true_residual(M, M->d_x, M->d_r, &rnorm, outer > 0 || x0 != nullptr);
        if (rc) return rc;
        if (rnorm <= tol || bnorm == 0.0) {
          converged = true;
          bad = false;
          break;
        }
        if (outer > 0 && !(rnorm < prev)) {
          // the last FP32 correction did not reduce the FP64 residual (the FP32 iteration
          // stagnated or diverged): undo it and finish in FP64 from the previous iterate
          HDG_CUDA_TRY(cudaMemcpyAsync(M->d_x, M->d_z, sizeof(double) * nv, cudaMemcpyDeviceToDevice, M->stream));
          rnorm = prev;
          fallback = true;
          break;
        }
        if (total_it >= maxit) break;
        // an inner breakdown still leaves a usable iterate: the outer step keeps it and restarts
        // the inner solve from the new FP64 residual
        bad = false;
        prev = rnorm;
        HDG_CUDA_TRY(cudaMemcpyAsync(M->d_z, M->d_x, sizeof(double) * nv, cudaMemcpyDeviceToDevice, M->stream));
        convert_kernel<float><<<304, 256, 0, M->stream>>>(M->d_r, M->d_r32, nv);
        M->launches++;
        int it;
        // each inner solve reduces its residual by inner_rtol, but no further than half the
        // remaining distance to the outer target (the last step stops as soon as it suffices)
        const double itol = std::max(M->inner_rtol * rnorm, 0.5 * tol);
        if (M->beta_q)  // convection: FP32 inner BiCGStab
          rc = bicg_run<float>(M, M->d_C32, M->d_BJ32, M->d_r32, bicg_vecs32(M), false, M->d_scal, itol * itol,
                               maxit - total_it, &M->graph_bicg32, &M->wgraph_bicg32, &it, &bad);
        else
          rc = pcg_run<float>(M, M->d_C32, M->d_BJ32, M->d_r32, M->d_x32, false, M->d_q32, M->d_z32, M->d_p32,
                              reinterpret_cast<float*>(M->d_q), M->d_scal, itol * itol, maxit - total_it,
                              &M->graph32, &it, &bad);
        if (rc) return rc;
        total_it += it;
        axpy_f32_kernel<<<nb, kNT, 0, M->stream>>>(nv, M->d_x32, M->d_x);
        M->launches++;
      }
      if (fallback && total_it < maxit) {
        rc = ensure_bj<double>(M);
        if (rc) return rc;
        int it64 = 0;
        rc = fp64_solve(M, true, tol, maxit - total_it, &it64, &converged, &bad, &rnorm);
        if (rc) return rc;
        total_it += it64;
      }
    }
    finish_kernel<<<nb, kNT, 0, M->stream>>>(nv, M->d_ftype, D2, M->d_x, M->d_uhatD, uhat);
    M->launches++;
    HDG_CUDA_TRY(cudaGetLastError());
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    if (iters) *iters = total_it;
    if (relres) *relres = bnorm > 0 ? rnorm / bnorm : 0.0;
    if (bad) return fail(HDG_ERR_NOT_CONVERGED, "Krylov breakdown");
    if (!converged)
      return fail(HDG_ERR_NOT_CONVERGED, "trace solve reached maxit with relative residual " +
                                             std::to_string(bnorm > 0 ? rnorm / bnorm : 0.0));
    return HDG_OK;
  }

  // Time one block-Jacobi PCG iteration (operator, update with its reductions, direction) in
  // FP64 for persistent grids of 4, 8, 16 and 32 blocks per SM; keep the fastest.  Cached
  // graphs are rebuilt when the grid changes.
  static int autotune(hdg_mesh* M, hdg_tuning* out) {
    int rc = ensure_workspace(M, false);
    if (rc) return rc;
    rc = prepare_rhs(M);
    if (rc) return rc;
    rc = ensure_bj<double>(M);
    if (rc) return rc;
    const int old = M->face_blocks;
    const int64_t nv = M->nfc * D2;
    const int cands[] = {152 * 4, 152 * 8, 152 * 16, 152 * 32};
    double* scal = M->d_scal + S_NSCAL;  // scratch scalars: never done, so every kernel runs
    double hs[S_NSCAL] = {0};
    hs[S_TOL2] = -1.0;
    hs[S_MAXIT] = 1e30;
    hs[S_RZ] = 1.0;
    HDG_CUDA_TRY(cudaMemcpyAsync(scal, hs, sizeof(hs), cudaMemcpyHostToDevice, M->stream));
    HDG_CUDA_TRY(cudaMemcpyAsync(M->d_p, M->d_b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, M->stream));
    HDG_CUDA_TRY(cudaMemcpyAsync(M->d_r, M->d_b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, M->stream));
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_x, 0, sizeof(double) * nv, M->stream));
    cudaEvent_t a, b;
    HDG_CUDA_TRY(cudaEventCreate(&a));
    HDG_CUDA_TRY(cudaEventCreate(&b));
    int best = old;
    float best_t = 1e30f;
    FaceArgs F = face_args(M);
    const int eg = em_grid<double, D2>(M), eg32 = em_grid<float, D2>(M);
    const int64_t nvp = bicg_stride(nv, 4);
    double* Y = M->d_Y;
    bool best_em = M->em64;
    auto iteration = [&](int nb, bool em) {
      if (em) {
        em_apply_kernel<double, D2><<<eg, EmPass<double, D2>::NTHR, EmPass<double, D2>::SMEM, M->stream>>>(
            M->d_C, M->d_p, M->d_fslot, M->nelt, nvp, Y, scal + S_DONE, M->d_status);
        pcg_matvec_em_kernel<double><<<nb, kNT, 0, M->stream>>>(nv, nvp, Y, M->d_p, M->d_q, M->d_red, M->d_counter,
                                                                scal);
      } else {
        pcg_matvec_kernel<double, D2><<<nb, kNT, 0, M->stream>>>(F, M->d_C, M->d_p, M->d_q, M->d_red, M->d_counter,
                                                                 scal);
      }
      pcg_update_kernel<double, D2><<<nb, kNT, 0, M->stream>>>(F, M->d_BJ, M->d_x, M->d_r, M->d_z, M->d_p, M->d_q,
                                                               M->d_red, M->d_counter, scal);
      pcg_dir_kernel<double><<<nb, kNT, 0, M->stream>>>(nv, M->d_z, M->d_p, scal);
    };
    for (int form = 0; form < 2; ++form) {
      const bool em = form == 1;
      if (M->em_forced && em != M->em64) continue;
      for (int cand : cands) {
        M->face_blocks = cand;
        const int nb = nblocks(M);
        iteration(nb, em);  // warm-up
        HDG_CUDA_TRY(cudaEventRecord(a, M->stream));
        for (int rep = 0; rep < 4; ++rep) iteration(nb, em);
        HDG_CUDA_TRY(cudaEventRecord(b, M->stream));
        HDG_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        HDG_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        M->launches += em ? 20 : 15;
        if (ms < best_t) {
          best_t = ms;
          best = cand;
          best_em = em;
        }
      }
    }
    M->face_blocks = best;
    // the same for the FP32 inner iteration (mixed precision), on FP32 copies of C^K and B^-1
    int best32 = M->face_blocks32;
    float best32_t = 1e30f;
    bool best32_em = M->em32;
    {
      rc = ensure_workspace(M, true);
      if (rc) return rc;
      if (!M->c32_ready) {
        convert_c32_kernel<D2><<<1216, 256, 0, M->stream>>>(M->d_C, M->d_C32, M->nelt);
        M->c32_ready = true;
      }
      rc = ensure_bj<float>(M);
      if (rc) return rc;
      convert_kernel<float><<<304, 256, 0, M->stream>>>(M->d_b, M->d_p32, nv);
      convert_kernel<float><<<304, 256, 0, M->stream>>>(M->d_b, M->d_r32, nv);
      HDG_CUDA_TRY(cudaMemsetAsync(M->d_x32, 0, sizeof(float) * nv, M->stream));
      HDG_CUDA_TRY(cudaMemcpyAsync(scal, hs, sizeof(hs), cudaMemcpyHostToDevice, M->stream));
      float* q32 = reinterpret_cast<float*>(M->d_q);
      float* Y32 = M->d_Y32;
      auto iteration32 = [&](int nb, bool em) {
        if (em) {
          em_apply_kernel<float, D2><<<eg32, EmPass<float, D2>::NTHR, EmPass<float, D2>::SMEM, M->stream>>>(
              M->d_C32, M->d_p32, M->d_fslot, M->nelt, nvp, Y32, scal + S_DONE, M->d_status);
          pcg_matvec_em_kernel<float><<<nb, kNT, 0, M->stream>>>(nv, nvp, Y32, M->d_p32, q32, M->d_red, M->d_counter,
                                                                 scal);
        } else {
          pcg_matvec_kernel<float, D2><<<nb, kNT, 0, M->stream>>>(F, M->d_C32, M->d_p32, q32, M->d_red,
                                                                  M->d_counter, scal);
        }
        pcg_update_kernel<float, D2><<<nb, kNT, 0, M->stream>>>(F, M->d_BJ32, M->d_x32, M->d_r32, M->d_z32,
                                                                M->d_p32, q32, M->d_red, M->d_counter, scal);
        pcg_dir_kernel<float><<<nb, kNT, 0, M->stream>>>(nv, M->d_z32, M->d_p32, scal);
      };
      const int keep = M->face_blocks;
      for (int form = 0; form < 2; ++form) {
        const bool em = form == 1;
        if (M->em_forced && em != M->em32) continue;
        for (int cand : cands) {
          M->face_blocks = cand;
          const int nb = nblocks(M);
          iteration32(nb, em);
          HDG_CUDA_TRY(cudaEventRecord(a, M->stream));
          for (int rep = 0; rep < 4; ++rep) iteration32(nb, em);
          HDG_CUDA_TRY(cudaEventRecord(b, M->stream));
          HDG_CUDA_TRY(cudaEventSynchronize(b));
          float ms = 0.f;
          HDG_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
          M->launches += em ? 20 : 15;
          if (ms < best32_t) {
            best32_t = ms;
            best32 = cand;
            best32_em = em;
          }
        }
      }
      M->face_blocks = keep;
      M->launches += 4;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const bool changed = best != old || best32 != M->face_blocks32 || best_em != M->em64 || best32_em != M->em32;
    M->face_blocks32 = best32;
    M->em64 = best_em;
    M->em32 = best32_em;
    if (changed) {
      cudaGraphExec_t* gs[] = {&M->graph64, &M->graph32, &M->wgraph64, &M->wgraph32, &M->graph_bicg,
                               &M->graph_bicg32, &M->wgraph_bicg, &M->wgraph_bicg32};
      for (cudaGraphExec_t* g : gs)
        if (*g) {
          cudaGraphExecDestroy(*g);
          *g = nullptr;
        }
    }
    if (out) {
      out->face_blocks = best;
      out->iter_ms = best_t / 4.0;
      out->face_blocks32 = best32;
      out->iter32_ms = best32_t < 1e29f ? best32_t / 4.0 : 0.0;
      out->matvec_em64 = best_em ? 1 : 0;
      out->matvec_em32 = best32_em ? 1 : 0;
    }
    return HDG_OK;
  }

  // z = B^-1 r + Pi V(Pi^T r): one application of the two-level preconditioner (FP64 vectors)
  static int precond_apply(hdg_mesh* M, const double* r, double* z) {
    int rc = ensure_workspace(M, false);
    if (rc) return rc;
    rc = prepare_rhs(M);
    if (rc) return rc;
    if (!M->coarse->ready) {
      rc = coarse_build(M);
      if (rc) return rc;
    }
    rc = ensure_bj<double>(M);
    if (rc) return rc;
    FaceArgs F = face_args(M);
    const int nb = nblocks(M);
    const CoarseArgs CA = coarse_args(M);
    double* scal = M->d_scal + S_NSCAL;
    HDG_CUDA_TRY(cudaMemsetAsync(scal, 0, sizeof(double) * S_NSCAL, M->stream));
    coarse_cycle<double, D2>(M, CA, r, M->stream, scal + S_DONE);
    pcg_zc_kernel<double, D2, true><<<nb, kNT, 0, M->stream>>>(F, CA, M->d_BJ, r, z, M->d_q, M->d_red, M->d_counter,
                                                               scal);
    M->launches += 1 + coarse_cycle_kernels(M->coarse);
    HDG_CUDA_TRY(cudaGetLastError());
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    return HDG_OK;
  }

  // y = H x in the operator form of the FP64 solve loops (face-major, or element pass + sum)
  static int apply(hdg_mesh* M, const double* x, double* y) {
    if (M->em64) {
      int rc = ensure_workspace(M, false);
      if (rc) return rc;
      double* never = M->d_scal + 2 * S_NSCAL - 1;  // a scratch slot, 0: the pass always runs
      HDG_CUDA_TRY(cudaMemsetAsync(never, 0, sizeof(double), M->stream));
      const int64_t nv = M->nfc * D2, nvp = bicg_stride(nv, 4);
      em_apply_kernel<double, D2><<<em_grid<double, D2>(M), EmPass<double, D2>::NTHR, EmPass<double, D2>::SMEM,
                                    M->stream>>>(M->d_C, x, M->d_fslot, M->nelt, nvp, M->d_Y, never, M->d_status);
      em_sum_kernel<double><<<nblocks(M), kNT, 0, M->stream>>>(nv, nvp, M->d_Y, y);
      M->launches += 2;
    } else {
      apply_kernel<D2><<<nblocks(M), kNT, 0, M->stream>>>(face_args(M), M->d_C, x, y);
      M->launches++;
    }
    HDG_CUDA_TRY(cudaGetLastError());
    return HDG_OK;
  }

  static int residual(hdg_mesh* M, const double* x, double* r, double* rnorm, double* bnorm) {
    int rc = ensure_workspace(M, false);
    if (rc) return rc;
    rc = prepare_rhs(M);
    if (rc) return rc;
    double rn;
    rc = true_residual(M, x, r, &rn);
    if (rc) return rc;
    if (rnorm) *rnorm = rn;
    if (bnorm) *bnorm = M->bnorm;
    return HDG_OK;
  }
};

// ------------------------------------------------------------------ batched graph
// Per-problem squared norms of a trace vector: out[p] += sum over the problem's free entries.
__global__ void prob_norms_kernel(const double* __restrict__ v, const int32_t* __restrict__ face_prob, int64_t nfc,
                                  int d2, double* out) {
  const int lane = threadIdx.x & 31;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nfc * d2; t += (int64_t)gridDim.x * blockDim.x) {
    const int p = face_prob[t / d2];
    double x = v[t] * v[t];
    // combine lanes of the same problem (problems occupy contiguous face ranges)
    const int p0 = __shfl_sync(0xffffffffu, p, 0);
    const bool uniform = __all_sync(__activemask(), p == p0);
    if (uniform && __activemask() == 0xffffffffu) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) atomicAdd(out + p, x);
    } else {
      atomicAdd(out + p, x);
    }
  }
}

// PCG scalars for the device-driven batch solve: the stopping threshold is
// (rtol * min_p ||b_p||)^2 so that every problem of the union meets rtol (||r_p|| <= ||r||).
__global__ void batch_scalars_kernel(double* scal, const double* bn2, int np, double rtol, int maxit, int graph_iters) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double mn = 1e300;
  for (int p = 0; p < np; ++p) mn = fmin(mn, bn2[p] > 0.0 ? bn2[p] : mn);
  if (!(mn < 1e300)) mn = 0.0;
  for (int i = 0; i < S_NSCAL; ++i) scal[i] = 0.0;
  scal[S_TOL2] = rtol * rtol * mn;
  scal[S_MAXIT] = (double)maxit;
  scal[S_MAXBODIES] = (double)(maxit / graph_iters + 2);
}

// Mixed-precision batch: control of the device-driven refinement loop.  After the FP64 residual
// r = b - H x (rr in so[S_RR]): stop when rr <= so[S_TOL2], after max_outer refinements or when
// the inner iterations reach so[S_MAXIT]; otherwise start an inner FP32 solve to inner_rtol.
__global__ void outer_check_kernel(cudaGraphConditionalHandle h_outer, cudaGraphConditionalHandle h_inner, double* so,
                                   double* si, double inner_rtol, int max_outer, int graph_iters) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double rr = so[S_RR];
  const double nb = so[S_BODIES] + 1.0;
  so[S_BODIES] = nb;
  const bool done = !(rr > so[S_TOL2]) || nb > (double)max_outer || so[S_ITERS] >= so[S_MAXIT];
  for (int i = 0; i < S_NSCAL; ++i) si[i] = 0.0;
  si[S_TOL2] = done ? 1e300 : inner_rtol * inner_rtol * rr;
  const double left = fmax(so[S_MAXIT] - so[S_ITERS], 1.0);
  si[S_MAXIT] = left;
  si[S_MAXBODIES] = floor(left / graph_iters) + 2.0;
  cudaGraphSetConditional(h_outer, done ? 0u : 1u);
  cudaGraphSetConditional(h_inner, done ? 0u : 1u);
}

// total inner iterations of the refinement
__global__ void outer_accum_kernel(double* so, const double* si) {
  if (blockIdx.x == 0 && threadIdx.x == 0) so[S_ITERS] += si[S_ITERS];
}

template <int D2>
static int record_group_mixed(hdg_mesh* M, cudaGraph_t graph, int asm_precision, const int32_t* face_prob, int np,
                              double* norms, double rtol, int maxit, double* q, double* u, double* uhat,
                              cudaGraphNode_t* last);

template <int D2>
static int record_group(hdg_mesh* M, cudaGraph_t graph, int asm_precision, int solve_precision,
                        const int32_t* face_prob, int np, double* norms, double rtol, int maxit, double* q, double* u,
                        double* uhat, cudaGraphNode_t* last) {
  if (solve_precision == HDG_MIXED_FP32)
    return record_group_mixed<D2>(M, graph, asm_precision, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
  FaceArgs F = face_args(M);
  const int nb = nblocks(M);
  const int64_t nv = M->nfc * D2;
  int rc = ensure_workspace(M, false);
  if (rc) return rc;
  if (!M->cap_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = M->cap_stream;
  cudaStream_t saved = M->stream;
  double* scal = M->d_scal;
  double* xD = M->d_uhatD;
  double* phiN = M->d_uhatD + nv;
  const bool tl = M->coarse != nullptr;
  const CoarseArgs CA = tl ? coarse_args(M) : CoarseArgs{};  // host set-up, before the capture
  // A: assembly, boundary data, right-hand side, block-Jacobi, per-problem ||b_p||, PCG start
  cudaGraph_t ga;
  HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  M->stream = cs;
  cudaMemsetAsync(M->d_status, 0, sizeof(int32_t) * 4, cs);
  cudaError_t e = (asm_precision == HDG_DF32) ? launch_k1(M) : launch_assemble(M);
  bdata_kernel<D2><<<nb, kNT, 0, cs>>>(F, M->d_fvx, M->d_vx, M->nelt, M->dt.D, M->dt.face_w, M->tab.nf, M->uD, M->gN,
                                       xD, phiN);
  rhs_kernel<D2><<<nb, kNT, 0, cs>>>(F, M->d_C, M->d_Cf, xD, phiN, M->d_b, M->d_red, M->d_counter,
                                     M->d_scal + S_NSCAL);
  bj_kernel<D2, double><<<(unsigned)((M->nfc + 63) / 64), 64, 0, cs>>>(F, M->d_C, M->d_BJ, M->d_status, false);
  int rcb = tl ? coarse_launch_build(M) : HDG_OK;  // Galerkin hierarchy of this assembly
  cudaMemsetAsync(norms, 0, sizeof(double) * 2 * np, cs);
  prob_norms_kernel<<<304, 256, 0, cs>>>(M->d_b, face_prob, M->nfc, D2, norms);
  batch_scalars_kernel<<<1, 32, 0, cs>>>(scal, norms, np, rtol, maxit, kGraphIters);
  pcg_init_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_C, M->d_b, M->d_x, false, M->d_r, M->d_red, M->d_counter,
                                                  scal);
  if (tl) {
    coarse_cycle<double, D2>(M, CA, M->d_r, cs, scal + S_DONE);
    pcg_zc_kernel<double, D2, true><<<nb, kNT, 0, cs>>>(F, CA, M->d_BJ, M->d_r, M->d_z, M->d_p, M->d_red,
                                                        M->d_counter, scal);
  } else {
    pcg_precond_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_BJ, M->d_r, M->d_z, M->d_p, M->d_red, M->d_counter,
                                                       scal);
  }
  M->stream = saved;
  if (rcb) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(cs, &junk);
    if (junk) cudaGraphDestroy(junk);
    return rcb;
  }
  cudaError_t e2 = cudaStreamEndCapture(cs, &ga);
  if (e != cudaSuccess || e2 != cudaSuccess) return fail(HDG_ERR_CUDA, "batch graph capture (assembly/setup) failed");
  cudaGraphNode_t na, nw, nc;
  HDG_CUDA_TRY(cudaGraphAddChildGraphNode(&na, graph, nullptr, 0, ga));
  cudaGraphDestroy(ga);
  // W: device-driven PCG loop
  cudaGraphConditionalHandle h;
  HDG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  HDG_CUDA_TRY(cudaGraphAddNode(&nw, graph, &na, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < kGraphIters; ++it) {
    pcg_matvec_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_C, M->d_p, M->d_q, M->d_red, M->d_counter, scal);
    if (tl) {
      pcg_update_tl_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_x, M->d_r, M->d_p, M->d_q, M->d_red, M->d_counter,
                                                           scal);
      coarse_cycle<double, D2>(M, CA, M->d_r, cs, scal + S_DONE);
      pcg_zc_kernel<double, D2, false><<<nb, kNT, 0, cs>>>(F, CA, M->d_BJ, M->d_r, M->d_z, M->d_p, M->d_red,
                                                           M->d_counter, scal);
    } else {
      pcg_update_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_BJ, M->d_x, M->d_r, M->d_z, M->d_p, M->d_q,
                                                        M->d_red, M->d_counter, scal);
    }
    pcg_dir_kernel<double><<<nb, kNT, 0, cs>>>(nv, M->d_z, M->d_p, scal);
  }
  loop_control_kernel<<<1, 32, 0, cs>>>(h, scal, S_DONE, S_BODIES, S_MAXBODIES);
  cudaGraph_t bout;
  HDG_CUDA_TRY(cudaStreamEndCapture(cs, &bout));
  // C: true residual, per-problem ||r_p||, trace with Dirichlet data, recovery
  cudaGraph_t gc;
  HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  M->stream = cs;
  pcg_init_kernel<double, D2><<<nb, kNT, 0, cs>>>(F, M->d_C, M->d_b, M->d_x, true, M->d_q, M->d_red, M->d_counter,
                                                  M->d_scal + S_NSCAL);
  prob_norms_kernel<<<304, 256, 0, cs>>>(M->d_q, face_prob, M->nfc, D2, norms + np);
  finish_kernel<<<nb, kNT, 0, cs>>>(nv, M->d_ftype, D2, M->d_x, M->d_uhatD, uhat);
  e = launch_recover(M, uhat, q, u);
  M->stream = saved;
  e2 = cudaStreamEndCapture(cs, &gc);
  if (e != cudaSuccess || e2 != cudaSuccess) return fail(HDG_ERR_CUDA, "batch graph capture (recovery) failed");
  HDG_CUDA_TRY(cudaGraphAddChildGraphNode(&nc, graph, &nw, 1, gc));
  cudaGraphDestroy(gc);
  *last = nc;
  M->rhs_ready = false;
  return HDG_OK;
}

// Part A, the refinement WHILE loop (FP64 residual, FP32 inner PCG in a nested WHILE loop,
// update) and part C of a mixed-precision group.
template <int D2>
static int record_group_mixed(hdg_mesh* M, cudaGraph_t graph, int asm_precision, const int32_t* face_prob, int np,
                              double* norms, double rtol, int maxit, double* q, double* u, double* uhat,
                              cudaGraphNode_t* last) {
  constexpr int kMaxOuter = 30;
  FaceArgs F = face_args(M);
  const int nb64 = nblocks(M);
  const int nb32 = nblocks_t<float>(M);
  const int64_t nv = M->nfc * D2;
  int rc = ensure_workspace(M, true);
  if (rc) return rc;
  if (!M->cap_stream) HDG_CUDA_TRY(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
  cudaStream_t cs = M->cap_stream;
  cudaStream_t saved = M->stream;
  double* so = M->d_scal;             // refinement scalars
  double* si = M->d_scal + S_NSCAL;   // inner FP32 PCG scalars
  double* xD = M->d_uhatD;
  double* phiN = M->d_uhatD + nv;
  float* q32 = reinterpret_cast<float*>(M->d_q);
  const bool tl = M->coarse != nullptr;
  M->c32_ready = true;  // the graph converts C^K before the coarse set-up reads it
  const CoarseArgs CA = tl ? coarse_args(M) : CoarseArgs{};
  // A: assembly, boundary data, right-hand side, FP32 operator and block inverses, coarse
  // hierarchy, per-problem ||b_p||, x = 0
  cudaGraph_t ga;
  HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  M->stream = cs;
  cudaMemsetAsync(M->d_status, 0, sizeof(int32_t) * 4, cs);
  cudaError_t e = (asm_precision == HDG_DF32) ? launch_k1(M) : launch_assemble(M);
  bdata_kernel<D2><<<nb64, kNT, 0, cs>>>(F, M->d_fvx, M->d_vx, M->nelt, M->dt.D, M->dt.face_w, M->tab.nf, M->uD,
                                         M->gN, xD, phiN);
  rhs_kernel<D2><<<nb64, kNT, 0, cs>>>(F, M->d_C, M->d_Cf, xD, phiN, M->d_b, M->d_red, M->d_counter, si);
  convert_c32_kernel<D2><<<1216, 256, 0, cs>>>(M->d_C, M->d_C32, M->nelt);
  bj_kernel<D2, float><<<(unsigned)((M->nfc + 63) / 64), 64, 0, cs>>>(F, M->d_C, M->d_BJ32, M->d_status, false);
  int rcb = tl ? coarse_launch_build(M) : HDG_OK;
  cudaMemsetAsync(norms, 0, sizeof(double) * 2 * np, cs);
  prob_norms_kernel<<<304, 256, 0, cs>>>(M->d_b, face_prob, M->nfc, D2, norms);
  batch_scalars_kernel<<<1, 32, 0, cs>>>(so, norms, np, rtol, maxit, kGraphIters);
  cudaMemsetAsync(M->d_x, 0, sizeof(double) * nv, cs);
  M->stream = saved;
  M->c32_ready = false;
  cudaError_t e2 = cudaStreamEndCapture(cs, &ga);
  if (rcb) {
    if (e2 == cudaSuccess) cudaGraphDestroy(ga);
    return rcb;
  }
  if (e != cudaSuccess || e2 != cudaSuccess) return fail(HDG_ERR_CUDA, "batch graph capture (assembly/setup) failed");
  cudaGraphNode_t na, nw, nc;
  HDG_CUDA_TRY(cudaGraphAddChildGraphNode(&na, graph, nullptr, 0, ga));
  cudaGraphDestroy(ga);
  // W: refinement loop
  cudaGraphConditionalHandle h_outer;
  HDG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_outer, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h_outer;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  HDG_CUDA_TRY(cudaGraphAddNode(&nw, graph, &na, nullptr, 1, &cp));
  cudaGraph_t obody = cp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle h_inner;
  HDG_CUDA_TRY(cudaGraphConditionalHandleCreate(&h_inner, obody, 1, cudaGraphCondAssignDefault));
  // outer body, first part: FP64 residual, control, FP32 start of the inner solve
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  pcg_init_kernel<double, D2><<<nb64, kNT, 0, cs>>>(F, M->d_C, M->d_b, M->d_x, true, M->d_r, M->d_red, M->d_counter,
                                                    so);
  outer_check_kernel<<<1, 32, 0, cs>>>(h_outer, h_inner, so, si, M->inner_rtol, kMaxOuter, kGraphIters);
  convert_kernel<float><<<304, 256, 0, cs>>>(M->d_r, M->d_r32, nv);
  pcg_init_kernel<float, D2><<<nb32, kNT, 0, cs>>>(F, M->d_C32, M->d_r32, M->d_x32, false, M->d_q32, M->d_red,
                                                   M->d_counter, si);
  if (tl) {
    coarse_cycle<float, D2>(M, CA, M->d_q32, cs, si + S_DONE);
    pcg_zc_kernel<float, D2, true><<<nb32, kNT, 0, cs>>>(F, CA, M->d_BJ32, M->d_q32, M->d_z32, M->d_p32, M->d_red,
                                                         M->d_counter, si);
  } else {
    pcg_precond_kernel<float, D2><<<nb32, kNT, 0, cs>>>(F, M->d_BJ32, M->d_q32, M->d_z32, M->d_p32, M->d_red,
                                                        M->d_counter, si);
  }
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  HDG_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  cudaGraph_t junk = nullptr;
  HDG_CUDA_TRY(cudaStreamEndCapture(cs, &junk));
  // the inner FP32 PCG loop, nested
  cudaGraphNode_t ni;
  cudaGraphNodeParams ci = {};
  ci.type = cudaGraphNodeTypeConditional;
  ci.conditional.handle = h_inner;
  ci.conditional.type = cudaGraphCondTypeWhile;
  ci.conditional.size = 1;
  HDG_CUDA_TRY(cudaGraphAddNode(&ni, obody, tail.data(), nullptr, tail.size(), &ci));
  cudaGraph_t ibody = ci.conditional.phGraph_out[0];
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < kGraphIters; ++it) {
    pcg_matvec_kernel<float, D2><<<nb32, kNT, 0, cs>>>(F, M->d_C32, M->d_p32, q32, M->d_red, M->d_counter, si);
    if (tl) {
      pcg_update_tl_kernel<float, D2><<<nb32, kNT, 0, cs>>>(F, M->d_x32, M->d_q32, M->d_p32, q32, M->d_red,
                                                            M->d_counter, si);
      coarse_cycle<float, D2>(M, CA, M->d_q32, cs, si + S_DONE);
      pcg_zc_kernel<float, D2, false><<<nb32, kNT, 0, cs>>>(F, CA, M->d_BJ32, M->d_q32, M->d_z32, M->d_p32, M->d_red,
                                                            M->d_counter, si);
    } else {
      pcg_update_kernel<float, D2><<<nb32, kNT, 0, cs>>>(F, M->d_BJ32, M->d_x32, M->d_q32, M->d_z32, M->d_p32, q32,
                                                         M->d_red, M->d_counter, si);
    }
    pcg_dir_kernel<float><<<nb32, kNT, 0, cs>>>(nv, M->d_z32, M->d_p32, si);
  }
  loop_control_kernel<<<1, 32, 0, cs>>>(h_inner, si, S_DONE, S_BODIES, S_MAXBODIES);
  HDG_CUDA_TRY(cudaStreamEndCapture(cs, &junk));
  // outer body, last part: x += x32, iteration count
  HDG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, obody, &ni, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  axpy_f32_kernel<<<nb64, kNT, 0, cs>>>(nv, M->d_x32, M->d_x);
  outer_accum_kernel<<<1, 32, 0, cs>>>(so, si);
  HDG_CUDA_TRY(cudaStreamEndCapture(cs, &junk));
  // C: true residual, per-problem ||r_p||, trace with Dirichlet data, recovery
  cudaGraph_t gc;
  HDG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  M->stream = cs;
  pcg_init_kernel<double, D2><<<nb64, kNT, 0, cs>>>(F, M->d_C, M->d_b, M->d_x, true, M->d_q, M->d_red, M->d_counter,
                                                    si);
  prob_norms_kernel<<<304, 256, 0, cs>>>(M->d_q, face_prob, M->nfc, D2, norms + np);
  finish_kernel<<<nb64, kNT, 0, cs>>>(nv, M->d_ftype, D2, M->d_x, M->d_uhatD, uhat);
  e = launch_recover(M, uhat, q, u);
  M->stream = saved;
  e2 = cudaStreamEndCapture(cs, &gc);
  if (e != cudaSuccess || e2 != cudaSuccess) return fail(HDG_ERR_CUDA, "batch graph capture (recovery) failed");
  HDG_CUDA_TRY(cudaGraphAddChildGraphNode(&nc, graph, &nw, 1, gc));
  cudaGraphDestroy(gc);
  *last = nc;
  M->rhs_ready = false;
  return HDG_OK;
}

int batch_record_group(hdg_mesh* M, cudaGraph_t graph, int asm_precision, int solve_precision,
                       const int32_t* face_prob, int np, double* norms, double rtol, int maxit, double* q, double* u,
                       double* uhat, cudaGraphNode_t* last) {
  const int sp = solve_precision;
  switch (M->tab.d2) {
    case 1: return record_group<1>(M, graph, asm_precision, sp, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
    case 3: return record_group<3>(M, graph, asm_precision, sp, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
    case 6: return record_group<6>(M, graph, asm_precision, sp, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
    case 10: return record_group<10>(M, graph, asm_precision, sp, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
    case 15: return record_group<15>(M, graph, asm_precision, sp, face_prob, np, norms, rtol, maxit, q, u, uhat, last);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

// iterations run by the last device-driven solve of M
int batch_group_iterations(hdg_mesh* M, int* iters, int* status) {
  double hv[S_NSCAL];
  HDG_CUDA_TRY(cudaMemcpy(hv, M->d_scal, sizeof(hv), cudaMemcpyDeviceToHost));
  *iters = (int)hv[S_ITERS];
  int32_t st[4];
  HDG_CUDA_TRY(cudaMemcpy(st, M->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  *status = (hv[S_BAD] != 0.0 || st[0] || st[1] || st[3]) ? 1 : 0;
  return HDG_OK;
}

int solve_trace(hdg_mesh* M, int precision, double rtol, int maxit, const double* x0, double* uhat, int* iters,
                double* relres) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "hdg_solve_trace before hdg_assemble_condense");
  if (precision != HDG_FP64 && precision != HDG_MIXED_FP32) return fail(HDG_ERR_ARG, "unknown precision");
  if (!(rtol > 0) || maxit < 1 || !uhat) return fail(HDG_ERR_ARG, "bad rtol/maxit/uhat");
  switch (M->tab.d2) {
    case 1: return Solver<1>::solve(M, precision, rtol, maxit, x0, uhat, iters, relres);
    case 3: return Solver<3>::solve(M, precision, rtol, maxit, x0, uhat, iters, relres);
    case 6: return Solver<6>::solve(M, precision, rtol, maxit, x0, uhat, iters, relres);
    case 10: return Solver<10>::solve(M, precision, rtol, maxit, x0, uhat, iters, relres);
    case 15: return Solver<15>::solve(M, precision, rtol, maxit, x0, uhat, iters, relres);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

int trace_apply(hdg_mesh* M, const double* x, double* y) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "operator before hdg_assemble_condense");
  switch (M->tab.d2) {
    case 1: return Solver<1>::apply(M, x, y);
    case 3: return Solver<3>::apply(M, x, y);
    case 6: return Solver<6>::apply(M, x, y);
    case 10: return Solver<10>::apply(M, x, y);
    case 15: return Solver<15>::apply(M, x, y);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

int autotune_face_grid(hdg_mesh* M, hdg_tuning* out) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "autotune before hdg_assemble_condense");
  switch (M->tab.d2) {
    case 1: return Solver<1>::autotune(M, out);
    case 3: return Solver<3>::autotune(M, out);
    case 6: return Solver<6>::autotune(M, out);
    case 10: return Solver<10>::autotune(M, out);
    case 15: return Solver<15>::autotune(M, out);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

int coarse_precond_apply(hdg_mesh* M, const double* r, double* z) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "preconditioner before hdg_assemble_condense");
  if ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(z)) % 16 != 0)
    return fail(HDG_ERR_ARG, "r and z must start on 16-byte boundaries");
  if (!M->coarse) return fail(HDG_ERR_STATE, "no coarse space: call hdg_set_coarse_space first");
  switch (M->tab.d2) {
    case 1: return Solver<1>::precond_apply(M, r, z);
    case 3: return Solver<3>::precond_apply(M, r, z);
    case 6: return Solver<6>::precond_apply(M, r, z);
    case 10: return Solver<10>::precond_apply(M, r, z);
    case 15: return Solver<15>::precond_apply(M, r, z);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

int trace_residual(hdg_mesh* M, const double* x, double* r, double* rnorm, double* bnorm) {
  if (!M->assembled) return fail(HDG_ERR_STATE, "residual before hdg_assemble_condense");
  switch (M->tab.d2) {
    case 1: return Solver<1>::residual(M, x, r, rnorm, bnorm);
    case 3: return Solver<3>::residual(M, x, r, rnorm, bnorm);
    case 6: return Solver<6>::residual(M, x, r, rnorm, bnorm);
    case 10: return Solver<10>::residual(M, x, r, rnorm, bnorm);
    case 15: return Solver<15>::residual(M, x, r, rnorm, bnorm);
  }
  return fail(HDG_ERR_UNSUPPORTED, "unsupported degree");
}

}  // namespace hdg
