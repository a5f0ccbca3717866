// The dense quadrature contraction of the volume masses (eq. 3.55) on the 5th-generation tensor
// cores, as a stand-alone measurement of that contraction:
//     Mass_e[p] = sum_q A[e][q] B[q][p],   A[e][q] = |K_e| omega_q g_e(p_q),
//                                          B[q][p] = P_i(p_hat_q) P_j(p_hat_q),  p = (i <= j),
// one GEMM [nelt x nq] . [nq x n(n+1)/2] for all elements at once.  The path that the solver
// uses forms the masses by sum factorisation in double-float arithmetic (assemble_df.cu) and
// keeps FP64-level accuracy; this kernel rounds A and B to BF16 and accumulates in FP32, so its
// masses carry BF16 rounding errors (about 2^-9 relative per operand).
//
// Kernel (one CTA of 128 threads per SM pair slot, persistent over tiles of 128 elements):
//  * B (the pair products, shared by every element) is written once per CTA into shared memory
//    in the canonical K-major core-matrix layout without swizzle: 8 rows x 16 bytes per core
//    matrix, core matrices adjacent in K 128 bytes apart (leading byte offset), adjacent in N
//    (K/8) 128 bytes apart (stride byte offset);
//  * per tile, the 128 threads form A (|K| omega_q g, rounded to BF16) in the same layout;
//  * one elected thread issues K/16 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
//    N = the padded pair count) into a tensor-memory accumulator and commits them to an
//    mbarrier;
//  * after the (bounded) wait each warp reads its 32 accumulator lanes (tcgen05.ld 32x32b) and
//    stores its elements' rows.
// A wait that runs out sets status[6] and the CTA frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "device_async.cuh"
#include "device_common.cuh"
#include "hdg_internal.h"

namespace hdg {
namespace tcm {

constexpr int kThreads = 128;          // = the MMA's M: one thread per accumulator lane (element)
constexpr int kWaitPolls = 1 << 22;     // bounded mbarrier waits

__host__ __device__ constexpr int round16(int x) { return (x + 15) / 16 * 16; }

// tensor-memory columns for an accumulator of n FP32 columns: a power of two >= 32
__host__ __device__ constexpr int tmem_cols(int n) {
  return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256;
}

// Shared-memory matrix descriptor of tcgen05 (K-major, no swizzle): start address, leading
// byte offset (between core matrices along K), stride byte offset (between 8-row groups), the
// fixed version bits 46-48 = 0b001, base offset 0, swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((a & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits
// 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// offset in bytes of element (row, k) in the K-major core-matrix layout of a rows x K BF16 tile
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K >> 3) + (k >> 3)) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct Args {
  const double* g;      // [nelt][nq] coefficient at the volume nodes
  const double* geo;    // [nelt][kGeoStride] (volume at 25)
  const double* w;      // [nq] reference weights
  const double* P;      // [nq][n] basis at the nodes
  const int16_t* pairs; // [np][2] (i <= j)
  float* out;           // [nelt][np]
  int32_t* status;
  int64_t nelt;
  int nq, n, np;
  int kpad, ntile, npad_tile;  // K padded to 16; columns per N tile; N tile padded to 16
};

// Tensor-core contraction: tiles of 128 elements, N tiles of at most 256 pair columns.
__global__ void __launch_bounds__(kThreads, 1) mass_tc_kernel(Args A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int K = A.kpad, NT = A.npad_tile;
  unsigned char* sA = smem;                        // 128 x K BF16
  unsigned char* sB = smem + 128 * K * 2;          // NT x K BF16
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols = tmem_cols(NT);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_fail = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = idesc_bf16_f32(128, NT);
  const int64_t ntiles_e = (A.nelt + 127) / 128;
  const int nnt = (A.np + A.ntile - 1) / A.ntile;
  uint32_t phase = 0;
  for (int nt = 0; nt < nnt && !s_fail; ++nt) {
    const int p0 = nt * A.ntile;
    const int pn = min(A.ntile, A.np - p0);
    // B tile: row = pair column (N), k = node; zero padding
    for (int t = tid; t < NT * K; t += kThreads) {
      const int row = t / K, k = t - row * K;
      float v = 0.f;
      if (row < pn && k < A.nq) {
        const int p = p0 + row;
        const int i = A.pairs[2 * p], j = A.pairs[2 * p + 1];
        v = (float)(A.P[k * A.n + i] * A.P[k * A.n + j]);
      }
      *reinterpret_cast<__nv_bfloat16*>(sB + kmajor_offset(row, k, K)) = __float2bfloat16_rn(v);
    }
    for (int64_t et = blockIdx.x; et < ntiles_e; et += gridDim.x) {
      const int64_t e0 = et * 128;
      // A tile: coalesced reads of the tile's contiguous coefficient block
      for (int t = tid; t < 128 * K; t += kThreads) {
        const int row = t / K, k = t - row * K;
        const int64_t e = e0 + row;
        float v = 0.f;
        if (e < A.nelt && k < A.nq) v = (float)(A.geo[e * kGeoStride + 25] * A.w[k] * A.g[e * A.nq + k]);
        *reinterpret_cast<__nv_bfloat16*>(sA + kmajor_offset(row, k, K)) = __float2bfloat16_rn(v);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
      fence_before();
      __syncthreads();
      fence_after();
      if (tid == 0) {
        for (int ks = 0; ks < K / 16; ++ks) {
          // K = 16 per instruction: two core matrices along K, 256 bytes further per step
          const uint64_t da = smem_desc(sA + ks * 256, 128, (K / 8) * 128);
          const uint64_t db = smem_desc(sB + ks * 256, 128, (K / 8) * 128);
          mma_bf16(tmem, da, db, idesc, ks > 0);
        }
        mma_commit(&bar);
      }
      __syncwarp();
      const bool ok = mbar_wait(&bar, phase, kWaitPolls);
      // every thread takes the same decision (a wait can run out on some threads only)
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          s_fail = 1;
          atomicAdd(A.status + 6, 1);
        }
        __syncthreads();
        break;
      }
      phase ^= 1u;
      fence_after();
      // warp w owns accumulator lanes 32 w .. 32 w + 31 (elements e0 + 32 w + lane)
      const int64_t e = e0 + warp * 32 + lane;
      for (int c0 = 0; c0 < NT; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (e < A.nelt) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c0 + c < pn) A.out[e * A.np + p0 + c0 + c] = v[c];
        }
      }
      fence_before();
      __syncthreads();  // every lane read before the next tile's MMAs overwrite the accumulator
      fence_after();
    }
    __syncthreads();
  }
  if (s_fail) {
    // an MMA that never completed: wait once more (bounded) for it before freeing the memory
    mbar_wait(&bar, phase, kWaitPolls);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// The same contraction on the CUDA cores in FP32, from the same BF16-rounded operands (the
// reference of the tensor-core result) or from FP32-rounded operands (round_bf16 = false).
__global__ void mass_fp32_kernel(Args A, bool round_bf16) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nelt * A.np) return;
  const int64_t e = t / A.np;
  const int p = (int)(t - e * A.np);
  const int i = A.pairs[2 * p], j = A.pairs[2 * p + 1];
  const double vol = A.geo[e * kGeoStride + 25];
  float s = 0.f;
  for (int q = 0; q < A.nq; ++q) {
    float a = (float)(vol * A.w[q] * A.g[e * A.nq + q]);
    float b = (float)(A.P[q * A.n + i] * A.P[q * A.n + j]);
    if (round_bf16) {
      a = __bfloat162float(__float2bfloat16_rn(a));
      b = __bfloat162float(__float2bfloat16_rn(b));
    }
    s = fmaf(a, b, s);
  }
  A.out[e * A.np + p] = s;
}

// ------------------------------------------------------------------ split-BF16 masses
// The masses of the HDG_MIXED_BF16 assembly, per element e
//     out[e] = [ M_{kappa^-1} pairs (i <= j) | M_c pairs | f^K (the pairs (0, j), P_0 = 1) ]
// (eq. 3.55 with g = |K| omega kappa^-1, |K| omega c and |K| omega f), FP32, on the tensor cores
// from three-way BF16 splits of both operands: x = x0 + x1 + x2 with x0 the BF16 rounding of x
// (taken in FP32) and x1, x2 the BF16 roundings of what the earlier parts leave.  The six products
// a_i b_j with i + j <= 2 carry every term above 2^-24 of |a b|; they accumulate in FP32 in
// tensor memory, so the masses carry FP32-level rounding (not the 2^-9 of single BF16 operands).
//
// Work per CTA (128 threads, persistent over tiles of 128 elements): jobs (coefficient, tile of
// at most 256 pair columns); per job the nodes in chunks of 32 (two K = 16 steps): the threads
// split their element's 32 coefficient values into sA (3 parts, K-major core layout, one 16-byte
// store per part and 8 nodes) and copy the chunk's block of the split pair-product table (built
// once per mesh on the host, L2-resident) into sB; one thread issues the 2 x 6 MMAs and commits
// them to an mbarrier; the next chunk waits for them (bounded wait).  After the last chunk each
// warp reads its 32 accumulator lanes.  Two CTAs per SM overlap one's split with the other's MMAs.
namespace m3 {
constexpr int KC = 32;                          // nodes per chunk
constexpr int NTMAX = 256;                      // pair columns per job (accumulator columns)
constexpr int kPartA = 128 * KC * 2;            // bytes of one BF16 part of the A chunk
constexpr int kBlockBytes = 3 * NTMAX * KC * 2; // stride of the (tile, chunk) blocks of the table
constexpr int kSmem = 3 * kPartA + kBlockBytes;

struct Args {
  const double *kappa, *c, *f, *geo;
  const float* wf;  // [nq][2] reference weights as double-float pairs: the hi part (nearest float) is read
  const unsigned char* B;  // [ntile][nchunk] blocks: [3 parts][rows_t][KC] BF16, K-major core layout
  float* out;              // [nelt][ostride]
  int32_t* status;
  int64_t nelt;
  int nq, n, np, nchunk, ntile, ostride;
};

__host__ __device__ inline int tile_rows(int np, int t) { return round16(np - t * NTMAX < NTMAX ? np - t * NTMAX : NTMAX); }

// xf = x0 + x1 + x2 exactly (BF16 parts of an FP32 value: 8 + 8 + 8 significant bits)
__device__ __forceinline__ void split3(float xf, __nv_bfloat16& x0, __nv_bfloat16& x1, __nv_bfloat16& x2) {
  x0 = __float2bfloat16_rn(xf);
  const float r1 = xf - __bfloat162float(x0);
  x1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(x1);
  x2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(kThreads, 1) mass3_tc_kernel(Args A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;               // [3][128][KC]
  unsigned char* sB = smem + 3 * kPartA;  // [3][rows][KC]
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(NTMAX)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init(&bar, 1);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const int64_t ntiles_e = (A.nelt + 127) / 128;
  const int njobs = 2 * A.ntile + 1;
  uint32_t phase = 0;
  bool failed = false;
  for (int64_t et = blockIdx.x; et < ntiles_e && !failed; et += gridDim.x) {
    const int64_t e = et * 128 + tid;  // this thread's element (row of A, lane of the accumulator)
    const bool act = e < A.nelt;
    const float volf = act ? (float)A.geo[e * kGeoStride + 25] : 0.f;
    bool bad = false;
    for (int j = 0; j < njobs && !failed; ++j) {
      const int coef = j < A.ntile ? 0 : j < 2 * A.ntile ? 1 : 2;
      const int t = coef < 2 ? j - coef * A.ntile : 0;
      const int p0 = t * NTMAX;
      const int pn = coef < 2 ? min(NTMAX, A.np - p0) : A.n;
      const int N = round16(pn);
      const int rows = tile_rows(A.np, t);
      const int col0 = coef * A.np + p0;
      const double* g = coef == 0 ? A.kappa : coef == 1 ? A.c : A.f;
      const uint32_t idesc = idesc_bf16_f32(128, N);
      for (int ch = 0; ch < A.nchunk && !failed; ++ch) {
        // A chunk: split |K| omega_q g(p_q) of this thread's element, 8 nodes per 16-byte store
#pragma unroll
        for (int kg = 0; kg < KC / 8; ++kg) {
          uint32_t w0[4], w1[4], w2[4];
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            __nv_bfloat16 h[2], m_[2], l[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const int q = ch * KC + kg * 8 + u + v;
              float a = 0.f;
              if (act && q < A.nq) {  // FP32 arithmetic: a carries at most 6 roundings of 2^-24
                const double gv = g[e * A.nq + q];
                const float vw = volf * __ldg(A.wf + 2 * q);
                if (coef == 0) {
                  if (!(gv > 0.0) || !isfinite(gv)) bad = true;
                  a = vw * __frcp_rn(gv > 0.0 ? (float)gv : 1.f);
                } else {
                  if (!isfinite(gv) || (coef == 1 && !(gv >= 0.0))) bad = true;
                  a = vw * (float)gv;
                }
              }
              split3(a, h[v], m_[v], l[v]);
            }
            w0[u / 2] = pack2(h[0], h[1]);
            w1[u / 2] = pack2(m_[0], m_[1]);
            w2[u / 2] = pack2(l[0], l[1]);
          }
          const uint32_t off = kmajor_offset(tid, kg * 8, KC);
          *reinterpret_cast<uint4*>(sA + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
          *reinterpret_cast<uint4*>(sA + kPartA + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
          *reinterpret_cast<uint4*>(sA + 2 * kPartA + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        }
        // B chunk: the table block of (tile t, chunk ch), rows x KC per part
        {
          const uint4* src = reinterpret_cast<const uint4*>(A.B + (size_t)(t * A.nchunk + ch) * kBlockBytes);
          uint4* dst = reinterpret_cast<uint4*>(sB);
          const int nvec = 3 * rows * KC * 2 / 16;
          for (int i = tid; i < nvec; i += kThreads) dst[i] = __ldg(src + i);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> async proxy
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
          // the small products first: (a2 b0), (a1 b1), (a0 b2), (a1 b0), (a0 b1), (a0 b0)
          const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks)
#pragma unroll
            for (int pr = 0; pr < 6; ++pr) {
              const uint64_t da = smem_desc(sA + pa[pr] * kPartA + ks * 256, 128, (KC / 8) * 128);
              const uint64_t db = smem_desc(sB + pb[pr] * rows * KC * 2 + ks * 256, 128, (KC / 8) * 128);
              mma_bf16(tmem, da, db, idesc, ch > 0 || ks > 0 || pr > 0);
            }
          mma_commit(&bar);
        }
        __syncwarp();
        const bool ok = mbar_wait(&bar, phase, kWaitPolls);
        if (__syncthreads_or(!ok)) {  // the same decision on every thread
          if (tid == 0) atomicAdd(A.status + 6, 1);
          failed = true;
          break;
        }
        phase ^= 1u;
        fence_after();
      }
      if (failed) break;
      // epilogue: warp w reads accumulator lanes 32 w .. 32 w + 31 (its threads' elements)
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (act) {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c0 + c < pn) A.out[e * A.ostride + col0 + c0 + c] = v[c];
        }
      }
      fence_before();
      __syncthreads();  // every lane read before the next job's MMAs overwrite the accumulator
      fence_after();
    }
    if (act && bad) atomicAdd(A.status + 1, 1);
  }
  if (failed) mbar_wait(&bar, phase, kWaitPolls);  // the MMAs in flight, once more (bounded)
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NTMAX) : "memory");
}
}  // namespace m3

}  // namespace tcm

// The split pair-product table of the current volume rule (host, once per mesh): per pair tile
// and node chunk, the three BF16 parts of P_i(p_q) P_j(p_q) in the K-major core layout.
static int ensure_mass3_table(hdg_mesh* M) {
  using namespace tcm;
  const Tables& T = M->tab;
  const int n = T.n, nq = T.nq, np = n * (n + 1) / 2;
  const int ntile = (np + m3::NTMAX - 1) / m3::NTMAX, nchunk = (nq + m3::KC - 1) / m3::KC;
  if (M->d_mass3B && M->mass3_rule == T.rule) return HDG_OK;
  if (M->d_mass3B) {
    cudaFree(M->d_mass3B);
    M->d_mass3B = nullptr;
  }
  std::vector<int> pi, pj;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) {
      pi.push_back(i);
      pj.push_back(j);
    }
  std::vector<uint16_t> h((size_t)ntile * nchunk * m3::kBlockBytes / 2, 0);
  auto bf16_bits = [](float x) {  // round to nearest even (the table entries are finite)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
  };
  auto bf16_val = [](uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
  };
  for (int t = 0; t < ntile; ++t) {
    const int rows = m3::tile_rows(np, t);
    for (int ch = 0; ch < nchunk; ++ch) {
      uint16_t* blk = h.data() + (size_t)(t * nchunk + ch) * m3::kBlockBytes / 2;
      for (int r = 0; r < rows; ++r) {
        const int p = t * m3::NTMAX + r;
        for (int kk = 0; kk < m3::KC; ++kk) {
          const int q = ch * m3::KC + kk;
          float x = 0.f;
          if (p < np && q < nq) x = (float)(T.P[(size_t)q * n + pi[p]] * T.P[(size_t)q * n + pj[p]]);
          const uint16_t b0 = bf16_bits(x);
          const float r1 = x - bf16_val(b0);
          const uint16_t b1 = bf16_bits(r1);
          const uint16_t b2 = bf16_bits(r1 - bf16_val(b1));
          const size_t off = (((size_t)(r >> 3) * (m3::KC >> 3) + (kk >> 3)) * 128 + (r & 7) * 16 + (kk & 7) * 2) / 2;
          blk[off] = b0;
          blk[(size_t)rows * m3::KC + off] = b1;
          blk[(size_t)2 * rows * m3::KC + off] = b2;
        }
      }
    }
  }
  HDG_CUDA_TRY(cudaMalloc(&M->d_mass3B, h.size() * 2));
  HDG_CUDA_TRY(cudaMemcpy(M->d_mass3B, h.data(), h.size() * 2, cudaMemcpyHostToDevice));
  M->mass3_rule = T.rule;
  return HDG_OK;
}

int mass3_stride(int k) {
  const int n = d3_of(k), np = n * (n + 1) / 2;
  return (2 * np + n + 3) / 4 * 4;
}

int mass3_contraction(hdg_mesh* M, float* out) {
  using namespace tcm;
  int rc = ensure_mass3_table(M);
  if (rc) return rc;
  const int n = M->tab.n, np = n * (n + 1) / 2;
  m3::Args a;
  a.kappa = M->kappa;
  a.c = M->c;
  a.f = M->f;
  a.geo = M->d_geo;
  a.wf = M->dt.vol_w_df;
  a.B = reinterpret_cast<const unsigned char*>(M->d_mass3B);
  a.out = out;
  a.status = M->d_status;
  a.nelt = M->nelt;
  a.nq = M->tab.nq;
  a.n = n;
  a.np = np;
  a.nchunk = (a.nq + m3::KC - 1) / m3::KC;
  a.ntile = (np + m3::NTMAX - 1) / m3::NTMAX;
  a.ostride = mass3_stride(M->k);
  // at least 80 KB per CTA, so that at most two CTAs (2 x 256 tensor-memory columns) share an SM
  const size_t req = std::max<size_t>(m3::kSmem, 80 * 1024);
  HDG_CUDA_TRY(cudaFuncSetAttribute(m3::mass3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req));
  const int64_t tiles = (M->nelt + 127) / 128;
  const int grid = (int)std::min<int64_t>(tiles, 2 * 152);
  HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 6, 0, sizeof(int32_t), M->stream));
  m3::mass3_tc_kernel<<<grid, kThreads, req, M->stream>>>(a);
  M->launches++;
  HDG_CUDA_TRY(cudaGetLastError());
  return HDG_OK;
}

int mass_contraction(hdg_mesh* M, const double* g, int mode, float* out) {
  using namespace tcm;
  const int nq = M->tab.nq, n = M->tab.n, np = n * (n + 1) / 2;
  Args a;
  a.g = g;
  a.geo = M->d_geo;
  a.w = M->dt.vol_w;
  a.P = M->dt.P;
  a.pairs = M->dt.pairs_n;
  a.out = out;
  a.status = M->d_status;
  a.nelt = M->nelt;
  a.nq = nq;
  a.n = n;
  a.np = np;
  a.kpad = round16(nq);
  const int nnt = (np + 255) / 256;
  a.ntile = (np + nnt - 1) / nnt;
  a.npad_tile = round16(a.ntile);
  if (mode == 0) {
    const size_t smem = (size_t)(128 + a.npad_tile) * a.kpad * 2;
    // at least 100 KB per CTA, so that at most two CTAs (2 x 256 tensor-memory columns) share an SM
    const size_t req = std::max<size_t>(smem, 100 * 1024);
    HDG_CUDA_TRY(cudaFuncSetAttribute(mass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req));
    const int64_t tiles = (M->nelt + 127) / 128;
    const int grid = (int)std::min<int64_t>(tiles, 2 * 152);
    HDG_CUDA_TRY(cudaMemsetAsync(M->d_status + 6, 0, sizeof(int32_t), M->stream));
    mass_tc_kernel<<<grid, kThreads, req, M->stream>>>(a);
  } else {
    const int64_t tot = M->nelt * np;
    mass_fp32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, M->stream>>>(a, mode == 1);
  }
  M->launches++;
  HDG_CUDA_TRY(cudaGetLastError());
  if (mode == 0) {
    int32_t st = 0;
    HDG_CUDA_TRY(cudaMemcpyAsync(&st, M->d_status + 6, sizeof(int32_t), cudaMemcpyDeviceToHost, M->stream));
    HDG_CUDA_TRY(cudaStreamSynchronize(M->stream));
    if (st) return fail(HDG_ERR_CUDA, "tensor-core contraction: an MMA did not complete within the wait limit");
  }
  return HDG_OK;
}

}  // namespace hdg

extern "C" int hdg_mixed_masses(hdg_mesh* mesh, float* out, int* stride) {
  if (!mesh) return hdg::fail(HDG_ERR_ARG, "NULL mesh");
  if (mesh->k < 1 || mesh->tab.rule != HDG_RULE_CONICAL)
    return hdg::fail(HDG_ERR_UNSUPPORTED, "the split-BF16 masses are built for k >= 1 on the conical volume rule");
  if (stride) *stride = hdg::mass3_stride(mesh->k);
  if (!out) return HDG_OK;
  if (!mesh->kappa) return hdg::fail(HDG_ERR_STATE, "hdg_set_coefficients was not called");
  HDG_CUDA_TRY(cudaMemsetAsync(mesh->d_status + 1, 0, sizeof(int32_t), mesh->stream));
  int rc = hdg::mass3_contraction(mesh, out);
  if (rc) return rc;
  int32_t st[7];
  HDG_CUDA_TRY(cudaMemcpyAsync(st, mesh->d_status, sizeof(st), cudaMemcpyDeviceToHost, mesh->stream));
  HDG_CUDA_TRY(cudaStreamSynchronize(mesh->stream));
  if (st[6]) return hdg::fail(HDG_ERR_CUDA, "tensor-core contraction: an MMA did not complete within the wait limit");
  if (st[1]) return hdg::fail(HDG_ERR_COEFF, std::to_string(st[1]) + " element(s) with kappa <= 0, c < 0 or non-finite data");
  return HDG_OK;
}

extern "C" int hdg_mass_contraction(hdg_mesh* mesh, const double* g, int mode, float* out) {
  if (!mesh || !g || !out) return hdg::fail(HDG_ERR_ARG, "NULL argument");
  if (mode < 0 || mode > 2) return hdg::fail(HDG_ERR_ARG, "mode must be 0 (tensor cores), 1 or 2 (CUDA cores)");
  if (mesh->k < 1) return hdg::fail(HDG_ERR_UNSUPPORTED, "the contraction is built for k >= 1");
  return hdg::mass_contraction(mesh, g, mode, out);
}
