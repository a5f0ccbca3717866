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

}  // namespace tcm

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

extern "C" int hdg_mass_contraction(hdg_mesh* mesh, const double* g, int mode, float* out) {
  if (!mesh || !g || !out) return hdg::fail(HDG_ERR_ARG, "NULL argument");
  if (mode < 0 || mode > 2) return hdg::fail(HDG_ERR_ARG, "mode must be 0 (tensor cores), 1 or 2 (CUDA cores)");
  if (mesh->k < 1) return hdg::fail(HDG_ERR_UNSUPPORTED, "the contraction is built for k >= 1");
  return hdg::mass_contraction(mesh, g, mode, out);
}
