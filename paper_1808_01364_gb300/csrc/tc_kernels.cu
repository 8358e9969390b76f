// Tensor-core (tcgen05) tile products for the dense Schur updates of large
// fronts (Sec. 2.1, C_BB -= W W^T and the trailing updates of the blocked
// elimination), with FP32 data on the 5th-generation tensor cores.
//
// One CTA of 128 threads (4 warps) computes a 128 x 64 tile D = A B^T with
// FP32 accumulation in tensor memory: operands are loaded by the threads in
// chunks of 32 along K, split into a TF32 high part and a TF32 remainder
// (a = hi + lo), stored in shared memory in the K-major no-swizzle core-matrix
// layout, and multiplied as hi*hi + hi*lo + lo*hi (12 MMAs of K = 8 per
// chunk), which keeps the products at about FP32 accuracy: the Schur updates
// of high-contrast problems cancel too much for plain TF32 inputs.  One
// elected thread issues the MMAs and commits them to an mbarrier; every wait
// is bounded, and on a timeout the CTA records RHIF_ERR_TIMEOUT, waits once
// more for its MMAs, frees its tensor memory and returns.
#include "common.cuh"
#include "kernels.h"
#include "tables.h"
#include "../../include/rhif.h"

namespace rhif {
namespace tc {

constexpr int kM = 128, kN = 64, kK = 32;   // tile and K chunk
constexpr int kThreadsTc = 128;
constexpr uint32_t kTmemCols = 64;

// Shared-memory matrix descriptor, K-major, no swizzle: 8-row x 16-byte core
// matrices; lbo = byte step between core matrices along K, sbo = along M/N.
__device__ inline uint64_t sdesc(const void* p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture family
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ inline void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ inline void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ inline void mma_tf32(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}

__device__ inline void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive accumulator columns of this thread's row (its warp's lanes).
__device__ inline void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// byte offset of element (r, k) of an R x 32 K-major no-swizzle tile
__device__ inline uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (kK / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

struct TileSmem {
  float a_hi[kM * kK], a_lo[kM * kK], b_hi[kN * kK], b_lo[kN * kK];
  uint64_t bar;
  uint32_t tmem;
};

// D (128 x 64) = sum_{k < K} fa(i, k) fb(j, k) over rows i < M of the tile,
// columns j < N (zero beyond), then epi(i, j, d) for every i < M, j < N.
// All 128 threads of the CTA must call it.  Returns false on a wait timeout.
template <class FA, class FB, class EPI>
__device__ bool tile_product_tf32x3(TileSmem& S, int M, int N, int K, FA fa, FB fb, EPI epi) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
  if (tid == 0) mbar_init(&S.bar, 1);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  constexpr uint32_t idesc = idesc_tf32(kM, kN);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < K && ok; k0 += kK) {
    const int kk = min(kK, K - k0);
    for (int idx = tid; idx < kM * kK; idx += kThreadsTc) {
      const int k = idx / kM, r = idx % kM;
      const float x = (r < M && k < kk) ? fa(r, k0 + k) : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t o = core_off(r, k) >> 2;
      S.a_hi[o] = hi;
      S.a_lo[o] = lo;
    }
    for (int idx = tid; idx < kN * kK; idx += kThreadsTc) {
      const int k = idx / kN, r = idx % kN;
      const float x = (r < N && k < kk) ? fb(r, k0 + k) : 0.f;
      float hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t o = core_off(r, k) >> 2;
      S.b_hi[o] = hi;
      S.b_lo[o] = lo;
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t sbo_a = 8 * 128, sbo_b = 8 * 128, lbo = 128;
#pragma unroll
      for (int s = 0; s < kK / 8; ++s) {
        const uint32_t koff = s * 2 * 128;   // two core matrices (8 TF32) per MMA
        const uint64_t ah = sdesc((const char*)S.a_hi + koff, lbo, sbo_a);
        const uint64_t al = sdesc((const char*)S.a_lo + koff, lbo, sbo_a);
        const uint64_t bh = sdesc((const char*)S.b_hi + koff, lbo, sbo_b);
        const uint64_t bl = sdesc((const char*)S.b_lo + koff, lbo, sbo_b);
        mma_tf32(tmem, ah, bh, idesc, (k0 > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      commit(&S.bar);
    }
    ok = __syncthreads_and(mbar_wait(&S.bar, phase)) != 0;   // CTA-uniform
    phase ^= 1;
    fence_after();
  }
  if (!ok) {
    mbar_wait(&S.bar, phase ^ 1);   // the MMAs still in flight, once more with the limit
  } else if (K > 0) {
    // epilogue: warp w owns accumulator rows 32w .. 32w+31
    const int row = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < kN; c0 += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < N) epi(row, c0 + j, v[j]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
  return ok;
}

// C (column-major, ldc) -= A B^T, A M x K (lda), B N x K (ldb), column-major.
__global__ void __launch_bounds__(kThreadsTc) k_tc_gemm_check(int M, int N, int K, const float* A,
                                                             int64_t lda, const float* B,
                                                             int64_t ldb, float* C, int64_t ldc,
                                                             int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smraw);
  const int i0 = blockIdx.x * kM, j0 = blockIdx.y * kN;
  auto fa = [&](int r, int k) { return A[(i0 + r) + (int64_t)k * lda]; };
  auto fb = [&](int r, int k) { return B[(j0 + r) + (int64_t)k * ldb]; };
  auto epi = [&](int r, int j, float d) { C[(i0 + r) + (int64_t)(j0 + j) * ldc] -= d; };
  if (!tile_product_tf32x3(S, min(kM, M - i0), min(kN, N - j0), K, fa, fb, epi) &&
      threadIdx.x == 0)
    report(status, RHIF_ERR_TIMEOUT, -1, kKindArg, blockIdx.x);
}

// Schur complement of every front of the level on the tensor cores:
// F[B, B] -= W W^T with W = F[B, I] (rows nI.. of the first nI columns), one
// CTA per 128 x 64 tile (a, b) of the boundary block; tiles entirely above
// the diagonal exit at once, tiles crossing it update only i >= j.
__global__ void __launch_bounds__(kThreadsTc) k_front_schur_tc(LevelDev Lv, int* status) {
  extern __shared__ __align__(128) unsigned char smraw[];
  TileSmem& S = *reinterpret_cast<TileSmem*>(smraw);
  int64_t bid = blockIdx.x;
  int c = 0;
  int rt = 0, ct = 0;
  for (; c < Lv.ncell; ++c) {
    const int nB = Lv.nB[c];
    rt = (nB + kM - 1) / kM;
    ct = (nB + kN - 1) / kN;
    const int64_t t = Lv.nI[c] > 0 ? (int64_t)rt * ct : 0;
    if (bid < t) break;
    bid -= t;
  }
  if (c >= Lv.ncell) return;
  const int a = (int)(bid / ct), b = (int)(bid % ct);
  if (b * kN > a * kM + kM - 1) return;   // above the diagonal (uniform per CTA)
  const int nI = Lv.nI[c], nB = Lv.nB[c], n = nI + nB;
  float* F = (float*)Lv.front + Lv.front_off[c];
  const int i0 = nI + a * kM, j0 = nI + b * kN;
  auto fa = [&](int r, int k) { return F[(i0 + r) + (int64_t)k * n]; };
  auto fb = [&](int r, int k) { return F[(j0 + r) + (int64_t)k * n]; };
  auto epi = [&](int r, int j, float d) {
    if (i0 + r >= j0 + j) F[(i0 + r) + (int64_t)(j0 + j) * n] -= d;
  };
  if (!tile_product_tf32x3(S, min(kM, n - i0), min(kN, n - j0), nI, fa, fb, epi) &&
      threadIdx.x == 0)
    report(status, RHIF_ERR_TIMEOUT, Lv.level, kKindCell, c);
}

}  // namespace tc

size_t tc_tile_smem_bytes() { return sizeof(tc::TileSmem) + 128; }

int64_t front_schur_tc_tiles(int nI, int nB) {
  if (nI == 0 || nB == 0) return 0;
  return (int64_t)((nB + tc::kM - 1) / tc::kM) * ((nB + tc::kN - 1) / tc::kN);
}

void launch_front_schur_tc(const LevelDev& Lv, int64_t tiles, int* status, cudaStream_t s) {
  if (tiles > 0)
    tc::k_front_schur_tc<<<(unsigned)tiles, tc::kThreadsTc, tc_tile_smem_bytes(), s>>>(Lv, status);
}

int configure_tc_kernels() {
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_gemm_check,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_tile_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc::k_front_schur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_tile_smem_bytes());
  return e == cudaSuccess ? 0 : -1;
}

void launch_tc_gemm_check(int M, int N, int K, const float* A, int64_t lda, const float* B,
                          int64_t ldb, float* C, int64_t ldc, int* status, cudaStream_t s) {
  dim3 grid((M + tc::kM - 1) / tc::kM, (N + tc::kN - 1) / tc::kN);
  tc::k_tc_gemm_check<<<grid, tc::kThreadsTc, tc_tile_smem_bytes(), s>>>(M, N, K, A, lda, B, ldb,
                                                                        C, ldc, status);
}

}  // namespace rhif
