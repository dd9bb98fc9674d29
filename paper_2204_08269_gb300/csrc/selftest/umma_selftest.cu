// Self-test of the tcgen05 / TMA building blocks (test infrastructure, built into its own
// library libjtfs_selftest.so): one CTA computes D[128 x 128] = A[128 x K] B[K x 128] in
// BF16 with FP32 accumulation, A K-major with a 32/64/128-byte swizzle, B either MN-major
// (rows of 128 time samples, 128-byte swizzle) or K-major.  The test compares D with a
// plain matrix product.
#include <stdint.h>

#include <string>

#include "../tma_host.h"
#include "../umma.cuh"

using namespace jtfs;
using namespace jtfs::umma;

namespace {

using __bf16_raw_t = uint16_t;

__global__ void k_umma_selftest(const __grid_constant__ CUtensorMap ta,
                                const __grid_constant__ CUtensorMap tb, float* D, int K,
                                int a_swz, int b_mn, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;
  uint8_t* sB = sA + 128 * K * 2;
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    failed = 0;
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 128);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  if (threadIdx.x == 0) {
    const int kb = a_swz / 2;
    mbar_arrive_expect_tx(&bar_tma, (uint32_t)(128 * K * 2 * 2));
    for (int k0 = 0; k0 < K; k0 += kb) tma_load_2d(sA + k0 * 256, &ta, k0, 0, &bar_tma);
    if (b_mn) {
      for (int n0 = 0; n0 < 128; n0 += 64) tma_load_2d(sB + (n0 / 64) * K * 128, &tb, n0, 0, &bar_tma);
    } else {
      for (int k0 = 0; k0 < K; k0 += 64) tma_load_2d(sB + k0 * 256, &tb, k0, 0, &bar_tma);
    }
    if (!mbar_wait(&bar_tma, 0, 2000000000ull)) {
      failed = 1;
    } else {
      const uint32_t lay = a_swz == 128 ? kSw128 : (a_swz == 64 ? kSw64 : kSw32);
      const uint32_t idesc = instr_desc(128, 128, 1, 1, 0, (uint32_t)b_mn, 0);
      for (int j = 0; j < K / 16; ++j) {
        const int box = (j * 16) / kb, off = ((j * 16) % kb) * 2;
        const uint64_t ad = smem_desc(smem_u32(sA + box * 128 * a_swz + off), 16, 8 * a_swz, lay);
        uint64_t bd;
        if (b_mn) {
          bd = smem_desc(smem_u32(sB + j * 16 * 128), (uint32_t)(K * 128), 1024, kSw128);
        } else {
          const int bb = (j * 16) / 64, bo = ((j * 16) % 64) * 2;
          bd = smem_desc(smem_u32(sB + bb * 128 * 128 + bo), 16, 1024, kSw128);
        }
        mma_f16(tbase, ad, bd, idesc, j > 0 ? 1u : 0u);
      }
      mma_commit(&bar_mma);
    }
  }
  __syncthreads();
  if (!failed) {
    if (!mbar_wait(&bar_mma, 0, 2000000000ull)) atomicExch(&failed, 1);
  }
  tc_fence_after();
  if (!failed) {
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < 128; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) D[row * 128 + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 128);
  if (threadIdx.x == 0) *status = failed;
}

// A from tensor memory: each thread stores its row of A (two BF16 per 32-bit column) with
// tcgen05.st, then one thread issues D = A B with B MN-major from shared memory (as above).
__global__ void k_umma_selftest_ta(const __bf16_raw_t* A, const __grid_constant__ CUtensorMap tb,
                                   float* D, int K, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sB = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    failed = 0;
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 256);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  // A columns start at 128: row r = 32 warp + lane, column c holds A[r][2c], A[r][2c + 1]
  {
    const int row = warp * 32 + lane;
    const uint32_t* arow = reinterpret_cast<const uint32_t*>(A + (size_t)row * K);
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    for (int c = 0; c < K / 2; c += 4)
      tmem_st4(tbase + lane_off + 128 + c, arow[c], arow[c + 1], arow[c + 2], arow[c + 3]);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_fence_after();
    mbar_arrive_expect_tx(&bar_tma, (uint32_t)(128 * K * 2));
    for (int n0 = 0; n0 < 128; n0 += 64) tma_load_2d(sB + (n0 / 64) * K * 128, &tb, n0, 0, &bar_tma);
    if (!mbar_wait(&bar_tma, 0, 2000000000ull)) {
      failed = 1;
    } else {
      const uint32_t idesc = instr_desc(128, 128, 1, 1, 0, 1, 0);
      for (int j = 0; j < K / 16; ++j) {
        const uint64_t bd = smem_desc(smem_u32(sB + j * 16 * 128), (uint32_t)(K * 128), 1024, kSw128);
        mma_f16_ta(tbase, tbase + 128 + j * 8, bd, idesc, j > 0 ? 1u : 0u);
      }
      mma_commit(&bar_mma);
    }
  }
  __syncthreads();
  if (!failed) {
    if (!mbar_wait(&bar_mma, 0, 2000000000ull)) atomicExch(&failed, 1);
  }
  tc_fence_after();
  if (!failed) {
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < 128; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) D[row * 128 + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
  if (threadIdx.x == 0) *status = failed;
}

// TF32 form: A [128 x K] FP32 K-major (rows of 32 values, 128-byte swizzle); B FP32, either
// MN-major (K rows of 128 values held as four 32-value atoms, 128-byte swizzle) or K-major;
// kind::tf32 MMAs of K = 8.
__global__ void k_umma_selftest_tf32(const __grid_constant__ CUtensorMap ta,
                                     const __grid_constant__ CUtensorMap tb, float* D, int K,
                                     int b_mn, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;                       // K / 32 atoms of 128 rows x 128 B
  uint8_t* sB = sA + 128 * K * 4;
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    failed = 0;
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_base, 128);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar_tma, (uint32_t)(128 * K * 4 * 2));
    for (int k0 = 0; k0 < K; k0 += 32) tma_load_2d(sA + (k0 / 32) * 128 * 128, &ta, k0, 0, &bar_tma);
    if (b_mn) {
      for (int n0 = 0; n0 < 128; n0 += 32) tma_load_2d(sB + (n0 / 32) * K * 128, &tb, n0, 0, &bar_tma);
    } else {
      for (int k0 = 0; k0 < K; k0 += 32) tma_load_2d(sB + (k0 / 32) * 128 * 128, &tb, k0, 0, &bar_tma);
    }
    if (!mbar_wait(&bar_tma, 0, 2000000000ull)) {
      failed = 1;
    } else {
      const uint32_t idesc = instr_desc(128, 128, 2, 2, 0, (uint32_t)b_mn, 0);
      for (int j = 0; j < K / 8; ++j) {
        const int atom = (j * 8) / 32, off = ((j * 8) % 32) * 4;
        const uint64_t ad = smem_desc(smem_u32(sA + atom * 128 * 128 + off), 16, 1024, kSw128);
        const uint64_t bd = b_mn
            ? smem_desc(smem_u32(sB + j * 8 * 128), (uint32_t)(K * 128), 1024, kSw128)
            : smem_desc(smem_u32(sB + atom * 128 * 128 + off), 16, 1024, kSw128);
        mma_tf32(tbase, ad, bd, idesc, j > 0 ? 1u : 0u);
      }
      mma_commit(&bar_mma);
    }
  }
  __syncthreads();
  if (!failed) {
    if (!mbar_wait(&bar_mma, 0, 2000000000ull)) atomicExch(&failed, 1);
  }
  tc_fence_after();
  if (!failed) {
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < 128; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) D[row * 128 + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 128);
  if (threadIdx.x == 0) *status = failed;
}

}  // namespace

// A pair of CTAs (cta_group::2, a cluster of two): D[256 x 128] = A[256 x K] B[K x 128] in
// BF16 with FP32 accumulation.  CTA r holds rows [128 r, +128) of A (K-major, 128-byte
// swizzle) and columns [64 r, +64) of B, MN-major (rows of 64 samples) or K-major (64 rows of
// B^T); the even CTA issues the M = 256 MMAs and commits to both CTAs' barriers, and each CTA
// reads its 128 rows of D from its own TMEM.  info[4 r + 0, 1] = TMEM base, cluster rank.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
k_umma2_selftest(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                 float* D, int K, int b_mn, int* status, uint32_t* info) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // each region is twice what this CTA loads, so that the operands stay inside the allocation
  // whatever the split of A and B between the two CTAs
  uint8_t* sA = sm;                       // K / 64 boxes of 128 rows x 128 B
  uint8_t* sB = sA + 256 * K * 2;         // MN-major: K rows x 128 B; K-major: K / 64 boxes of 64 rows
  __shared__ uint64_t bar_tma, bar_peer, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const uint32_t rank = cluster_rank();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    failed = 0;
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_peer, 1);
    mbar_init(&bar_mma, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc2(&tmem_base, 128);
    tmem_relinquish2();
  }
  __syncthreads();
  cluster_sync_all();   // both CTAs' barriers exist before the peer arrives on them
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  if (threadIdx.x == 0) {
    info[rank * 4 + 0] = tbase;
    info[rank * 4 + 1] = rank;
    mbar_arrive_expect_tx(&bar_tma, (uint32_t)(128 * K * 2 + 64 * K * 2));
    for (int k0 = 0; k0 < K; k0 += 64) tma_load_2d(sA + k0 * 256, &ta, k0, 128 * (int)rank, &bar_tma);
    if (b_mn) {
      tma_load_2d(sB, &tb, 64 * (int)rank, 0, &bar_tma);
    } else {
      for (int k0 = 0; k0 < K; k0 += 64) tma_load_2d(sB + k0 * 128, &tb, k0, 64 * (int)rank, &bar_tma);
    }
    bool ok = mbar_wait(&bar_tma, 0, 2000000000ull);
    if (!ok) failed = 1;
    if (rank == 1) {
      if (ok) mbar_arrive_cluster(mapa_rank(&bar_peer, 0));
    } else {
      if (ok && !mbar_wait_cluster(&bar_peer, 0, 2000000000ull)) {
        failed = 2;
        ok = false;
      }
      if (ok) {
        tc_fence_after();
        const uint32_t idesc = instr_desc(256, 128, 1, 1, 0, (uint32_t)b_mn, 0);
        for (int j = 0; j < K / 16; ++j) {
          const int box = j / 4, off = (j % 4) * 32;
          const uint64_t ad = smem_desc(smem_u32(sA + box * 128 * 128 + off), 16, 1024, kSw128);
          const uint64_t bd =
              b_mn ? smem_desc(smem_u32(sB + j * 16 * 128), (uint32_t)(K * 128), 1024, kSw128)
                   : smem_desc(smem_u32(sB + box * 64 * 128 + off), 16, 1024, kSw128);
          mma2_f16(tbase, ad, bd, idesc, j > 0 ? 1u : 0u);
        }
        mma2_commit_mc(&bar_mma, (uint16_t)3);
      }
    }
  }
  __syncthreads();
  if (!failed) {
    if (!mbar_wait_cluster(&bar_mma, 0, 2000000000ull)) atomicExch(&failed, 3);
  }
  tc_fence_after();
  if (!failed) {
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < 128; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) D[(128 * rank + row) * 128 + c0 + i] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // the peer's MMAs and reads are done before the pair frees its TMEM
  if (warp == 0) tmem_dealloc2(tbase, 128);
  if (threadIdx.x == 0) status[rank] = failed;
}

extern "C" int jtfs_selftest_umma_tf32(const float* A, const float* B, float* D, int K, int b_mn,
                                       int* status_dev, void* stream) {
  if (K < 32 || K > 64 || K % 32) return 1;
  CUtensorMap ta, tb;
  std::string err;
  {
    cuuint64_t dims[2] = {(cuuint64_t)K, 128};
    cuuint64_t str[1] = {(cuuint64_t)K * 4};
    cuuint32_t box[2] = {32, 128};
    if (!make_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A, dims, str, box, 128, &err)) return 2;
  }
  if (b_mn) {
    cuuint64_t dims[2] = {128, (cuuint64_t)K};
    cuuint64_t str[1] = {128 * 4};
    cuuint32_t box[2] = {32, (cuuint32_t)K};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, B, dims, str, box, 128, &err)) return 2;
  } else {
    cuuint64_t dims[2] = {(cuuint64_t)K, 128};
    cuuint64_t str[1] = {(cuuint64_t)K * 4};
    cuuint32_t box[2] = {32, 128};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, B, dims, str, box, 128, &err)) return 2;
  }
  const size_t smem = 1024 + (size_t)128 * K * 4 * 2;
  cudaFuncSetAttribute(k_umma_selftest_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_umma_selftest_tf32<<<1, 128, smem, (cudaStream_t)stream>>>(ta, tb, D, K, b_mn, status_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int jtfs_selftest_umma(const void* A, const void* B, float* D, int K, int a_swz,
                                  int b_mn, int* status_dev, void* stream) {
  if (K < 16 || K > 128 || K % 16 || (a_swz != 32 && a_swz != 64 && a_swz != 128)) return 1;
  if (K % (a_swz / 2)) return 1;
  if (!b_mn && K % 64) return 1;
  CUtensorMap ta, tb;
  std::string err;
  {
    cuuint64_t dims[2] = {(cuuint64_t)K, 128};
    cuuint64_t str[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {(cuuint32_t)(a_swz / 2), 128};
    if (!make_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, str, box, a_swz, &err))
      return 2;
  }
  if (b_mn) {
    cuuint64_t dims[2] = {128, (cuuint64_t)K};
    cuuint64_t str[1] = {128 * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)K};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, str, box, 128, &err)) return 2;
  } else {
    cuuint64_t dims[2] = {(cuuint64_t)K, 128};
    cuuint64_t str[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {64, 128};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, str, box, 128, &err)) return 2;
  }
  const size_t smem = 1024 + (size_t)128 * K * 2 * 2;
  cudaFuncSetAttribute(k_umma_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_umma_selftest<<<1, 128, smem, (cudaStream_t)stream>>>(ta, tb, D, K, a_swz, b_mn, status_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int jtfs_selftest_umma_ta(const void* A, const void* B, float* D, int K,
                                     int* status_dev, void* stream) {
  if (K < 16 || K > 128 || K % 16) return 1;
  CUtensorMap tb;
  std::string err;
  cuuint64_t dims[2] = {128, (cuuint64_t)K};
  cuuint64_t str[1] = {128 * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)K};
  if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, str, box, 128, &err)) return 2;
  const size_t smem = 1024 + (size_t)128 * K * 2;
  cudaFuncSetAttribute(k_umma_selftest_ta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_umma_selftest_ta<<<1, 128, smem, (cudaStream_t)stream>>>((const __bf16_raw_t*)A, tb, D, K,
                                                              status_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

extern "C" int jtfs_selftest_umma2(const void* A, const void* B, float* D, int K, int b_mn,
                                   int* status_dev, uint32_t* info_dev, void* stream) {
  if (K < 64 || K > 128 || K % 64) return 1;
  CUtensorMap ta, tb;
  std::string err;
  {
    cuuint64_t dims[2] = {(cuuint64_t)K, 256};
    cuuint64_t str[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {64, 128};
    if (!make_tmap(&ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, str, box, 128, &err)) return 2;
  }
  if (b_mn) {
    cuuint64_t dims[2] = {128, (cuuint64_t)K};
    cuuint64_t str[1] = {128 * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)K};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, str, box, 128, &err)) return 2;
  } else {
    cuuint64_t dims[2] = {(cuuint64_t)K, 128};
    cuuint64_t str[1] = {(cuuint64_t)K * 2};
    cuuint32_t box[2] = {64, 64};
    if (!make_tmap(&tb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, B, dims, str, box, 128, &err)) return 2;
  }
  const size_t smem = 1024 + (size_t)256 * K * 2 + (size_t)128 * K * 2;
  cudaFuncSetAttribute(k_umma2_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_umma2_selftest<<<2, 128, smem, (cudaStream_t)stream>>>(ta, tb, D, K, b_mn, status_dev, info_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
