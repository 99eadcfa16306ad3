// Dense bf16 matrix product on the fifth-generation tensor cores:
//
//   C[M x N] = epilogue(A[M x K] B[N x K]^T),  A, B bf16 row-major (K contiguous),
//   float32 accumulation in tensor memory.
//
// One CTA of four warps per 128 x 128 tile of C.  Warp 0 (one thread) streams
// 128 x 64 tiles of A and B into a four-stage shared-memory ring with TMA
// (128-byte swizzle, out-of-range rows and columns read as zero); warp 1 (one
// thread) waits for each stage and issues four tcgen05.mma (K = 16 each) into
// a 128 x 128 float32 accumulator in tensor memory, releasing the stage with
// tcgen05.commit when its products are done; then all four warps read the
// accumulator back (warp w owns rows 32w..32w+31), apply the epilogue and
// store.  Every wait is bounded: a wait that gives up sets the error flag,
// the CTA drains its copies in flight, frees its tensor memory and returns.
//
// The epilogue (all optional): + bias[n], ReLU, x [mask[m, n] > 0],
// x oscale[n] + oshift[n]; the result is stored in float32 and, optionally,
// rounded to bf16 as a row-major and as a transposed copy (the operands of
// the next products).  It is the one the learned warm start's network
// needs (Sec. "learned warm start" of the library: not in the paper).
#include "mls_internal.cuh"
#include "umma.cuh"

#include <mutex>

namespace mls {

constexpr int kGemmBM = 128, kGemmBN = 128, kGemmBK = 64, kGemmStages = 4;
constexpr int kGemmTileA = kGemmBM * kGemmBK * 2;  // bytes per stage
constexpr int kGemmTileB = kGemmBN * kGemmBK * 2;
constexpr int kGemmSmem = kGemmStages * (kGemmTileA + kGemmTileB) + 1024;  // + alignment slack
constexpr uint32_t kGemmWaitLimit = 1u << 22;

__global__ void __launch_bounds__(128, 1) k_gemm_umma(const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                                                      float* __restrict__ C, int ldc, GemmEpilogue ep,
                                                      int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + kGemmStages * kGemmTileA;
  __shared__ uint64_t full_bar[kGemmStages], empty_bar[kGemmStages], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * kGemmBN;
  const int nk = (K + kGemmBK - 1) / kGemmBK;
  if (ep.lower && n0 > m0 + kGemmBM - 1) return;  // tile strictly above the diagonal (uniform per CTA)
  if (threadIdx.x == 0) {
    for (int s = 0; s < kGemmStages; ++s) {
      umma::mbar_init(&full_bar[s], 1);
      umma::mbar_init(&empty_bar[s], 1);
    }
    umma::mbar_init(&done_bar, 1);
    umma::mbar_fence_init();
    s_fail = 0;
    umma::tma_prefetch_map(&tmA);
    umma::tma_prefetch_map(&tmB);
  }
  if (warp == 0) {
    umma::tmem_alloc(&tmem_base, kGemmBN);
    umma::tmem_relinquish();
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tacc = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: stage kb % S holds the K-block kb; its use number is kb / S
    int issued = 0;
    bool failed = false;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kGemmStages;
      if (kb >= kGemmStages && !umma::mbar_wait(&empty_bar[s], ((kb / kGemmStages) - 1) & 1, kGemmWaitLimit)) {
        failed = true;
        break;
      }
      umma::mbar_arrive_expect_tx(&full_bar[s], kGemmTileA + kGemmTileB);
      umma::tma_load_2d(sA + s * kGemmTileA, &tmA, &full_bar[s], kb * kGemmBK, m0);
      umma::tma_load_2d(sB + s * kGemmTileB, &tmB, &full_bar[s], kb * kGemmBK, n0);
      ++issued;
    }
    if (failed) {
      s_fail = 1;
      // copies that may still be in flight: the last S issued
      for (int kb = issued > kGemmStages ? issued - kGemmStages : 0; kb < issued; ++kb)
        umma::mbar_wait(&full_bar[kb % kGemmStages], (kb / kGemmStages) & 1, kGemmWaitLimit);
    }
  } else if (warp == 1 && lane == 0) {
    // tensor-core issuer
    const uint32_t idesc = umma::idesc_bf16_f32(kGemmBM, kGemmBN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kGemmStages;
      if (!umma::mbar_wait(&full_bar[s], (kb / kGemmStages) & 1, kGemmWaitLimit)) {
        s_fail = 1;
        break;
      }
      umma::tc_fence_after();
      const uint32_t a0 = umma::smem_u32(sA + s * kGemmTileA), b0 = umma::smem_u32(sB + s * kGemmTileB);
#pragma unroll
      for (int k = 0; k < kGemmBK / 16; ++k)
        umma::mma_bf16(tacc, umma::sdesc_k_sw128(a0 + 32 * k), umma::sdesc_k_sw128(b0 + 32 * k), idesc,
                       (kb | k) ? 1u : 0u);
      umma::mma_commit(&empty_bar[s]);
    }
    umma::mma_commit(&done_bar);
  }
  __syncwarp();

  // epilogue: thread (warp, lane) owns row m0 + 32 warp + lane
  const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&done_bar, 0, kGemmWaitLimit) ? 1 : 0);
  umma::tc_fence_after();
  if (!ok) {
    if (lane == 0) s_fail = 1;
  } else if (nk > 0) {
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < kGemmBN && n0 + c0 < N; c0 += 16) {
      float v[16];
      umma::tmem_ld16(tacc + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (ep.acc64) {
        if (m < M) {
          double* arow = ep.acc64 + (int64_t)m * ep.ld64;
          const int em = ep.ea[m] - ep.ebias;
          const unsigned flip = ep.sign < 0.0 ? 0x80000000u : 0u;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + c0 + j;
            const unsigned fb = __float_as_uint(v[j]) ^ flip;
            if (n < N && (!ep.lower || n <= m) && (fb & 0x7fffffffu)) {
              // sign x 2^e x v as a double built from v's bits with integer
              // instructions (v is an integer below 2^24, a normal float;
              // float64 instructions issue at 1/64 rate here), then one add
              const int ex = (int)((fb >> 23) & 0xffu) - 127 + 1023 + em + ep.eb[n];
              const unsigned long long db = ((unsigned long long)(fb >> 31) << 63) |
                                            ((unsigned long long)(ex < 1 ? 0 : (ex > 2046 ? 2047 : ex)) << 52) |
                                            ((unsigned long long)(fb & 0x7fffffu) << 29);
              arow[n] += __longlong_as_double((long long)db);
            }
          }
        }
        continue;
      }
      if (m < M) {
        float* crow = C + (int64_t)m * ldc;
        const float* mrow = ep.mask ? ep.mask + (int64_t)m * ldc : nullptr;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c0 + j;
          if (n < N) {
            float x = v[j];
            if (ep.bias) x += ep.bias[n];
            if (ep.relu) x = fmaxf(x, 0.f);
            if (mrow && !(mrow[n] > 0.f)) x = 0.f;
            if (ep.oscale) x = x * ep.oscale[n] + ep.oshift[n];
            crow[n] = x;
            if (ep.out16) ep.out16[(int64_t)m * ep.ld16 + n] = __float2bfloat16(x);
            if (ep.out16t) ep.out16t[(int64_t)n * ep.ld16t + m] = __float2bfloat16(x);
          }
        }
      }
    }
  } else if (!ep.acc64) {
    // K = 0: the product is zero
    const int m = m0 + warp * 32 + lane;
    if (m < M)
      for (int n = n0; n < min(N, n0 + kGemmBN); ++n) {
        float x = 0.f;
        if (ep.bias) x += ep.bias[n];
        if (ep.relu) x = fmaxf(x, 0.f);
        if (ep.mask && !(ep.mask[(int64_t)m * ldc + n] > 0.f)) x = 0.f;
        if (ep.oscale) x = x * ep.oscale[n] + ep.oshift[n];
        C[(int64_t)m * ldc + n] = x;
        if (ep.out16) ep.out16[(int64_t)m * ep.ld16 + n] = __float2bfloat16(x);
        if (ep.out16t) ep.out16t[(int64_t)n * ep.ld16t + m] = __float2bfloat16(x);
      }
  }
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tacc, kGemmBN);
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ---- split-product trailing update of the coarse Cholesky ------------------------------
// A22 -= L21 L21^T on its lower triangle from the bf16 slices of L21's rows
// (the splitting of multilevel.cu: slice p of row i at columns p 128 ..
// p 128 + 127 of fwd, row exponents e).  One CTA per 128 x 64 tile of A22:
// the 64-row slices of the tile's columns (all eight, both 64-wide K blocks)
// stay in shared memory, the 128-row slices of its rows stream through a
// four-stage ring, and slice p of the rows times slice q of the columns
// accumulates into tensor-memory accumulator p + q (eight of 64 columns:
// all 512).  The epilogue sums accumulators 0..3 and 4..7 exactly in two
// 64-bit integers, scales each by a power of two, adds them in float64 (one
// rounding) and subtracts the result from A22 once; the tile's old values
// are loaded before the accumulators are read, and the tile is staged
// through shared memory so that rows are written whole.
// d 2^k for a double d that is zero or an integer below 2^53 in magnitude
// and a scaled result in the normal range: the exponent field moved by k
__device__ __forceinline__ double pow2_scale(double d, int k) {
  if (d == 0.0) return 0.0;
  return __longlong_as_double(__double_as_longlong(d) + ((long long)k << 52));
}

constexpr int kOzBM = 128, kOzBN = 64, kOzKB = kOzPanel / 64, kOzStagesA = 4;
constexpr int kOzTileA = kOzBM * 64 * 2;
constexpr int kOzTileB = kOzBN * 64 * 2;
constexpr int kOzSmemB = kOzSlices * kOzKB * kOzTileB;
constexpr int kOzSmem = kOzSmemB + kOzStagesA * kOzTileA + 1024;
static_assert(kOzSmem <= 227 * 1024, "split-product update: shared memory");
static_assert(kOzSlices * kOzBN <= 512, "split-product update: tensor memory");

__global__ void __launch_bounds__(128, 1) k_ozaki_syrk(const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB, int n,
                                                       const int* __restrict__ e, double* __restrict__ A, int lda,
                                                       int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sB = base;
  uint8_t* sA = base + kOzSmemB;
  __shared__ uint64_t bfull, full_bar[kOzStagesA], empty_bar[kOzStagesA], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kOzBM, n0 = blockIdx.x * kOzBN;
  if (n0 > m0 + kOzBM - 1) return;  // tile strictly above the diagonal (uniform per CTA)
  constexpr int na = kOzSlices * kOzKB;
  if (threadIdx.x == 0) {
    umma::mbar_init(&bfull, 1);
    for (int s = 0; s < kOzStagesA; ++s) {
      umma::mbar_init(&full_bar[s], 1);
      umma::mbar_init(&empty_bar[s], 1);
    }
    umma::mbar_init(&done_bar, 1);
    umma::mbar_fence_init();
    s_fail = 0;
    umma::tma_prefetch_map(&tmA);
    umma::tma_prefetch_map(&tmB);
  }
  if (warp == 0) {
    umma::tmem_alloc(&tmem_base, 512);
    umma::tmem_relinquish();
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tacc = tmem_base;

  if (warp == 0 && lane == 0) {
    umma::mbar_arrive_expect_tx(&bfull, kOzSmemB);
    for (int q = 0; q < kOzSlices; ++q)
      for (int kk = 0; kk < kOzKB; ++kk)
        umma::tma_load_2d(sB + (q * kOzKB + kk) * kOzTileB, &tmB, &bfull, q * kOzPanel + kk * 64, n0);
    int issued = 0;
    bool failed = false;
    for (int a = 0; a < na; ++a) {
      const int s = a % kOzStagesA;
      if (a >= kOzStagesA && !umma::mbar_wait(&empty_bar[s], ((a / kOzStagesA) - 1) & 1, kGemmWaitLimit)) {
        failed = true;
        break;
      }
      umma::mbar_arrive_expect_tx(&full_bar[s], kOzTileA);
      umma::tma_load_2d(sA + s * kOzTileA, &tmA, &full_bar[s], (a / kOzKB) * kOzPanel + (a % kOzKB) * 64, m0);
      ++issued;
    }
    if (failed) {
      s_fail = 1;
      umma::mbar_wait(&bfull, 0, kGemmWaitLimit);
      for (int a = issued > kOzStagesA ? issued - kOzStagesA : 0; a < issued; ++a)
        umma::mbar_wait(&full_bar[a % kOzStagesA], (a / kOzStagesA) & 1, kGemmWaitLimit);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = umma::idesc_bf16_f32(kOzBM, kOzBN);
    bool ok = umma::mbar_wait(&bfull, 0, kGemmWaitLimit);
    for (int a = 0; ok && a < na; ++a) {
      const int s = a % kOzStagesA;
      if (!umma::mbar_wait(&full_bar[s], (a / kOzStagesA) & 1, kGemmWaitLimit)) {
        ok = false;
        break;
      }
      umma::tc_fence_after();
      const int p = a / kOzKB, kk = a % kOzKB;
      const uint32_t a0 = umma::smem_u32(sA + s * kOzTileA);
      for (int q = 0; q < kOzSlices - p; ++q) {
        const uint32_t b0 = umma::smem_u32(sB + (q * kOzKB + kk) * kOzTileB);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          umma::mma_bf16(tacc + (uint32_t)(kOzBN * (p + q)), umma::sdesc_k_sw128(a0 + 32 * k),
                         umma::sdesc_k_sw128(b0 + 32 * k), idesc, (p | kk | k) ? 1u : 0u);
      }
      umma::mma_commit(&empty_bar[s]);
    }
    if (!ok) s_fail = 1;
    umma::mma_commit(&done_bar);
  }
  __syncthreads();
  const bool ok = __all_sync(0xffffffffu, umma::mbar_wait(&done_bar, 0, kGemmWaitLimit) ? 1 : 0);
  umma::tc_fence_after();
  if (!ok && lane == 0) s_fail = 1;
  __syncthreads();
  if (!s_fail) {
    const int m = m0 + warp * 32 + lane;
    const int em = m < n ? e[m] : 0;
    double* stage = (double*)sA + warp * 32 * 17;  // 32 rows x 16 columns (+1 pad) per warp
    for (int c0 = 0; c0 < kOzBN && n0 + c0 < n; c0 += 16) {
      int en[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) en[j] = n0 + c0 + j < n ? e[n0 + c0 + j] : 0;
      // this chunk's old values of A22, loaded now so that their latency
      // hides behind the accumulator reads and the sums below
      double old[16];
#pragma unroll
      for (int it = 0; it < 16; ++it) {
        const int row = 2 * it + (lane >> 4), col = lane & 15;
        const int mm = m0 + warp * 32 + row, nn = n0 + c0 + col;
        old[it] = (mm < n && nn < n && nn <= mm) ? A[(int64_t)mm * lda + nn] : 0.0;
      }
      // S_0..S_3 and S_4..S_7 summed exactly in two 64-bit integers
      // (sum_d S_d 2^(7 (3 - d)) stays below 2^46), then each scaled by a power
      // of two and added in float64 once
      long long hi[16], lo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
      for (int d = 0; d < kOzSlices; ++d) {
        float v[16];
        umma::tmem_ld16(tacc + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kOzBN * d + c0), v);
        const int sh = kOzBits * ((kOzSlices / 2 - 1) - (d % (kOzSlices / 2)));
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long t = (long long)__float2int_rz(v[j]) << sh;
          if (d < kOzSlices / 2) hi[j] += t;
          else lo[j] += t;
        }
      }
      double acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        // -(hi 2^(e - 35) + lo 2^(e - 63)), e = e_i + e_j: exact scalings, one rounding
        const int e = em + en[j];
        acc[j] = -(pow2_scale((double)hi[j], e - kOzBits * (kOzSlices / 2 + 1)) +
                   pow2_scale((double)lo[j], e - kOzBits * (kOzSlices + 1)));
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) stage[lane * 17 + j] = acc[j];
      __syncwarp();
#pragma unroll
      for (int it = 0; it < 16; ++it) {
        const int row = 2 * it + (lane >> 4), col = lane & 15;
        const int mm = m0 + warp * 32 + row, nn = n0 + c0 + col;
        if (mm < n && nn < n && nn <= mm) A[(int64_t)mm * lda + nn] = old[it] + stage[row * 17 + col];
      }
      __syncwarp();
    }
  }
  umma::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tacc, 512);
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

// ---- host side ------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// tensor map of a row-major bf16 matrix [rows][pitch] read as [rows][cols]
// tiles of box_rows x 64 with the 128-byte swizzle
static bool bf16_map(CUtensorMap* map, const void* ptr, int rows, int cols, int pitch, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

mls_status gemm_bf16_tn(cudaStream_t stream, int M, int N, int K, const __nv_bfloat16* A, int lda,
                        const __nv_bfloat16* B, int ldb, float* C, int ldc, const GemmEpilogue& ep, int* err) {
  if (M < 1 || N < 1 || K < 0 || !A || !B || (!C && !ep.acc64) || !err) return MLS_EINVAL;
  if (ep.acc64 && (!ep.ea || !ep.eb || ep.ld64 < N)) return MLS_EINVAL;
  if (lda < K || ldb < K || (!ep.acc64 && ldc < N) || (lda % 8) || (ldb % 8)) return MLS_EINVAL;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return MLS_EINVAL;
  CUtensorMap ma, mb;
  const int kk = K > 0 ? K : 8;
  if (!bf16_map(&ma, A, M, kk, lda, kGemmBM) || !bf16_map(&mb, B, N, kk, ldb, kGemmBN)) return MLS_ECUDA;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(k_gemm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  });
  if (attr_err != cudaSuccess) return MLS_ECUDA;
  const dim3 grid((N + kGemmBN - 1) / kGemmBN, (M + kGemmBM - 1) / kGemmBM);
  k_gemm_umma<<<grid, 128, kGemmSmem, stream>>>(ma, mb, M, N, K, C, ldc, ep, err);
  return cudaGetLastError() == cudaSuccess ? MLS_OK : MLS_ECUDA;
}

// A[i][j] -= (L21 L21^T)[i][j] for j <= i < n from the slices fwd [n][opitch]
// (slice p at columns p 128) and row exponents e; A row-major with pitch lda
mls_status ozaki_syrk(cudaStream_t stream, int n, const __nv_bfloat16* fwd, int opitch, const int* e, double* A,
                      int lda, int* err) {
  if (n < 1 || !fwd || !e || !A || !err || opitch < kOzSlices * kOzPanel || (opitch % 8) || lda < n) return MLS_EINVAL;
  CUtensorMap ma, mb;
  if (!bf16_map(&ma, fwd, n, kOzSlices * kOzPanel, opitch, kOzBM) ||
      !bf16_map(&mb, fwd, n, kOzSlices * kOzPanel, opitch, kOzBN))
    return MLS_ECUDA;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [] {
    attr_err = cudaFuncSetAttribute(k_ozaki_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  });
  if (attr_err != cudaSuccess) return MLS_ECUDA;
  const dim3 grid((n + kOzBN - 1) / kOzBN, (n + kOzBM - 1) / kOzBM);
  k_ozaki_syrk<<<grid, 128, kOzSmem, stream>>>(ma, mb, n, e, A, lda, err);
  return cudaGetLastError() == cudaSuccess ? MLS_OK : MLS_ECUDA;
}

}  // namespace mls

using namespace mls;

namespace {
// error flag of the public product entry point (one per device, looked up once)
__device__ int g_gemm_err;
std::mutex g_gemm_mutex;
}  // namespace

extern "C" mls_status mls_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                                    int32_t ldb, float* C, int32_t ldc, void* stream) {
  std::lock_guard<std::mutex> lock(g_gemm_mutex);
  int* err = nullptr;
  if (cudaGetSymbolAddress((void**)&err, g_gemm_err) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  const mls_status st = gemm_bf16_tn(s, M, N, K, (const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)B, ldb, C, ldc,
                                     GemmEpilogue{}, err);
  if (st != MLS_OK) return st;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  return h ? MLS_ETIMEOUT : MLS_OK;
}
