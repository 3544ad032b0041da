// rhd_tc.cuh -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores.
//
//   D[m][n] = epilogue( sum_k A[m][k] * B[n][k] )     (A: M x K, B: N x K, both
//                                                      row-major = K-major)
//
// One CTA of 128 threads per 128-row tile of D, all N (<= 256) columns at
// once.  K is staged through shared memory in chunks of 64: the threads copy
// the chunk into the no-swizzle K-major core-matrix layout (8 rows x 16 bytes
// per core matrix), one elected thread issues four tcgen05.mma (K = 16 each)
// into a TMEM accumulator and commits them to an mbarrier, and the CTA waits
// on that barrier before the next chunk overwrites the staging buffers.  The
// epilogue reads the accumulator back with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31 = rows of the tile).  Every wait is bounded: on timeout the CTA
// raises an error flag and skips the rest (the context stays usable).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rhd {
namespace tc {

constexpr int kTileM = 128;
constexpr int kChunkK = 64;
// staging: A chunk 128 x 64 bf16 = 16 KB, B chunk up to 256 x 64 bf16 = 32 KB
constexpr int kStageA = kTileM * kChunkK * 2;
constexpr int kStageB = 256 * kChunkK * 2;
// the two core-matrix strides of a staged operand with R rows:
// K-adjacent core matrices are R/8 * 128 bytes apart (LBO), row-adjacent
// (8-row groups) 128 bytes apart (SBO)
__host__ __device__ constexpr uint32_t lbo_bytes(int rows) { return (uint32_t)(rows / 8) * 128u; }
constexpr uint32_t kSbo = 128u;
constexpr long long kWaitLimit = 1ll << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4, 14 bits each), descriptor version 1 at bit
// 46, base offset 0, no swizzle (layout type 0 in bits 61..63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

// Poll the barrier's phase `parity` until it completes, at most `limit`
// times; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          long long limit = kWaitLimit) {
  const uint32_t a = smem_addr(bar);
  for (long long k = 0; k < limit; ++k) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Whole warp: allocate ncols TMEM columns (power of two >= 32); the address
// is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// One MMA: D[tmem] (+)= A[sdesc] * B[sdesc]^T.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Copy rows [r0, r0 + R) x columns [k0, k0 + 64) of a row-major bf16 matrix
// (leading dimension ld elements, a multiple of 8; rows >= nrows and columns
// >= ncols read as 0) into the core-matrix layout at dst: element (r, k) at
// byte (k / 8) * lbo_bytes(R) + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
template <int R>
__device__ __forceinline__ void stage(uint8_t *dst, const __nv_bfloat16 *src, int64_t ld,
                                      int64_t r0, int64_t nrows, int64_t k0, int64_t ncols) {
  constexpr int kUnits = R * (kChunkK / 8);  // 16-byte units
  for (int u = threadIdx.x; u < kUnits; u += blockDim.x) {
    const int kc = u % (kChunkK / 8), r = u / (kChunkK / 8);
    const int64_t row = r0 + r, col = k0 + kc * 8;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (row < nrows) {
      const __nv_bfloat16 *p = src + row * ld + col;
      if (col + 8 <= ncols) {
        val = *reinterpret_cast<const uint4 *>(p);
      } else if (col < ncols) {
        __align__(16) __nv_bfloat16 t[8];
        for (int j = 0; j < 8; ++j) t[j] = col + j < ncols ? p[j] : __float2bfloat16(0.0f);
        val = *reinterpret_cast<const uint4 *>(t);
      }
    }
    *reinterpret_cast<uint4 *>(dst + kc * lbo_bytes(R) + (r / 8) * 128 + (r % 8) * 16) = val;
  }
}

// Epilogue kinds
enum Epi : int {
  kEpiStore = 0,      // D = acc (FP32)
  kEpiBiasGelu = 1,   // Z = acc + bias (FP32, kept for the backward pass);
                      // H = gelu(Z) (BF16, the next layer's input)
  kEpiBias = 2,       // D = acc + bias (FP32)
};

struct GemmArgs {
  const __nv_bfloat16 *A;  // [M][lda]
  const __nv_bfloat16 *B;  // [N][ldb]
  int64_t M, N, K, lda, ldb;
  float *D;                // [M][ldd] FP32 (Z for kEpiBiasGelu; may be null there)
  int64_t ldd;
  const float *bias;       // [N]
  __nv_bfloat16 *H;        // [M][ldh] (kEpiBiasGelu)
  int64_t ldh;
  int epi;
  int accumulate;          // D += result (kEpiStore only; split-K partial sums)
  unsigned *err;           // set to 1 on a wait timeout
  int wait_test;           // test only (0 otherwise): issue no MMA, so the first barrier
                           // wait runs out (after kTestWaitLimit polls) with nothing in flight
};
constexpr long long kTestWaitLimit = 64;

// tanh form of GELU, 0.5 z (1 + tanh(u)) with u = k0 (z + k1 z^3), written as
// z / (1 + e^-2u) (0.5 (1 + tanh u) is the logistic function of 2u): one fast
// exponential and one division, relative error ~1e-6 -- far below the BF16
// rounding the activation gets next.  e^-2u overflows to inf for z << 0, where
// the quotient is the correct 0.
__device__ __forceinline__ float gelu(float z) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (z + k1 * z * z * z);
  return __fdividef(z, 1.0f + __expf(-2.0f * u));
}

// NT = padded N (multiple of 16, <= 256); TCOLS = TMEM columns (power of 2 >= NT, >= 32).
template <int NT, int TCOLS>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  static_assert(NT % 16 == 0 && NT <= 256 && TCOLS >= NT && TCOLS >= 32, "tile");
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStageA;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int failed;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t m0 = (int64_t)blockIdx.x * kTileM;

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    failed = 0;
  }
  if (warp == 0) tmem_alloc(&tslot, TCOLS);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;

  constexpr uint32_t idesc = idesc_bf16(kTileM, NT);
  const int nchunks = (int)((g.K + kChunkK - 1) / kChunkK);
  unsigned phase = 0;
  for (int c = 0; c < nchunks; ++c) {
    const int64_t k0 = (int64_t)c * kChunkK;
    stage<kTileM>(sA, g.A, g.lda, m0, g.M, k0, g.K);
    stage<NT>(sB, g.B, g.ldb, 0, g.N, k0, g.K);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && !g.wait_test) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < kChunkK / 16; ++ks) {
        // K step ks covers core-matrix columns 2 ks and 2 ks + 1
        const uint64_t da = sdesc(smem_addr(sA) + 2 * ks * lbo_bytes(kTileM), lbo_bytes(kTileM), kSbo);
        const uint64_t db = sdesc(smem_addr(sB) + 2 * ks * lbo_bytes(NT), lbo_bytes(NT), kSbo);
        mma_bf16(tmem, da, db, idesc, c > 0 || ks > 0);
      }
      mma_commit(&bar);
    }
    const bool ok = mbar_wait(&bar, phase, g.wait_test ? kTestWaitLimit : kWaitLimit);
    phase ^= 1u;
    if (!ok) failed = 1;
    tc_fence_after();
    __syncthreads();
    if (failed) break;
  }

  if (!failed) {
    const int64_t row = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < NT; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      if (row < g.M) {
        for (int j = 0; j < 32; ++j) {
          const int64_t col = c0 + j;
          if (col >= g.N) break;
          float z = v[j];
          if (g.epi != kEpiStore) z += g.bias[col];
          if (g.epi == kEpiStore && g.accumulate) z += g.D[row * g.ldd + col];
          if (g.D) g.D[row * g.ldd + col] = z;
          if (g.epi == kEpiBiasGelu) g.H[row * g.ldh + col] = __float2bfloat16(gelu(z));
        }
      }
    }
  } else {
    // the MMAs of the abandoned chunk may still be in flight: give them one
    // more bounded wait before the accumulator is released (none were issued
    // in the wait test)
    mbar_wait(&bar, phase ^ 1u, g.wait_test ? kTestWaitLimit : kWaitLimit);
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(tmem, TCOLS);
}

__host__ constexpr size_t gemm_smem_bytes(int NT) { return (size_t)kStageA + (size_t)NT * kChunkK * 2; }

template <int NT, int TCOLS>
cudaError_t launch_nt(const GemmArgs &g, cudaStream_t st) {
  const size_t smem = gemm_smem_bytes(NT);
  const cudaError_t e = allow_smem<gemm_bf16_kernel<NT, TCOLS>>(smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (g.M + kTileM - 1) / kTileM;
  gemm_bf16_kernel<NT, TCOLS><<<(unsigned)tiles, 128, smem, st>>>(g);
  return cudaGetLastError();
}

// D = epi(A B^T) for 1 <= N <= 160 (the MLP's widths); lda, ldb multiples of 8.
inline cudaError_t gemm(const GemmArgs &g, cudaStream_t st) {
  if (g.M <= 0) return cudaSuccess;
  switch ((g.N + 15) / 16) {
    case 1: return launch_nt<16, 32>(g, st);
    case 2: return launch_nt<32, 32>(g, st);
    case 3: return launch_nt<48, 64>(g, st);
    case 4: return launch_nt<64, 64>(g, st);
    case 5: return launch_nt<80, 128>(g, st);
    case 6: return launch_nt<96, 128>(g, st);
    case 7: return launch_nt<112, 128>(g, st);
    case 8: return launch_nt<128, 128>(g, st);
    case 9: return launch_nt<144, 256>(g, st);
    case 10: return launch_nt<160, 256>(g, st);
    default: return cudaErrorInvalidValue;
  }
}

// out[c][r] = in[r][c] for a rows x cols bf16 matrix (leading dims ldi, ldo),
// through a 32 x 32 shared-memory tile.
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, int64_t rows,
                                      int64_t cols, int64_t ldi, __nv_bfloat16 *__restrict__ out,
                                      int64_t ldo) {
  __shared__ __nv_bfloat16 t[32][34];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    t[k][threadIdx.x] = (r < rows && c < cols) ? in[r * ldi + c] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < rows) out[c * ldo + r] = t[threadIdx.x][k];
  }
}

inline cudaError_t transpose(const __nv_bfloat16 *in, int64_t rows, int64_t cols, int64_t ldi,
                             __nv_bfloat16 *out, int64_t ldo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(in, rows, cols, ldi, out, ldo);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace rhd
