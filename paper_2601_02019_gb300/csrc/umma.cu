// tcgen05 tensor-core GEMM for sm_103a: TMA-fed, TMEM-accumulated, BF16 in,
// FP32 out, optional split-BF16 (three products) for near-FP32 accuracy.
//
//   D(m, n) = sum_{k in split z} A(m, k) B(n, k)         (both K-major, "TN")
//   out[z*plane + m*som + n*son] = D(m, n)
//
// A and B are read through 2-D TMA tensor maps (BF16, K innermost, 128-byte
// swizzle, box 64 x rows).  With npass = 3 the maps come in (hi, lo) pairs,
// x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and the block accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below FP32 resolution).
//
// Split-BF16 passes accumulate in two TMEM accumulators: the hi*hi products in
// one, every lower-order product in the other, added in the epilogue.  The
// tensor core's FP32 accumulation does not round to nearest, so each
// accumulate step can lose up to an ulp of the running sum; keeping the small
// correction terms out of the large accumulator makes their steps cost an ulp
// of a value ~2^8 smaller.
//
// One CTA computes a 128 x BN tile for one K split with 4 warps:
//   warp 0 (one lane)  TMA producer over a STAGES-deep shared-memory ring,
//   warp 1 (one lane)  issues tcgen05.mma (cta_group::1, kind::f16, M = 128),
//   warp 2             allocates / frees the TMEM accumulator (BN columns),
//   warps 0-3          epilogue: tcgen05.ld 32x32b, one accumulator row per thread.
// Every mbarrier wait is bounded: on a timeout the kernel records an error in
// *err and falls through, so a fault in the pipeline cannot hang the GPU.
#include <cuda.h>

#include <atomic>

#include "kernels.cuh"
#include "tc.cuh"

namespace as {

namespace {

constexpr int STAGES = 4;
// PRECISE (state-writing products, BN <= 64): each of the four K = 16 MMAs of
// a stage has its own hi*hi accumulator, so a K split of t tiles costs every
// accumulator t - 1 accumulate steps (the engine uses splits of at most four
// tiles) and the rest of the sum happens in FP32 registers (round to nearest)
// and in the FP64 plane reduction.
template <int BN, int NPASS, bool PRECISE>
__global__ void __launch_bounds__(128, 1) umma_gemm_kernel(const __grid_constant__ UmmaOperand opA,
                                                           const __grid_constant__ UmmaOperand opB, int M, int N,
                                                           int K, int klen, int b_row0, float* out, long long som,
                                                           long long son, long long plane, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr uint32_t A_BYTES = UM * UK * 2;
  constexpr uint32_t B_BYTES = BN * UK * 2;
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int fail_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * UM, n0 = blockIdx.y * BN, z = blockIdx.z;
  const int kb = z * klen, ke = min(K, kb + klen);
  const int ktiles = (ke > kb) ? (ke - kb + UK - 1) / UK : 0;
  const int niter = ktiles * NPASS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&done_bar, 1);
    fail_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr int NACC = PRECISE ? ((NPASS > 1) ? 5 : 4) : ((NPASS > 1) ? 2 : 1);
  static_assert(NACC * BN <= 512, "TMEM holds 512 columns");
  if (warp == 2) {
    // TMEM accumulators: NACC x BN columns, allocated as a power of two >= 32
    constexpr uint32_t need = (uint32_t)(NACC * BN);
    constexpr uint32_t ncols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0 && niter > 0) {
    // TMA producer
    for (int it = 0; it < niter; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u)) { atomicExch(&fail_s, 1); break; }
      const int kt = it / NPASS, pass = it % NPASS;
      const int kx = kb + kt * UK;
      const int la = (NPASS == 1) ? 0 : kPassA[pass], lb = (NPASS == 1) ? 0 : kPassB[pass];
      const CUtensorMap* ma = &opA.m[la];
      const CUtensorMap* mb = &opB.m[lb];
      mbar_expect_tx(&full_bar[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, ma, &full_bar[s], kx, m0);
      tma_load_2d(sB + s * B_BYTES, mb, &full_bar[s], kx, b_row0 + n0);
    }
  } else if (warp == 1 && lane == 0 && niter > 0) {
    // MMA issuer
    constexpr uint32_t idesc = idesc_bf16(BN);
    bool ok = true;
    for (int it = 0; it < niter; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!mbar_wait(&full_bar[s], ph)) { atomicExch(&fail_s, 1); ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
      const int pass = it % NPASS;
#pragma unroll
      for (int kk = 0; kk < UK / 16; ++kk) {
        // accumulator of this MMA and whether this is its first write
        int aidx;
        bool first;
        if (pass == 0) {
          aidx = PRECISE ? kk : 0;
          first = (it == 0) && (PRECISE || kk == 0);
        } else {
          aidx = PRECISE ? 4 : 1;
          first = (it == 1) && (kk == 0);
        }
        const uint32_t dst = tmem + (uint32_t)(aidx * BN);
        const uint64_t da = smem_desc(a0 + kk * 32), db = smem_desc(b0 + kk * 32);
        const uint32_t acc = first ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty_bar[s]))
                   : "memory");
    }
    (void)ok;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&done_bar))
                 : "memory");
  }
  __syncwarp();
  // epilogue: thread (warp w, lane l) owns accumulator row 32w + l
  const int row = warp * 32 + lane;
  const int gm = m0 + row;
  bool have = niter > 0;
  if (have && !mbar_wait(&done_bar, 0)) { atomicExch(&fail_s, 1); have = false; }
  have = __all_sync(0xffffffffu, have);   // tcgen05.ld below is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float* o = out + (long long)z * plane;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 16) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = 0.f;
    if (have) {
#pragma unroll
      for (int a = 0; a < NACC; ++a) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + a * BN);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(r[j]);
      }
    }
    if (gm < M) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int gn = n0 + c0 + j;
        if (gn < N) o[(long long)gm * som + (long long)gn * son] = v[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    constexpr uint32_t need = (uint32_t)(NACC * BN);
    constexpr uint32_t ncols = need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : (need <= 256 ? 256 : 512)));
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
  if (threadIdx.x == 0 && fail_s && err) atomicExch(err, AS_ETIMEOUT);
}

}  // namespace

namespace {

// x -> BF16 levels: l0 = bf16(x), l1 = bf16(x - l0), l2 = bf16(x - l0 - l1)
// (each residual is exact in FP32).  Source row-major (rows x cols, lds);
// destinations row-major with ldd; l1 / l2 may be null.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__global__ void split_bf16_kernel(const float* __restrict__ src, long long lds, int rows, int cols,
                                  __nv_bfloat16* __restrict__ l0, __nv_bfloat16* __restrict__ l1,
                                  __nv_bfloat16* __restrict__ l2, long long ldd) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e - (long long)r * cols);
    __nv_bfloat16 a, b, d;
    split3(src[(long long)r * lds + c], a, b, d);
    const long long o = (long long)r * ldd + c;
    l0[o] = a;
    if (l1) l1[o] = b;
    if (l2) l2[o] = d;
  }
}

// Transposing split: dst(c, r) = src(r, c); 32 x 32 tiles through shared memory.
__global__ void split_bf16_t_kernel(const float* __restrict__ src, long long lds, int rows, int cols,
                                    __nv_bfloat16* __restrict__ l0, __nv_bfloat16* __restrict__ l1,
                                    __nv_bfloat16* __restrict__ l2, long long ldd) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(long long)r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      __nv_bfloat16 a, b, d;
      split3(tile[threadIdx.x][i], a, b, d);
      const long long o = (long long)c * ldd + r;
      l0[o] = a;
      if (l1) l1[o] = b;
      if (l2) l2[o] = d;
    }
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  // looked up once; a function-local static is initialised thread-safely
  static const EncodeFn fn = []() -> EncodeFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeFn)p;
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

template <int BN, int NPASS, bool PRECISE>
as_status launch_umma_t(cudaStream_t s, const UmmaOperand& A, const UmmaOperand& B, int M, int N, int K, int splits,
                        int b_row0, float* out, long long som, long long son, long long plane, int* err) {
  const int ktiles = (K + UK - 1) / UK;
  int S = std::max(1, std::min(splits, ktiles));
  int klen = ((ktiles + S - 1) / S) * UK;
  S = (K + klen - 1) / klen;
  dim3 grid((M + UM - 1) / UM, (N + BN - 1) / BN, S);
  const size_t smem = (size_t)STAGES * (UM * UK * 2 + BN * UK * 2) + 1024;
  static std::atomic<int> configured_device{-1};   // the attribute is per device; set it once
  int dev = 0;
  AS_CUDA_TRY(cudaGetDevice(&dev));
  if (configured_device.load() != dev) {   // setting it twice from two threads is harmless
    AS_CUDA_TRY(cudaFuncSetAttribute(umma_gemm_kernel<BN, NPASS, PRECISE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    configured_device.store(dev);
  }
  umma_gemm_kernel<BN, NPASS, PRECISE><<<grid, 128, smem, s>>>(A, B, M, N, K, klen, b_row0, out, som, son, plane, err); count_launches(1);
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace

bool umma_available() { return encode_fn() != nullptr; }

as_status umma_make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int kdim, long long ld, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return AS_ENOTSUP;
  if (((uintptr_t)base & 15) || ((ld * 2) & 15) || (kdim % 8)) return AS_EINVAL;
  const cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)UK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? AS_OK : AS_EINVAL;
}

as_status launch_umma_gemm(cudaStream_t s, const UmmaOperand& A, const UmmaOperand& B, int M, int N, int K, int bn,
                           int npass, int splits, int b_row0, float* out, long long som, long long son, long long plane,
                           int* err, bool precise) {
  if (M <= 0 || N <= 0) return AS_OK;
  if (npass != 1 && npass != 3 && npass != 6) return AS_EINVAL;
  if (precise) {
    if (bn != 64) return AS_EINVAL;
    return npass == 6   ? launch_umma_t<64, 6, true>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err)
           : npass == 3 ? launch_umma_t<64, 3, true>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err)
                        : launch_umma_t<64, 1, true>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err);
  }
#define AS_UMMA_CASE(BNV)                                                                                          \
  if (bn == BNV)                                                                                                   \
    return npass == 6   ? launch_umma_t<BNV, 6, false>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err) \
           : npass == 3 ? launch_umma_t<BNV, 3, false>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err) \
                        : launch_umma_t<BNV, 1, false>(s, A, B, M, N, K, splits, b_row0, out, som, son, plane, err);
  AS_UMMA_CASE(32)
  AS_UMMA_CASE(64)
  AS_UMMA_CASE(128)
  AS_UMMA_CASE(192)
  AS_UMMA_CASE(256)
#undef AS_UMMA_CASE
  return AS_EINVAL;
}

int umma_bn_for(int N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  if (N <= 192) return 192;
  return 256;
}

as_status launch_split_bf16(cudaStream_t s, const float* src, long long lds, int rows, int cols, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, long long ldd, bool transpose, __nv_bfloat16* lo2) {
  if (rows <= 0 || cols <= 0) return AS_OK;
  if (transpose) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    split_bf16_t_kernel<<<grid, dim3(32, 8), 0, s>>>(src, lds, rows, cols, hi, lo, lo2, ldd); count_launches(1);
  } else {
    const long long tot = (long long)rows * cols;
    const int blocks = (int)std::min<long long>((tot + 255) / 256, 8192);
    split_bf16_kernel<<<blocks, 256, 0, s>>>(src, lds, rows, cols, hi, lo, lo2, ldd); count_launches(1);
  }
  AS_CUDA_TRY(cudaGetLastError());
  return AS_OK;
}

}  // namespace as
