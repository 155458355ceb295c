// BF16 tensor-core GEMM on tcgen05 for the token GEMMs of the transformer blocks
// (QKV, attention projection + residual, MLP fc1 + GELU, fc2 + residual).
//
//   C[M, N] = epilogue(A[M, K] . Bt[N, K]^T),  A and Bt bf16 with K contiguous,
//   FP32 accumulation in tensor memory.
//
// Persistent, warp-specialized CTA (one per SM):
//   warp 0      TMA producer: A and B tiles (BK = 64 -> one 128-byte swizzle row per
//               tile row) into a STAGES-deep shared-memory ring;
//   warp 1      TMEM owner and MMA issuer: 4 x tcgen05.mma (M=128, N=BN, K=16) per
//               stage, accumulating into one of two TMEM buffers;
//   warps 2..5  epilogue: tcgen05.ld of the finished accumulator, bias / GELU /
//               residual, vector stores; the other accumulator buffer is filled by
//               the next tile's MMAs meanwhile.
// Output tiles are visited N-fastest so consecutive CTAs reuse the same A rows from L2.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BK = 64;
constexpr int THREADS = 192;

template <int BN>
struct TcCfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (BN == 256) ? 4 : (BN == 128 ? 6 : 8);
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
};

__device__ __forceinline__ void store_row_chunk(int epi, void* C, int ldc, int row, int col, const float* bias,
                                                const float* resid, const float (&f)[32]) {
  if (epi == EPI_BIAS || epi == EPI_BIAS_GELU) {
    bf16* dst = reinterpret_cast<bf16*>(C) + (size_t)row * ldc + col;
    uint32_t packed[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float a = f[2 * i] + __ldg(bias + col + 2 * i);
      float b = f[2 * i + 1] + __ldg(bias + col + 2 * i + 1);
      if (epi == EPI_BIAS_GELU) { a = gelu_erf(a); b = gelu_erf(b); }
      __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      packed[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    uint4* d4 = reinterpret_cast<uint4*>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d4[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
  } else {
    float* dst = reinterpret_cast<float*>(C) + (size_t)row * ldc + col;
    float4* d4 = reinterpret_cast<float4*>(dst);
    if (epi == EPI_BIAS_RESID) {
      const float4* r4 = reinterpret_cast<const float4*>(resid + (size_t)row * ldc + col);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 r = r4[i];
        float4 o;
        o.x = r.x + (f[4 * i + 0] + __ldg(bias + col + 4 * i + 0));
        o.y = r.y + (f[4 * i + 1] + __ldg(bias + col + 4 * i + 1));
        o.z = r.z + (f[4 * i + 2] + __ldg(bias + col + 4 * i + 2));
        o.w = r.w + (f[4 * i + 3] + __ldg(bias + col + 4 * i + 3));
        d4[i] = o;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) d4[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(THREADS, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmB, void* C,
                                                             int ldc, int M, int N, int K, int epi,
                                                             const float* __restrict__ bias, const float* resid,
                                                             int* err) {
  using Cfg = TcCfg<BN>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;   // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;  // [2] epilogue -> MMA
  uint64_t* teardown = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(teardown + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = N / BN, tiles = ((M + BM - 1) / BM) * tiles_n, nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { tc::mbar_init(&acc_full[a], 1); tc::mbar_init(&acc_empty[a], 4); }
    tc::mbar_init(teardown, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (g >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((g / S) & 1) ^ 1, abort_flag)) goto producer_abort;
          uint8_t* sa = smem + s * Cfg::STAGE_BYTES;
          tc::mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
          tc::tma_load_2d(sa, &tmA, &full[s], kb * BK, m0);
          tc::tma_load_2d(sa + Cfg::A_BYTES, &tmB, &full[s], kb * BK, n0);
        }
      }
      // let the last copies land before the CTA may exit
      for (uint32_t h = (g > (uint32_t)S ? g - S : 0); h < g; ++h)
        if (!tc::mbar_wait_timed(&full[h % S], (h / S) & 1)) break;
      goto producer_done;
    producer_abort:
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      *abort_flag = 1;
    producer_done:;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
      uint32_t g = 0, i = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++i) {
        const uint32_t acc = i & 1, use = i >> 1;
        if (use >= 1 && !tc::mbar_wait(&acc_empty[acc], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dtm = tmem_base + acc * BN;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (!tc::mbar_wait(&full[s], (g / S) & 1, abort_flag)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * Cfg::STAGE_BYTES);
          const uint64_t ad = tc::desc_kmajor_sw128(sa);
          const uint64_t bd = tc::desc_kmajor_sw128(sa + Cfg::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            tc::mma_f16(dtm, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&acc_full[acc]);
      }
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
      // every issued MMA has finished before TMEM can be released
      tc::mma_commit(teardown);
      tc::mbar_wait_timed(teardown, 0);
    }
    __syncwarp();
  } else {
    // epilogue warps 2..5: TMEM sub-partition (warp % 4) holds rows 32*(warp%4) ...
    const int quarter = warp & 3;
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
      const uint32_t acc = i & 1, use = i >> 1;
      if (!tc::mbar_wait(&acc_full[acc], use & 1, abort_flag)) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      __syncwarp();
      tc::fence_after_sync();
      const int m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
      const int row = m0 + quarter * 32 + lane;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tbase + c0, r);
        tc::tmem_ld_wait();
        float f[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(r[j]);
        if (row < M) store_row_chunk(epi, C, ldc, row, n0 + c0, bias, resid, f);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// rows x inner bf16 matrix, inner contiguous; box = box_inner x box_rows, 128-byte swizzle.
bool make_map_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                 uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int BN>
cudaError_t launch_bn(const bf16* A, const bf16* Bt, void* C, int ldc, int M, int N, int K, int epi,
                      const float* bias, const float* resid, int* err, cudaStream_t st) {
  using Cfg = TcCfg<BN>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ma, mb;
  if (!make_map_2d(&ma, A, (uint64_t)K, (uint64_t)M, BK, BM)) return cudaErrorInvalidValue;
  if (!make_map_2d(&mb, Bt, (uint64_t)K, (uint64_t)N, BK, BN)) return cudaErrorInvalidValue;
  const int tiles = ((M + BM - 1) / BM) * (N / BN);
  const int grid = tiles < num_sms() ? tiles : num_sms();
  gemm_tc_kernel<BN><<<grid, THREADS, Cfg::SMEM_BYTES, st>>>(ma, mb, C, ldc, M, N, K, epi, bias, resid, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(const bf16* A, const bf16* Bt, void* C, int ldc, int M, int N, int K, int epi,
                           const float* bias, const float* resid, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || K % BK || N % 64 || ldc % 8) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt)) & 15) return cudaErrorInvalidValue;
  if (N % 256 == 0) return launch_bn<256>(A, Bt, C, ldc, M, N, K, epi, bias, resid, err, st);
  if (N % 128 == 0) return launch_bn<128>(A, Bt, C, ldc, M, N, K, epi, bias, resid, err, st);
  return launch_bn<64>(A, Bt, C, ldc, M, N, K, epi, bias, resid, err, st);
}

}  // namespace inpaint
