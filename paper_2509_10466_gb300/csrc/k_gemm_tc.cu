// 16-bit tensor-core GEMM on tcgen05 for the token GEMMs of the transformer blocks
// (QKV, attention projection + residual, MLP fc1 + GELU, fc2 + residual).
//
//   C[M, N] = epilogue(A[M, K] . Bt[N, K]^T),  A and Bt in T (bf16 or f16) with K
//   contiguous, FP32 accumulation in tensor memory.
//
// Persistent, warp-specialized CTA (one per SM):
//   warp 0        TMA producer: A and B tiles (BK = 64 -> one 128-byte swizzle row per
//                 tile row) into a STAGES-deep shared-memory ring;
//   warp 1        TMEM owner and MMA issuer: 4 x tcgen05.mma (M=128, N=BN, K=16) per
//                 stage, accumulating into one of two TMEM buffers;
//   warps 2..9    epilogue: two warps per TMEM lane quarter (32 rows each), splitting
//                 the tile's columns; tcgen05.ld of the finished accumulator, bias /
//                 GELU / residual / LayerNorm; global rows are read and written through a
//                 per-warp shared-memory tile so that every access instruction covers
//                 whole 64-byte row segments.  The other accumulator is filled by the
//                 next tile's MMAs meanwhile.
// Output tiles are visited N-fastest so consecutive CTAs reuse the same A rows from L2.
//
// EPI_RESID_LN (N == BN, a whole row per tile) also normalizes the new residual row:
// x = resid + acc + bias is stored (FP32) and y = LayerNorm(x) (eps 1e-5, biased
// variance, FP32 statistics) is stored in T for the next GEMM.  Each thread reduces
// its half row chunk by chunk (exact mean and squared deviations per 32 values, merged
// with Chan's pairwise formula), the two halves of a row are merged through shared
// memory, and the stored x is re-read (the warp's own rows) to normalize.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"
#include "warp_rows.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BK = 64;
constexpr int EW = 2;                       // epilogue warps per TMEM lane quarter
constexpr int EPI_WARPS = 4 * EW;
constexpr int THREADS = 64 + 32 * EPI_WARPS;

template <int BN>
struct TcCfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (BN == 256) ? 3 : (BN == 192 ? 4 : (BN == 128 ? 5 : 6));
  // two accumulators of BN columns, in an allocation of a power of two columns
  static constexpr int TMEM_COLS = 2 * BN <= 128 ? 2 * BN : (2 * BN <= 256 ? 256 : 512);
  static constexpr int COLS_PER_WARP = BN / EW;
  static constexpr int PARAM_FLOATS = 1024 + 2 * BN;       // bias (N <= 1024) and LayerNorm scale/shift
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align slack*/ + 256 /*barriers*/ +
                                    EPI_WARPS * 32 * 2 * 4 /*LayerNorm partial statistics*/ +
                                    PARAM_FLOATS * 4 + 1024 /*tile alignment*/ +
                                    EPI_WARPS * 3 * rows::TILE_BYTES /*two store tiles + a load tile per warp*/;
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB dynamic shared memory of an sm_100-family CTA");
};

struct GemmArgs {
  void* C;
  int ldc, M, N, K, epi;
  const float* bias;
  const float* resid;
  const float* ln_g;
  const float* ln_b;
  void* ln_out;
  int* err;
  int splits;  // split-K (EPI_NONE only): work item = (tile, split), split s sums k-blocks
               // [s nk / splits, (s + 1) nk / splits) into rows s * m_pad + m of C
  int m_pad;
};

// scalar loads: parameter vectors sit at any offset of the weight blob
__device__ __forceinline__ void load32(const float* __restrict__ p, float (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __ldg(p + i);
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int BN, typename T>
__global__ void __launch_bounds__(THREADS, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmB,
                                                             const __grid_constant__ CUtensorMap tmC,
                                                             const __grid_constant__ CUtensorMap tmLN,
                                                             const GemmArgs args) {
  using Cfg = TcCfg<BN>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * Cfg::STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;      // [2] MMA -> epilogue
  uint64_t* acc_empty = acc_full + 2;  // [2] epilogue -> MMA
  uint64_t* teardown = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(teardown + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ln_stats = reinterpret_cast<float*>(smem + S * Cfg::STAGE_BYTES + 256);  // [EPI_WARPS][32][2]
  float* s_bias = ln_stats + EPI_WARPS * 32 * 2;                                     // [1024]
  float* s_lng = s_bias + 1024;                                                      // [BN]
  float* s_lnb = s_lng + BN;                                                         // [BN]
  uint8_t* s_tile = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_lnb + BN) + 1023) &
                                               ~uintptr_t(1023));                  // [EPI_WARPS][3][2 KB]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = args.M, N = args.N;
  const int splits = args.splits > 1 ? args.splits : 1;
  const int tiles_n = N / BN, tiles = ((M + BM - 1) / BM) * tiles_n * splits, nk = args.K / BK;
  // work item -> output tile (N fastest, so consecutive CTAs share A rows in L2), split, k-blocks
  auto item = [&](int w, int& m0, int& n0, int& sp, int& kb0, int& kb1) {
    const int tt = w / splits;
    sp = w - tt * splits;
    m0 = (tt / tiles_n) * BM;
    n0 = (tt % tiles_n) * BN;
    kb0 = (int)((long long)sp * nk / splits);
    kb1 = (int)((long long)(sp + 1) * nk / splits);
  };
  int* err = args.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { tc::mbar_init(&acc_full[a], 1); tc::mbar_init(&acc_empty[a], EPI_WARPS); }
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
  // per-column epilogue parameters, read once per CTA
  const bool bias_smem = args.epi != EPI_NONE && N <= 1024;
  if (bias_smem)
    for (int c = threadIdx.x; c < N; c += blockDim.x) s_bias[c] = args.bias[c];
  if (args.epi == EPI_RESID_LN)
    for (int c = threadIdx.x; c < BN; c += blockDim.x) { s_lng[c] = args.ln_g[c]; s_lnb[c] = args.ln_b[c]; }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();
  pdl_wait();

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        int m0, n0, sp, kb0, kb1;
        item(tile, m0, n0, sp, kb0, kb1);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = g % S;
          if (g >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((g / S) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * Cfg::STAGE_BYTES;
          tc::mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
          tc::tma_load_2d(sa, &tmA, &full[s], kb * BK, m0);
          tc::tma_load_2d(sa + Cfg::A_BYTES, &tmB, &full[s], kb * BK, n0);
        }
      }
      // let the last copies land before the CTA may exit
      for (uint32_t h = (g > (uint32_t)S ? g - S : 0); h < g; ++h)
        if (!tc::mbar_wait_timed(&full[h % S], (h / S) & 1)) break;
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f32acc(H16<T>::kMmaFmt, BM, BN);
      uint32_t g = 0, i = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++i) {
        const uint32_t acc = i & 1, use = i >> 1;
        if (use >= 1 && !tc::mbar_wait(&acc_empty[acc], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dtm = tmem_base + acc * BN;
        int m0, n0, sp, kb0, kb1;
        item(tile, m0, n0, sp, kb0, kb1);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = g % S;
          if (!tc::mbar_wait(&full[s], (g / S) & 1, abort_flag)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * Cfg::STAGE_BYTES);
          const uint64_t ad = tc::desc_kmajor_sw128(sa);
          const uint64_t bd = tc::desc_kmajor_sw128(sa + Cfg::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            tc::mma_f16(dtm, ad + 2 * kk, bd + 2 * kk, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
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
    // epilogue: TMEM sub-partition (warp % 4) holds rows 32*(warp%4) .. +31; column group cg
    const int quarter = warp & 3, cg = (warp - 2) >> 2;
    const int epi = args.epi;
    const int c_lo = cg * Cfg::COLS_PER_WARP, c_hi = c_lo + Cfg::COLS_PER_WARP;
    const bool resid = epi == EPI_BIAS_RESID || epi == EPI_RESID_LN;
    rows::AsyncRows st{s_tile + (size_t)(warp - 2) * 3 * rows::TILE_BYTES, 0};
    uint8_t* tl = st.tiles + 2 * rows::TILE_BYTES;  // residual loads
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
      const uint32_t acc = i & 1, use = i >> 1;
      int m0, n0, sp, kb0, kb1;
      item(tile, m0, n0, sp, kb0, kb1);
      const int row0 = m0 + quarter * 32;    // this warp's 32 rows; the thread owns row0 + lane
      const int nvalid = M - row0;
      const int crow0 = sp * args.m_pad + row0;  // the row in C (split slices of m_pad rows)
      if (resid && lane < nvalid)  // the residual rows into L2 while the tile's MMAs run
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(args.resid + (size_t)(row0 + lane) * args.ldc +
                                                                        n0 + c_lo),
                     "r"(Cfg::COLS_PER_WARP * 4)
                     : "memory");
      if (!tc::mbar_wait(&acc_full[acc], use & 1, abort_flag)) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      __syncwarp();
      tc::fence_after_sync();
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * BN;
      float run_n = 0.f, run_mean = 0.f, run_m2 = 0.f;  // LayerNorm statistics of this part of the row
      float4 gn[8];  // residual loads of the next chunk, issued one chunk ahead
      if (resid) rows::load32_issue(args.resid + (size_t)row0 * args.ldc + n0 + c_lo, args.ldc, nvalid, lane, gn);
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
        const int col = n0 + c0;
        float rv[32];
        if (resid) {
          rows::load32_finish(tl, lane, gn, rv);
          if (c0 + 32 < c_hi) rows::load32_issue(args.resid + (size_t)row0 * args.ldc + col + 32, args.ldc, nvalid, lane, gn);
        }
        uint32_t r[32];
        tc::tmem_ld_32x32b_x32(tbase + c0, r);
        tc::tmem_ld_wait();
        float f[32];
        if (epi == EPI_NONE) {
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(r[j]);
          rows::store32_f32_async(&tmC, st, col, crow0, nvalid, lane, f);
          continue;
        }
        if (bias_smem) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 t = *reinterpret_cast<const float4*>(s_bias + col + j);
            f[j] = __uint_as_float(r[j]) + t.x;
            f[j + 1] = __uint_as_float(r[j + 1]) + t.y;
            f[j + 2] = __uint_as_float(r[j + 2]) + t.z;
            f[j + 3] = __uint_as_float(r[j + 3]) + t.w;
          }
        } else {
          float bv[32];
          load32(args.bias + col, bv);
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = __uint_as_float(r[j]) + bv[j];
        }
        if (epi == EPI_BIAS || epi == EPI_BIAS_GELU) {
          if (epi == EPI_BIAS_GELU) {
#pragma unroll
            for (int j = 0; j < 32; ++j) f[j] = gelu_as(f[j]);
          }
          rows::store32_h16_async<T>(&tmC, st, col, row0, nvalid, lane, f);
        } else if (epi == EPI_BIAS_F32) {
          rows::store32_f32_async(&tmC, st, col, row0, nvalid, lane, f);
        } else {  // residual (+ LayerNorm statistics; x stays in TMEM for the normalisation)
#pragma unroll
          for (int j = 0; j < 32; ++j) f[j] = rv[j] + f[j];
          rows::store32_f32_async(&tmC, st, col, row0, nvalid, lane, f);
          if (epi == EPI_RESID_LN) {
            uint32_t xr[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) xr[j] = __float_as_uint(f[j]);
            tc::tmem_st_32x32b_x32(tbase + c0, xr);
            float cm = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) cm += f[j];
            cm *= (1.f / 32.f);
            float cq = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) cq = fmaf(f[j] - cm, f[j] - cm, cq);
            const float nn = run_n + 32.f;
            const float dl = cm - run_mean;
            run_mean += dl * (32.f / nn);
            run_m2 += cq + dl * dl * (run_n * 32.f / nn);
            run_n = nn;
          }
        }
      }
      if (epi == EPI_RESID_LN) {
        tc::tmem_st_wait();
        // merge the EW column groups of each row (fixed order), then normalize the row held in TMEM
        float* sts = ln_stats + ((size_t)(warp - 2) * 32 + lane) * 2;
        sts[0] = run_mean;
        sts[1] = run_m2;
        named_sync(1 + quarter, 32 * EW);
        float mean = 0.f, m2 = 0.f, n = 0.f;
#pragma unroll
        for (int g2 = 0; g2 < EW; ++g2) {
          // the warp of column group g2 in this quarter is 2 + 4*g2 + ((quarter - 2) & 3)
          const float* o = ln_stats + ((size_t)(4 * g2 + ((quarter - 2) & 3)) * 32 + lane) * 2;
          const float om = o[0], oq = o[1], on = (float)Cfg::COLS_PER_WARP;
          const float nn = n + on;
          const float dl = om - mean;
          mean += dl * (on / nn);
          m2 += oq + dl * dl * (n * on / nn);
          n = nn;
        }
        named_sync(1 + quarter, 32 * EW);  // the statistics slots are reused by the next tile
        const float rstd = rsqrtf(m2 / n + 1e-5f);
#pragma unroll 1
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
          uint32_t xr[32];
          tc::tmem_ld_32x32b_x32(tbase + c0, xr);
          tc::tmem_ld_wait();
          float xv[32];
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 tg = *reinterpret_cast<const float4*>(s_lng + c0 + j);
            const float4 tb = *reinterpret_cast<const float4*>(s_lnb + c0 + j);
            xv[j] = (__uint_as_float(xr[j]) - mean) * rstd * tg.x + tb.x;
            xv[j + 1] = (__uint_as_float(xr[j + 1]) - mean) * rstd * tg.y + tb.y;
            xv[j + 2] = (__uint_as_float(xr[j + 2]) - mean) * rstd * tg.z + tb.z;
            xv[j + 3] = (__uint_as_float(xr[j + 3]) - mean) * rstd * tg.w + tb.w;
          }
          rows::store32_h16_async<T>(&tmLN, st, n0 + c0, row0, nvalid, lane, xv);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
    }
    rows::async_drain(lane);
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

// rows x inner matrix of 16-bit elements (tensor-map type dt), inner contiguous; box =
// box_inner x box_rows, 128-byte swizzle.
bool make_map_2d(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t rows,
                 uint32_t box_inner, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 2};
  cuuint32_t box[2] = {box_inner, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es,
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

// Store map of a [rows][inner] matrix (row pitch ld elements of es bytes; f32, else the
// 16-bit type dt16): 32-row boxes of 64 bytes in the 64-byte swizzle that the epilogue's
// staging tiles use.
bool make_store_map(CUtensorMap* m, const void* base, bool f32, CUtensorMapDataType dt16, uint64_t inner,
                    uint64_t rows, uint64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  const uint32_t es = f32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld * es};
  cuuint32_t box[2] = {64 / es, 32};
  cuuint32_t ess[2] = {1, 1};
  return fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : dt16, 2, const_cast<void*>(base), dims,
            strides, box, ess, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, typename T>
cudaError_t launch_bn(const T* A, const T* Bt, const GemmArgs& args, cudaStream_t st) {
  using Cfg = TcCfg<BN>;
  constexpr CUtensorMapDataType dt = tc::tma_dtype<T>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<BN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap ma, mb;
  if (!make_map_2d(&ma, dt, A, (uint64_t)args.K, (uint64_t)args.M, BK, BM)) return cudaErrorInvalidValue;
  if (!make_map_2d(&mb, dt, Bt, (uint64_t)args.K, (uint64_t)args.N, BK, BN)) return cudaErrorInvalidValue;
  const int tiles = ((args.M + BM - 1) / BM) * (args.N / BN) * (args.splits > 1 ? args.splits : 1);
  const int grid = tiles < num_sms() ? tiles : num_sms();
  // outputs: C (f32 for the residual epilogues and EPI_NONE, else T) and the LayerNorm output
  CUtensorMap mc, ml;
  const bool c32 = args.epi == EPI_NONE || args.epi == EPI_BIAS_RESID || args.epi == EPI_RESID_LN ||
                   args.epi == EPI_BIAS_F32;
  if ((reinterpret_cast<uintptr_t>(args.C) & 15) || (args.ldc * (c32 ? 4 : 2)) % 16) return cudaErrorInvalidValue;
  const uint64_t c_rows = args.splits > 1 ? (uint64_t)args.splits * args.m_pad : (uint64_t)args.M;
  if (!make_store_map(&mc, args.C, c32, dt, (uint64_t)args.N, c_rows, (uint64_t)args.ldc))
    return cudaErrorInvalidValue;
  ml = mc;
  if (args.epi == EPI_RESID_LN &&
      ((reinterpret_cast<uintptr_t>(args.ln_out) & 15) ||
       !make_store_map(&ml, args.ln_out, false, dt, (uint64_t)args.N, (uint64_t)args.M, (uint64_t)args.N)))
    return cudaErrorInvalidValue;
  cudaError_t le = launch_pdl(gemm_tc_kernel<BN, T>, grid, dim3(THREADS), Cfg::SMEM_BYTES, st, ma, mb, mc, ml, args);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_any(const T* A, const T* Bt, const GemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0 || a.K % BK || a.N % 64 || a.ldc % 8) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt)) & 15) return cudaErrorInvalidValue;
  if (a.epi != EPI_NONE && !a.bias) return cudaErrorInvalidValue;
  if (a.splits > 1 && (a.epi != EPI_NONE || a.m_pad < (a.M + BM - 1) / BM * BM || a.splits > a.K / BK))
    return cudaErrorInvalidValue;
  if (a.epi == EPI_RESID_LN) {  // a whole row per tile
    if (a.N == 256) return launch_bn<256, T>(A, Bt, a, st);
    if (a.N == 128) return launch_bn<128, T>(A, Bt, a, st);
    if (a.N == 64) return launch_bn<64, T>(A, Bt, a, st);
    return cudaErrorInvalidValue;
  }
  if (a.N % 256 == 0) return launch_bn<256, T>(A, Bt, a, st);
  if (a.N % 128 == 0) return launch_bn<128, T>(A, Bt, a, st);
  if (a.N % 192 == 0) return launch_bn<192, T>(A, Bt, a, st);  // d = 192 models: 192, 576
  return launch_bn<64, T>(A, Bt, a, st);
}

}  // namespace

bool gemm_tc_ln_supported(int N) { return N == 64 || N == 128 || N == 256; }

template <typename T>
cudaError_t launch_gemm_tc(const T* A, const T* Bt, void* C, int ldc, int M, int N, int K, int epi,
                           const float* bias, const float* resid, int* err, cudaStream_t st) {
  GemmArgs a{C, ldc, M, N, K, epi, bias, resid, nullptr, nullptr, nullptr, err, 1, 0};
  return launch_any<T>(A, Bt, a, st);
}

template <typename T>
cudaError_t launch_gemm_tc_resid_ln(const T* A, const T* Bt, float* X, int M, int N, int K, const float* bias,
                                    const float* ln_g, const float* ln_b, T* ln_out, int* err, cudaStream_t st) {
  GemmArgs a{X, N, M, N, K, EPI_RESID_LN, bias, X, ln_g, ln_b, ln_out, err, 1, 0};
  return launch_any<T>(A, Bt, a, st);
}

cudaError_t launch_gemm_tc_splitk(const bf16* A, const bf16* Bt, float* C, int M, int N, int K, int splits, int* err,
                                  cudaStream_t st) {
  const int m_pad = (M + BM - 1) / BM * BM;
  GemmArgs a{C, N, M, N, K, EPI_NONE, nullptr, nullptr, nullptr, nullptr, nullptr, err, splits, m_pad};
  return launch_any<bf16>(A, Bt, a, st);
}

#define INSTANTIATE(T)                                                                                           \
  template cudaError_t launch_gemm_tc<T>(const T*, const T*, void*, int, int, int, int, int, const float*,        \
                                         const float*, int*, cudaStream_t);                                       \
  template cudaError_t launch_gemm_tc_resid_ln<T>(const T*, const T*, float*, int, int, int, const float*,       \
                                                  const float*, const float*, T*, int*, cudaStream_t);
INSTANTIATE(bf16)
INSTANTIATE(f16)
#undef INSTANTIATE

}  // namespace inpaint
