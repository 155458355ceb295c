// Decoder stages on tcgen05 tensor cores (BF16 form):
//   out = gelu(conv3x3(upsample2(in)) + bias),  in NHWC [B, Hi, Wi, Cin] bf16,
//   out NHWC [B, 2Hi, 2Wi, Cout] bf16.
//
// Nearest x2 upsampling followed by a 3x3 conv is, for each output parity (a, b) of
// pixel (2i+a, 2j+b), a 2x2 conv on the low-resolution input with merged weights:
// input rows {i-1, i} for a = 0 (taps ky {0} and {1,2}) and {i, i+1} for a = 1 (taps
// {0,1} and {2}); the same for columns.  So each parity is an implicit GEMM with
// M = B*Hi*Wi pixels, N = Cout, K = 4*Cin (2.25x fewer products than 9*Cin).  The A
// tile of one (tap, 64-channel chunk) is a 4D TMA box {64 ch, 16 cols, 8 rows, 1 frame}
// of the NHWC input shifted by the tap offset; TMA's out-of-bounds fill supplies the
// conv's zero padding.  The merged weights are a K-major [4][Cout][4*Cin] bf16 matrix.
//
// Same persistent warp-specialized structure as the token GEMM: warp 0 TMA, warp 1
// MMA (M=128, N=Cout), two TMEM accumulators; the epilogue (bias, GELU, bf16, NHWC
// scatter to the parity's pixels) has two groups of 4 warps, group g draining the
// tiles that land in accumulator g, so two tiles are drained at once.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "tc_primitives.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BK = 64, TW = 16, TH = 8;  // tile = 8 rows x 16 cols of input pixels
constexpr int THREADS = 320;  // warp 0 TMA, warp 1 MMA, warps 2-5 and 6-9: one epilogue group per accumulator
constexpr int STAGES = 6;

template <int COUT>
struct DecCfg {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = COUT * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TMEM_COLS = (2 * COUT <= 32) ? 32 : (2 * COUT <= 64 ? 64 : (2 * COUT <= 128 ? 128 : (2 * COUT <= 256 ? 256 : 512)));
  static constexpr int ACC_STRIDE = TMEM_COLS / 2;  // second accumulator starts on a power-of-two column
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB dynamic shared memory of an sm_100-family CTA");
};

template <int COUT>
__global__ void __launch_bounds__(THREADS, 1) upconv_tc_kernel(const __grid_constant__ CUtensorMap tmIn,
                                                               const __grid_constant__ CUtensorMap tmW, bf16* out,
                                                               int B, int Hi, int Wi, int Cin,
                                                               const float* __restrict__ bias, int* err) {
  using Cfg = DecCfg<COUT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* teardown = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(teardown + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx_n = (Wi + TW - 1) / TW, ty_n = (Hi + TH - 1) / TH;
  const int tiles = B * ty_n * tx_n * 4;
  const int kc = Cin / BK, nk = 4 * kc;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { tc::mbar_init(&acc_full[a], 1); tc::mbar_init(&acc_empty[a], 4); }
    tc::mbar_init(teardown, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmIn);
    tc::prefetch_tmap(&tmW);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();
  pdl_wait();

  // tile -> (parity p fastest, then column tile, row tile, frame)
  auto decode = [&](int tile, int& p, int& j0, int& i0, int& img) {
    p = tile & 3;
    int r = tile >> 2;
    j0 = (r % tx_n) * TW;
    r /= tx_n;
    i0 = (r % ty_n) * TH;
    img = r / ty_n;
  };

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        int p, j0, i0, img;
        decode(tile, p, j0, i0, img);
        const int a = p >> 1, b = p & 1;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          if (g >= (uint32_t)STAGES && !tc::mbar_wait(&empty[s], ((g / STAGES) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          const int tap = kb / kc, c0 = (kb - tap * kc) * BK;
          const int dy = tap >> 1, dx = tap & 1;
          const int oy = a == 0 ? dy - 1 : dy, ox = b == 0 ? dx - 1 : dx;
          uint8_t* sa = smem + s * Cfg::STAGE_BYTES;
          tc::mbar_expect_tx(&full[s], Cfg::STAGE_BYTES);
          tc::tma_load_4d(sa, &tmIn, &full[s], c0, j0 + ox, i0 + oy, img);
          tc::tma_load_2d(sa + Cfg::A_BYTES, &tmW, &full[s], kb * BK, p * COUT);
        }
      }
      for (uint32_t h = (g > (uint32_t)STAGES ? g - STAGES : 0); h < g; ++h)
        if (!tc::mbar_wait_timed(&full[h % STAGES], (h / STAGES) & 1)) break;
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, COUT);
      uint32_t g = 0, i = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++i) {
        const uint32_t acc = i & 1, use = i >> 1;
        if (use >= 1 && !tc::mbar_wait(&acc_empty[acc], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dtm = tmem_base + acc * Cfg::ACC_STRIDE;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % STAGES;
          if (!tc::mbar_wait(&full[s], (g / STAGES) & 1, abort_flag)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * Cfg::STAGE_BYTES);
          const uint64_t ad = tc::desc_kmajor_sw128(sa);
          const uint64_t bd = tc::desc_kmajor_sw128(sa + Cfg::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) tc::mma_f16(dtm, ad + 2 * kk, bd + 2 * kk, idesc, (kb | kk) != 0);
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&acc_full[acc]);
      }
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
      tc::mma_commit(teardown);
      tc::mbar_wait_timed(teardown, 0);
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3, grp = (warp - 2) >> 2;
    const int Ho = 2 * Hi, Wo = 2 * Wi;
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
      const uint32_t acc = i & 1, use = i >> 1;
      if ((int)acc != grp) continue;  // the other group drains this accumulator
      if (!tc::mbar_wait(&acc_full[acc], use & 1, abort_flag)) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      __syncwarp();
      tc::fence_after_sync();
      int p, j0, i0, img;
      decode(tile, p, j0, i0, img);
      const int r = quarter * 32 + lane;            // tile row = TMA box position (x fastest)
      const int pi = i0 + r / TW, pj = j0 + r % TW;
      const bool valid = pi < Hi && pj < Wi;
      const int oy = 2 * pi + (p >> 1), ox = 2 * pj + (p & 1);
      bf16* dst = out + (((size_t)img * Ho + oy) * Wo + ox) * COUT;
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * Cfg::ACC_STRIDE;
#pragma unroll 1
      for (int c0 = 0; c0 < COUT; c0 += 32) {
        uint32_t v[32];
        tc::tmem_ld_32x32b_x32(tbase + c0, v);
        tc::tmem_ld_wait();
        if (valid) {
          uint32_t packed[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const float x0 = gelu_as(__uint_as_float(v[2 * k]) + __ldg(bias + c0 + 2 * k));
            const float x1 = gelu_as(__uint_as_float(v[2 * k + 1]) + __ldg(bias + c0 + 2 * k + 1));
            __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            packed[k] = *reinterpret_cast<uint32_t*>(&h2);
          }
          uint4* d4 = reinterpret_cast<uint4*>(dst + c0);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            d4[k] = make_uint4(packed[4 * k], packed[4 * k + 1], packed[4 * k + 2], packed[4 * k + 3]);
        }
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

// Merged sub-pixel weights: wp[p][co][tap*Cin + ci] (bf16), p = a*2 + b, tap = dy*2 + dx,
// summing the 3x3 taps that land on the same low-resolution input pixel.
__global__ void subpixel_weights_kernel(const float* __restrict__ w, int Cout, int Cin, bf16* __restrict__ wp) {
  const size_t n = (size_t)4 * Cout * 4 * Cin;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % Cin);
    const int tap = (int)((e / Cin) % 4);
    const int co = (int)((e / (4 * (size_t)Cin)) % Cout);
    const int p = (int)(e / (4 * (size_t)Cin * Cout));
    const int a = p >> 1, b = p & 1, dy = tap >> 1, dx = tap & 1;
    // rows of the 3x3 kernel merged into input-row offset dy for parity a
    const int ky0 = (a == 0) ? (dy == 0 ? 0 : 1) : (dy == 0 ? 0 : 2);
    const int ky1 = (a == 0) ? (dy == 0 ? 0 : 2) : (dy == 0 ? 1 : 2);
    const int kx0 = (b == 0) ? (dx == 0 ? 0 : 1) : (dx == 0 ? 0 : 2);
    const int kx1 = (b == 0) ? (dx == 0 ? 0 : 2) : (dx == 0 ? 1 : 2);
    float s = 0.f;
    for (int ky = ky0; ky <= ky1; ++ky)
      for (int kx = kx0; kx <= kx1; ++kx) s += w[((size_t)co * Cin + ci) * 9 + ky * 3 + kx];
    wp[e] = __float2bfloat16_rn(s);
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

template <int COUT>
cudaError_t launch_cout(const bf16* in, int B, int Hi, int Wi, int Cin, const bf16* wp, const float* bias, bf16* out,
                        int* err, cudaStream_t st) {
  using Cfg = DecCfg<COUT>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(upconv_tc_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  auto fn = encode_fn();
  if (!fn) return cudaErrorInvalidValue;
  CUtensorMap mi, mw;
  {
    cuuint64_t dims[4] = {(cuuint64_t)Cin, (cuuint64_t)Wi, (cuuint64_t)Hi, (cuuint64_t)B};
    cuuint64_t strides[3] = {(cuuint64_t)Cin * 2, (cuuint64_t)Wi * Cin * 2, (cuuint64_t)Hi * Wi * Cin * 2};
    cuuint32_t box[4] = {BK, TW, TH, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (fn(&mi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)4 * Cin, (cuuint64_t)4 * COUT};
    cuuint64_t strides[1] = {(cuuint64_t)4 * Cin * 2};
    cuuint32_t box[2] = {BK, COUT};
    cuuint32_t es[2] = {1, 1};
    if (fn(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(wp), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int tiles = B * ((Hi + TH - 1) / TH) * ((Wi + TW - 1) / TW) * 4;
  const int grid = tiles < num_sms() ? tiles : num_sms();
  cudaError_t le = launch_pdl(upconv_tc_kernel<COUT>, grid, dim3(THREADS), Cfg::SMEM_BYTES, st, mi, mw, out, B, Hi,
                              Wi, Cin, bias, err);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

}  // namespace

bool upconv_tc_supported(int Cin, int Cout) {
  return Cin % 64 == 0 && (Cout == 32 || Cout == 64 || Cout == 96 || Cout == 128);
}

cudaError_t launch_subpixel_weights(const float* w, int Cout, int Cin, bf16* wp, cudaStream_t st) {
  subpixel_weights_kernel<<<256, 256, 0, st>>>(w, Cout, Cin, wp);
  return cudaGetLastError();
}

cudaError_t launch_upconv_tc(const bf16* in, int B, int Hi, int Wi, int Cin, const bf16* wp, const float* bias,
                             bf16* out, int Cout, int* err, cudaStream_t st) {
  if (!upconv_tc_supported(Cin, Cout)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(wp)) & 15) return cudaErrorInvalidValue;
  switch (Cout) {
    case 32: return launch_cout<32>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    case 64: return launch_cout<64>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    case 96: return launch_cout<96>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    default: return launch_cout<128>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
  }
}

}  // namespace inpaint
