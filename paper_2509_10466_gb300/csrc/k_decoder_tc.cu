// Decoder stages on tcgen05 tensor cores (BF16 form):
//   out = gelu(conv3x3(upsample2(in)) + bias),  in NHWC [B, Hi, Wi, Cin] in T,
//   out NHWC [B, 2Hi, 2Wi, Cout] in T (T = bf16 or f16: the 16-bit forms).
//
// Nearest x2 upsampling followed by a 3x3 conv is, for each output parity (a, b) of
// pixel (2i+a, 2j+b), a 2x2 conv on the low-resolution input with merged weights:
// input rows {i-1, i} for a = 0 (taps ky {0} and {1,2}) and {i, i+1} for a = 1 (taps
// {0,1} and {2}); the same for columns.  So each parity is an implicit GEMM with
// M = B*Hi*Wi pixels, N = Cout, K = 4*Cin (2.25x fewer products than 9*Cin).  The A
// tile of one (tap, 64-channel chunk) is a 4D TMA box {64 ch, 16 cols, 8 rows, 1 frame}
// of the NHWC input shifted by the tap offset; TMA's out-of-bounds fill supplies the
// conv's zero padding.  The merged weights are a K-major [4][Cout][4*Cin] matrix in T.
//
// Same persistent warp-specialized structure as the token GEMM: warp 0 TMA, warp 1
// MMA (M=128, N=Cout), two TMEM accumulators; the epilogue (bias, GELU, 16-bit, NHWC
// scatter to the parity's pixels) has two groups of 4 warps, group g draining the
// tiles that land in accumulator g, so two tiles are drained at once.  This M = pixels
// form (upconv_tc_kernel) serves inputs under 16 x 16 pixels and Cout of 96 or 128; at
// Cout = 32 and 64 the transposed form below (upconv_t_kernel) stacks the parities on M
// so that every MMA is 128 x 256 x 16.
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

template <int COUT, typename T>
__global__ void __launch_bounds__(THREADS, 1) upconv_tc_kernel(const __grid_constant__ CUtensorMap tmIn,
                                                               const __grid_constant__ CUtensorMap tmW, T* out,
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
      constexpr uint32_t idesc = tc::idesc_f32acc(H16<T>::kMmaFmt, BM, COUT);
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
      T* dst = out + (((size_t)img * Ho + oy) * Wo + ox) * COUT;
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
            packed[k] = H16<T>::pack2(x0, x1);
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

// Merged sub-pixel weights: wp[p][co][tap*Cin + ci] (in T), p = a*2 + b, tap = dy*2 + dx,
// summing the 3x3 taps that land on the same low-resolution input pixel.
template <typename T>
__global__ void subpixel_weights_kernel(const float* __restrict__ w, int Cout, int Cin, T* __restrict__ wp) {
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
    wp[e] = from_f32<T>(s);
  }
}

// ---------------------------------------------------------------------------------
// Transposed form for Cout = 32 or 64, with the parities stacked on the MMA's M side.
// The form above (M = pixels, N = Cout) issues narrow MMAs (N = 32 or 64), which keep
// the tensor core below its rate and need many more instructions per output.  Here a tile is a
// 16 x 16 block of input pixels (N = 256, pixel q = 16 py + px) and the accumulator row
// g * Cout + co holds output channel co of parity g of a group of NG = 128 / Cout parities
// (all four at Cout = 32; the two of output-row parity a at Cout = 64):
//   D[g Cout + co][q] = sum over input shifts (sy, sx) and channels ci of
//                       Ws[s][g Cout + co][ci] . in[i0 + py + sy][j0 + px + sx][ci]
// over the shifts any parity of the group uses (9 at Cout = 32, 6 at Cout = 64), with Ws
// the parity's merged 2 x 2-tap weight for that shift, or 0 where the parity does not
// read that shift (stacked_weights_kernel).  Every MMA is 128 x 256 x 16.  The epilogue
// thread of accumulator row (g, co) turns 32 pixels at a time into 16-bit GELU outputs,
// transposes them through a 2 KB shared tile (32 pixels x 32 channels) and stores 16-byte
// channel chunks of each output pixel (2 (i0 + py) + a, 2 (j0 + px) + b).
constexpr int TQ = 16;            // tile = TQ x TQ input pixels
constexpr int TB_ROWS = TQ + 2;   // a column-shifted pixel box spans the three row shifts
constexpr int A_STAGES = 4, B_STAGES = 2;
constexpr int T_THREADS = 320;    // warp 0 TMA, warp 1 MMA, warps 2-5 and 6-9: one epilogue group per accumulator

template <int COUT>
struct DecTCfg {
  static constexpr int NG = 128 / COUT;                 // parities per group (stacked on M)
  static constexpr int GROUPS = 4 / NG;
  static constexpr int NSH = NG == 4 ? 9 : 6;           // input shifts per group
  static constexpr int NY = NSH / 3;                    // row shifts per group (3 column shifts each)
  static constexpr int A_BYTES = 128 * BK * 2;          // stacked weights of one (shift, chunk)
  static constexpr int B_BYTES = TB_ROWS * TQ * BK * 2; // pixel rows i0 - 1 .. i0 + TQ at one column shift
  static constexpr int SMEM_BYTES = A_STAGES * A_BYTES + B_STAGES * B_BYTES + 1024 + 256 + 8 * 2048;
  static_assert(COUT == 32 || COUT == 64, "stacked parities need Cout = 32 or 64");
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB dynamic shared memory of an sm_100-family CTA");
};

// Input offset of 3x3 row tap ky for output-row parity a after nearest x2 upsampling:
// floor((a + ky - 1) / 2), in {-1, 0, 1}.
__host__ __device__ __forceinline__ int tap_offset(int a, int k) { return (a + k + 1) / 2 - 1; }

// Shift s of group grp as (sy, sx) and whether parity (a, b) reads it.
__device__ __forceinline__ void group_shift(int ng, int grp, int s, int& sy, int& sx) {
  if (ng == 4) { sy = s / 3 - 1; sx = s % 3 - 1; }
  else { sy = s / 3 + grp - 1; sx = s % 3 - 1; }
}

// ws[(grp * NSH + s) * 128 + g * Cout + co][ci] (in T): the sum of the 3x3 taps (ky, kx)
// of w[co][ci][ky][kx] whose inputs land on shift s for parity g of group grp, 0 where the
// parity does not read that shift.
template <typename T>
__global__ void stacked_weights_kernel(const float* __restrict__ w, int Cout, int Cin, T* __restrict__ ws) {
  const int ng = 128 / Cout, nsh = ng == 4 ? 9 : 6, groups = 4 / ng;
  const size_t n = (size_t)groups * nsh * 128 * Cin;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % Cin);
    const int row = (int)((e / Cin) % 128);
    const int gs = (int)(e / ((size_t)Cin * 128));
    const int s = gs % nsh, grp = gs / nsh;
    const int g = row / Cout, co = row % Cout;
    const int a = ng == 4 ? g >> 1 : grp, b = ng == 4 ? g & 1 : g;
    int sy, sx;
    group_shift(ng, grp, s, sy, sx);
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky)
      for (int kx = 0; kx < 3; ++kx)
        if (tap_offset(a, ky) == sy && tap_offset(b, kx) == sx) acc += w[((size_t)co * Cin + ci) * 9 + ky * 3 + kx];
    ws[e] = from_f32<T>(acc);
  }
}

// Per tile and 64-channel chunk, the pixel boxes are loaded once per column shift sx, 18
// rows high (rows i0 - 1 .. i0 + 16); the product of row shift sy reads the 16 x 16 block
// starting (sy + 1) pixel rows into the box, a contiguous run of 256 K-major rows, so
// the three (or two) row shifts share one box.  Stacked weights and pixel boxes stream
// through separate rings.
template <int COUT, typename T>
__global__ void __launch_bounds__(T_THREADS, 1) upconv_t_kernel(const __grid_constant__ CUtensorMap tmIn,
                                                                const __grid_constant__ CUtensorMap tmW, T* out,
                                                                int B, int Hi, int Wi, int Cin,
                                                                const float* __restrict__ bias, int* err) {
  using Cfg = DecTCfg<COUT>;
  constexpr int NG = Cfg::NG, GROUPS = Cfg::GROUPS, NSH = Cfg::NSH, NY = Cfg::NY;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;                                // [A_STAGES][128 x 64] stacked weights
  uint8_t* sB = smem + A_STAGES * Cfg::A_BYTES;      // [B_STAGES][18 x 16 pixels x 64]
  uint64_t* afull = reinterpret_cast<uint64_t*>(sB + B_STAGES * Cfg::B_BYTES);
  uint64_t* aempty = afull + A_STAGES;
  uint64_t* bfull = aempty + A_STAGES;
  uint64_t* bempty = bfull + B_STAGES;
  uint64_t* acc_full = bempty + B_STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* teardown = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(teardown + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint8_t* stage_tiles = sB + B_STAGES * Cfg::B_BYTES + 256;  // [8 epilogue warps][32 pixels][64 B]
  static_assert((2 * A_STAGES + 2 * B_STAGES + 5) * 8 + 8 <= 256, "barrier area");

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx_n = (Wi + TQ - 1) / TQ, by_n = (Hi + TQ - 1) / TQ;
  const int tiles = B * by_n * bx_n * GROUPS;
  const int kc = Cin / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < A_STAGES; ++s) { tc::mbar_init(&afull[s], 1); tc::mbar_init(&aempty[s], 1); }
    for (int s = 0; s < B_STAGES; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
    for (int a = 0; a < 2; ++a) { tc::mbar_init(&acc_full[a], 1); tc::mbar_init(&acc_empty[a], 4); }
    tc::mbar_init(teardown, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmIn);
    tc::prefetch_tmap(&tmW);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();
  pdl_wait();

  // tile -> (group fastest, then column block, row block, frame)
  auto decode = [&](int tile, int& grp, int& j0, int& i0, int& img) {
    grp = tile % GROUPS;
    int r = tile / GROUPS;
    j0 = (r % bx_n) * TQ;
    r /= bx_n;
    i0 = (r % by_n) * TQ;
    img = r / by_n;
  };

  if (warp == 0) {
    if (lane == 0) {
      uint32_t ga = 0, gb = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        int grp, j0, i0, img;
        decode(tile, grp, j0, i0, img);
        for (int ck = 0; ck < kc && ok; ++ck)
          for (int sxi = 0; sxi < 3 && ok; ++sxi) {
            const int c0 = ck * BK;
            {  // the pixel box of column shift sxi - 1
              const int s = gb % B_STAGES;
              if (gb >= (uint32_t)B_STAGES && !tc::mbar_wait(&bempty[s], ((gb / B_STAGES) & 1) ^ 1, abort_flag)) {
                ok = false;
                break;
              }
              tc::mbar_expect_tx(&bfull[s], Cfg::B_BYTES);
              tc::tma_load_4d(sB + s * Cfg::B_BYTES, &tmIn, &bfull[s], c0, j0 + sxi - 1, i0 - 1, img);
              ++gb;
            }
            for (int yi = 0; yi < NY; ++yi) {  // the stacked weights of shift (row shift yi, column shift sxi)
              const int s = ga % A_STAGES;
              if (ga >= (uint32_t)A_STAGES && !tc::mbar_wait(&aempty[s], ((ga / A_STAGES) & 1) ^ 1, abort_flag)) {
                ok = false;
                break;
              }
              tc::mbar_expect_tx(&afull[s], Cfg::A_BYTES);
              tc::tma_load_2d(sA + s * Cfg::A_BYTES, &tmW, &afull[s], c0, (grp * NSH + yi * 3 + sxi) * 128);
              ++ga;
            }
          }
      }
      // the loads land before the CTA may exit
      for (uint32_t h = (ga > (uint32_t)A_STAGES ? ga - A_STAGES : 0); h < ga; ++h)
        if (!tc::mbar_wait_timed(&afull[h % A_STAGES], (h / A_STAGES) & 1)) break;
      for (uint32_t h = (gb > (uint32_t)B_STAGES ? gb - B_STAGES : 0); h < gb; ++h)
        if (!tc::mbar_wait_timed(&bfull[h % B_STAGES], (h / B_STAGES) & 1)) break;
      if (!ok) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f32acc(H16<T>::kMmaFmt, 128, TQ * TQ);
      uint32_t ga = 0, gb = 0, i = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x, ++i) {
        int grp, j0, i0, img;
        decode(tile, grp, j0, i0, img);
        const uint32_t acc = i & 1, use = i >> 1;
        if (use >= 1 && !tc::mbar_wait(&acc_empty[acc], (use & 1) ^ 1, abort_flag)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dtm = tmem_base + acc * (TQ * TQ);
        bool first = true;
        for (int ck = 0; ck < kc && ok; ++ck)
          for (int sxi = 0; sxi < 3 && ok; ++sxi) {
            const int sb = gb % B_STAGES;
            if (!tc::mbar_wait(&bfull[sb], (gb / B_STAGES) & 1, abort_flag)) { ok = false; break; }
            ++gb;
            for (int yi = 0; yi < NY; ++yi) {
              const int sa = ga % A_STAGES;
              if (!tc::mbar_wait(&afull[sa], (ga / A_STAGES) & 1, abort_flag)) { ok = false; break; }
              ++ga;
              tc::fence_after_sync();
              // row shift sy = yi - 1 (four parities) or grp - 1 + yi (two): the block starts
              // sy + 1 pixel rows (of 16 x 128 B) into the box
              const int r0 = NG == 4 ? yi : grp + yi;
              const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sA + sa * Cfg::A_BYTES));
              const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sB + sb * Cfg::B_BYTES + r0 * TQ * 128));
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                tc::mma_f16(dtm, ad + 2 * kk, bd + 2 * kk, idesc, first ? 0u : 1u);
                first = false;
              }
              tc::mma_commit(&aempty[sa]);
            }
            tc::mma_commit(&bempty[sb]);
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
    const int quarter = warp & 3, grp_e = (warp - 2) >> 2;
    const int Ho = 2 * Hi, Wo = 2 * Wi;
    const int row = quarter * 32 + lane;             // accumulator row: parity g, channel co
    const int co = row % COUT;
    const int cbase = (quarter * 32) % COUT;         // first channel of this warp's rows
    uint8_t* tl = stage_tiles + (size_t)(warp - 2) * 2048;
    uint32_t i = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
      const uint32_t acc = i & 1, use = i >> 1;
      if ((int)acc != grp_e) continue;  // the other group drains this accumulator
      if (!tc::mbar_wait(&acc_full[acc], use & 1, abort_flag)) {
        if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      __syncwarp();
      tc::fence_after_sync();
      int grp, j0, i0, img;
      decode(tile, grp, j0, i0, img);
      // every row of a warp belongs to the same parity (a, b) = (wa, wb)
      const int wa = NG == 4 ? quarter >> 1 : grp, wb = NG == 4 ? quarter & 1 : quarter >> 1;
      const float bv = __ldg(bias + co);
      const uint32_t tbase = tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * (TQ * TQ);
#pragma unroll 1
      for (int c = 0; c < TQ * TQ; c += 32) {
        uint32_t v[32];
        tc::tmem_ld_32x32b_x32(tbase + c, v);
        tc::tmem_ld_wait();
        if (c + 32 >= TQ * TQ) {  // the accumulator is free once its last columns are read
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
        }
        // pixel c + k of channel co -> tile[k][lane] (16-bit)
#pragma unroll
        for (int k = 0; k < 32; ++k)
          *reinterpret_cast<T*>(tl + k * 64 + lane * 2) = from_f32<T>(gelu_as(__uint_as_float(v[k]) + bv));
        __syncwarp();
        // 16-byte chunk ch of pixel k: channels cbase + 8 ch .. +7 of output pixel (2 (i0 + py) + wa, 2 (j0 + px) + wb)
#pragma unroll
        for (int r4 = 0; r4 < 4; ++r4) {
          const int k = r4 * 8 + (lane >> 2), ch = lane & 3;
          const int q = c + k, py = q / TQ, px = q % TQ;
          const int pi = i0 + py, pj = j0 + px;
          if (pi < Hi && pj < Wi) {
            const uint4 val = *reinterpret_cast<const uint4*>(tl + k * 64 + ch * 16);
            T* dst = out + (((size_t)img * Ho + 2 * pi + wa) * Wo + 2 * pj + wb) * COUT + cbase + ch * 8;
            *reinterpret_cast<uint4*>(dst) = val;
          }
        }
        __syncwarp();
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 512);
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

template <int COUT, typename T>
cudaError_t launch_cout(const T* in, int B, int Hi, int Wi, int Cin, const T* wp, const float* bias, T* out, int* err,
                        cudaStream_t st) {
  using Cfg = DecCfg<COUT>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(upconv_tc_kernel<COUT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    if (fn(&mi, tc::tma_dtype<T>(), 4, const_cast<T*>(in), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)4 * Cin, (cuuint64_t)4 * COUT};
    cuuint64_t strides[1] = {(cuuint64_t)4 * Cin * 2};
    cuuint32_t box[2] = {BK, COUT};
    cuuint32_t es[2] = {1, 1};
    if (fn(&mw, tc::tma_dtype<T>(), 2, const_cast<T*>(wp), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int tiles = B * ((Hi + TH - 1) / TH) * ((Wi + TW - 1) / TW) * 4;
  const int grid = tiles < num_sms() ? tiles : num_sms();
  cudaError_t le = launch_pdl(upconv_tc_kernel<COUT, T>, grid, dim3(THREADS), Cfg::SMEM_BYTES, st, mi, mw, out, B, Hi,
                              Wi, Cin, bias, err);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

template <int COUT, typename T>
cudaError_t launch_t_cout(const T* in, int B, int Hi, int Wi, int Cin, const T* ws, const float* bias, T* out,
                          int* err, cudaStream_t st) {
  using Cfg = DecTCfg<COUT>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(upconv_t_kernel<COUT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    cuuint32_t box[4] = {BK, TQ, TB_ROWS, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (fn(&mi, tc::tma_dtype<T>(), 4, const_cast<T*>(in), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)Cin, (cuuint64_t)Cfg::GROUPS * Cfg::NSH * 128};
    cuuint64_t strides[1] = {(cuuint64_t)Cin * 2};
    cuuint32_t box[2] = {BK, 128};
    cuuint32_t es[2] = {1, 1};
    if (fn(&mw, tc::tma_dtype<T>(), 2, const_cast<T*>(ws), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int tiles = B * ((Hi + TQ - 1) / TQ) * ((Wi + TQ - 1) / TQ) * Cfg::GROUPS;
  const int grid = tiles < num_sms() ? tiles : num_sms();
  cudaError_t le = launch_pdl(upconv_t_kernel<COUT, T>, grid, dim3(T_THREADS), Cfg::SMEM_BYTES, st, mi, mw, out, B, Hi,
                              Wi, Cin, bias, err);
  if (le != cudaSuccess) return le;
  return cudaGetLastError();
}

}  // namespace

bool upconv_tc_supported(int Cin, int Cout) {
  return Cin % 64 == 0 && (Cout == 32 || Cout == 64 || Cout == 96 || Cout == 128);
}

template <typename T>
cudaError_t launch_subpixel_weights(const float* w, int Cout, int Cin, T* wp, cudaStream_t st) {
  subpixel_weights_kernel<T><<<256, 256, 0, st>>>(w, Cout, Cin, wp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_upconv_tc(const T* in, int B, int Hi, int Wi, int Cin, const T* wp, const float* bias, T* out,
                             int Cout, int* err, cudaStream_t st) {
  if (!upconv_tc_supported(Cin, Cout)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(wp)) & 15) return cudaErrorInvalidValue;
  switch (Cout) {
    case 32: return launch_cout<32, T>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    case 64: return launch_cout<64, T>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    case 96: return launch_cout<96, T>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
    default: return launch_cout<128, T>(in, B, Hi, Wi, Cin, wp, bias, out, err, st);
  }
}

}  // namespace inpaint

namespace inpaint {

bool upconv_t_supported(int Cin, int Cout, int Hi, int Wi) {
  return Cin % 64 == 0 && (Cout == 32 || Cout == 64) && Hi >= TQ && Wi >= TQ;
}

size_t upconv_t_weight_elems(int Cin, int Cout) {
  if (Cin % 64 || (Cout != 32 && Cout != 64)) return 0;
  const int ng = 128 / Cout;
  return (size_t)(4 / ng) * (ng == 4 ? 9 : 6) * 128 * Cin;
}

template <typename T>
cudaError_t launch_stacked_weights(const float* w, int Cout, int Cin, T* ws, cudaStream_t st) {
  if (!upconv_t_weight_elems(Cin, Cout)) return cudaErrorInvalidValue;
  stacked_weights_kernel<T><<<256, 256, 0, st>>>(w, Cout, Cin, ws);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_upconv_t(const T* in, int B, int Hi, int Wi, int Cin, const T* ws, const float* bias, T* out,
                            int Cout, int* err, cudaStream_t st) {
  if (!upconv_t_supported(Cin, Cout, Hi, Wi)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(ws) | reinterpret_cast<uintptr_t>(out)) & 15)
    return cudaErrorInvalidValue;
  if (Cout == 32) return launch_t_cout<32, T>(in, B, Hi, Wi, Cin, ws, bias, out, err, st);
  return launch_t_cout<64, T>(in, B, Hi, Wi, Cin, ws, bias, out, err, st);
}

#define INSTANTIATE(T)                                                                                              \
  template cudaError_t launch_subpixel_weights<T>(const float*, int, int, T*, cudaStream_t);                        \
  template cudaError_t launch_upconv_tc<T>(const T*, int, int, int, int, const T*, const float*, T*, int, int*,     \
                                           cudaStream_t);                                                           \
  template cudaError_t launch_stacked_weights<T>(const float*, int, int, T*, cudaStream_t);                         \
  template cudaError_t launch_upconv_t<T>(const T*, int, int, int, int, const T*, const float*, T*, int, int*,      \
                                          cudaStream_t);
INSTANTIATE(bf16)
INSTANTIATE(f16)
#undef INSTANTIATE

}  // namespace inpaint
