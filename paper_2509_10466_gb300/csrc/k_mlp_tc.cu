// Fused attention projection + MLP of a transformer block on tcgen05 (the 16-bit forms:
// operands in T = bf16 or f16, FP32 accumulation), for a tile of token rows:
//   x1   = x + A . Wp + bp                      (MMA_P into TMEM; A = attention output)
//   Y    = normalized x1                         (T, written into the SMEM A buffer;
//                                                 LayerNorm2's affine part is folded into W1)
//   for hidden chunks j of 128 columns:
//     H_j  = gelu(Y . W1[:, j] + b1[j])         (MMA1 into TMEM, epilogue back into TMEM)
//     OUT += H_j . W2[j, :]                      (MMA2, A operand from TMEM; OUT holds x1)
//   x = OUT + b2, ln_out = normalized x: the next block's LN1 without its affine part
//   (folded into that block's QKV weights), or the final LN with it.
// Neither x1, its LayerNorm nor the hidden activations leave the SM: the intermediate
// residual row goes from the projection's accumulator into the output accumulator (as
// its starting value), so the only HBM traffic is the attention output and the residual
// row in, the new residual row and its LayerNorm out.
//
// CTA pairs (clusters of two SMs) run 2-SM MMAs (cta_group::2) over 256-row tiles: each
// CTA holds its own 128 rows of A / Y and of H_j and half of every weight block, the even
// CTA issues the MMAs for both, and each CTA's TMEM receives the accumulator rows of its
// own 128 rows.  Per SM this halves the weight bytes that stream from L2 for the same
// tensor work.
//
// A is loaded once per tile by TMA into SMEM; after MMA_P the drain warps overwrite it
// with Y in the 128-byte-swizzled K-major layout of a TMA load, the A operand of every
// MMA1.  Wp^T, W1^T ([hid][D]) and W2^T ([D][hid]) k-blocks stream through a ring of
// 16 KB stages in the order the MMA warp consumes them (MMA1 of chunk j+1 is issued
// before MMA2 of chunk j, so the tensor core works while the epilogue warps turn H_j
// into 16-bit values); the ring takes what shared memory is left.  TMEM: OUT (D cols) + two H
// buffers (128 cols each); MMA_P accumulates into the H buffers' columns, so the next
// tile's projection runs while the final drain still reads OUT.  The epilogue writes the 16-bit H_j over the FP32 columns it
// has just read (two hidden columns per 32-bit TMEM column, the tcgen05 A-operand
// layout).  Barriers that the MMA warp waits on live in the even CTA and count both CTAs'
// arrivals and TMA bytes; MMA completions are signalled to both CTAs.
//
// Warps: 0 TMA producer, 1 TMEM owner + MMA issuer (even CTA only; 2, 3 idle:
// warpgroup 0 hands its registers to the final warps), 4..11 hidden-chunk epilogue (two
// per TMEM lane quarter, splitting the chunk's columns), 12..15 final epilogue (one per
// lane quarter).  The tensor core idles while the accumulator is drained, twice per tile
// (after MMA_P: residual, LayerNorm2 into SMEM; after the last MMA2: store, LayerNorm),
// so three warps per lane quarter share both drains by columns (at D = 256: 64 columns
// for the final warp, 96 for each GELU warp; at D = 128: half and two quarters).  The three exchange per-row
// partial statistics (Welford) through shared memory and merge them in one fixed order.
// Residual rows are prefetched to L2 a tile ahead; the first 32-column block of each GELU
// warp's slice (all 128 rows of the CTA) is loaded by TMA into shared memory a tile ahead,
// the other blocks one block ahead into registers; rows move in whole 64-byte segments
// (warp_rows.cuh) and leave by TMA stores.  CTA pairs that get one tile fewer than the
// others start about half a tile late, so that their drains (all of a tile's HBM traffic)
// fall between those of the other pairs rather than on every SM at once.
#include <cuda.h>
#include <cudaTypedefs.h>


#include "common.cuh"
#include "tc_primitives.cuh"
#include "warp_rows.cuh"

namespace inpaint {

namespace {

constexpr int BM = 128, BK = 64, HC = 128;   // rows per CTA, k-block, hidden chunk
constexpr int NB = 2;                         // H buffers in TMEM (FP32, then 16-bit in place)
constexpr int LOOK = NB - 1;                  // MMA1 runs this many chunks ahead of MMA2
constexpr int ROLE_WARPS = 4;                 // warpgroup 0: TMA producer, MMA issuer, two idle
constexpr int EPI_WARPS = 8;                  // GELU warps: two per TMEM lane quarter
constexpr int OUT_WARPS = 4;                  // final-epilogue warps: one per lane quarter
constexpr int THREADS = 32 * (ROLE_WARPS + EPI_WARPS + OUT_WARPS);
constexpr uint16_t PAIR = 0x3;                // both CTAs of the cluster
// Registers per thread: launched with 65536 / THREADS; warpgroup 0 gives most of its share
// to the final-epilogue warpgroup.
constexpr int REG_LAUNCH = 65536 / THREADS / 8 * 8;
constexpr int REG_ROLE = 72, REG_FINAL = 184, REG_EPI = REG_LAUNCH;
static_assert(ROLE_WARPS * REG_ROLE + EPI_WARPS * REG_EPI + OUT_WARPS * REG_FINAL <=
                  (ROLE_WARPS + EPI_WARPS + OUT_WARPS) * REG_LAUNCH,
              "register reallocation exceeds the launch allotment");
constexpr int EPI_COLS = HC / (EPI_WARPS / 4);  // hidden columns of a chunk per GELU warp
static_assert(EPI_COLS % 32 == 0 && EPI_COLS <= 64, "GELU warp column split");
static_assert(EPI_WARPS == 8, "the output drain is shared by the final warp and two GELU warps per lane quarter");
constexpr int DRAIN_WARPS = EPI_WARPS + OUT_WARPS;
// Each drain warp stores by TMA from two staging tiles; residual rows are loaded through
// the first of them once the previous stores have read it.
constexpr int DRAIN_TILES = 2 * DRAIN_WARPS;

template <int D>
struct MlpCfg {
  static constexpr int A_BYTES = BM * D * 2;                  // this CTA's A (then Y) rows, D/64 atoms of 16 KB
  static constexpr int KA = D / BK;                           // k-blocks of MMA_P and MMA1
  static constexpr int KH = HC / BK;                          // k-blocks of MMA2 per chunk
  static constexpr int STAGE_BYTES = 16384;
  static constexpr int W1_BOX = (HC / 2) * BK * 2;            // this CTA's half of a W1 k-block (HC/2 rows)
  static constexpr int W1_KB = KA < STAGE_BYTES / W1_BOX ? KA : STAGE_BYTES / W1_BOX;  // k-blocks per stage
  static constexpr int W1_STAGES = KA / W1_KB;                // W1 stages per chunk
  static constexpr int W2_BOX = (D / 2) * BK * 2;             // this CTA's half of a Wp or W2 k-block (D/2 rows)
  static constexpr int PARAM_FLOATS = 1024 + 2 * D;          // b1 (hid <= 1024), b2, bp
  // 16 KB weight stages: as many as fit (up to two chunks' worth; four, one chunk, at D = 256)
  // Drain column slices, in 32-column blocks: the final warp takes the first FS blocks,
  // each GELU warp GS blocks (none when D = 64), as even as 32-column blocks allow.
  static constexpr int NCH = D / 32, GS = NCH == 8 ? 3 : NCH / 4, FS = NCH - 2 * GS;
  // the first residual block of each GELU warp's slice (all 128 rows), loaded by TMA a tile
  // ahead: two blocks of 128 rows x 32 FP32 columns
  static constexpr int RES_BYTES = GS > 0 ? 2 * BM * 32 * 4 : 0;
  static constexpr int FIXED_BYTES = A_BYTES + 1024 /*align slack*/ + 512 /*barriers*/ + (1024 + 2 * D) * 4 +
                                     1024 /*tile alignment*/ + DRAIN_TILES * rows::TILE_BYTES + 3 * BM * 2 * 4 +
                                     RES_BYTES;
  static constexpr int RING_FIT = (232448 - FIXED_BYTES) / STAGE_BYTES;
  static constexpr int RING = RING_FIT < 8 ? RING_FIT : 8;
  static_assert(RING >= 4, "weight ring too shallow");
  static constexpr int SMEM_BYTES = A_BYTES + RING * STAGE_BYTES + RES_BYTES + 1024 /*align slack*/ +
                                    512 /*barriers*/ + PARAM_FLOATS * 4 + 1024 /*tile alignment*/ +
                                    DRAIN_TILES * rows::TILE_BYTES /*staging tiles of the drain warps*/ +
                                    3 * BM * 2 * 4 /*partial row statistics of the three drain slices*/;
  static constexpr int H_COL0 = 256;                          // H buffers at TMEM columns 256 + HC b
  static_assert(H_COL0 + D <= 512 && NB * HC >= D, "MMA_P's accumulator lives in the H buffers' columns");
  static_assert(W1_KB * W1_BOX <= STAGE_BYTES && W2_BOX <= STAGE_BYTES, "stage too small");
  static_assert(SMEM_BYTES <= 232448, "exceeds the 227 KB dynamic shared memory of an sm_100-family CTA");
};

struct MlpArgs {
  float* X;              // residual stream [M, D] f32, updated in place
  void* ln_out;          // [M, D] of the operand type
  const float* bp;       // [D] projection bias
  const float* b1;       // [hid]
  const float* b2;       // [D]
  const float* ln_g;     // [D] affine part of the LayerNorm of ln_out, or null
  const float* ln_b;
  int M, hid;
  int* err;
  unsigned stagger_ns;   // start delay of the CTA pairs that get one tile fewer than the others
};


template <int D, typename T>
__global__ void __launch_bounds__(THREADS, 1) proj_mlp_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmWp,
                                                                 const __grid_constant__ CUtensorMap tmW1,
                                                            const __grid_constant__ CUtensorMap tmW2,
                                                            const __grid_constant__ CUtensorMap tmX,
                                                            const __grid_constant__ CUtensorMap tmLN,
                                                            const __grid_constant__ CUtensorMap tmXr,
                                                            const MlpArgs args) {
  using Cfg = MlpCfg<D>;
  constexpr int RING = Cfg::RING;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sR = sA + Cfg::A_BYTES;                      // ring
  uint8_t* s_res = sR + RING * Cfg::STAGE_BYTES;       // [2][128 rows x 128 B], 128-byte swizzle
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_res + Cfg::RES_BYTES);
  uint64_t* full = bar;                 // [RING]  even CTA: both CTAs' weight bytes
  uint64_t* empty = full + RING;        // [RING]  both: stage consumed by the pair's MMAs
  uint64_t* a_full = empty + RING;      //         even CTA: both CTAs' A bytes
  uint64_t* a_empty = a_full + 1;       //         both: Y no longer read
  uint64_t* p_full = a_empty + 1;       //         both: projection accumulator in OUT
  uint64_t* a_ready = p_full + 1;       //         even CTA: both CTAs wrote Y (SMEM) and x1 (OUT)
  uint64_t* h_full = a_ready + 1;       // [NB]    both: H_j in TMEM
  uint64_t* h_done = h_full + NB;       // [NB]    even CTA: both CTAs turned H_j into 16-bit values (in TMEM)
  uint64_t* o_full = h_done + NB;       //         both: OUT complete
  uint64_t* teardown = o_full + 1;
  uint64_t* stat_bar = teardown + 1;    // [4]     per lane quarter: the three drain slices' statistics
  uint64_t* res_full = stat_bar + 4;    //         this CTA: the GELU warps' first residual blocks landed
  uint64_t* res_empty = res_full + 1;   //         this CTA: the GELU warps read them
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(res_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* s_b1 = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bar) + 512);  // [hid]
  float* s_b2 = s_b1 + 1024;                                                      // [D]
  float* s_bp = s_b2 + D;
  uint8_t* s_tile = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(s_bp + D) + 1023) &
                                               ~uintptr_t(1023));  // [DRAIN_WARPS][2 KB]
  float* s_stat = reinterpret_cast<float*>(s_tile + DRAIN_TILES * rows::TILE_BYTES);  // [3][BM][mean, M2]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = args.M, NJ = args.hid / HC;
  const int tiles = (M + BM - 1) / BM;
  int* err = args.err;
  // Pair p covers tiles 2p (even CTA) and 2p+1 (odd CTA); the odd tile may lie past the
  // last one, the odd CTA then loads no Y rows and stores nothing.
  const int rank = (int)tc::cluster_ctarank();
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const int pairs = (tiles + 1) >> 1;
  // the even CTA's copy of a barrier (shared::cluster address): the pair's arrivals go there
  auto lead = [](const void* p) { return tc::mapa_shared(tc::smem_u32(p), 0); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < RING; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    tc::mbar_init(p_full, 1);
    tc::mbar_init(a_ready, 2 * DRAIN_WARPS);
    for (int b = 0; b < NB; ++b) {
      tc::mbar_init(&h_full[b], 1);
      tc::mbar_init(&h_done[b], 2 * EPI_WARPS);
    }
    tc::mbar_init(o_full, 1);
    for (int k = 0; k < 4; ++k) tc::mbar_init(&stat_bar[k], 3 * 32);
    tc::mbar_init(res_full, 1);
    tc::mbar_init(res_empty, EPI_WARPS);
    tc::mbar_init(teardown, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmWp);
    tc::prefetch_tmap(&tmW1);
    tc::prefetch_tmap(&tmW2);
    tc::prefetch_tmap(&tmXr);
  }
  if (warp == 1) {  // one warp of each CTA allocates the pair's TMEM together
    tc::tmem_alloc_pair(tmem_slot, 512);
    tc::tmem_relinquish_pair();
  }
  for (int c = threadIdx.x; c < args.hid; c += blockDim.x) s_b1[c] = args.b1[c];
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    s_b2[c] = args.b2[c];
    s_bp[c] = args.bp[c];
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::cluster_sync();  // both CTAs' barriers exist before any remote arrival
  tc::fence_after_sync();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();
  pdl_wait();
  // Every pair runs the same sequence of phases, and the drains (tensor core idle, all of the
  // tile's HBM traffic) would otherwise start on every SM at the same moment.  The pairs that
  // get one tile fewer than the others start about half a tile late: that costs them nothing
  // (they still finish before the others) and puts their drains between those of the others.
  if (args.stagger_ns && pairs % ncl != 0 && cid >= pairs % ncl) {
    const uint64_t t0 = tc::globaltimer();
    while (tc::globaltimer() - t0 < args.stagger_ns) __nanosleep(256);
  }

  // Both drains of pair p's tile (the t-th of this CTA) run in three warps per lane
  // quarter (warp & 3, 32 rows, the thread owning row row0 + lane), each over its slice of
  // nch 32-column blocks from column c_lo (slice `role`: 0 final warp, 1 and 2 the GELU
  // warps).  Rows move in whole 64-byte segments through the warp's two staging tiles:
  // stores go out by TMA from both (`st`), and `tl`, the first, serves the residual loads.

  // The slices' Welford partials of each row, merged by all three warps in one fixed
  // order (phase: the barrier's phase parity); mean and 1 / std of the whole row.
  auto row_stats = [&](int quarter, int role, uint32_t phase, float run_mean, float run_m2, float& mean,
                       float& rstd) -> bool {
    float* sr = s_stat + (size_t)(quarter * 32 + lane) * 2;
    sr[role * BM * 2] = run_mean;
    sr[role * BM * 2 + 1] = run_m2;
    tc::mbar_arrive(&stat_bar[quarter]);
    if (!tc::mbar_wait(&stat_bar[quarter], phase, abort_flag)) return false;
    float n = 0.f, m2 = 0.f;
    mean = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int nk = 32 * (k == 0 ? Cfg::FS : Cfg::GS);
      if (nk == 0) continue;
      const float mk = sr[k * BM * 2], qk = sr[k * BM * 2 + 1];
      const float nn = __fadd_rn(n, (float)nk);
      const float dl = __fsub_rn(mk, mean);
      mean = __fadd_rn(mean, __fmul_rn(dl, __fdiv_rn((float)nk, nn)));
      m2 = __fadd_rn(__fadd_rn(m2, qk), __fmul_rn(__fmul_rn(dl, dl), __fdiv_rn(__fmul_rn(n, (float)nk), nn)));
      n = nn;
    }
    rstd = rsqrtf(__fadd_rn(__fdiv_rn(m2, n), 1e-5f));
    return true;
  };
  // Exact mean and squared deviations of 32 values, merged into the running partial
  // (Chan's pairwise formula).
  auto block_stats = [](const float (&f)[32], float& run_n, float& run_mean, float& run_m2) {
    float cm = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) cm += f[k];
    cm *= (1.f / 32.f);
    float cq = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) cq = fmaf(f[k] - cm, f[k] - cm, cq);
    const float nn = run_n + 32.f;
    const float dl = cm - run_mean;
    run_mean += dl * (32.f / nn);
    run_m2 += cq + dl * dl * (run_n * 32.f / nn);
    run_n = nn;
  };

  // After MMA_P: x1 = x + P + bp into OUT (P: MMA_P's accumulator in the H columns; x1 is
  // the starting value of MMA2's accumulation), Y = (x1 - mean) / std in T into the
  // SMEM A buffer.  A warp's OUT columns are its own final-drain slice of the previous
  // tile, which it has finished.  Each residual
  // block is loaded while the previous one is processed, the first while MMA_P runs.
  auto mid = [&](int t, int p, int role, int c_lo, int nch, uint8_t* tl) -> bool {
    const int quarter = warp & 3, r = quarter * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    const int row0 = (2 * p + rank) * BM + quarter * 32;
    const int nvalid = M - row0;
    const float* xb = args.X + (size_t)row0 * D;
    // a GELU warp's first block comes from the TMA-loaded residual tile; the next block's
    // residual is loaded one block ahead (the first of them while MMA_P runs)
    const bool pre = Cfg::GS > 0 && role > 0;
    float4 gn[8];
    if (nch > (pre ? 1 : 0)) rows::load32_issue(xb + c_lo + (pre ? 32 : 0), D, nvalid, lane, gn);
    if (lane == 0) tc::bulk_wait_read<0>();  // the previous tile's stores are done with `tl`
    if (!tc::mbar_wait(p_full, t & 1, abort_flag)) return false;
    __syncwarp();
    tc::fence_after_sync();
    float run_n = 0.f, run_mean = 0.f, run_m2 = 0.f;
    if (nch > 0) {
#pragma unroll 1
      for (int c0 = c_lo; c0 < c_lo + 32 * nch; c0 += 32) {
        uint32_t v[32];
        tc::tmem_ld_32x32b_x32(lane_base + Cfg::H_COL0 + c0, v);
        float f[32];
        if (pre && c0 == c_lo) {  // row r of the prefetched block (128-byte rows, 128-byte swizzle)
          if (!tc::mbar_wait(res_full, t & 1, abort_flag)) return false;
          const uint8_t* rb = s_res + (role - 1) * (BM * 128) + r * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 q4 = *reinterpret_cast<const float4*>(rb + ((c ^ (r & 7)) << 4));
            f[4 * c] = q4.x; f[4 * c + 1] = q4.y; f[4 * c + 2] = q4.z; f[4 * c + 3] = q4.w;
          }
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(res_empty);  // read: the next tile's block may land
        } else {
          rows::load32_finish(tl, lane, gn, f);
          if (c0 + 32 < c_lo + 32 * nch) rows::load32_issue(xb + c0 + 32, D, nvalid, lane, gn);
        }
        tc::tmem_ld_wait();
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
          const float4 b = *reinterpret_cast<const float4*>(s_bp + c0 + k);
          f[k] += __uint_as_float(v[k]) + b.x;
          f[k + 1] += __uint_as_float(v[k + 1]) + b.y;
          f[k + 2] += __uint_as_float(v[k + 2]) + b.z;
          f[k + 3] += __uint_as_float(v[k + 3]) + b.w;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = __float_as_uint(f[k]);
        tc::tmem_st_32x32b_x32(lane_base + c0, v);
        block_stats(f, run_n, run_mean, run_m2);
      }
      tc::tmem_st_wait();
    }
    float mean, rstd;
    if (!row_stats(quarter, role, 0, run_mean, run_m2, mean, rstd)) return false;
#pragma unroll 1
    for (int c0 = c_lo; c0 < c_lo + 32 * nch; c0 += 32) {
      uint32_t xr[32];
      tc::tmem_ld_32x32b_x32(lane_base + c0, xr);
      tc::tmem_ld_wait();
      uint32_t pk[16];
#pragma unroll
      for (int k = 0; k < 32; k += 2)
        pk[k / 2] = H16<T>::pack2((__uint_as_float(xr[k]) - mean) * rstd, (__uint_as_float(xr[k + 1]) - mean) * rstd);
      // columns c0 .. c0+31 of row r: atom c0/64, 16-byte chunks (c0%64)/8 .. +3, swizzled by r%8
      uint8_t* rowp = sA + (c0 >> 6) * (BM * BK * 2) + r * 128;
      const int ch0 = (c0 & 63) >> 3;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        *reinterpret_cast<uint4*>(rowp + (((ch0 + k) ^ (r & 7)) << 4)) =
            make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
    }
    tc::fence_proxy_async_smem();  // Y is read by the tensor core (async proxy)
    tc::fence_before_sync();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive_cluster(lead(a_ready));
    return true;
  };

  // After the last MMA2: x = OUT + b2 stored and written back into OUT, ln_out =
  // (x - mean) / std (times ln_g plus ln_b for the final LayerNorm) stored; then OUT is free.
  const bool affine = args.ln_g != nullptr;
  auto fin = [&](int t, int p, int role, int c_lo, int nch, rows::AsyncRows& st) -> bool {
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    const int row0 = (2 * p + rank) * BM + quarter * 32;
    const int nvalid = M - row0;
    if (!tc::mbar_wait(o_full, t & 1, abort_flag)) return false;
    __syncwarp();
    tc::fence_after_sync();
    float run_n = 0.f, run_mean = 0.f, run_m2 = 0.f;
#pragma unroll 1
    for (int c0 = c_lo; c0 < c_lo + 32 * nch; c0 += 32) {
      uint32_t v[32];
      tc::tmem_ld_32x32b_x32(lane_base + c0, v);
      tc::tmem_ld_wait();
      float f[32];
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const float4 b = *reinterpret_cast<const float4*>(s_b2 + c0 + k);
        f[k] = __uint_as_float(v[k]) + b.x;
        f[k + 1] = __uint_as_float(v[k + 1]) + b.y;
        f[k + 2] = __uint_as_float(v[k + 2]) + b.z;
        f[k + 3] = __uint_as_float(v[k + 3]) + b.w;
      }
      rows::store32_f32_async_wide(&tmX, st, c0, row0, nvalid, lane, f);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = __float_as_uint(f[k]);
      tc::tmem_st_32x32b_x32(lane_base + c0, v);
      block_stats(f, run_n, run_mean, run_m2);
    }
    tc::tmem_st_wait();
    float mean, rstd;
    if (!row_stats(quarter, role, 1, run_mean, run_m2, mean, rstd)) return false;
#pragma unroll 1
    for (int c0 = c_lo; c0 < c_lo + 32 * nch; c0 += 32) {
      uint32_t v[32];
      tc::tmem_ld_32x32b_x32(lane_base + c0, v);
      tc::tmem_ld_wait();
      float xv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) xv[k] = (__uint_as_float(v[k]) - mean) * rstd;
      if (affine) {  // scalar loads: the parameters' offset in the weight blob has no alignment
#pragma unroll
        for (int k = 0; k < 32; ++k) xv[k] = xv[k] * __ldg(args.ln_g + c0 + k) + __ldg(args.ln_b + c0 + k);
      }
      rows::store32_h16_async<T>(&tmLN, st, c0, row0, nvalid, lane, xv);
    }
    tc::fence_before_sync();
    __syncwarp();
    return true;
  };

  if (warp < ROLE_WARPS) {
    tc::setmaxnreg_dec<REG_ROLE>();
    if (warp == 0) {
      if (lane == 0) {
        uint32_t g = 0;  // ring slot counter
        bool ok = true;
        // each CTA loads its half of every weight stage into its own ring slot; the even
        // CTA's barrier expects both halves
        auto push = [&](const CUtensorMap* map, int nbox, int c0, int c1, int box_bytes) {
          const int s = g % RING;
          if (g >= (uint32_t)RING && !tc::mbar_wait(&empty[s], ((g / RING) & 1) ^ 1, abort_flag)) return false;
          if (rank == 0) tc::mbar_expect_tx(&full[s], 2 * nbox * box_bytes);
          for (int b = 0; b < nbox; ++b)
            tc::tma_load_2d_pair(sR + s * Cfg::STAGE_BYTES + b * box_bytes, map, lead(&full[s]), c0 + b * BK, c1);
          ++g;
          return true;
        };
        int t = 0;
        for (int p = cid; p < pairs && ok; p += ncl, ++t) {
          const int m0 = (2 * p + rank) * BM;
          if (t >= 1 && !tc::mbar_wait(a_empty, (t - 1) & 1, abort_flag)) { ok = false; break; }
          if (rank == 0) tc::mbar_expect_tx(a_full, ((2 * p + 1) * BM < M ? 2 : 1) * Cfg::A_BYTES);
          if (m0 < M)
            for (int kb = 0; kb < Cfg::KA; ++kb)
              tc::tma_load_2d_pair(sA + kb * (BM * BK * 2), &tmA, lead(a_full), kb * BK, m0);
          if constexpr (Cfg::GS > 0) {  // the GELU warps' first residual blocks of this tile
            if (t >= 1 && !tc::mbar_wait(res_empty, (t - 1) & 1, abort_flag)) { ok = false; break; }
            if (m0 < M) {
              tc::mbar_expect_tx(res_full, Cfg::RES_BYTES);
              for (int g = 0; g < 2; ++g)
                tc::tma_load_2d(s_res + g * (BM * 128), &tmXr, res_full, 32 * (Cfg::FS + g * Cfg::GS), m0);
            } else {
              tc::mbar_arrive(res_full);  // no rows: the phase completes without bytes
            }
          }
          for (int kb = 0; kb < Cfg::KA && ok; ++kb)  // the projection's k-blocks first
            ok = push(&tmWp, 1, kb * BK, rank * (D / 2), Cfg::W2_BOX);
          for (int j = 0; j < NJ + LOOK && ok; ++j) {  // the MMA warp's consumption order
            if (j < NJ)
              for (int st = 0; st < Cfg::W1_STAGES && ok; ++st)
                ok = push(&tmW1, Cfg::W1_KB, st * Cfg::W1_KB * BK, j * HC + rank * (HC / 2), Cfg::W1_BOX);
            if (j >= LOOK)
              for (int kb = 0; kb < Cfg::KH && ok; ++kb)
                ok = push(&tmW2, 1, (j - LOOK) * HC + kb * BK, rank * (D / 2), Cfg::W2_BOX);
          }
        }
        // every signal addressed to this CTA has landed before it may exit: the pair's
        // releases of the last stages and of the last A / Y tile
        for (uint32_t h = (g > (uint32_t)RING ? g - RING : 0); h < g; ++h)
          if (!tc::mbar_wait_timed(&empty[h % RING], (h / RING) & 1)) break;
        if (t >= 1) tc::mbar_wait_timed(a_empty, (t - 1) & 1);
        if (Cfg::GS > 0 && t >= 1) tc::mbar_wait_timed(res_full, (t - 1) & 1);
        if (!ok) {
          if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
          *abort_flag = 1;
        }
      }
      __syncwarp();
    } else if (warp == 1 && rank == 0) {
      if (lane == 0) {
        constexpr uint32_t id1 = tc::idesc_f32acc(H16<T>::kMmaFmt, 2 * BM, HC);
        constexpr uint32_t id2 = tc::idesc_f32acc(H16<T>::kMmaFmt, 2 * BM, D);
        uint32_t g = 0, q = 0;  // ring slot counter, hidden-chunk counter (across tiles)
        bool ok = true;
        auto pop = [&](int& s) {
          s = g % RING;
          // weight bytes of both CTAs, counted by the TMA transactions themselves
          if (!tc::mbar_wait(&full[s], (g / RING) & 1, abort_flag)) return false;
          tc::fence_after_sync();
          ++g;
          return true;
        };
        auto mma1 = [&](uint32_t qq) {  // H[qq % NB] = Y . W1_chunk^T
          const uint32_t hb = qq % NB, use = qq / NB;
          // H buffer free: the previous use's GELU read it (h_done cannot run two phases
          // ahead: its next phase needs this very MMA1), and that use's MMA2, issued
          // before this MMA1, read the 16-bit values before this MMA1 overwrites them
          if (use >= 1 && !tc::mbar_wait(&h_done[hb], (use & 1) ^ 1, abort_flag)) return false;
          tc::fence_after_sync();
          const uint32_t dt = tmem_base + Cfg::H_COL0 + hb * HC;
          for (int st = 0; st < Cfg::W1_STAGES; ++st) {
            int s;
            if (!pop(s)) return false;
            for (int b = 0; b < Cfg::W1_KB; ++b) {
              const int kb = st * Cfg::W1_KB + b;
              const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sA + kb * (BM * BK * 2)));
              const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sR + s * Cfg::STAGE_BYTES + b * Cfg::W1_BOX));
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) tc::mma_f16_pair(dt, ad + 2 * kk, bd + 2 * kk, id1, (kb | kk) != 0);
            }
            tc::mma_commit_pair(&empty[s], PAIR);
          }
          tc::mma_commit_pair(&h_full[hb], PAIR);
          return true;
        };
        auto mma2 = [&](uint32_t qq, bool last) {  // OUT += 16-bit H[qq % NB] . W2_chunk^T
          const uint32_t hb = qq % NB, use = qq / NB;
          if (!tc::mbar_wait(&h_done[hb], use & 1, abort_flag)) return false;
          tc::fence_after_sync();
          for (int kb = 0; kb < Cfg::KH; ++kb) {
            int s;
            if (!pop(s)) return false;
            const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sR + s * Cfg::STAGE_BYTES));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // hidden column k lives in GELU warp k / EPI_COLS's columns, two per TMEM column
              const int k = kb * BK + kk * 16;
              const uint32_t at = tmem_base + Cfg::H_COL0 + hb * HC + (k / EPI_COLS) * EPI_COLS + (k % EPI_COLS) / 2;
              tc::mma_f16_pair_ta(tmem_base, at, bd + 2 * kk, id2, 1u);
            }
            tc::mma_commit_pair(&empty[s], PAIR);
          }
          if (last) tc::mma_commit_pair(o_full, PAIR);
          return true;
        };
        // P = A . Wp^T into the H columns: the previous tile's MMA2s, issued before, have
        // read them (tcgen05 MMAs run in issue order); its final drain may still read OUT
        auto mma_p = [&](int t) {
          if (!tc::mbar_wait(a_full, t & 1, abort_flag)) return false;
          tc::fence_after_sync();
          for (int kb = 0; kb < Cfg::KA; ++kb) {
            int s;
            if (!pop(s)) return false;
            const uint64_t ad = tc::desc_kmajor_sw128(tc::smem_u32(sA + kb * (BM * BK * 2)));
            const uint64_t bd = tc::desc_kmajor_sw128(tc::smem_u32(sR + s * Cfg::STAGE_BYTES));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              tc::mma_f16_pair(tmem_base + Cfg::H_COL0, ad + 2 * kk, bd + 2 * kk, id2, (kb | kk) != 0);
            tc::mma_commit_pair(&empty[s], PAIR);
          }
          tc::mma_commit_pair(p_full, PAIR);
          // Y in SMEM and x1 in OUT, from both CTAs
          if (!tc::mbar_wait_cluster(a_ready, t & 1, abort_flag)) return false;
          tc::fence_after_sync();
          return true;
        };
        int t = 0;
        for (int p = cid; p < pairs && ok; p += ncl, ++t) {
          ok = mma_p(t);
          const uint32_t q0 = q;
          for (int j = 0; j < NJ + LOOK && ok; ++j) {
            if (j < NJ) {
              ok = mma1(q0 + j);
              if (ok && j == NJ - 1) tc::mma_commit_pair(a_empty, PAIR);  // Y no longer read after the last MMA1
            }
            if (ok && j >= LOOK) ok = mma2(q0 + j - LOOK, j == NJ + LOOK - 1);
          }
          q = q0 + NJ;
        }
        if (!ok) {
          if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
          *abort_flag = 1;
        }
        // every issued MMA has finished (and signalled) before TMEM can be released
        tc::mma_commit_pair(teardown, 0x1);
        tc::mbar_wait_timed(teardown, 0);
      }
      __syncwarp();
    }
  } else if (warp < ROLE_WARPS + EPI_WARPS) {
    // ---- hidden chunks: TMEM H -> bias + GELU -> T in TMEM (the A operand of MMA2);
    // before and after them, this warp's slices of the tile's two drains
    const int quarter = warp & 3, cg = (warp - ROLE_WARPS) >> 2;
    const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
    rows::AsyncRows st{s_tile + (size_t)(warp - ROLE_WARPS) * 2 * rows::TILE_BYTES, 0};
    uint8_t* tl = st.tiles;
    const int d_lo = 32 * (Cfg::FS + cg * Cfg::GS);
    constexpr int NL = EPI_COLS / 32;   // 32-column TMEM loads per chunk, issued before one wait
    uint32_t q = 0;
    bool ok = true;
    int t = 0;
    for (int p = cid; p < pairs && ok; p += ncl, ++t) {
      ok = mid(t, p, 1 + cg, d_lo, Cfg::GS, tl);
      for (int j = 0; j < NJ && ok; ++j, ++q) {
        const uint32_t hb = q % NB, use = q / NB;
        if (!tc::mbar_wait(&h_full[hb], use & 1, abort_flag)) { ok = false; break; }
        __syncwarp();
        tc::fence_after_sync();
        const int cb = cg * EPI_COLS;
        uint32_t v[NL][32];
#pragma unroll
        for (int l = 0; l < NL; ++l) tc::tmem_ld_32x32b_x32(lane_base + Cfg::H_COL0 + hb * HC + cb + 32 * l, v[l]);
        tc::tmem_ld_wait();
        // 16-bit GELU values back into the first EPI_COLS / 2 columns this warp just read
        // (pairs of hidden columns per 32-bit TMEM column): MMA2's A operand
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          const float* bp = s_b1 + j * HC + cb + 32 * l;
          uint32_t pk[16];
#pragma unroll
          for (int k = 0; k < 16; k += 2) {
            const float4 b4 = *reinterpret_cast<const float4*>(bp + 2 * k);
            const uint32_t* x = &v[l][2 * k];
            pk[k] = gelu2_pack<T>(__uint_as_float(x[0]) + b4.x, __uint_as_float(x[1]) + b4.y);
            pk[k + 1] = gelu2_pack<T>(__uint_as_float(x[2]) + b4.z, __uint_as_float(x[3]) + b4.w);
          }
          tc::tmem_st_32x32b_x16(lane_base + Cfg::H_COL0 + hb * HC + cb + 16 * l, pk);
        }
        tc::tmem_st_wait();
        tc::fence_before_sync();
        __syncwarp();
        // the 16-bit H values are complete in this CTA's tensor memory (tcgen05.wait::st)
        if (lane == 0) tc::mbar_arrive_remote(lead(&h_done[hb]));
      }
      if (ok) ok = fin(t, p, 1 + cg, d_lo, Cfg::GS, st);
    }
    rows::async_drain(lane);
    if (!ok) {
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      *abort_flag = 1;
    }
  } else {
    // ---- final: the first slice of both drains of every tile
    tc::setmaxnreg_inc<REG_FINAL>();
    const int quarter = warp & 3;
    rows::AsyncRows st{s_tile + (size_t)(warp - ROLE_WARPS) * 2 * rows::TILE_BYTES, 0};
    uint8_t* tl = st.tiles;
    bool ok = true;
    int t = 0;
    // a tile's residual rows head for L2 while the previous tile's MMAs run
    auto prefetch = [&](int p) {
      const int row0 = (2 * p + rank) * BM + quarter * 32;
      if (p < pairs && lane < M - row0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(args.X + (size_t)(row0 + lane) * D),
                     "r"(D * 4)
                     : "memory");
    };
    prefetch(cid);
    for (int p = cid; p < pairs && ok; p += ncl, ++t) {
      ok = mid(t, p, 0, 0, Cfg::FS, tl);
      prefetch(p + ncl);
      if (ok) ok = fin(t, p, 0, 0, Cfg::FS, st);
    }
    rows::async_drain(lane);
    if (!ok) {
      if (err) atomicExch(err, DEV_MBAR_TIMEOUT);
      *abort_flag = 1;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  tc::cluster_sync();  // no CTA leaves while its peer may still signal it or read its memory
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc_pair(tmem_base, 512);
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

bool map2d(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t rows, uint32_t box_inner,
           uint32_t box_rows) {
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

// Store map of a dense [rows][inner] matrix: 32-row boxes of 64 bytes, 64-byte swizzle
// (the layout of the drain warps' staging tiles), or with `wide` 32-row boxes of 128 bytes,
// 128-byte swizzle (a wide box over both tiles).
bool store_map(CUtensorMap* m, const void* base, bool f32, CUtensorMapDataType dt16, uint64_t inner, uint64_t rows,
               bool wide = false) {
  auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const uint32_t es = f32 ? 4 : 2;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * es};
  cuuint32_t box[2] = {(wide ? 128u : 64u) / es, 32};
  cuuint32_t ess[2] = {1, 1};
  return fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : dt16, 2, const_cast<void*>(base), dims,
            strides, box, ess, CU_TENSOR_MAP_INTERLEAVE_NONE, wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Load map of the FP32 residual stream [rows][inner]: boxes of 32 columns (128 bytes) x 128
// rows, 128-byte swizzle (the GELU warps' prefetched first residual block).
bool residual_map(CUtensorMap* m, const float* base, uint64_t inner, uint64_t rows) {
  auto fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner * 4};
  cuuint32_t box[2] = {32, BM};
  cuuint32_t ess[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, ess,
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

template <int D, typename T>
cudaError_t launch_d(const T* A, const T* Wpt, const T* W1t, const T* W2t, const MlpArgs& a, cudaStream_t st) {
  using Cfg = MlpCfg<D>;
  constexpr CUtensorMapDataType dt = tc::tma_dtype<T>();
  auto kern = proj_mlp_tc_kernel<D, T>;
  cudaLaunchConfig_t lc = {};
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  lc.blockDim = dim3(THREADS);
  lc.dynamicSmemBytes = Cfg::SMEM_BYTES;
  lc.stream = st;
  lc.attrs = at;
  lc.numAttrs = 1;  // occupancy query without the stream attribute
  static int max_pairs = 0;  // co-resident CTA pairs at one CTA per SM
  if (!max_pairs) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    lc.gridDim = dim3(num_sms() / 2 * 2);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &lc);
    if (e != cudaSuccess) return e;
    max_pairs = n > 0 ? n : 1;
  }
  CUtensorMap ma, mp, m1, m2, mx, mln, mxr;
  if (!map2d(&ma, dt, A, D, (uint64_t)a.M, BK, BM)) return cudaErrorInvalidValue;
  if (!map2d(&mp, dt, Wpt, D, D, BK, D / 2)) return cudaErrorInvalidValue;
  if (!store_map(&mx, a.X, true, dt, D, (uint64_t)a.M, true) || !store_map(&mln, a.ln_out, false, dt, D, (uint64_t)a.M))
    return cudaErrorInvalidValue;
  if (!map2d(&m1, dt, W1t, D, (uint64_t)a.hid, BK, HC / 2)) return cudaErrorInvalidValue;
  if (!map2d(&m2, dt, W2t, (uint64_t)a.hid, D, BK, D / 2)) return cudaErrorInvalidValue;
  if (!residual_map(&mxr, a.X, D, (uint64_t)a.M)) return cudaErrorInvalidValue;
  const int pairs = ((a.M + BM - 1) / BM + 1) / 2;
  lc.gridDim = dim3((pairs < max_pairs ? pairs : max_pairs) * 2);
  lc.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelEx(&lc, kern, ma, mp, m1, m2, mx, mln, mxr, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

bool mlp_tc_supported(int d, int hid) {
  return (d == 64 || d == 128 || d == 256) && hid % HC == 0 && hid >= HC && hid <= 1024;
}

template <typename T>
cudaError_t launch_proj_mlp_tc(const T* A, const T* Wpt, const float* bp, const T* W1t, const T* W2t,
                               const float* b1, const float* b2, float* X, const float* ln_g, const float* ln_b,
                               T* ln_out, int M, int d, int hid, int* err, cudaStream_t st) {
  if (!mlp_tc_supported(d, hid) || M <= 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Wpt) | reinterpret_cast<uintptr_t>(W1t) |
       reinterpret_cast<uintptr_t>(W2t) | reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(ln_out)) & 15)
    return cudaErrorInvalidValue;
  if ((ln_g == nullptr) != (ln_b == nullptr)) return cudaErrorInvalidValue;
  // about half of a tile's time: 256 rows x D x (D + 2 hid) multiply-adds at 10.8 TFLOP/s
  // per CTA pair, the rate that the D = 256, hid = 1024 tiles reach
  const unsigned stagger = (unsigned)(2.0 * 256 * d * (d + 2.0 * hid) / 10.8e12 * 0.5 * 1e9);
  MlpArgs a{X, ln_out, bp, b1, b2, ln_g, ln_b, M, hid, err, stagger};
  if (d == 256) return launch_d<256, T>(A, Wpt, W1t, W2t, a, st);
  if (d == 128) return launch_d<128, T>(A, Wpt, W1t, W2t, a, st);
  return launch_d<64, T>(A, Wpt, W1t, W2t, a, st);
}

template cudaError_t launch_proj_mlp_tc<bf16>(const bf16*, const bf16*, const float*, const bf16*, const bf16*,
                                              const float*, const float*, float*, const float*, const float*, bf16*,
                                              int, int, int, int*, cudaStream_t);
template cudaError_t launch_proj_mlp_tc<f16>(const f16*, const f16*, const float*, const f16*, const f16*,
                                             const float*, const float*, float*, const float*, const float*, f16*, int,
                                             int, int, int*, cudaStream_t);

}  // namespace inpaint
