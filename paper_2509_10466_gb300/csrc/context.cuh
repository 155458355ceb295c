// Library context and shared runtime helpers (internal).
#pragma once

#include <vector>

#include "common.cuh"

namespace inpaint {

// Offsets (in floats) of every tensor of the weight blob, in blob order.
struct BlockOff {
  size_t ln1g, ln1b, qkvw, qkvb, projw, projb, ln2g, ln2b, fc1w, fc1b, fc2w, fc2b;
  size_t relpos = 0;  // [heads][15][15] when the config has a relative-position bias
};
struct Offsets {
  size_t embw, embb;
  std::vector<BlockOff> blk;
  size_t lnfg, lnfb, d1w, d1b, d2w, d2b, hw, hb;
  size_t total;
};


}  // namespace inpaint

// ------------------------------------------------------------------------- context

using inpaint::Offsets;
using inpaint::BlockOff;

struct Plan {
  int B, H, W, Hp, Wp, Ht, Wt, Nt, M;
  size_t tok, ln, qkv, o, hid, masks, f1, f2, err, end;
};

// One frame's memory tensor (temporal blocks l = 1, 3, ...; block l at (l / 2) * stride):
// k | v rows [Nt][2d] of the activation type, then the block's usable-key mask [Nt].
struct MemLayout {
  size_t kv_bytes = 0, stride = 0, total = 0;
};

// Memory slots of one batched call: tab = table [B][m] of previous frames' buffers (null
// entries = empty slots, the table itself null = no memory), out = host array [B] of this
// call's output buffers (null = do not record).
struct MemArgs {
  const inpaint::MemTab* tab = nullptr;
  uint8_t* const* out = nullptr;
  MemLayout lay;
};

struct EventPair {
  cudaEvent_t a, b;
  int cls;
};

// Host-buffer calls: frame f's inputs are on the device once in_ready[f] (recorded on the
// copy stream) completes; the forward then embeds frame by frame, and records out_ready[f]
// on the compute stream once frame f's output is written, so that the copies overlap the
// first and the last kernels.
struct FramePipe {
  const cudaEvent_t* in_ready = nullptr;
  const cudaEvent_t* out_ready = nullptr;
};

struct inpaint_ctx {
  inpaint_config cfg;
  int d, heads, L, r, c1, c2, hid;
  bool use_tc;  // a 16-bit tensor-core form (BF16 or FP16); else the FP32 SIMT form
  bool fp16;    // the 16-bit operand type is FP16 (else BF16)
  Offsets off;
  size_t nparams;
  float* w32 = nullptr;        // float32 blob (device)
  float* embed_wt = nullptr;   // [64][d]
  float* dec1_wt = nullptr;    // [9][d][c1]
  float* dec2_wt = nullptr;    // [9][c1][c2]
  // Derived weight copies of the 16-bit forms, in the operand type (bf16 or f16 bits):
  uint16_t* lin16 = nullptr;    // per block: qkv^T [3d][d], proj^T [d][d], fc1^T [rd][d], fc2^T [d][rd]
  // BF16 form with the fused projection + MLP: the affine part of LN1 and LN2 is folded
  // into the QKV and fc1 weights (lin16) and biases (fold_b, per block qkv [3d] then
  // fc1 [rd]); the LayerNorm producers then write the normalized rows only
  bool fold_ln = false;
  float* fold_b = nullptr;
  size_t lin_block_elems = 0;
  uint16_t* embed_w16 = nullptr;  // embed.w [d][64]
  uint16_t* dec1_wp = nullptr;    // merged sub-pixel weights [4][c1][4d]
  uint16_t* dec2_wp = nullptr;    // [4][c2][4c1]
  uint16_t* dec1_ws = nullptr;    // parity-stacked sub-pixel weights (transposed stage)
  uint16_t* dec2_ws = nullptr;
  size_t weight_bytes = 0;
  int* dev_err = nullptr;
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  // last internal-workspace forward, for inpaint_token_masks
  bool have_masks = false;
  Plan last{};
  // host e2e staging, its copy stream and per-frame events
  uint8_t* stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> in_ev, out_ev;
  cudaEvent_t start_ev = nullptr, done_ev = nullptr;
  // half-resolution buffers of inpaint_fullres
  uint8_t* pp = nullptr;
  size_t pp_bytes = 0;
  // backward scratch
  uint8_t* bws = nullptr;
  size_t bws_bytes = 0;
  // z-buffer keys of inpaint_point_splat
  uint8_t* zbuf = nullptr;
  size_t zbuf_bytes = 0;
  // profiling
  bool prof = false;
  std::vector<EventPair> events;
  size_t ev_used = 0;
  int64_t launches = 0;
};

namespace inpaint {

// Bracket one kernel launch with events when profiling is on; counts launches.
struct LaunchScope {
  inpaint_ctx* c;
  cudaStream_t st;
  int cls;
  EventPair* ep = nullptr;
  LaunchScope(inpaint_ctx* c_, cudaStream_t s, int k) : c(c_), st(s), cls(k) {
    c->launches++;
    if (!c->prof) return;
    if (c->ev_used == c->events.size()) {
      EventPair p;
      if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return;
      c->events.push_back(p);
    }
    ep = &c->events[c->ev_used++];
    ep->cls = k;
    cudaEventRecord(ep->a, st);
  }
  ~LaunchScope() {
    if (ep) cudaEventRecord(ep->b, st);
  }
};

inline int grow(uint8_t** buf, size_t* cap, size_t need, const inpaint_ctx* c, size_t other_bytes) {
  if (need <= *cap) return INPAINT_OK;
  if (c->cfg.hbm_budget_bytes && c->weight_bytes + other_bytes + need > c->cfg.hbm_budget_bytes) return INPAINT_E_NOMEM;
  if (*buf) {
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
  }
  if (cudaMalloc(buf, need) != cudaSuccess) {
    cudaGetLastError();
    *buf = nullptr;
    return INPAINT_E_NOMEM;
  }
  *cap = need;
  return INPAINT_OK;
}

}  // namespace inpaint

