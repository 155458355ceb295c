/*
 * inpaint.h - C ABI of the GB300 mask-aware windowed-transformer inpainting library.
 *
 * The library runs the per-frame inpainting pass of the privacy pipeline of arXiv
 * 2509.10466: the model receives a frame whose private (masked) regions are set to 0
 * and returns the completed frame ("Inpainting Manager" section).  The network is a
 * hybrid CNN/transformer derived from DSTT ("Real-time Digital Inpainting"), with
 * scaled-dot-product attention ("Inpainting Model", item "Distinct Transformer Blocks")
 * and a convolutional reconstruction with a final crop (item "Modified Vec2Patch").
 *
 * The pass, per frame (H, W padded internally to multiples of 32 with x = 0, hole = 1):
 *   1. m = 1 - hole; input = [x*m (RGB), m]; 4x4 stride-4 conv patch embedding to
 *      tokens [N, dim]; token mask v0[t] = 1 if any pixel of the patch is known.
 *   2. `blocks` pre-LN transformer blocks.  Block l: LN -> QKV -> multi-head attention
 *      inside 8x8-token windows (offset by 4 tokens on odd blocks when shift = 1; slots
 *      outside the grid are void).  Keys are the tokens with v_l = 1; a window with no
 *      such key outputs 0.  v_{l+1}[t] = OR of v_l over t's window (bit-exact).  Then
 *      proj + residual, LN -> MLP (exact-erf GELU) -> residual.
 *   3. Final LN; two stages of nearest x2 upsample + 3x3 conv + GELU (dim/4, dim/8
 *      channels); 3x3 conv to RGB = pred.
 *   4. out = hole ? pred : x, cropped to H x W (known pixels copied exactly).
 *
 * Conventions
 *   - Every device pointer is caller-owned and must stay valid until the work queued
 *     on `stream` has finished.  x, out, pred, target, grad_out: float32 NCHW
 *     [B, 3, H, W], contiguous.  hole: uint8 [B, H, W], nonzero = private pixel.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls only enqueue
 *     work unless stated otherwise; completion is stream-ordered.
 *   - Every function returns INPAINT_OK (0) or an error code; nothing throws across
 *     the ABI.  A failed call leaves caller buffers in an unspecified state.
 *   - One context may be used by one host thread at a time.  Calls that use the
 *     context's internal workspace (inpaint_frame/batch/batch_host/backward) must not
 *     overlap on different streams; inpaint_batch_ws takes a caller workspace and may
 *     run concurrently on different streams with different workspaces.
 *   - Requirements: window = 8, patch = 4, dim / heads = 32; dim % 64 == 0 for BF16 / FP16.
 */
#ifndef INPAINT_H
#define INPAINT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define INPAINT_API __attribute__((visibility("default")))
#else
#define INPAINT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  INPAINT_OK = 0,
  INPAINT_E_INVAL = 1,    /* bad argument or unsupported configuration            */
  INPAINT_E_NOMEM = 2,    /* device allocation failed or exceeds hbm_budget_bytes */
  INPAINT_E_CUDA = 3,     /* a CUDA runtime call failed                           */
  INPAINT_E_TIMEOUT = 4,  /* inpaint_sync deadline passed before the work finished */
  INPAINT_E_STATE = 5,    /* call not valid in the context's current state        */
  INPAINT_E_DEVICE = 6    /* a kernel reported an error (e.g. a bounded wait ran out) */
};

/* Precision forms: FP32 on the SIMT pipes; BF16 or FP16 operands on the tensor cores
 * with FP32 accumulation, softmax statistics, LayerNorms and residual stream.  The
 * paper's engine runs in FP16 ("Inpainting Model", "Hardware"). */
enum { INPAINT_FP32 = 0, INPAINT_BF16 = 1, INPAINT_FP16 = 2 };

typedef struct inpaint_config {
  int32_t dim;        /* token channels d                                   */
  int32_t heads;      /* attention heads (dim / heads must be 32)           */
  int32_t window;     /* window side in tokens (must be 8)                  */
  int32_t blocks;     /* transformer blocks L                               */
  int32_t mlp_ratio;  /* MLP hidden = mlp_ratio * dim                       */
  int32_t patch;      /* patch-embedding stride (must be 4)                 */
  int32_t dec_c1;     /* decoder stage-1 channels, 0 = dim / 4              */
  int32_t dec_c2;     /* decoder stage-2 channels, 0 = dim / 8              */
  int32_t precision;  /* INPAINT_FP32 (SIMT FP32), INPAINT_BF16 or INPAINT_FP16 (16-bit
                         tensor-core operands, FP32 accumulation, softmax statistics
                         and LayerNorms) */
  int32_t shift;      /* 1 = odd blocks use windows offset by half a window  */
  uint64_t seed;      /* seed of the default weights (inpaint_init with NULL
                         weights, inpaint_default_weights); unused otherwise   */
  size_t hbm_budget_bytes; /* cap on the context's device memory, 0 = none   */
  int32_t mem_slots;  /* temporal memory slots m (0-4).  With m > 0 the odd blocks are
                         temporal: their queries also attend to the keys / values that up
                         to m previous frames produced in the same block (memory tensors;
                         see inpaint_batch_mem).  0 = single-frame spatial model. */
  int32_t pos_bias;   /* 1 = learned relative-position bias in every window softmax: a
                         per-head table [15][15] (blob: after each block's fc2.b) added
                         to the score of query (qy, qx) and key (ky, kx) of a window at
                         [ky - qy + 7][kx - qx + 7].  0 = none. */
} inpaint_config;

typedef struct inpaint_ctx inpaint_ctx;

/* Number of float32 values in the weight blob for `cfg`.  Blob order (each tensor
 * row-major): embed.w [d,4,4,4] (out, in = R,G,B,mask, ky, kx), embed.b [d]; per block:
 * ln1.g, ln1.b [d], qkv.w [d,3d] (in, out; out = q | k | v, head h at columns
 * 32h.. of each third), qkv.b [3d], proj.w [d,d], proj.b [d], ln2.g, ln2.b [d],
 * fc1.w [d, r*d], fc1.b [r*d], fc2.w [r*d, d], fc2.b [d] (then relpos [heads,15,15]
 * when pos_bias = 1); then lnf.g, lnf.b [d],
 * dec1.w [c1,d,3,3], dec1.b [c1], dec2.w [c2,c1,3,3], dec2.b [c2], head.w [3,c2,3,3],
 * head.b [3].  Errors: E_INVAL for a NULL or unsupported config. */
INPAINT_API int inpaint_num_params(const inpaint_config* cfg, size_t* n_params);

/* The default weight blob of `cfg` for `seed`, written to host_out (host float32, n >=
 * inpaint_num_params values).  The paper trains its own inpainter and publishes no
 * weights; the workloads run on random-init weights N(0, 0.02).  Host code only: it
 * needs no GPU.  Value i of the blob depends on (seed, i) alone (counter-based):
 *   mix(z): z += 0x9E3779B97F4A7C15; z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9;
 *           z = (z ^ z >> 27) * 0x94D049BB133111EB; return z ^ z >> 31   (SplitMix64)
 *   r = mix(mix(seed) + i)                                  (64-bit wrap-around)
 *   u1 = ((r >> 32) + 0.5) / 2^32,  u2 = ((r & 0xFFFFFFFF) + 0.5) / 2^32
 *   z = sqrt(-2 ln u1) cos(2 pi u2)   (Box-Muller, double precision)
 * Matrices, conv kernels and relative-position tables get (float)(0.02 z); LayerNorm
 * scales 1; biases and LayerNorm shifts 0.  Errors: E_INVAL (config, NULL, n too small). */
INPAINT_API int inpaint_default_weights(const inpaint_config* cfg, uint64_t seed, float* host_out, size_t n);

/* Create a context on the current CUDA device and upload `weights` (host float32,
 * `n_weights` values in blob order; must equal inpaint_num_params).  With weights =
 * NULL the context takes the default blob of cfg->seed (inpaint_default_weights;
 * n_weights 0 or num_params); inpaint_get_weights exports it.  The context owns its
 * copy of the weights and a device workspace that grows on demand up to
 * hbm_budget_bytes.  Blocks until the upload is done.  Errors: E_INVAL (config, count
 * mismatch), E_NOMEM, E_CUDA.  *out is NULL on error. */
INPAINT_API int inpaint_init(const inpaint_config* cfg, const float* weights, size_t n_weights,
                 inpaint_ctx** out);

/* Replace the weights (float32 blob).  weights_on_device = 1: `weights` is a device
 * pointer and the update is enqueued on `stream`; 0: host pointer, copied before
 * returning.  Used by fine-tuning after an optimizer step. */
INPAINT_API int inpaint_set_weights(inpaint_ctx* ctx, const float* weights, int weights_on_device,
                        void* stream);

/* Copy the context's float32 weight blob to host memory (num_params values). Blocking. */
INPAINT_API int inpaint_get_weights(inpaint_ctx* ctx, float* host_out);

/* Device workspace bytes one forward call of this shape needs (inpaint_batch_ws). */
INPAINT_API int inpaint_workspace_bytes(inpaint_ctx* ctx, int B, int H, int W, size_t* bytes);

/* Forward pass of one frame (B = 1); see inpaint_batch. */
INPAINT_API int inpaint_frame(inpaint_ctx* ctx, const float* x, const uint8_t* hole, int H, int W,
                  float* out, void* stream);

/* Forward pass of B frames of equal size (steps 1-4 above).  Device pointers:
 * x [B,3,H,W], hole [B,H,W], out [B,3,H,W]; pred_or_null, if not NULL, receives the
 * decoder output (before compositing) [B,3,H,W].  Uses the context's workspace
 * (grown if needed: E_NOMEM beyond the budget).  Errors: E_INVAL for B < 1, H or
 * W < 1, NULL pointers; E_CUDA on a launch failure. */
INPAINT_API int inpaint_batch(inpaint_ctx* ctx, const float* x, const uint8_t* hole, int B, int H,
                  int W, float* out, float* pred_or_null, void* stream);

/* Same as inpaint_batch but every intermediate lives in the caller's device
 * `workspace` (256-byte aligned, >= inpaint_workspace_bytes).  Calls with distinct
 * workspaces may run concurrently on distinct streams; the weights are shared
 * read-only.  Token masks of such calls are not kept for inpaint_token_masks. */
INPAINT_API int inpaint_batch_ws(inpaint_ctx* ctx, void* workspace, size_t workspace_bytes,
                     const float* x, const uint8_t* hole, int B, int H, int W, float* out,
                     float* pred_or_null, void* stream);

/* End-to-end form with HOST buffers: copies x and hole host->device, runs
 * inpaint_batch, copies out device->host and waits for completion.  The copies run on a
 * stream of the context, frame by frame, overlapped with the kernels: each frame is
 * embedded once its inputs have landed and copied back once its output is written.
 * The forward itself runs on `stream`, which at return has also waited for the copies.
 * Pinned host memory gives asynchronous copies; pageable memory works but is slower.
 * Token masks of the call are kept for inpaint_token_masks, as with inpaint_batch. */
INPAINT_API int inpaint_batch_host(inpaint_ctx* ctx, const float* x_host, const uint8_t* hole_host,
                       int B, int H, int W, float* out_host, void* stream);

/* Full-resolution path with the pre/post processing on the GPU.  The paper runs
 * segmentation and inpainting at half resolution and scales the outputs by 2
 * ("Upscaling"), and builds the hole from the masks of the objects the user selected
 * ("Object Control").  Inputs (device): x [B,3,H,W] float32 full-resolution frames (H,
 * W even); obj_masks uint8 [B,K,H/2,W/2] per-object masks at model resolution (nonzero
 * = object pixel); selected uint8 [B,K] (nonzero = the object is private).  Steps:
 * hole_half = OR of the selected masks (bit-exact); x_half = 2x2 mean of x; inpaint at
 * H/2 x W/2; out [B,3,H,W] = hole_half[y/2][x/2] ? pred_half[y/2][x/2] : x[y][x]
 * (nearest x2 upscale; known pixels copied exactly).  hole_half_out (device uint8
 * [B,H/2,W/2]) receives the hole if not NULL.  Uses the context's workspace.
 * Errors: E_INVAL for odd H or W, K < 1, NULL pointers. */
INPAINT_API int inpaint_fullres(inpaint_ctx* ctx, const float* x, const uint8_t* obj_masks,
                                const uint8_t* selected, int B, int K, int H, int W, float* out,
                                uint8_t* hole_half_out, void* stream);

/* Token masks v0 ... vL of the last inpaint_frame/inpaint_batch call, copied to host:
 * uint8 [(L+1), B, Ht*Wt] (Ht = H_pad/4, Wt = W_pad/4, row-major tokens).  `n` is
 * the capacity of `host_out` in bytes; E_INVAL if too small, E_STATE if no forward
 * call has run.  Blocking. */
INPAINT_API int inpaint_token_masks(inpaint_ctx* ctx, uint8_t* host_out, size_t n);

/* Hole-L1 fine-tuning loss (the paper trains with a per-pixel L1 loss weighted
 * towards the masked region, "Training structure"; this path keeps the hole term):
 * loss = sum over hole pixels and channels |out - target| / (3 * n_hole), 0 when
 * there are no hole pixels; grad_out = dloss/dout (sign(0) = 0, 0 on known pixels).
 * loss_dev: one device float; grad_out_dev: device [B,3,H,W] or NULL.  The sum is
 * reduced in a fixed order (deterministic). */
INPAINT_API int inpaint_l1_hole_loss(inpaint_ctx* ctx, const float* out, const float* target,
                         const uint8_t* hole, int B, int H, int W, float* loss_dev,
                         float* grad_out_dev, void* stream);

/* Allocation-free form of inpaint_l1_hole_loss for callers that must not allocate
 * device memory: processes whose device memory belongs to another allocator, per-frame
 * real-time loops where cudaMalloc/cudaFree would synchronize the device and stall
 * other streams, and deployments that forbid allocation after start-up.  The paper has
 * no counterpart; this is a property of the library, not of the method.
 * Same arguments, result and fixed-order reduction as inpaint_l1_hole_loss, but no
 * context and no allocation: its scratch (32 KiB of partial sums) is a fixed array in
 * the library's device module, present on every device that loads the library until
 * the process exits.  Each call looks up that array's device address with the device
 * current (cudaGetSymbolAddress), so make the first call on each device before any
 * stream capture.  Under CUDA's lazy module loading that first call on a device also
 * loads the library's device module, which reserves the 32 KiB there (a driver-side
 * allocation that may synchronize the device): callers that must not allocate at all
 * once running make one warm-up call per device at start-up.  Every call on a device
 * shares the one array:
 * calls that overlap on the GPU (other streams, other host threads) race and must be
 * ordered by the caller; each call rewrites every scratch value it reads, so leftovers
 * of an earlier call never leak into a result.  Returns INPAINT_E_INVAL, launching
 * nothing, when B*H*W exceeds INPAINT_L1_NOALLOC_MAX_PIXELS (4096 x 4096 pixels), and
 * INPAINT_E_CUDA (with inpaint_last_cuda_error set) when a CUDA call fails. */
#define INPAINT_L1_NOALLOC_MAX_PIXELS (4096 * 4096)
INPAINT_API int inpaint_l1_hole_loss_noalloc(const float* out, const float* target,
                                             const uint8_t* hole, int B, int H, int W,
                                             float* loss_dev, float* grad_out_dev, void* stream);

/* Gradient of sum(out * grad_out) with respect to the weight blob, written to
 * grad_weights (device float32, num_params values, overwritten).  Recomputes the
 * forward, keeping only each block's input, and recomputes each block again during
 * the reverse sweep (per-block activation recomputation).  The token masks carry no
 * gradient.  FP32-accurate in every precision setting: statistics, adjoints and
 * accumulation in FP32, every matrix product as three bf16 tensor-core products of the
 * split x = hi + lo (hi.hi + hi.lo + lo.hi, FP32 accumulation; about 1e-5 relative per
 * product), reduced in a fixed order (bit-reproducible). */
INPAINT_API int inpaint_backward(inpaint_ctx* ctx, const float* x, const uint8_t* hole,
                     const float* grad_out, int B, int H, int W, float* grad_weights,
                     void* stream);

/* One fine-tuning step's gradient in one call (the paper fine-tunes with an L1 loss that
 * weights the masked region, "Training structure"): the forward in the backward's own
 * FP32-accurate form, keeping each block's input, the hole-L1 loss of its output against
 * target (as inpaint_l1_hole_loss), and the gradient of that loss with respect to the
 * weight blob (as inpaint_backward with grad_out = dloss/dout); the forward is not run a
 * second time.  target: device [B,3,H,W] float32; loss_dev: one device float;
 * grad_weights: device float32, num_params values (overwritten); out_or_null: device
 * [B,3,H,W] float32 receiving the forward's output, or NULL. */
INPAINT_API int inpaint_train_step(inpaint_ctx* ctx, const float* x, const uint8_t* hole, const float* target,
                                   int B, int H, int W, float* loss_dev, float* grad_weights,
                                   float* out_or_null, void* stream);

/* Wait for `stream` with a host deadline (timeout_ms < 0: wait forever), then check
 * the context's device error flag.  E_TIMEOUT if the deadline passed (the work keeps
 * running), E_DEVICE if a kernel raised the flag (the flag is then cleared). */
INPAINT_API int inpaint_sync(inpaint_ctx* ctx, void* stream, int timeout_ms);

/* Per-kernel-class timing with CUDA events on the launching stream.  While enabled,
 * each kernel launch of the context is bracketed by an event pair.  Classes:
 * 0 embed, 1 layernorm, 2 qkv gemm, 3 attention, 4 proj gemm, 5 fc1 gemm, 6 fc2 gemm,
 * 7 decoder stage 1, 8 decoder stage 2, 9 head + composite, 10 other, 11 fused
 * projection + MLP (proj + residual + LN2 + fc1 + GELU + fc2 + residual + LayerNorm in
 * one kernel), 12 point cloud, 13 splat, 14 fused QKV + window attention (spatial blocks
 * of the 16-bit forms).
 * inpaint_profile_read synchronizes and returns total milliseconds and launch
 * counts per class (arrays of INPAINT_PROFILE_CLASSES), then clears them. */
#define INPAINT_PROFILE_CLASSES 15
INPAINT_API int inpaint_profile_enable(inpaint_ctx* ctx, int on);
INPAINT_API int inpaint_profile_read(inpaint_ctx* ctx, float* ms, int64_t* launches);

/* Temporal memory (cfg.mem_slots = m > 0).  A frame's memory tensor holds, for every
 * temporal block (odd l), the k | v rows of its own tokens in that block and their
 * usable-key mask: what a later frame of the same stream attends to.
 * inpaint_memory_bytes gives the size of one frame's memory buffer for an H x W stream
 * (0 when m = 0).  The paper keeps a fixed number of memory tensors of previous outputs
 * as model inputs and outputs (Sections "Inpainting Manager", "Minimal memory slots"). */
INPAINT_API int inpaint_memory_bytes(inpaint_ctx* ctx, int H, int W, size_t* bytes);

/* As inpaint_batch (workspace NULL: the context's own; else as inpaint_batch_ws, with
 * ws_bytes >= inpaint_workspace_bytes), with memory.  mem_in: host array [B * m] of device pointers, frame
 * b's slots at [b*m .. b*m + m-1], each a previous frame's memory buffer of the same
 * H x W, or NULL for an empty slot (the array itself may be NULL: no memory).  mem_out:
 * host array [B] of device buffers (inpaint_memory_bytes each, NULL = not recorded) that
 * receive each frame's own memory tensor.  Buffers must be 256-byte aligned and are
 * owned by the caller; an output buffer must not also be an input of the same call.
 * B * m may be at most 512 (the slot table travels in the kernel parameters, so the call
 * makes no host-to-device copy).  With every slot empty the result equals inpaint_batch.
 * Errors: E_INVAL (m = 0 with memory arguments, B * m > 512, misaligned buffers,
 * shapes), E_NOMEM, E_CUDA. */
INPAINT_API int inpaint_batch_mem(inpaint_ctx* ctx, void* workspace, size_t ws_bytes, const float* x,
                                  const uint8_t* hole, int B, int H, int W, float* out, float* pred,
                                  const void* const* mem_in, void* const* mem_out, void* stream);

/* Coloured point cloud of an inpainted frame (the paper transplants the inpainted RGB
 * onto the depth measurements, Section "Point Cloud Visualisation", and maps camera
 * points into the viewer's world with p' = R p + t, Section "Perspective Alignment").
 * depth: device float [H][W] (a pixel is a point when its depth is finite and > 0);
 * rgb: device float [3][H][W]; cam: host float[4] = fx, fy, cx, cy of the pinhole
 * camera (pixel centres at +0.5); rt: host float[12] = R (row-major) then t, camera to
 * world.  points: device float [H*W][6] = world x, y, z (NaN for non-points), r, g, b.
 * Back-projection x = d (u + 0.5 - cx) / fx, y = d (v + 0.5 - cy) / fy, z = d; every
 * operation rounded separately (no fused multiply-add), so results are reproducible bit
 * for bit.  Errors: E_INVAL, E_CUDA. */
INPAINT_API int inpaint_point_cloud(inpaint_ctx* ctx, const float* depth, const float* rgb, int H, int W,
                                    const float* cam, const float* rt, float* points, void* stream);

/* Headless z-buffered splat of a point cloud (device [n_points][6] as above) into an
 * Ho x Wo image at a remote viewpoint: q = R p + t with rt = world to viewer (host
 * float[12]); points with q_z > 1e-3 cover pixel (floor(fy q_y / q_z + cy),
 * floor(fx q_x / q_z + cx)) of the view camera (host float[4]) when inside the image;
 * per pixel the nearest point wins, equal depths the lower point index.  Outputs
 * (device): img float [3][Ho][Wo] (0 where empty), depth_out float [Ho][Wo] (q_z, +inf
 * where empty) and index_out int32 [Ho][Wo] (winning point, -1 where empty); the last
 * two may be NULL.  Uses a scratch buffer of the context (one splat in flight per
 * context).  The paper renders with OpenGL; this path has no graphics API.  Errors:
 * E_INVAL, E_NOMEM, E_CUDA. */
INPAINT_API int inpaint_point_splat(inpaint_ctx* ctx, const float* points, int64_t n_points, const float* view,
                                    const float* rt, int Ho, int Wo, float* img, float* depth_out, int32_t* index_out,
                                    void* stream);

/* Number of kernels this context has launched since creation. */
INPAINT_API int inpaint_launch_count(inpaint_ctx* ctx, int64_t* count);

/* Release every device resource of the context.  Waits for its work to finish. */
INPAINT_API void inpaint_destroy(inpaint_ctx* ctx);

/* Static description of an error code. */
INPAINT_API const char* inpaint_strerror(int code);

/* The CUDA runtime error (cudaError_t value and its name) behind the last
 * INPAINT_E_CUDA that a call on this host thread returned; 0 and "cudaSuccess" if none. */
INPAINT_API int inpaint_last_cuda_error(void);
INPAINT_API const char* inpaint_cuda_error_name(int cuda_error);

/* --- unit-test hooks for single kernels (used by the test suite) ---------------- */

/* C[M,N] = A[M,K] . B[K,N] on the BF16 tensor-core GEMM (tcgen05, FP32 accumulate).
 * A: bf16 row-major [M,K]; Bt: bf16 row-major [N,K] (B transposed, K contiguous);
 * C: float32 row-major [M,N].  M >= 1 (rows of the last 128-row tile past M are read as
 * zeros and not stored), N % 64 == 0, K % 64 == 0. */
INPAINT_API int inpaint_test_gemm_bf16(const void* A, const void* Bt, float* C, int M, int N, int K,
                           void* stream);

/* Failure detection on the device, exercised without a fault: one thread waits on an
 * mbarrier that nothing arrives at, with the same bounded wait the tensor-core kernels
 * use but a limit of limit_us microseconds (1 to 1000000) instead of their 2 s.  When the
 * limit passes it writes the device error code of an expired wait into the context's
 * error word, as those kernels do, and returns; inpaint_sync then reports E_DEVICE and
 * clears the word.  Errors: E_INVAL, E_CUDA. */
INPAINT_API int inpaint_test_wait_expiry(inpaint_ctx* ctx, int limit_us, void* stream);

/* Two GELU evaluations of the library on device floats x[n]: y_bf16_form[i] as the
 * 16-bit forms' decoder epilogues compute it (0.5 x (1 + tanh(x P(x^2))) with a fitted degree-4
 * P and the approximate hardware tanh: |error| <= 6e-6 + 2.5e-4 |x| absolute on [-12, 12],
 * saturating beyond) and y_fp32_form[i] with CUDA's erff (the FP32 form). */
INPAINT_API int inpaint_test_gelu(const float* x, float* y_bf16_form, float* y_fp32_form, int n,
                                  void* stream);

/* The GELU of the 16-bit forms' hidden activations (the fused projection + MLP kernel), on
 * device floats x[n]: the same 0.5 x (1 + tanh(x P(x^2))) evaluated in FP16 arithmetic on
 * pairs (x rounded to FP16 saturating at +-65504, packed FP16 multiply-adds, the
 * approximate FP16 tanh), y[i] its FP16 result as a float.  The kernel rounds that result
 * to the operand type.  Errors: E_INVAL, E_CUDA. */
INPAINT_API int inpaint_test_gelu_h16(const float* x, float* y, int n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* INPAINT_H */
