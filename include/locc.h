/*
 * locc.h -- C ABI of the B300 (sm_103a) local-crop contact detector.
 *
 * Method: "Local object crop collision network for efficient simulation of
 * non-convex objects in GPU-based simulators" (Son & Kim, RSS 2023).  Given two
 * posed objects, the detector looks only at the local crops of the two shapes
 * where they may touch (Sec. III, collision predictor: cells of each object's
 * pose-transformed grid that lie in the intersection region of the two boxes;
 * appendix: "intersection region of two AABB"), encodes each crop with a
 * point-wise MLP and pooling (Sec. III, shape encoder; appendix: point-wise
 * MLP, ReLU everywhere) and predicts the contact with an MLP head.
 *
 * This library computes, for every candidate pair:
 *   1. pose composition:   R_rel = R_A^T R_B, t_rel = R_A^T (t_B - t_A);
 *   2. crop centre:        centre of (A's body box) n (B's box seen in A's
 *                          frame), in A's body frame;
 *   3. crop gather:        per object, the <= 64 surface points nearest to the
 *                          centre inside a ball of radius r (ties to the lower
 *                          point index), in the canonical crop frame (A's axes,
 *                          origin at the centre), zero padded;
 *   4. encoder:            3 -> 64 -> 128 -> 256 (ReLU) per point, max-pool over
 *                          the valid points of each object;
 *   5. head:               [f_A, f_B] 512 -> 256 -> 256 (ReLU) -> 8;
 *   6. epilogue:           out = {logit, contact point (world), unit normal
 *                          (world, from A towards B), penetration depth}.
 * plus an AABB broadphase that turns environments of objects into pairs (the
 * broad phase that rules out far-apart pairs, Sec. II footnote 1).
 *
 * Conventions
 *   - Every array argument of locc_detect / locc_crop / locc_network /
 *     locc_broadphase is a DEVICE pointer owned by the caller (for example the
 *     data pointer of a CUDA tensor).  locc_detect_host takes HOST pointers.
 *   - A pose is 7 float32: unit quaternion (w, x, y, z) then translation;
 *     p_world = R(q) p_body + t.  Quaternions are used as given (not
 *     renormalised).
 *   - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is
 *     the legacy default stream).  Nothing blocks except locc_status,
 *     locc_detect_host and locc_create / locc_destroy.
 *   - A pair whose object index or shape id is out of range gets an all-NaN
 *     output row and raises a device error flag; locc_status reports it.  No
 *     kernel traps.
 *   - Return codes: 0 on success, otherwise one of LOCC_ERR_*; the message of
 *     the last failing call on this host thread is locc_last_error().
 *   - A handle is not thread-safe: one host thread (or external locking) per
 *     handle.  Its scratch buffers are reused by every call, so calls on
 *     different streams of one handle must not overlap in time.
 */
#ifndef LOCC_H_
#define LOCC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOCC_OK 0
#define LOCC_ERR_INVALID_ARG (-1)  /* bad argument (NULL, size, range) */
#define LOCC_ERR_OOM (-2)          /* device or host allocation failed */
#define LOCC_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define LOCC_ERR_TIMEOUT (-4)      /* a bounded device wait ran out */
#define LOCC_ERR_BAD_WEIGHTS (-5)  /* weights blob malformed */
#define LOCC_ERR_BAD_INDEX (-6)    /* a kernel met an out-of-range index */
#define LOCC_ERR_BUSY (-7)         /* server queue full: request rejected */

#define LOCC_CROP_POINTS 64        /* points kept per object */
#define LOCC_CROP_LOCAL 0          /* crop mode: nearest samples in the crop ball */
#define LOCC_CROP_GLOBAL 1         /* crop mode: the first 64 samples of each shape */
#define LOCC_OUT_DIM 8             /* logit, point xyz, normal xyz, depth */
#define LOCC_N_PARAMS 240776       /* parameters of the crop network */

typedef struct locc_handle locc_handle;

/* Shape library: surface samples and box of every shape, in body frames.
 *   points: host float32 [n_shapes][n_points][3]
 *   aabb:   host float32 [n_shapes][6] = (lo.x, lo.y, lo.z, hi.x, hi.y, hi.z)
 * 1 <= n_points <= 65536.  locc_create copies both; the caller keeps
 * ownership of its arrays. */
typedef struct {
  int32_t n_shapes;
  int32_t n_points;
  const float *points;
  const float *aabb;
} locc_shape_library;

/* Arithmetic of the encoder and head matrix products.  Pose composition and
 * crop selection are float32 in every mode.
 *   LOCC_FP32: float32 CUDA-core products (the plain path);
 *   LOCC_BF16: bf16 operands on the tensor cores, float32 accumulation;
 *              the biases of encoder layers 1 and 2 enter the accumulation
 *              as bf16 hi + lo pairs (exact to about 2^-17 relative);
 *   LOCC_FP8:  e4m3 operands on the tensor cores, float32 accumulation;
 *              per-output-channel weight scales, and static per-channel
 *              activation scales (bounds that follow from the crop radius and
 *              the weights) folded into the next layer's weights; encoder
 *              layer 1 stays bf16 (hi/lo split), with its scale and bias
 *              folded in the same way. */
typedef enum { LOCC_FP32 = 0, LOCC_BF16 = 1, LOCC_FP8 = 2 } locc_precision;

/* Create a detector on the current CUDA device.
 *   lib:          shape library (host memory, copied).
 *   weights_blob: host bytes of a "LOCCW001" parameter blob: 8-byte magic,
 *                 uint32 version (1), uint32 n_layers (6), 6 x (uint32 in,
 *                 uint32 out) = (3,64) (64,128) (128,256) (512,256) (256,256)
 *                 (256,8), then for each layer float32 W[out][in] followed by
 *                 float32 b[out], little endian.  Copied.
 *   crop_radius:  radius r of the crop ball, > 0 (body-frame units).
 *   prec:         arithmetic of the network products (see above).
 *   out:          receives the handle; *out is NULL on failure.
 * Also sets up the library's kernels on this device once per handle (their
 * shared-memory limits, module loads and the device address of
 * locc_detect_noalloc's scratch array), so that no later call on the handle
 * loads a module.
 * Errors: INVALID_ARG, BAD_WEIGHTS, OOM, CUDA. */
int locc_create(const locc_shape_library *lib, const void *weights_blob,
                size_t blob_bytes, float crop_radius, locc_precision prec,
                locc_handle **out);

/* Switch the arithmetic used by later calls (weights are kept for all modes). */
int locc_set_precision(locc_handle *h, locc_precision prec);

/* Contact detection for n_pairs pairs (all device pointers, steps 1-6).
 *   poses:     float32 [n_obj][7]
 *   obj_shape: int32 [n_obj], shape id of each object
 *   pairs:     int32 [n_pairs][2], object indices (A, B)
 *   out:       float32 [n_pairs][8] = {logit, px, py, pz, nx, ny, nz, depth};
 *              collision <=> logit > 0.
 * n_pairs == 0 is a no-op.  Scratch grows on demand: when n_pairs exceeds
 * the handle's capacity the call synchronises the stream and re-allocates
 * with cudaMalloc (not graph-capturable); call locc_reserve first to keep
 * every later call free of allocations and synchronisation. */
int locc_detect(locc_handle *h, const float *poses, const int32_t *obj_shape,
                int32_t n_obj, const int32_t *pairs, int32_t n_pairs,
                float *out, void *stream);

/* Same as locc_detect with HOST arrays: copies inputs to the device, runs,
 * copies out back, and waits for the stream.  Page-locked (pinned) arrays are
 * copied directly; pageable ones go through pinned staging owned by the
 * handle. */
int locc_detect_host(locc_handle *h, const float *poses,
                     const int32_t *obj_shape, int32_t n_obj,
                     const int32_t *pairs, int32_t n_pairs, float *out,
                     void *stream);

/* Steps 1-3 only (device pointers).  Outputs (idx_out / centre_out may be NULL):
 *   xyz_out:    float32 [n_pairs][2][64][4]: canonical x, y, z and 1.0 for a
 *               selected point, all zeros for padding; object A then B.  The
 *               selected set is the min(64, n) in-ball samples nearest to the
 *               centre (ties to the lower sample index); their order within a
 *               crop is deterministic but not part of the result (the encoder
 *               max-pools over points);
 *   idx_out:    int32 [n_pairs][2][64] library point index, -1 for padding;
 *   cnt_out:    int32 [n_pairs][2] number of selected points;
 *   centre_out: float32 [n_pairs][4] crop centre in A's body frame (w = 0). */
int locc_crop(locc_handle *h, const float *poses, const int32_t *obj_shape,
              int32_t n_obj, const int32_t *pairs, int32_t n_pairs,
              float *xyz_out, int32_t *idx_out, int32_t *cnt_out,
              float *centre_out, void *stream);

/* Steps 4-5 only, on crops in locc_crop's layout (device pointers):
 *   xyz: float32 [n_pairs][2][64][4] (w = 1 marks a valid point);
 *   y_out: float32 [n_pairs][8] raw head outputs in the crop frame;
 *   feat_out (may be NULL): float32 [n_pairs][512] pooled [f_A, f_B]. */
int locc_network(locc_handle *h, const float *xyz, int32_t n_pairs,
                 float *y_out, float *feat_out, void *stream);

/* AABB broadphase (device pointers): objects of environment e are
 * env_offsets[e] .. env_offsets[e+1]-1.  Writes every pair (i, j), i < j, of
 * one environment whose world boxes (the axis-aligned box of each object's
 * posed body box) overlap into pairs_out (int32 [max_pairs][2]), in order of
 * environment then i then j, and the total count into *n_pairs_out (device
 * int32).  If the total exceeds max_pairs, only the first max_pairs are
 * written and *n_pairs_out holds the full count. */
int locc_broadphase(locc_handle *h, const float *poses, const int32_t *obj_shape,
                    const int32_t *env_offsets, int32_t n_env, int32_t *pairs_out,
                    int32_t *n_pairs_out, int32_t max_pairs, void *stream);

/* One simulator step on the device (all device pointers): locc_broadphase of
 * the environments, then contact detection (as locc_detect) of every candidate
 * pair, with out: float32 [max_pairs][8]; rows at and beyond *n_pairs_out are
 * left untouched, and only the first max_pairs pairs are detected.  The pair
 * count stays on the device and launch shapes depend only on max_pairs and
 * n_env, so after locc_reserve(h, max_pairs, n_env) the call allocates nothing,
 * never synchronises the host and can be captured in a CUDA graph. */
int locc_step(locc_handle *h, const float *poses, const int32_t *obj_shape,
              int32_t n_obj, const int32_t *env_offsets, int32_t n_env,
              int32_t *pairs_out, int32_t *n_pairs_out, int32_t max_pairs,
              float *out, void *stream);

/* locc_step with HOST arrays: copies poses [n_obj][7], obj_shape [n_obj] and
 * env_offsets [n_env+1] to the device, runs the step, waits, and copies back
 * the pair count (*n_pairs_out, host), the first min(count, max_pairs) pairs
 * (pairs_out, host int32 [max_pairs][2]) and their outputs (out, host float32
 * [max_pairs][8]).  Page-locked arrays are copied directly, pageable ones
 * through the handle's pinned staging. */
int locc_step_host(locc_handle *h, const float *poses, const int32_t *obj_shape,
                   int32_t n_obj, const int32_t *env_offsets, int32_t n_env,
                   int32_t *pairs_out, int32_t *n_pairs_out, int32_t max_pairs,
                   float *out, void *stream);

/* ------------------------------------------------------- pipelined stepping
 * Host-buffer steps with up to `depth` steps in flight (1..LOCC_STEPPER_MAX_
 * DEPTH): each step's inputs are copied in, and its results copied out, on
 * copy streams of their own while the neighbouring steps run on the device.
 * The steps run one after another (they share the handle's scratch), so the
 * handle must not be used by other calls while a stepper has steps in flight.
 *
 * locc_stepper_create: reserves the handle for max_pairs / max_env
 *   (locc_reserve) and allocates depth slots of device staging (inputs for
 *   max_obj objects and max_env environments, max_pairs pairs and outputs).
 *   Errors: LOCC_ERR_INVALID_ARG (a size < 1, depth out of range), LOCC_ERR_OOM.
 * locc_stepper_submit: enqueues one step (as locc_step) and returns at once
 *   with a ticket.  poses [n_obj][7], obj_shape [n_obj], env_offsets
 *   [n_env + 1], pairs_out [max_pairs][2] and out [max_pairs][8] are
 *   page-locked HOST arrays that must stay valid, and the inputs unchanged,
 *   until locc_stepper_wait returns for the ticket.  The pair list and the
 *   outputs are copied back at the stepper's full max_pairs capacity: the
 *   first min(count, max_pairs) rows are the step's, rows beyond are
 *   unspecified.  LOCC_ERR_BUSY when depth steps are in flight (wait for one
 *   first); LOCC_ERR_INVALID_ARG for pageable arrays or sizes beyond the
 *   stepper's.  Index errors of the step are reported by locc_status.
 * locc_stepper_wait: blocks until the ticket's step and its copies are done
 *   and writes its pair count to *n_pairs_out (host); tickets may be waited
 *   for in any order, each once (else LOCC_ERR_INVALID_ARG).
 * locc_stepper_destroy: waits for everything in flight, then frees. */
#define LOCC_STEPPER_MAX_DEPTH 4
typedef struct locc_stepper locc_stepper;
int locc_stepper_create(locc_handle *h, int32_t max_pairs, int32_t max_env, int32_t max_obj,
                        int32_t depth, locc_stepper **out);
int locc_stepper_submit(locc_stepper *t, const float *poses, const int32_t *obj_shape,
                        int32_t n_obj, const int32_t *env_offsets, int32_t n_env,
                        int32_t *pairs_out, int32_t *n_pairs_out, float *out, int64_t *ticket);
int locc_stepper_wait(locc_stepper *t, int64_t ticket);
void locc_stepper_destroy(locc_stepper *t);

/* Pre-allocate scratch for up to max_pairs pairs and max_envs environments
 * per call (blocking).  Later calls within these sizes allocate nothing. */
int locc_reserve(locc_handle *h, int32_t max_pairs, int32_t max_envs);

/* Stage timing: with enable != 0, later locc_step / locc_detect calls record
 * CUDA events on their streams around each stage.  locc_stage_times waits for
 * the last call's final event and writes up to n durations in milliseconds:
 * [0] broadphase, [1] crop gather, [2] encoder, [3] head + epilogue (each
 * summed over the pipeline chunks; chunks of different stages overlap), [4]
 * the whole call.  Returns the number written (>= 0) or an error code. */
int locc_profile(locc_handle *h, int enable);
int locc_stage_times(locc_handle *h, float *ms_out, int n);

/* Pipelining of locc_detect / locc_step: the pairs are cut into n_chunks
 * (1..16) parts; the crop gather of part i + 1 runs on the caller's stream
 * while the network of part i runs on a stream owned by the handle (forked
 * from and joined back into the caller's stream, so the call stays
 * capturable).  crop_ctas_per_sm caps the resident crop CTAs per SM (0 = no
 * cap) so they fit beside a network CTA.  Defaults: 1 chunk, no cap.  Results
 * do not depend on these settings. */
int locc_set_pipeline(locc_handle *h, int32_t n_chunks, int32_t crop_ctas_per_sm);
/*   n_chunks == 0 selects instead the fused launch of the BF16 path: one
 *   persistent kernel in which crop warps on the CUDA cores hand each
 *   object's crop rows through shared memory to the tensor-core encoder of
 *   the same SM (crop_ctas_per_sm is then the number of crop warps per CTA,
 *   6 or 8); used for BF16 with local crops, the other modes run separate
 *   kernels. */

/* Autotuner: times locc_step (reps repetitions after one warm-up) for each
 * pipelining setting in {1, 2, 4, 8} chunks x {no cap, 8, 6, 4} crop CTAs per
 * SM, and for BF16 with local crops the fused launch with 6 or 8 crop warps
 * per CTA, on the given step inputs (as locc_step), keeps the fastest and
 * writes it to best_out[2] = {n_chunks, crop_ctas_per_sm} (n_chunks 0: the
 * fused launch, see locc_set_pipeline) and its mean step time in ms to
 * *best_ms_out (either may be NULL).  Blocking. */
int locc_autotune(locc_handle *h, const float *poses, const int32_t *obj_shape,
                  int32_t n_obj, const int32_t *env_offsets, int32_t n_env,
                  int32_t *pairs_out, int32_t *n_pairs_out, int32_t max_pairs,
                  float *out, int32_t reps, int32_t *best_out, float *best_ms_out,
                  void *stream);

/* Wait for `stream`, then report and clear the device error flag:
 * 0, LOCC_ERR_TIMEOUT (a bounded device wait ran out) or LOCC_ERR_BAD_INDEX. */
int locc_status(locc_handle *h, void *stream);

/* Test entry for the failure path of the tensor-core kernels, which the paper
 * does not have: launches one CTA on `stream` that allocates TMEM and waits
 * on an mbarrier that nothing completes, bounded by max_cycles SM cycles
 * (1 <= max_cycles <= 2e9, else LOCC_ERR_INVALID_ARG).  The wait runs out;
 * the CTA raises the timeout bit of the handle's device error flag,
 * releases its TMEM and returns -- the path every bounded wait of the
 * encoder and head kernels takes.  The next locc_status reports
 * LOCC_ERR_TIMEOUT and clears the flag; the CUDA context stays usable.
 * Nothing traps or faults. */
int locc_selftest_wait_timeout(locc_handle *h, int64_t max_cycles, void *stream);

/* Allocation-free detection, for callers that may not allocate device memory
 * while they run: a simulator whose own pool allocator owns all of HBM after
 * start-up, or a latency-critical loop where cudaMalloc / cudaFree (which can
 * synchronise the device) are not allowed.  The paper has no counterpart; this
 * is a deployment variant of locc_detect.
 *   Same arguments and outputs as locc_detect (device pointers), computed with
 *   the float32 network whatever the handle's precision.  n_pairs must be
 *   <= LOCC_NOALLOC_MAX_PAIRS, else LOCC_ERR_INVALID_ARG with a message.
 *   Scratch: one library-owned __device__ array of about 4 MiB, resident on
 *   every device that loads the library until the process exits.  The call
 *   allocates nothing (no cudaMalloc / cudaFree, no allocating library call)
 *   and loads nothing: locc_create already looked up that array's device
 *   address (cudaGetSymbolAddress, with the handle's device current) and
 *   loaded the kernels this call launches.
 *   All calls share the array: calls whose kernels may overlap on the GPU
 *   (other streams, handles or host threads) race and must be ordered by the
 *   caller.  The current device must be the handle's device. */
#define LOCC_NOALLOC_MAX_PAIRS 1024
int locc_detect_noalloc(locc_handle *h, const float *poses,
                        const int32_t *obj_shape, int32_t n_obj,
                        const int32_t *pairs, int32_t n_pairs, float *out,
                        void *stream);

/* ---------------------------------------------------------------- training
 * The crop network is trained on the GPU with this library's own forward and
 * backward kernels (float32): binary cross-entropy on the collision logit plus
 * alpha * mean(f^2) on the pooled embedding (Sec. III-A loss, alpha = 0.5),
 * regression terms on the contact point, normal and depth (collisions only for
 * point and normal; Huber loss on depth), w_len (|n| - 1)^2 on the length of
 * the raw normal output of every pair (this library's term: the epilogue
 * normalises n, and a short raw n would amplify the rounding of the BF16 /
 * FP8 paths), Adam with bias correction (Sec. IV-A and the hyper-parameter
 * table: lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8). */
typedef struct locc_trainer locc_trainer;
typedef struct {
  float lr, beta1, beta2, eps;       /* Adam */
  float w_pt, w_n, w_d, huber_beta;  /* regression weights, Huber width */
  float alpha;                       /* embedding regulariser */
  float w_len;                       /* raw-normal length term (0 = off) */
} locc_train_config;

/* Trainer for the handle's network; parameters start from the handle's
 * current weights.  max_batch: largest n_pairs of a step.  Blocking.  The
 * first LOCC_FP32 step also allocates that pass's own activation buffers
 * (about 192 KB per pair of max_batch) and waits for the allocation; a
 * trainer that only runs LOCC_BF16 steps never holds them. */
int locc_trainer_create(locc_handle *h, int32_t max_batch,
                        const locc_train_config *cfg, locc_trainer **out);

/* One step on n_pairs (1..max_batch) pairs, device pointers:
 *   poses / obj_shape / pairs: as locc_detect;
 *   targets: float32 [n_pairs][8] world-frame {label (0/1), contact point xyz,
 *            normal xyz (A towards B), depth (> 0 overlap, < 0 gap)};
 *   rot:     float32 [n_pairs][9] row-major rotation of each pair's canonical
 *            crop frame (rotation augmentation, Sec. III-A), or NULL;
 *   loss_out: device float32 [1] mean loss of the batch, or NULL;
 *   update:  nonzero -> Adam step; zero -> gradients only.
 * Asynchronous on `stream`. */
int locc_train_step(locc_trainer *t, const float *poses, const int32_t *obj_shape,
                    int32_t n_obj, const int32_t *pairs, int32_t n_pairs,
                    const float *targets, const float *rot, float *loss_out,
                    int32_t update, void *stream);

/* Copy the last step's gradient / the current parameters (device float32
 * [LOCC_N_PARAMS], per layer W[out][in] then b[out]), or set the parameters. */
int locc_trainer_grad(locc_trainer *t, float *grad_out, void *stream);
int locc_trainer_params(locc_trainer *t, float *params_out, void *stream);
int locc_trainer_set_params(locc_trainer *t, const float *params, void *stream);

/* Optimizer state for training checkpoints (the paper has no counterpart):
 * copy out / restore Adam's first and second moments (device float32
 * [LOCC_N_PARAMS] each, same layout as the parameters) and the number of
 * Adam steps taken (the bias-correction exponent).  Together with the
 * parameters this is everything a resumed run needs to continue exactly where
 * the checkpoint was taken.  Asynchronous on `stream` except for the step
 * count, which is host state (step >= 0, else LOCC_ERR_INVALID_ARG). */
int locc_trainer_get_state(locc_trainer *t, float *m_out, float *v_out, int64_t *step_out,
                           void *stream);
int locc_trainer_set_state(locc_trainer *t, const float *m, const float *v, int64_t step,
                           void *stream);

/* Install the trainer's parameters as the handle's inference weights (all
 * precisions); blocking. */
int locc_trainer_commit(locc_trainer *t);

/* Learning rate of the following steps (learning-rate schedules); host-side,
 * takes effect at the next locc_train_step.  lr >= 0 and finite, else
 * LOCC_ERR_INVALID_ARG. */
int locc_trainer_set_lr(locc_trainer *t, float lr);
/* Arithmetic of the following steps (host-side; default LOCC_FP32):
 *   LOCC_FP32: float32 CUDA-core products (gradients to float32 rounding);
 *   LOCC_BF16: the dense products of forward and backward on the tensor
 *     cores with bf16 operands and float32 accumulation; parameters, Adam
 *     moments, activations and gradients stay float32.  Layer 3's backward
 *     is computed sparsely (its gradient is non-zero only at each channel's
 *     argmax row, Sec. III-A max-pooling) in float32.
 * Other values: LOCC_ERR_INVALID_ARG. */
int locc_trainer_set_precision(locc_trainer *t, int32_t precision);
void locc_trainer_destroy(locc_trainer *t);

/* ---------------------------------------------------------------- serving
 * A request server on one handle: simulator clients submit contact-query
 * batches of any size (their own objects, poses and pair lists) from any host
 * thread, and a scheduler thread owned by the server runs them with continuous
 * batching.  The paper runs the detector for thousands of simulated
 * environments in parallel on one GPU (Sec. I; Sec. IV, Claim 3); the server
 * is the deployment form of locc_detect for many simulators sharing a GPU,
 * which the paper does not describe.
 *   - Admission by device memory: a request's inputs are copied into a device
 *     arena of arena_bytes (a budget of HBM) when a block large enough is
 *     free; queued requests are admitted in arrival order as blocks free up,
 *     at most max_active at once and while the admitted requests' pairs left
 *     to launch (each counted up to one launch) stay below max_active_pairs.
 *   - Continuous batching: every launch packs the pending pairs of all
 *     admitted requests, up to max_batch_pairs: each request first gets an
 *     equal share, the room left goes in admission order.  A large request
 *     spans several launches; requests that arrive meanwhile join the next
 *     launch.  Host->device copies of newly admitted requests, the launches
 *     and the device->host copies of results run on three streams and overlap.
 *   - A pair's result does not depend on which launch or batch mates it got:
 *     every output row is computed from that pair's inputs alone, with the
 *     same arithmetic as locc_detect at the handle's precision.
 * While a server exists it owns the handle: make no other call on the handle
 * until locc_server_destroy returns. */
typedef struct locc_server locc_server;
typedef struct {
  int64_t arena_bytes;      /* device bytes for admitted requests' inputs;
                               0 -> half of the device's free memory */
  int32_t max_batch_pairs;  /* pairs per launch, >= 1 (0 -> 131072) */
  int32_t max_active;       /* admitted requests at once, 1..1024 (0 -> 256) */
  int64_t max_queued_pairs; /* pairs waiting for admission beyond which
                               locc_server_submit rejects (an empty queue
                               always accepts); 0 -> no limit */
  int64_t max_active_pairs; /* admission pauses while the admitted requests'
                               pairs still to launch, each counted up to
                               max_batch_pairs, reach this (one request is
                               always admitted): bounds how many requests
                               share the launches without keeping small
                               requests out behind a large one;
                               0 -> 4 x max_batch_pairs */
} locc_server_config;

/* A request: HOST arrays, read until the request completes; `out` is written
 * when it completes.  Page-locked (pinned) memory lets the copies overlap.
 *   poses [n_obj][7], obj_shape [n_obj], pairs [n_pairs][2] (object indices
 *   of this request, 0 <= index < n_obj), out float32 [n_pairs][8] as
 *   locc_detect. */
typedef struct {
  const float *poses;
  const int32_t *obj_shape;
  int32_t n_obj;
  const int32_t *pairs;
  int32_t n_pairs;
  float *out;
} locc_request;

/* Timeline of one completed request, microseconds since its submission. */
typedef struct {
  double admit_us;     /* admitted (inputs placed in the arena) */
  double done_us;      /* last result row copied to `out` */
  int32_t launches;    /* launches that carried some of its pairs */
  int32_t status;      /* 0, or the error code of a failed launch */
} locc_request_info;

typedef struct {
  int64_t submitted, rejected, completed, failed;
  int64_t queued, active;          /* now: waiting for admission / admitted */
  int64_t pairs_completed, launches;
  int64_t arena_bytes, arena_used, arena_peak;
  double latency_p50_us, latency_p99_us, latency_max_us;  /* completed requests */
  double mean_pairs_per_launch;
  int32_t max_active_seen;         /* most requests admitted at once */
} locc_server_counters;

/* Start a server on h (reserves the handle's scratch for max_batch_pairs).
 * cfg may be NULL (all defaults).  Errors: INVALID_ARG, OOM, CUDA. */
int locc_server_create(locc_handle *h, const locc_server_config *cfg,
                       locc_server **out);

/* Queue a request; thread-safe, never blocks on the GPU.  *id_out receives
 * its id.  n_pairs == 0 completes at once.  Checks every pair index and shape
 * id on the host: INVALID_ARG for a bad one.  OOM when the request's inputs
 * could never fit in the arena; BUSY when requests are waiting for admission
 * and their pairs plus this request's would exceed max_queued_pairs (the
 * request is not queued; counted as rejected). */
int locc_server_submit(locc_server *s, const locc_request *req, int64_t *id_out);

/* Wait up to timeout_ms (< 0: no limit) for request `id`.  On completion
 * fills *info (may be NULL), forgets the id and returns the request's status
 * (0 or the failed launch's error code); TIMEOUT if it is still running
 * (the id stays valid); INVALID_ARG for an unknown id. */
int locc_server_wait(locc_server *s, int64_t id, int32_t timeout_ms,
                     locc_request_info *info);

/* Counters and latency percentiles since creation or the last reset. */
int locc_server_stats(locc_server *s, locc_server_counters *st, int32_t reset);

/* Finish every queued and admitted request, stop the scheduler and free the
 * server (the handle stays).  Blocking. */
void locc_server_destroy(locc_server *s);

/* Crop mode of every later call on the handle (detection, crops, training):
 * LOCC_CROP_LOCAL (default: the method's local crops) or LOCC_CROP_GLOBAL,
 * the ablation without locality (Sec. IV-B, GLOBAL-OCN): each object keeps its
 * first 64 surface samples -- an area-uniform subset of the whole surface,
 * whatever the crop ball -- in the same canonical frame, count 64 (fewer if
 * the shapes have fewer samples).  Errors: LOCC_ERR_INVALID_ARG. */
int locc_set_crop_mode(locc_handle *h, int32_t mode);

/* Release all device and host memory of the handle (blocking). */
void locc_destroy(locc_handle *h);

/* ------------------------------------------------------ simulation step ----
 * Contact resolution driven by the detector (Sec. IV-C: the network inside a
 * GPU simulator's step; Table 2: |signed distance| whenever a contact
 * arises).  Penalty method (the paper cites its solver without describing
 * it): a contact row {logit, point, normal (A -> B), depth} with logit > 0
 * pushes B by F = max(0, k_contact max(depth, 0) - c_contact v_n) n at the
 * point and A by -F, v_n the normal speed of B relative to A there; each body
 * box corner below the ground plane z = 0 adds max(0, k_plane pen - c_plane
 * v_z) upwards and -mu_plane (v_x, v_y); gravity; unit mass and the inertia
 * of a solid box filling the body AABB; semi-implicit Euler with damping,
 * quaternion renormalised. */
typedef struct {
  float dt, gravity;
  float k_contact, c_contact;
  float k_plane, c_plane, mu_plane;
  float lin_damp, ang_damp;
} locc_sim_params;

/* One step of every object, in place: poses [n_obj][7] and velocities
 * vel [n_obj][6] (linear, angular, world) on the device.  Contacts: the first
 * min(*n_pairs_dev, max_pairs) rows (all max_pairs when n_pairs_dev is NULL)
 * of pairs [.][2] and contacts [.][8] (the format of locc_detect's output,
 * world frame).  acc: device scratch float32 [n_obj][6], zero on entry and
 * left zero.  Asynchronous on `stream`. */
int locc_sim_step(locc_handle *h, const locc_sim_params *prm, float *poses, float *vel,
                  const int32_t *obj_shape, int32_t n_obj, const int32_t *pairs,
                  const int32_t *n_pairs_dev, int32_t max_pairs, const float *contacts,
                  float *acc, void *stream);

/* Proxy-geometry contacts in the same row format from bounding spheres of
 * radius radius[shape] (device float32 [n_shapes]) about each object's
 * origin: logit = depth = r_A + r_B - |t_B - t_A|, normal along t_B - t_A,
 * point halfway between the sphere surfaces.  A baseline contact source for
 * locc_sim_step. */
int locc_sphere_contacts(locc_handle *h, const float *poses, const int32_t *obj_shape,
                         int32_t n_obj, const int32_t *pairs, const int32_t *n_pairs_dev,
                         int32_t max_pairs, const float *radius, float *out, void *stream);

/* --------------------------------------------------------------- UCF-GJK ----
 * The analytical comparator (Sec. IV-B, Claim 1; "range of parameters in
 * UCF-GJK" of the hyper-parameter table): each shape is a union of convex
 * elements given by their vertices (a convex decomposition; body frame); a
 * pair collides when any pair of elements intersects, each element pair being
 * tested by GJK on the Minkowski difference for exactly `iterations`
 * iterations (a uniform computational flow).  A pair the iterations leave
 * undecided counts as colliding.  Float32. */
typedef struct locc_gjk locc_gjk;

/* Copy a convex decomposition to the device: shape s owns elements
 * [elem_off[s], elem_off[s + 1]), element e owns vertices
 * [vert_off[e], vert_off[e + 1]) of verts (host float32 [n][3]); every shape
 * needs >= 1 element and every element >= 1 vertex.  Blocking.  Errors:
 * LOCC_ERR_INVALID_ARG, LOCC_ERR_OOM. */
int locc_gjk_create(int32_t n_shapes, const int32_t *elem_off, const int32_t *vert_off,
                    const float *verts, locc_gjk **out);

/* collide [n_pairs] uint8 (device): 1 collision, 0 none, 0xff out-of-range
 * pair (which also raises the flag locc_gjk_status reports).  poses, obj_shape,
 * pairs as for locc_detect; 1 <= iterations <= 1024.  Asynchronous. */
int locc_gjk_detect(locc_gjk *h, const float *poses, const int32_t *obj_shape, int32_t n_obj,
                    const int32_t *pairs, int32_t n_pairs, int32_t iterations,
                    uint8_t *collide, void *stream);

/* Synchronise `stream`; 0 or LOCC_ERR_BAD_INDEX (flag then cleared). */
int locc_gjk_status(locc_gjk *h, void *stream);

void locc_gjk_destroy(locc_gjk *h);

/* ------------------------------------------------ voxel-latent variant ----
 * The paper's own design (Sec. III "Local Crop Collision Network"; appendix
 * "Architecture Details"): a shape encoder computes, once per library shape,
 * a latent of 6 x 6 x 6 cells x 16 features over the shape's AABB (per-point
 * MLP 3 -> 256 -> 256 -> 256, cell-wise max pooling, a 3-D U-Net of four
 * 128-channel 3x3x3 convolutions -- the first unpadded -- and four transposed
 * convolutions with concatenated skips, a global [max || mean] feature tiled
 * onto every cell, a linear layer to 16).  Per pair, each object's cells whose
 * centre lies in the intersection of its box with the other object's box
 * (seen as an axis-aligned box of its frame), widened by the cell's
 * half-diagonal so that no cell touching the region is missed, are average
 * pooled (no cell: 0); [pooled (16) || pose in A's frame (7)] of each object
 * goes through 23 -> 128 -> 128 -> 128 (ReLU), the two results are max pooled,
 * then 128 -> 128 -> 128 -> 128 (ReLU) -> 1 gives the collision logit
 * (collision <=> logit > 0, i.e. sigmoid > 0.5).  A's pose input is
 * (1, 0, 0, 0, 0, 0, 0), B's (q_A* q_B, R_A^T (t_B - t_A)).  Cells are
 * numbered (i * 6 + j) * 6 + k along body axes 0, 1, 2.  Float32 on the CUDA
 * cores; the cell selection is bit-reproducible (explicitly rounded float32 in
 * a fixed order).  Same conventions as above: device pointers, asynchronous
 * on `stream`, out-of-range indices give a NaN logit and raise the flag that
 * locc_voxel_status reports. */
#define LOCC_VOXEL_N_PARAMS 5533969 /* parameters of the voxel network */
#define LOCC_VOXEL_CELLS 216        /* 6 x 6 x 6 cells per shape */
#define LOCC_VOXEL_F 16             /* latent features per cell */

typedef struct locc_voxel locc_voxel;

/* Copy the library to the device, read the "LOCCV001" blob (8-byte magic,
 * uint32 version 1, uint32 LOCC_VOXEL_N_PARAMS, then float32 parameters:
 * e1 W[256][3] b, e2 W[256][256] b, e3 likewise, c1 W[128][256][3][3][3] b,
 * c2..c4 W[128][128][3][3][3] b, d1 W[128][128][3][3][3] b (transposed
 * convolutions are [in][out][3][3][3]), d2..d4 W[256][128][3][3][3] b,
 * f W[16][384] b, p1 W[128][23] b, p2, p3, q1, q2, q3 W[128][128] b,
 * q4 W[1][128] b) and encode every shape (blocking).  Errors:
 * LOCC_ERR_INVALID_ARG, LOCC_ERR_BAD_WEIGHTS, LOCC_ERR_OOM, LOCC_ERR_CUDA. */
int locc_voxel_create(const locc_shape_library *lib, const void *weights_blob,
                      size_t blob_bytes, locc_voxel **out);

/* Re-run the shape encoder on `stream` (the latents are already computed by
 * locc_voxel_create; this is for timing and for callers that reload). */
int locc_voxel_encode(locc_voxel *h, void *stream);

/* Copy the latents to out: device float32 [n_shapes][216][16]. */
int locc_voxel_latents(locc_voxel *h, float *out, void *stream);

/* Collision logits of n_pairs pairs: poses [n_obj][7], obj_shape [n_obj],
 * pairs [n_pairs][2] (A, B), logit [n_pairs] float32 (all device). */
int locc_voxel_detect(locc_voxel *h, const float *poses, const int32_t *obj_shape,
                      int32_t n_obj, const int32_t *pairs, int32_t n_pairs,
                      float *logit, void *stream);

/* locc_voxel_detect plus, when not NULL, the selected cells of each object as
 * index ranges cell_ranges [n_pairs][2][6] int32 = (i0, i1, j0, j1, k0, k1),
 * inclusive, i0 > i1 on an empty axis; and the pooled features
 * pooled [n_pairs][2][16] float32. */
int locc_voxel_detect_ex(locc_voxel *h, const float *poses, const int32_t *obj_shape,
                         int32_t n_obj, const int32_t *pairs, int32_t n_pairs,
                         float *logit, int32_t *cell_ranges, float *pooled,
                         void *stream);

/* Arithmetic of the predictor: LOCC_FP32 (CUDA cores, default) or LOCC_BF16
 * (tcgen05 tensor cores: bf16 operands -- pooled features and pose included --
 * with float32 accumulation; selection and pooling stay float32).  Errors:
 * LOCC_ERR_INVALID_ARG. */
int locc_voxel_set_precision(locc_voxel *h, int32_t precision);

/* Synchronise `stream` and report (then clear) the device error flag:
 * 0 or LOCC_ERR_BAD_INDEX. */
int locc_voxel_status(locc_voxel *h, void *stream);

/* Release the handle (blocking). */
void locc_voxel_destroy(locc_voxel *h);

/* Message of the last failing call on this host thread ("" if none). */
const char *locc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LOCC_H_ */
