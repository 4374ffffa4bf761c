/*
 * anim.h -- C ABI of the GB300 skeletal-animation library.
 *
 * The library evaluates, for thousands of characters per frame, the three
 * stages of GPU skeletal animation described in Sec. 1 of "A GPU-based
 * solution for large-scale skeletal animation simulation" (arXiv 2505.06703):
 *   1. Simulation: sample keyframes and interpolate/blend them into local
 *      poses (Sec. 1 step 1; Sec. 2 requires that interpolation and blending
 *      are kept);
 *   2. Hierarchy-Scan: local -> model space, the tree prefix product of
 *      Eq. 1 (Sec. 3);
 *   3. Bind MeshPose: skin = model x inverse bind (Sec. 1 step 3);
 * plus the adjoint of stages 2-3 for position losses and batched IK built on
 * it (extensions of the path, not in the paper).
 *
 * Conventions
 *   - Column vectors; 3x4 row-major affine matrices [R | t] (12 floats,
 *     48 bytes) stand for 4x4 matrices with last row (0 0 0 1).
 *   - Quaternions are stored (x, y, z, w), Hamilton product.
 *   - Local pose L = [R(q/|q|) | t]; model M_i = M_parent(i) L_i (roots:
 *     M_i = L_i); skin S_i = M_i B_i with B_i the inverse bind pose.
 *   - A skeleton type is a parent array with parent[i] < i (the paper's
 *     "traversing the tree in order", Sec. 3.2.1); parent[i] = -1 marks a
 *     root.  Depth counts levels, a root has depth 1.
 *   - Per-joint arrays of a batch of characters are [sum of joint counts][k]
 *     with character c's joints at rows off[c] .. off[c]+n-1, off the
 *     exclusive prefix of the joint counts in character order
 *     (anim_plan_row_offsets).
 *
 * Ownership and threading
 *   - Host arrays passed to create/upload calls are copied; the caller keeps
 *     ownership.  Device pointers passed to the evaluation calls belong to the
 *     caller; the library never frees them.  They must be 16-byte aligned.
 *   - Evaluation calls are asynchronous on the given CUDA stream (`stream`
 *     is a cudaStream_t; NULL is the legacy default stream).  They allocate
 *     nothing and never synchronize, so they can be captured into a CUDA
 *     graph once the plan has been tuned/built.
 *   - A context is not thread-safe; use one per host thread.
 *
 * Errors
 *   Every call returns ANIM_OK (0) or a negative ANIM_E* code and records a
 *   message retrievable with anim_last_error().  No exception crosses the
 *   ABI.  Invalid input data that only the GPU sees (non-finite times, out of
 *   range blend weights are NOT errors; they are used as given) sets bits of
 *   a device status word read by anim_get_status().
 */
#ifndef ANIM_H
#define ANIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ANIM_API __attribute__((visibility("default")))
#else
#define ANIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ANIM_OK = 0,
  ANIM_EINVAL = -1,      /* bad argument (null pointer, size, parent array, alignment) */
  ANIM_ENOMEM = -2,      /* device or host allocation failed */
  ANIM_ECUDA = -3,       /* a CUDA runtime call failed */
  ANIM_ETIMEOUT = -4,    /* a bounded device-side wait expired */
  ANIM_EDEVICE = -5,     /* no usable device / wrong architecture */
  ANIM_ESTATE = -6,      /* call out of order (e.g. clips missing for a type) */
  ANIM_EUNSUPPORTED = -7 /* size beyond a documented limit */
};

/* Device status word bits (anim_get_status). */
enum {
  ANIM_STATUS_NONFINITE_TIME = 1, /* a character time was NaN/Inf; sampled at key 0 */
  ANIM_STATUS_QUEUE = 2           /* a work item was malformed (library bug guard) */
};

/* Limits.  A skeleton type has at most ANIM_MAX_JOINTS joints. */
#define ANIM_MAX_JOINTS 2048
#define ANIM_MAX_KEYS 1024
#define ANIM_MAX_CLIPS 4
#define ANIM_MAX_VERTS (1 << 20)

typedef struct anim_ctx anim_ctx;
typedef struct anim_plan anim_plan;
typedef struct anim_ik anim_ik;

/* Create a context on CUDA device `device` (must be compute capability 10.3,
 * the sm_103a target the kernels are built for).  *out receives the handle. */
ANIM_API int anim_create(anim_ctx **out, int device);

/* Destroy a context and every plan/IK object still owned by it. */
ANIM_API int anim_destroy(anim_ctx *ctx);

/* Message of the last error on this context ("" if none).  Valid until the
 * next call on the context.  ctx may be NULL (then: last create error). */
ANIM_API const char *anim_last_error(const anim_ctx *ctx);

/* Register n_types skeleton types (the joint lists of Sec. 3.2.1).
 *   joint_counts[t]  : 1 .. ANIM_MAX_JOINTS joints of type t;
 *   parents          : concatenated parent arrays, parent[i] in [-1, i-1],
 *                      else ANIM_EINVAL;
 *   inv_bind         : concatenated [n][12] inverse bind poses B_i, or NULL to
 *                      derive them on the GPU as the inverse of the model
 *                      pose of the rest pose (rest_q, rest_t required then);
 *   rest_q, rest_t   : concatenated [n][4] / [n][3] rest pose, or NULL;
 *   out_type_ids     : receives the ids of the new types (n_types entries).
 * Synchronous (returns after the device tables are built). */
ANIM_API int anim_create_skeletons(anim_ctx *ctx, int n_types, const int32_t *joint_counts, const int32_t *parents,
                          const float *inv_bind, const float *rest_q, const float *rest_t,
                          int32_t *out_type_ids);

/* Upload the clips sampled by the Simulation stage (Sec. 1 step 1) for a
 * type: keys is host [n_clips][n_keys][n][8] = qx qy qz qw tx ty tz pad,
 * 1 <= n_clips <= ANIM_MAX_CLIPS (anim_evaluate_frame blends clip 0 -> clip
 * 1 by the per-character weight; anim_evaluate_frame_layers blends all of
 * them), 2 <= n_keys <= ANIM_MAX_KEYS, keys looping with period n_keys /
 * rate_hz seconds.  Replaces earlier clips of the type (and drops an
 * additive layer whose key count or rate no longer matches).  Synchronous. */
ANIM_API int anim_upload_clips(anim_ctx *ctx, int32_t type_id, int n_clips, int n_keys, float rate_hz, const float *keys);

/* An additive layer for a type (the paper asks for the clip blending of an
 * animation state machine to be kept, Sec. 2, without defining layers):
 * host keys [n_keys][n][8] in the clip format, with the clips' n_keys and
 * rate_hz (clips first: ANIM_ESTATE otherwise); applied by
 * anim_evaluate_frame_layers.  Synchronous. */
ANIM_API int anim_upload_additive(anim_ctx *ctx, int32_t type_id, int n_keys, float rate_hz, const float *keys);

/* A plan fixes the characters of a batch: char_type[c] (host, n_chars
 * entries) is each character's type.  The plan holds the row offsets, the
 * per-type work lists and the device scratch of the frame's work queue.
 * n_chars may be 0 (then evaluation calls are no-ops). */
ANIM_API int anim_plan_create(anim_ctx *ctx, int64_t n_chars, const int32_t *char_type, anim_plan **out);
ANIM_API int anim_plan_destroy(anim_ctx *ctx, anim_plan *plan);

/* Total joints of the plan (rows of the per-joint arrays). */
ANIM_API int anim_plan_total_joints(const anim_plan *plan, int64_t *out_total);

/* Host copy of the row offsets: out[0..n_chars] (exclusive prefix). */
ANIM_API int anim_plan_row_offsets(const anim_plan *plan, int64_t *out);

/* Skinned mesh of a type (no counterpart in the paper beyond the skinning
 * step its pipeline ends with, Sec. 1, and Table 1's 1,000-3,000-face
 * meshes): n_verts in [1, ANIM_MAX_VERTS] vertices in bind space, host
 * arrays copied in: rest_pos [n_verts][3], rest_nrm [n_verts][3] (unit),
 * bones [n_verts][4] joint ids in [0, n), weights [n_verts][4] (finite,
 * summing to 1; zero-weight slots are skipped).  Replaces an earlier mesh of
 * the type.  ANIM_EINVAL on an out-of-range bone or a non-finite weight. */
ANIM_API int anim_upload_mesh(anim_ctx *ctx, int32_t type_id, int n_verts, const float *rest_pos,
                              const float *rest_nrm, const int32_t *bones, const float *weights);

/* Triangles of a type's mesh for anim_raster: host faces [n_faces][3]
 * vertex indices in [0, n_verts) of the mesh uploaded before (ANIM_ESTATE
 * without one), 1 <= n_faces <= 4,096.  Replaces earlier faces. */
ANIM_API int anim_upload_faces(anim_ctx *ctx, int32_t type_id, int n_faces, const int32_t *faces);

/* Host copy of the plan's vertex offsets: out[0..n_chars], the exclusive
 * prefix of the characters' vertex counts (0 for a type without a mesh). */
ANIM_API int anim_plan_vertex_offsets(anim_ctx *ctx, const anim_plan *plan, int64_t *out);

/* The fused frame (Sec. 1 steps 1-3): for each character c, sample its
 * type's clips at d_time[c] seconds, blend clip 0 -> clip 1 with
 * d_blend_w[c], compose down the hierarchy (Eq. 1) and multiply by the inverse
 * bind.  d_time, d_blend_w: device [n_chars] float; d_skin: device
 * [total][12] float (written).  A small work-queue launch, then the frame
 * kernels: the segmented persistent kernel for the types without a
 * chain-walk schedule and, under a schedule that enables it, the chain-walk
 * kernel for the others -- one after the other on `stream` when the
 * segmented part holds at most 16 work items, otherwise side by side on a
 * second stream of the context that `stream` forks to and joins back. */
ANIM_API int anim_evaluate_frame(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_blend_w,
                        float *d_skin, void *stream);

/* The fused frame from and to host memory, for callers whose inputs and
 * outputs live on the host: h_time and h_blend_w (host [n_chars] float) are
 * copied in, the frame runs as in anim_evaluate_frame, and the skin matrices
 * are copied back into h_skin (host [total][12] float), all in order on
 * `stream`; the output is complete once `stream` has synchronized.
 * Page-locked buffers (cudaMallocHost, cudaHostRegister) make the copies
 * asynchronous; pageable ones work through the driver's staging.  A plan of
 * at least 1,024 characters is evaluated in up to 4 contiguous ranges of
 * nearly equal joint counts, each range's skin matrices copied back on a
 * second stream of the plan while the next range's frame runs (the call's
 * `stream` waits for those copies, so the rule above holds).  The device
 * staging buffers (n_chars x 8 B + total x 48 B), the ranges' own plans, the
 * copy stream and its events belong to the plan and are created by the
 * first call, which is therefore not capturable in a CUDA graph; later calls
 * with page-locked buffers are. */
ANIM_API int anim_evaluate_frame_host(anim_ctx *ctx, anim_plan *plan, const float *h_time, const float *h_blend_w,
                             float *h_skin, void *stream);

/* The fused frame followed by linear blend skinning of every character's
 * mesh, fused into the same kernel: vertex v of character c goes to
 * sum_k w_k S_{b_k} [p; 1] with normal normalize(sum_k w_k R_{b_k} n), where
 * S = [R | t] are the character's skin matrices (rigid), still in shared
 * memory.  d_verts: device [total vertices][6] float (position, normal) at
 * the plan's vertex offsets, 16-byte aligned; d_skin may be NULL, and then
 * the skin matrices never reach memory.  Every type runs on the segmented
 * kernel here (the chain-walk kernel has no skinning pass). */
ANIM_API int anim_evaluate_frame_skinned(anim_ctx *ctx, const anim_plan *plan, const float *d_time,
                                         const float *d_blend_w, float *d_skin, float *d_verts, void *stream);

/* The fused frame with layered blending: every clip of a character's type
 * is sampled at d_time[c] (slerp between keys, lerp for translations), the
 * rotations are blended by incremental slerp -- q = q_0, W = w_0, then for
 * each further clip i: W += w_i and, while W > 0, q = slerp(q, q_i, w_i / W)
 * -- and the translations by their weighted mean (clip 0's when all weights
 * are 0); two clips with weights (1 - w, w) give anim_evaluate_frame's
 * blend.  A type with an additive layer then takes q * slerp(1, q_a, a) and
 * t + a t_a with a = d_add_w[c] (d_add_w NULL: a = 0).  d_weights: device
 * [n_chars][4] float (weights of clips beyond the type's count are
 * ignored), non-negative; d_skin as in anim_evaluate_frame.  Every type
 * runs on the segmented kernel here. */
ANIM_API int anim_evaluate_frame_layers(anim_ctx *ctx, const anim_plan *plan, const float *d_time,
                                        const float *d_weights, const float *d_add_w, float *d_skin, void *stream);

/* Camera and crowd layout of anim_raster. */
typedef struct anim_raster_params {
  int32_t width, height;  /* image size in pixels */
  int32_t cols;           /* characters per grid row */
  float spacing;          /* world distance between grid cells */
  float ox, oy, scale;    /* screen = (ox + scale X, oy - scale Y) */
} anim_raster_params;

/* Headless rasterization of the skinned crowd (the paper renders its crowd,
 * Sec. 4 and Fig. 6, through a graphics API; no graphics stack here):
 * character c stands at world offset (col * spacing, -row * spacing, 0),
 * col = c % cols, row = c / cols; an orthographic camera looking down -Z
 * maps (X, Y, Z) to screen (ox + scale X, oy - scale Y), depth (2 - Z) / 4.
 * Positions snapped to 1/256 pixel; a pixel is covered when its centre is
 * inside a triangle by integer edge functions, ties on an edge a->b going to
 * the triangle when b - a points down or horizontally left; the nearest
 * depth wins, then the smaller id c * 4096 + face.  d_verts: the skinned
 * vertices of anim_evaluate_frame_skinned; d_vis: device scratch
 * [height][width] uint64; d_ids (nullable): [height][width] winning ids,
 * 0xFFFFFFFF where empty; d_rgba (nullable): [height][width] flat-shaded
 * RGBA8.  At most 1,048,575 characters.  Three launches on `stream`. */
ANIM_API int anim_raster(anim_ctx *ctx, const anim_plan *plan, const float *d_verts, const anim_raster_params *params,
                         uint64_t *d_vis, uint32_t *d_ids, uint32_t *d_rgba, void *stream);

/* The two launches of anim_evaluate_frame, for callers that schedule them
 * apart (e.g. to time the persistent kernel alone): build_queue buckets the
 * characters by (type, key index) into the plan's work queue from d_time;
 * run_queue is the persistent frame kernel consuming that queue.  run_queue
 * must follow a build_queue with the same d_time in stream order. */
ANIM_API int anim_frame_build_queue(anim_ctx *ctx, const anim_plan *plan, const float *d_time, void *stream);
ANIM_API int anim_frame_run_queue(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_blend_w,
                                  float *d_skin, void *stream);

/* The same frame computed by the plain comparator: one CTA per character,
 * one launch per skeleton type, one barrier per tree level (the
 * level-synchronous schedule).  Same arguments and results. */
ANIM_API int anim_evaluate_frame_levelsync(anim_ctx *ctx, const anim_plan *plan, const float *d_time,
                                  const float *d_blend_w, float *d_skin, void *stream);

/* Hierarchy-Scan (Eq. 1) + Bind from given local poses: d_q [total][4]
 * (unnormalized allowed, normalized internally), d_t [total][3].  Writes
 * d_skin [total][12] and/or d_model [total][12] (either may be NULL, not
 * both). */
ANIM_API int anim_forward_local(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t, float *d_skin,
                       float *d_model, void *stream);

/* Level-synchronous comparator of anim_forward_local (skin output only). */
ANIM_API int anim_forward_local_levelsync(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t,
                                 float *d_skin, void *stream);

/* The paper's own Hierarchy-Scan schedules as GPU comparators of
 * anim_forward_local (skin output only): one CTA per character, one thread
 * per joint, joints in shared memory, a block barrier between phases.
 * algorithm 1: every joint walks to the root multiplying its ancestors'
 * local matrices (Sec. 2, Alg. 1); 2: pointer doubling over joints,
 * ceil(log2 depth) rounds (Sec. 3.1, Alg. 2 and Eq. 2); 3: 64-node blocks,
 * 6 in-block doubling rounds, then a walk over the nearest out-of-block
 * ancestors' partial products (Sec. 3.2.1, Alg. 3); 4: a joint and up to 7
 * in-block ancestors serially, up to 7 jumps of stride 8, then the
 * out-of-block walk (Sec. 3.2.2, Alg. 4); 5: threads for the leaf joints
 * only, each composing down its root path and writing every joint on it
 * (the scheme Sec. 2 attributes to KIYA).  Same inputs and outputs as
 * anim_forward_local.  ANIM_EUNSUPPORTED if a type of the plan has more than
 * 1,024 joints; ANIM_EINVAL for another algorithm number. */
ANIM_API int anim_forward_local_paper(anim_ctx *ctx, const anim_plan *plan, int algorithm, const float *d_q,
                                      const float *d_t, float *d_skin, void *stream);

/* Adjoint of anim_forward_local's model positions p_j (translation column
 * of M_j): given d_grad_pos [total][3] = dLoss/dp, writes d_grad_q [total][4]
 * (w.r.t. the unnormalized q) and d_grad_t [total][3].  The forward pass is
 * recomputed inside the kernel; nothing is stored between the calls.
 * Rigid poses only (unit quaternion rotations, unit scale). */
ANIM_API int anim_backward(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t,
                  const float *d_grad_pos, float *d_grad_q, float *d_grad_t, void *stream);

/* Fused forward + adjoint of the loss sum_j |p_j - target_j|^2: d_target
 * [total][3]; writes d_grad_q, d_grad_t and, if d_loss != NULL, each
 * character's loss d_loss[n_chars]. */
ANIM_API int anim_loss_backward(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t,
                       const float *d_target, float *d_grad_q, float *d_grad_t, float *d_loss, void *stream);

/* Batched IK: n_eff effector joints per type (host [n_types_of_ctx][n_eff],
 * entries for types the plan does not use are ignored).  The IK object owns
 * the active-subtree tables, a device step counter and its own Adam state
 * for the active joints only (2 x 16 B per active joint, zeroed here). */
ANIM_API int anim_ik_create(anim_ctx *ctx, const anim_plan *plan, int n_eff, const int32_t *effectors, anim_ik **out);
ANIM_API int anim_ik_destroy(anim_ctx *ctx, anim_ik *ik);

/* Reset the IK step counter to 0 and zero the object's own Adam state
 * (asynchronous on stream). */
ANIM_API int anim_ik_reset(anim_ctx *ctx, anim_ik *ik, void *stream);

/* One IK step, all in one kernel: forward over the effectors' ancestors,
 * loss sum_e |p_e - target_e|^2, adjoint, and an Adam update (PyTorch's
 * definition, step counter kept on the device and incremented) of d_q
 * ([total][4], updated in place) with the moments in d_m, d_v ([total][4],
 * updated in place), or -- both NULL -- in the object's own state, which
 * holds the active joints only, contiguous in the active subtree's order
 * (whole 32-byte sectors instead of the caller's scattered 16-byte rows).
 * Only the active joints' rows of d_q, d_m, d_v are read or written.  d_t [total][3] fixed; d_targets
 * [n_chars][n_eff][3]; d_loss[n_chars] (nullable) receives each
 * character's loss before the update.  ANIM_EINVAL if exactly one of d_m,
 * d_v is NULL. */
ANIM_API int anim_ik_step(anim_ctx *ctx, anim_ik *ik, float *d_q, float *d_m, float *d_v, const float *d_t,
                 const float *d_targets, float lr, float beta1, float beta2, float eps, float *d_loss,
                 void *stream);

/* Autotuner (no counterpart in the paper; it picks the schedule of the
 * scan): times every candidate schedule -- segment length 4/8/16/32 for the
 * pointer-jumping scan, 1, 2 or 3 resident CTAs per SM of the persistent
 * kernels, work items of about 1,024/2,048/4,096 joints, and for the
 * frame whether walkable types (chain schedules of at most 160 steps with
 * most lanes busy) run on one of the two chain-walk kernels beside the
 * segmented kernel -- of
 * `which` (0 = fused frame, 1 = forward_local, 2 = loss_backward, 3 = frame
 * with skinning, 4 = frame with layered blending) with CUDA events on scratch
 * inputs it allocates, and keeps the fastest.  The result
 * is cached in the context per hash of (which, type ids, joint counts,
 * depths, character counts); calling anim_tune again for the same mix
 * applies the cached schedule without timing.  The schedule is per context
 * (segment lengths of the plan's types, CTAs per SM, item size), so it also
 * applies to other plans of the context.  Synchronous; not capturable;
 * which = 0, 3 and 4 need clips for every type of the plan (3 skins the
 * meshes uploaded, 4 blends the clips and additive layers uploaded). */
ANIM_API int anim_tune(anim_ctx *ctx, anim_plan *plan, int which);

/* The same search for the fused IK step (anim_ik_step): each candidate
 * schedule gets a temporary IK object for `effectors` (as in anim_ik_create)
 * and is timed on scratch state it allocates; the fastest is applied and
 * cached per (type mix, effectors).  An IK object created afterwards keeps
 * that schedule.  The IK step runs on the effectors' ancestors only, much
 * smaller than the whole skeletons anim_tune(which = 2) times, so its best
 * schedule differs.  Synchronous; not capturable. */
ANIM_API int anim_tune_ik(anim_ctx *ctx, anim_plan *plan, int n_eff, const int32_t *effectors);

/* The schedule the autotuner picked, as 5 integers: segment length, resident
 * CTAs per SM, work-item size in joints, chain-walk kernel for the frame
 * (0: none, 1: one warp per item, 2: three warps per item, two of them
 * sampling the local transforms and writing the skin rows out, one walking
 * the chains), adjoint kernel (0: persistent, k = 1..8: one work item per CTA,
 * items sized so k CTAs share an SM) -- read with anim_get_schedule (segment
 * length of the plan's first type) and re-applied without timing by
 * anim_set_schedule (for example in another process); CTAs per SM is 1, 2
 * or 3.  anim_set_schedule returns ANIM_EUNSUPPORTED and keeps the previous
 * schedule when one character of a type does not fit in a CTA's shared
 * memory under the new one; a schedule that fits the forward kernels but
 * not the adjoint (which keeps two more vectors per joint) is accepted, and
 * anim_backward / anim_loss_backward then return ANIM_EUNSUPPORTED until a
 * schedule that fits is set.  An IK object keeps the adjoint kernel of the
 * schedule it was created under.  Synchronous; not capturable. */
ANIM_API int anim_get_schedule(anim_ctx *ctx, const anim_plan *plan, int32_t *out5);
ANIM_API int anim_set_schedule(anim_ctx *ctx, anim_plan *plan, const int32_t *in5);

/* Read and clear the device status word (synchronizes `stream`). */
ANIM_API int anim_get_status(anim_ctx *ctx, void *stream, int *out_status);

/* Host-only skeleton analysis (no GPU needed): the segment decomposition the
 * scan uses for a maximum segment length seg_len.  Outputs: *out_nseg,
 * out_seg_start[nseg+1] (caller provides n+1 entries), *out_rounds (pointer
 * jumping rounds over segments), *out_depth (tree depth, root = 1). */
ANIM_API int anim_analyze_skeleton(int n, const int32_t *parents, int seg_len, int32_t *out_nseg,
                          int32_t *out_seg_start, int32_t *out_rounds, int32_t *out_depth);

/* Forward scan + bind for callers that cannot allocate device memory.
 * (No counterpart in the paper: this is a deployment variant of
 * anim_forward_local.)  Some callers may not call cudaMalloc at all: code
 * running under a fixed device-memory budget or a custom allocator that owns
 * every byte, plug-ins handed only pre-allocated buffers by their host, or
 * processes that must not grow their footprint after start-up.  This entry
 * point creates no context or plan and allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call): its scratch -- the skeleton's segment
 * tables, the record the kernel reads and the work-queue counter -- lives in
 * a 96 KB static device array that every GPU loading the library holds
 * until the process exits.
 *   n_joints            : 1 .. ANIM_MAX_JOINTS joints of the one skeleton type;
 *   parents             : host [n_joints], parent[i] in [-1, i-1];
 *   n_chars             : 0 .. 16,777,216 characters of that type, character c
 *                         at rows c*n_joints .. c*n_joints + n_joints - 1;
 *   d_q, d_t            : device [n_chars*n_joints][4] (unnormalized allowed) and
 *                         [n_chars*n_joints][3] local poses;
 *   d_inv_bind          : device [n_joints][12] inverse bind poses;
 *   d_skin              : device [n_chars*n_joints][12], written.
 * d_q, d_inv_bind and d_skin must be 16-byte aligned.  Besides the joint
 * count, the skeleton's shape is limited by shared memory: one character's
 * work item takes 16 * (3 n + 1 + 6 nseg) bytes plus its tables, nseg the
 * number of segments (natural chains, parent[i+1] == i, cut into pieces of at
 * most 16 joints), and must fit one CTA's opt-in shared memory (about 213 KB
 * here): a 2,048-joint chain fits, a 2,048-joint star (nseg about n) does not.
 * Returns ANIM_EINVAL (NULL pointer, bad parent, misalignment),
 * ANIM_EUNSUPPORTED (a size beyond the limits above, or `stream` is being
 * captured into a CUDA graph) or ANIM_ECUDA; there is no message string.
 * n_chars == 0 returns ANIM_OK and touches nothing.  The first call on a
 * device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Each call writes the tables into the array
 * with an asynchronous copy from a host staging buffer of the calling thread
 * on `stream` and launches the kernel after it, which is why a capturing
 * stream is refused: the recorded copy would replay the buffer's contents at
 * replay time.  Every call shares the one array, so calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialized by the caller. */
ANIM_API int anim_forward_local_noalloc(int n_joints, const int32_t *parents, int64_t n_chars, const float *d_q,
                                        const float *d_t, const float *d_inv_bind, float *d_skin, void *stream);

/* Library version (major * 10000 + minor * 100 + patch). */
ANIM_API int anim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ANIM_H */
