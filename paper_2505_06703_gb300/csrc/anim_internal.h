// Internal declarations shared by the host runtime (host.cu) and the kernel
// translation units.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace anim {

// Per-type device tables (all pointers are device memory owned by the
// context).  The joint order is the caller's order; the scan works on
// "segments": maximal runs of consecutive joints i, i+1, ... with
// parent[i+1] == i (natural chains), cut into pieces of at most seg_len
// joints.  Segments partition [0, n) into intervals.
struct TypeDev {
  int n;           // joints
  int nseg;        // segments
  int rounds;      // pointer-jumping rounds over the segment tree
  int max_depth;   // tree depth (root = 1)
  int n_clips;     // 0 if no clips uploaded
  int n_keys;
  float rate;
  int chain;       // 1: the joints form one natural chain (parent[i] = i - 1 for i > 0)
  const int32_t *parent;     // [n]
  const int32_t *depth;      // [n]
  const int32_t *seg_start;  // [nseg + 1]
  const int32_t *seg_link;   // [nseg]  parent joint of the segment's first joint, -1 for roots
  const uint32_t *jinfo;     // [n] segment of the joint (bits 0-15) | kJStart | kJLink
  // The same tables in the 16-bit form the kernels keep in shared memory,
  // staged there by cp.async: jinfo16 [n rounded up to even] = segment |
  // kJ16Start | kJ16Link; sub16, par16, gat16 [n] = sub_end, parent and
  // gather (identity for a type) as int16.
  const uint16_t *jinfo16;
  const int16_t *sub16, *par16, *gat16;
  const float4 *inv_bind;    // [n][3] rows of B_i
  const float4 *keys;        // [n_clips][n_keys][n][2]: (qx qy qz qw), (tx ty tz theta); theta's sign
                             // bit: the next key lies on the other hemisphere
  const float4 *add_keys;    // additive layer [n_keys][n][2] in the same format, or nullptr
  // adjoint (on views numbered in depth-first pre-order, so a joint's slot
  // is its index and its subtree is [j, sub_end[j]))
  const int32_t *sub_end;    // [n] one past the subtree of joint j
  // IK views: the active subtree of a type; view joint j reads row gather[j]
  // of the full type (nullptr = identity).
  const int32_t *gather;
  // A view that renumbers every joint of its type: the view slot of each of
  // the type's joints (the inverse of gather), else nullptr.
  const int32_t *inv_gather;
  // The paper's 64-node blocks (comparator kernels): nearest ancestor of
  // each joint outside its block of 64 consecutive indices, -1 at the top.
  const int32_t *blk_out;
  // Skinned mesh (linear blend skinning after the bind product): 3 float4
  // per vertex: (px py pz nx), (ny nz w0 w1), (w2 w3 bones01 bones23) with
  // the bone ids as 16-bit pairs in the last two words' bits.
  int n_verts;
  int n_faces;
  const float4 *mesh;
  const int32_t *faces;      // [n_faces][3] vertex indices (raster)
  // Chain-walk frame kernel (k_walk): a static lane schedule of wk_S steps
  // for wk_P lanes per character, staged in chunks of wk_K steps (the table
  // is padded with idle entries to whole chunks); entry [s][slot] names the
  // joint lane `slot` composes at step s (kWInvalid: idle).  wk_mode 1:
  // natural chains walked parent-first, branch-point matrices passed through
  // shared memory; 0: the type runs on the segmented CTA kernels only.
  int wk_mode, wk_P, wk_logP, wk_S;
  int wk_nbs;                // branch-point slots per character (mode 1)
  int wk_K;
  const uint32_t *wk_tab;    // [wk_S][wk_P]
  // key-pair records in schedule order with the inverse binds folded in
  // (skin-space walk), clips 0 and 1: [clip][key][wk_S][4][wk_P] float4 =
  // (q0', q_perp', (t0', theta), (t1' - t0', 0)); nullptr: the type does not
  // run on the walk kernel (no clips yet, or inverse binds that are not rigid)
  const float4 *wk_keys;
  const float4 *wk_u;        // [wk_S][wk_P] (u = R_B^T t_B of the slot's joint, 0)
};
// Chain-walk schedule entries: joint | flags | load slot | store slot; bit 31
// set marks an idle entry.
constexpr uint32_t kWInvalid = 0xFFFFFFFFu;
constexpr uint32_t kWJoint = 0xFFFu;        // bits 0-11
constexpr uint32_t kWStart = 1u << 12;      // first joint of a chain: M = slot[load] * L (or L at a root)
constexpr uint32_t kWStore = 1u << 13;      // branch point: keep M in slot[store]
constexpr int kWLoadShift = 15;             // bits 15-22
constexpr int kWStoreShift = 23;            // bits 23-30
constexpr uint32_t kWRootSlot = 255;        // load slot of a chain that starts at a root
constexpr int kWalkMaxSteps = 160;          // longest schedule the walk kernel takes (latency bound)
constexpr int kWalkMaxSmem = 32 * 1024;     // shared memory of one walk CTA (staging + branch slots)
// Static shared memory the persistent kernels may use besides the dynamic
// item buffers (two staged work items, scan scratch); the host subtracts it
// from the per-CTA budget.
constexpr int kStaticSmemAllowance = 14 * 1024;

// Device status word bits (ANIM_STATUS_* in the ABI).
constexpr int kStatusNonfiniteTime = 1;
constexpr int kStatusTimeout = 4;

constexpr uint32_t kJStart = 1u << 16;  // joint opens its segment
constexpr uint32_t kJLink = 1u << 17;   // the joint's segment hangs from a parent joint
// 16-bit joint info (shared memory): segment (14 bits) | start | link.
constexpr uint16_t kJ16Seg = 0x3FFFu, kJ16Start = 0x4000u, kJ16Link = 0x8000u;

// One unit of work: `count` characters of one type.  For the frame the
// characters share the key index k0 (so they read the same key records).
struct WorkItem {
  int32_t start;  // index into the item character list
  int32_t count;
  int32_t type;
  int32_t k0;
};

// Persistent kernels: 8 compute warps + 1 producer warp per CTA.
constexpr int kPersistentThreads = 288;
// One-item adjoint kernel: 4 warps, no producer; its static shared memory.
constexpr int kAdjSmallThreads = 128;
constexpr int kAdjSmallStatic = 4 * 1024;

struct LaunchCfg {
  int threads;       // CTA size
  int ctas;          // persistent grid size
  size_t smem;       // dynamic shared memory per CTA (bytes)
  int min_blocks = 2;  // resident CTAs per SM the kernel variant is compiled for (2 or 3)
};

// ---------------------------------------------------------------- kernels
// Arguments of the persistent scan kernels (k_scan_qt's modes, k_scan).
struct ScanArgs {
  const TypeDev *types;
  const WorkItem *items;
  int n_items;
  const int32_t *item_chars;   // character ids referenced by items
  const int64_t *row_off;      // [n_chars + 1]
  int *queue_head;             // device work-queue counter (0 at launch)
  int *done;                   // finish counter for the last-CTA reset (nullptr: no reset)
  int *status;
  // sampled mode
  const float *time;
  const float *blend_w;
  // local-pose mode
  const float *q;
  const float *t;
  // outputs
  float *skin;
  float *model;
  int C_max_unused;
  // frame with skinning: vertices [sum of vertex counts][6] (position,
  // normal) at the characters' vertex offsets; skin may then be nullptr
  float *verts;
  const int64_t *vert_off;  // [n_chars + 1]
  // frame with layered blending: clip weights [n_chars][4] and additive
  // weights [n_chars] (nullable); blend_w is unused then
  const float *layer_w;
  const float *add_w;
};

// The matrix frame kernel with the skinning pass (a.verts).
cudaError_t launch_scan(const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t s);

// Frame work queue.  The plan cuts the characters of each type (types in
// cost order) into ranges of at most kRangeChars (kRangeCharsMax for the
// walk kernel's types, whose items hold 32 / P characters: larger ranges
// leave fewer part-filled items per key bin), each owning a region of
// item slots large enough for any key distribution.  One CTA per range sorts
// its characters by key index k0 (counting sort in shared memory) and writes
// work items of at most cap[type] characters sharing (type, k0) into its
// region, then empty items (count 0) into the rest of the region.
constexpr int kRangeChars = 256;
constexpr int kRangeCharsMax = 1024;
constexpr int kMaxRanges = 4096;  // so at most ~900,000 characters per plan
struct RangeDev {
  int32_t type;
  int32_t start;   // first index into the type-grouped character list
  int32_t count;   // characters (<= kRangeCharsMax)
  int32_t region;  // first item slot of the range
};
struct BucketArgs {
  const RangeDev *ranges;
  int n_ranges;
  int n_slots;                // total item slots (end of the last region)
  const int32_t *type_chars;  // characters grouped by type, plan order
  const float *time;          // [n_chars]
  const TypeDev *types;
  const int32_t *cap;         // [n_types] characters per item
  int32_t *sorted;            // same indexing as type_chars, sorted by k0 within each range
  WorkItem *items;            // [n_slots]
  int *queue_head;            // [1] reset to 0
  int *status;
};
constexpr int kMaxTypes = 512;
cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t s);

// Plain level-synchronous comparator: one CTA per character of one type.
struct LevelArgs {
  TypeDev type;
  const int32_t *chars;  // characters of this type
  int n_chars;
  const int64_t *row_off;
  const float *time, *blend_w;
  const float *q, *t;
  float *skin;
  int *status;
};
cudaError_t launch_levelsync(int mode, const LevelArgs &a, int threads, cudaStream_t s);

// Adjoint.  mode: 0 = grad_pos given, 1 = loss vs targets, 2 = IK step, 3 =
// IK step with the IK object's own Adam state.
struct AdjointArgs {
  const TypeDev *types;
  const WorkItem *items;
  int n_items;
  const int32_t *item_chars;
  const int64_t *row_off;
  int *queue_head;         // 0 at launch; reset by the last CTA
  int *done;               // finish counter for that reset
  int *status;
  const float *q, *t;
  const float *grad_pos;   // mode 0
  const float *target;     // mode 1: [total][3]; mode 2: [n_chars][n_eff][3]
  float *grad_q, *grad_t;  // modes 0, 1
  float *loss;             // per character, nullable
  // IK (mode 2): types are active-subtree views (TypeDev::gather maps view
  // joints to rows of the full type); effectors are view joint ids.
  const int32_t *eff_slot;       // [n_types][n_eff] view joint ids
  int n_eff;
  float *m, *v;
  // mode 3 (IK with the object's own Adam state): m, v hold one row per
  // view joint in view order, character c's rows from state_off[c]; in mode
  // 2 they are the caller's [total][4] rows
  const int64_t *state_off;
  float *q_mut;
  int *step;         // device step counter (read at start, incremented by the last CTA)
  float lr, beta1, beta2, eps;
};
cudaError_t launch_adjoint(int mode, const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t s);

// Chain-walk frame kernel: one-warp CTAs, CTA i running work-queue slot i
// (at most 32 / wk_P characters of one walk type sharing the key index k0;
// empty slots exit), composing them lane-parallel along the type's schedule.
struct WalkArgs {
  const TypeDev *types;
  const WorkItem *items;
  int n_items;                 // slots (the grid)
  int nbs_max;                 // branch-point slot capacity per character
  const int32_t *item_chars;
  const int64_t *row_off;
  int *status;
  const float *time, *blend_w;
  float *skin;
  // 0: wait for the preceding grid (the work-queue kernel) before reading
  // the item.  1 (k_walk2 only): the preceding grid is the segmented frame
  // kernel, which lets this launch start only after its own wait for the
  // work queue; the item and the inputs are read from L2 at once, and each
  // CTA waits for that grid at its end, so that the next launch in the
  // stream (the next frame's work queue) still follows both.
  int pred_waited;
};
size_t walk_smem_bytes(int chars_per_item, int nbs);
// The warp-specialized variant (three warps per item: two sample and write
// out, one walks), same arguments and tables.
size_t walk2_smem_bytes(int chars_per_item, int nbs);
cudaError_t launch_walk2(const WalkArgs &a, size_t smem, cudaStream_t s);
int walk2_blocks_per_sm(size_t smem);
// Shared memory per CTA of the warp-specialized walk, padded up from `smem`
// so that at most ceil(n_items / sm_count) CTAs are resident per SM: the
// block scheduler then spreads the items evenly instead of stacking one
// more on some SMs (the frame ends with its most loaded SM).
size_t walk2_spread_smem(size_t smem, int n_items, int sm_count);
cudaError_t launch_walk(const WalkArgs &a, size_t smem, cudaStream_t s);
int walk_blocks_per_sm(size_t smem);  // resident one-warp CTAs per SM at this shared-memory size

// The paper's Algorithms 1-4 (comparators): one CTA per character.
constexpr int kPaperMaxJoints = 1024;
struct PaperArgs {
  const TypeDev *types;
  const int32_t *char_type;
  const int64_t *row_off;
  int algo;  // 1..4
  const float *q, *t;
  float *skin;
};
size_t paper_smem_bytes(int n);
cudaError_t launch_paper(const PaperArgs &a, int n_chars, int threads, size_t smem, cudaStream_t s);

// Headless rasterization of skinned characters (comparator picture of the
// paper's rendering): clear, one CTA per character rasterizing its faces
// into the 64-bit visibility buffer, resolve to ids / RGBA.
struct RasterArgs {
  const TypeDev *types;
  const int32_t *char_type;
  const int64_t *vert_off;
  const float *verts;             // [total vertices][6]
  unsigned long long *vis;        // [height][width]
  uint32_t *ids;                  // nullable
  uint32_t *rgba;                 // nullable
  int width, height, cols;
  float spacing, ox, oy, scale;
};
cudaError_t launch_raster(const RasterArgs &a, int n_chars, cudaStream_t s);

// Setup kernels.
cudaError_t launch_prepare_keys(float4 *keys, int n_clips, int n_keys, int n, cudaStream_t s);
cudaError_t launch_bind_from_rest(const int32_t *parent, const float *rest_q, const float *rest_t, int n,
                                  float4 *inv_bind, cudaStream_t s);

// Shared-memory footprint of one work item of C characters (bytes).
size_t scan_smem_bytes(int n, int nseg, int C);
size_t adjoint_smem_bytes(int n, int nseg, int C);
size_t scan_qt_smem_bytes(int n, int nseg, int C);

// The scan on (quaternion, translation) items: mode 0 the plain frame (skin
// matrices out), mode 1 the forward from local poses (skin and / or model
// matrices out), mode 2 the frame with layered blending.
cudaError_t launch_scan_qt(int mode, const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t s);

}  // namespace anim
