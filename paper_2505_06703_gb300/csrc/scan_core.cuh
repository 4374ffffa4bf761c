// The segmented Hierarchy-Scan shared by the forward and adjoint kernels.
//
// Eq. 1 defines the model pose of joint i as the product of the local
// matrices on the root-to-i path.  The paper evaluates it with one thread per
// joint, pointer jumping and block barriers (Sec. 3, Algs. 2-4).  Here the
// tree is cut into segments (runs of consecutive joints where each joint is
// the parent of the next, at most seg_len long) and a work item of C
// characters is processed in shared memory:
//   pass 1a  every (joint, character) builds its local matrix L_j: the
//            Simulation math, fully parallel;
//   pass 1b  one lane per (segment, character) walks its segment and
//            replaces L_j by the running product P_j = L_first ... L_j
//            (work-efficient: one 3x4 product per joint, light serial work);
//   pass 2   pointer jumping over the segment tree (the paper's doubling idea
//            applied to segments instead of joints): Y_g starts as the
//            partial product at the joint the segment hangs from and, after
//            ceil(log2(segment depth)) rounds, is the model pose of that joint;
//   pass 3   M_j = Y_seg(j) P_j, then the Bind MeshPose product S_j = M_j B_j,
//            written back in place; one thread per joint walks a group of the
//            item's characters so B_j is loaded once per group.
//
// CTA layout: kComputeWarps warps run the passes and synchronize among
// themselves on named barrier 1; one producer warp fetches the next work
// item (queue counter, descriptor, type table, per-character data) into the
// other half of a double buffer and hands it over on named barrier 2.
#pragma once
#include "anim_internal.h"
#include "dev_math.cuh"

namespace anim {

constexpr int kComputeWarps = 8;
constexpr int kComputeThreads = kComputeWarps * 32;
constexpr int kCtaThreads = kComputeThreads + 32;
static_assert(kCtaThreads == kPersistentThreads, "CTA shape");
constexpr int kCMax = 64;  // characters per work item

__device__ __forceinline__ void compute_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kComputeThreads) : "memory");
}
__device__ __forceinline__ void handoff_sync() { asm volatile("bar.sync 2, %0;" ::"n"(kCtaThreads) : "memory"); }
// Barrier among the NT threads that run the passes: the persistent kernels'
// compute warps (named barrier 1), or the whole CTA of a kernel whose
// threads all compute.
template <int NT>
__device__ __forceinline__ void pass_sync() {
  if constexpr (NT == kComputeThreads)
    compute_sync();
  else
    __syncthreads();
}

// cp.async global -> shared copy of 4 bytes (both addresses 4-byte aligned);
// the issuing thread waits for its copies with cp_async_wait_all.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Everything one work item needs besides the big buffers (double-buffered).
struct ItemBuf {
  TypeDev T;
  FastDiv divC, divS, divN;  // by C, by nseg, by n
  int item;                  // -1: no more work
  int C, k0, type;
  int cgroups, cpt;          // pass 3: character groups and characters per group
  long long off[kCMax];      // first row of each character
  long long voff[kCMax];     // first skinned vertex of each character (frame with skinning)
  int cid[kCMax];
  float alpha[kCMax];        // frame: fraction between keys k0 and k0+1
  float blend[kCMax];        // frame: clip blend weight
  float lw[kCMax][4];        // frame with layers: clip weights
  float law[kCMax];          // frame with layers: additive weight
};
static_assert(2 * sizeof(ItemBuf) + 2048 <= kStaticSmemAllowance, "item buffers exceed the static allowance");

struct LayerIn {
  const float *w;    // [n_chars][4]
  const float *add;  // [n_chars] or nullptr
};

template <int MODE>
__device__ __forceinline__ void stage_item(ItemBuf &b, int it, const WorkItem &wi, const TypeDev *types,
                                           const int32_t *item_chars, const int64_t *row_off, const float *time,
                                           const float *blend_w, int *status, const int64_t *vert_off = nullptr,
                                           LayerIn layers = LayerIn{nullptr, nullptr});

// Producer warp: grab the next item from the queue and stage its data.
// MODE 0 (frame) also computes each character's key fraction.
template <int MODE>
__device__ __forceinline__ void fetch_item(ItemBuf &b, int *queue_head, int n_items, const WorkItem *items,
                                           const TypeDev *types, const int32_t *item_chars, const int64_t *row_off,
                                           const float *time, const float *blend_w, int *status,
                                           const int64_t *vert_off, LayerIn layers) {
  const int lane = threadIdx.x & 31;
  int it = 0;
  WorkItem wi;
  for (;;) {  // skip empty slots of the frame's work queue
    if (lane == 0) it = atomicAdd(queue_head, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) {
      if (lane == 0) b.item = -1;
      __syncwarp();
      return;
    }
    wi = items[it];
    if (wi.count > 0) break;
  }
  stage_item<MODE>(b, it, wi, types, item_chars, row_off, time, blend_w, status, vert_off, layers);
}

// One warp stages work item `it` (descriptor wi) into b.
template <int MODE>
__device__ __forceinline__ void stage_item(ItemBuf &b, int it, const WorkItem &wi, const TypeDev *types,
                                           const int32_t *item_chars, const int64_t *row_off, const float *time,
                                           const float *blend_w, int *status, const int64_t *vert_off,
                                           LayerIn layers) {
  const int lane = threadIdx.x & 31;
  // the type record by cp.async, overlapping the character loads below
  const int *src = reinterpret_cast<const int *>(types + wi.type);
  int *dst = reinterpret_cast<int *>(&b.T);
  for (int k = lane; k < (int)(sizeof(TypeDev) / 4); k += 32) cp_async4(dst + k, src + k);
  cp_async_commit();
  const float rate = types[wi.type].rate;
  for (int c = lane; c < wi.count; c += 32) {
    const int cid = __ldg(item_chars + wi.start + c);
    b.cid[c] = cid;
    b.off[c] = row_off[cid];
    if (vert_off) b.voff[c] = vert_off[cid];
    if (MODE == 0) {
      const float tm = __ldg(time + cid);
      float al = 0.f;
      if (isfinite(tm)) {
        const float u = __fmul_rn(tm, rate);
        al = u - floorf(u);
      } else {
        atomicOr(status, 1);
      }
      b.alpha[c] = al;
      if (layers.w) {
        for (int i = 0; i < 4; ++i) b.lw[c][i] = __ldg(layers.w + 4 * (size_t)cid + i);
        b.law[c] = layers.add ? __ldg(layers.add + cid) : 0.f;
      } else {
        b.blend[c] = __ldg(blend_w + cid);
      }
    }
  }
  if (lane == 0) {
    const int n = types[wi.type].n, nseg = types[wi.type].nseg;
    b.item = it;
    b.C = wi.count;
    b.k0 = wi.k0;
    b.type = wi.type;
    b.divC.init(wi.count);
    b.divS.init(nseg);
    b.divN.init(n);
    int g = (kComputeThreads + n - 1) / n;
    g = g < 1 ? 1 : (g > wi.count ? wi.count : g);
    b.cpt = (wi.count + g - 1) / g;
    b.cgroups = (wi.count + b.cpt - 1) / b.cpt;
  }
  cp_async_wait_all();  // the type record's copies
  __syncwarp();
}

// Per-joint input arrays that the compute warps read from global memory,
// row r of array i at base[i] + floats[i] * r (unused slots nullptr).
// perm: a view's rows are a permutation of the character's n rows (the
// adjoint's depth-first views), so the contiguous range covers them.
struct RowPrefetch {
  const float *base[4];
  int floats[4];
  int perm;
};

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

// One warp: hint L2 to fetch the rows of item b's characters (rows off..off+n
// of each, or off + gather[j] for a view) of every array of pf.  A prefetch
// returns nothing to the kernel, so it may run ahead of the wait for a
// preceding grid: L2 is the point of coherence for that grid's writes.
__device__ __forceinline__ void prefetch_rows(const ItemBuf &b, const RowPrefetch &pf) {
  const int lane = threadIdx.x & 31;
  const int n = b.T.n;
  const int32_t *gat = b.T.gather;
  for (int c = 0; c < b.C; ++c) {
    const long long off = b.off[c];
    if (!gat || pf.perm) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!pf.base[i]) continue;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(pf.base[i] + pf.floats[i] * off);
        const uintptr_t hi = lo + (uintptr_t)(4 * pf.floats[i]) * (uintptr_t)n;
        for (uintptr_t p = (lo & ~(uintptr_t)127) + 128 * (uintptr_t)lane; p < hi; p += 32 * 128)
          prefetch_l2(reinterpret_cast<const void *>(p));
      }
    } else {
      // a view's rows: one hint per 128-byte line where the row starts it
      // (the previous joint's row from the lane below)
      long long carry = -1;
#pragma unroll 4
      for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        const long long r = j < n ? off + __ldg(gat + j) : -1;
        long long rp = __shfl_up_sync(0xffffffffu, r, 1);
        if (lane == 0) rp = carry;
        carry = __shfl_sync(0xffffffffu, r, 31);
        if (r < 0) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!pf.base[i]) continue;
          const long long bytes = 4LL * pf.floats[i];
          if (rp < 0 || ((r * bytes) >> 7) != ((rp * bytes) >> 7)) prefetch_l2(pf.base[i] + pf.floats[i] * r);
        }
      }
    }
  }
}

// Producer warp main loop: keep one item ahead of the compute warps, and
// (pf non-empty) warm L2 with the next item's rows while the current one
// runs.
template <int MODE>
__device__ __forceinline__ void producer_loop(ItemBuf *bufs, int *queue_head, int n_items, const WorkItem *items,
                                              const TypeDev *types, const int32_t *item_chars,
                                              const int64_t *row_off, const float *time, const float *blend_w,
                                              int *status, const int64_t *vert_off = nullptr,
                                              LayerIn layers = LayerIn{nullptr, nullptr},
                                              const RowPrefetch &pf = RowPrefetch{}) {
  int cur = 0;
  fetch_item<MODE>(bufs[0], queue_head, n_items, items, types, item_chars, row_off, time, blend_w, status,
                   vert_off, layers);
  __threadfence_block();
  handoff_sync();
  while (bufs[cur].item >= 0) {
    cur ^= 1;
    fetch_item<MODE>(bufs[cur], queue_head, n_items, items, types, item_chars, row_off, time, blend_w, status,
                     vert_off, layers);
    if (pf.base[0] && bufs[cur].item >= 0) prefetch_rows(bufs[cur], pf);
    __threadfence_block();
    handoff_sync();
  }
}

// Before the wait for a preceding grid: stage item blockIdx.x (the first
// wave of the queue holds items 0 .. gridDim.x - 1, in some order across the
// CTAs) into scratch buffer b and prefetch its rows.  Only for queues and
// tables that no preceding grid writes, and only when the CTAs get more than
// one item each: with one, the compute warps read the rows right after the
// wait anyway, and the extra staging measured slower (a persistent fwd+bwd
// launch of one 8-character item per CTA: 18.4 -> 22.8 us).
__device__ __forceinline__ void prefetch_first_wave(ItemBuf &b, int n_items, const WorkItem *items,
                                                    const TypeDev *types, const int32_t *item_chars,
                                                    const int64_t *row_off, const RowPrefetch &pf) {
  if (n_items <= (int)gridDim.x) return;
  const WorkItem wi = items[blockIdx.x];
  if (wi.count <= 0) return;
  stage_item<1>(b, (int)blockIdx.x, wi, types, item_chars, row_off, nullptr, nullptr, nullptr);
  prefetch_rows(b, pf);
}

// Dynamic shared memory of one work item:
//   P        [C][3n+1] float4   local -> running -> model/skin matrices
//   Y0, Y1   [C][nseg][3] float4  pass-2 buffers
//   ptr0/1   int16 [nseg] each    pass-2 jumping pointers (type-level)
//   seg_start int32 [nseg+1], seg_link int32 [nseg], jinfo uint16 [n]
//            the type's tables, staged once per item so the serial passes
//            read shared memory instead of waiting on global loads.
struct ItemLayout {
  float4 *P, *Y0, *Y1;
  int16_t *ptr0, *ptr1;
  int32_t *seg_start, *seg_link;
  uint16_t *jinfo;
  float4 *end;  // first float4 after the layout
};
__host__ __device__ inline size_t item_table_bytes(int n, int nseg) {
  return (4ull * nseg + 4ull * (2ull * nseg + 1) + 2ull * n + 15) / 16 * 16;
}
__device__ __forceinline__ ItemLayout item_layout(float4 *sm, int C, int n, int nseg) {
  ItemLayout L;
  L.P = sm;
  L.Y0 = L.P + C * (3 * n + 1);
  L.Y1 = L.Y0 + 3 * C * nseg;
  char *t = reinterpret_cast<char *>(L.Y1 + 3 * C * nseg);
  L.ptr0 = reinterpret_cast<int16_t *>(t);
  L.ptr1 = L.ptr0 + nseg;
  L.seg_start = reinterpret_cast<int32_t *>(t + 4 * nseg);
  L.seg_link = L.seg_start + nseg + 1;
  L.jinfo = reinterpret_cast<uint16_t *>(L.seg_link + nseg);
  L.end = reinterpret_cast<float4 *>(t + item_table_bytes(n, nseg));
  return L;
}
// Stage the type's segment tables (the parent structure of the scan) into
// the item's shared memory by cp.async: seg_start, seg_link and the 16-bit
// joint info in 4-byte words (an odd last entry by a plain load, so nothing
// is written past the table).  Issued at the start of pass 1a; every thread
// calls cp_async_wait_all before the barrier that precedes the tables' first
// use, so the copies overlap pass 1a's work.  ASYNC false: plain loads,
// the joint info converted here (the allocation-free entry's type record,
// which has no 16-bit tables).
template <int NT = kComputeThreads, bool ASYNC = true>
__device__ __forceinline__ void stage_tables(const ItemBuf &b, const ItemLayout &L, int tid) {
  const int n = b.T.n, nseg = b.T.nseg;
  if (!ASYNC) {
    for (int k = tid; k <= nseg; k += NT) L.seg_start[k] = __ldg(b.T.seg_start + k);
    for (int k = tid; k < nseg; k += NT) L.seg_link[k] = __ldg(b.T.seg_link + k);
    for (int j = tid; j < n; j += NT) {
      const uint32_t i = __ldg(b.T.jinfo + j);
      L.jinfo[j] = (uint16_t)((i & kJ16Seg) | ((i & kJStart) ? kJ16Start : 0u) | ((i & kJLink) ? kJ16Link : 0u));
    }
    return;
  }
  for (int k = tid; k <= nseg; k += NT) cp_async4(L.seg_start + k, b.T.seg_start + k);
  for (int k = tid; k < nseg; k += NT) cp_async4(L.seg_link + k, b.T.seg_link + k);
  if (b.T.jinfo16) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(b.T.jinfo16);
    uint32_t *dst = reinterpret_cast<uint32_t *>(L.jinfo);
    for (int k = tid; k < n / 2; k += NT) cp_async4(dst + k, src + k);
    if ((n & 1) && tid == 0) L.jinfo[n - 1] = __ldg(b.T.jinfo16 + n - 1);
  } else {
    for (int j = tid; j < n; j += NT) {
      const uint32_t i = __ldg(b.T.jinfo + j);
      L.jinfo[j] = (uint16_t)((i & kJ16Seg) | ((i & kJStart) ? kJ16Start : 0u) | ((i & kJLink) ? kJ16Link : 0u));
    }
  }
  cp_async_commit();
}

// Pass 1a from given local poses (q normalized here, t), optionally through a
// gather map (IK views).  Character-major so consecutive lanes read
// consecutive rows.
template <int NT = kComputeThreads>
__device__ __forceinline__ void pass1a_qt(const ItemBuf &b, float4 *P, int cs4, const float *q_all,
                                          const float *t_all, int tid) {
  const int n = b.T.n, CN = b.C * n;
  const int32_t *gat = b.T.gather;
  const float4 *q4 = reinterpret_cast<const float4 *>(q_all);
#pragma unroll 2
  for (int idx = tid; idx < CN; idx += NT) {
    const int c = (int)b.divN.div(idx), j = idx - c * n;
    const long long row = b.off[c] + (gat ? __ldg(gat + j) : j);
    const float4 q = normalize4(__ldg(q4 + row));
    const float *tp = t_all + 3 * row;
    sts_aff(P + c * cs4 + 3 * j, aff_from_qt(q, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2)));
  }
}

// Pass 1b: running products along each segment, in place.
template <int NT = kComputeThreads>
__device__ __forceinline__ void pass1b(const ItemBuf &b, const ItemLayout &Lt, float4 *P, int cs4, int tid) {
  const int C = b.C, NS = b.T.nseg * C;
  for (int idx = tid; idx < NS; idx += NT) {
    const int g = (int)b.divC.div(idx), c = idx - g * C;
    const int a0 = Lt.seg_start[g], a1 = Lt.seg_start[g + 1];
    float4 *Pc = P + c * cs4;
    Aff acc = lds_aff(Pc + 3 * a0);
    if (a0 + 1 >= a1) continue;
    Aff nxt = lds_aff(Pc + 3 * (a0 + 1));
    for (int j = a0 + 1; j < a1; ++j) {
      const Aff L = nxt;
      if (j + 1 < a1) nxt = lds_aff(Pc + 3 * (j + 1));
      acc = aff_mul(acc, L);
      sts_aff(Pc + 3 * j, acc);
    }
  }
}

// Pass 2 + its barriers.  Returns the buffer holding the final Y.  The
// jumping pointers depend only on the skeleton, so one copy per item lives
// in shared memory (ptr0/ptr1, double-buffered) next to the Y buffers.
template <int NT = kComputeThreads>
__device__ __forceinline__ float4 *pass2(const ItemBuf &b, const ItemLayout &Lt, float4 *P, int cs4, int tid) {
  const int nseg = b.T.nseg;
  const int CS = b.C * nseg;
  float4 *Y0 = Lt.Y0, *Y1 = Lt.Y1;
  int16_t *ptr0 = Lt.ptr0, *ptr1 = Lt.ptr1;
  for (int idx = tid; idx < CS; idx += NT) {
    const int c = (int)b.divS.div(idx), g = idx - c * nseg;
    const int lk = Lt.seg_link[g];
    const Aff y = lk < 0 ? aff_identity() : lds_aff(P + c * cs4 + 3 * lk);
    sts_aff(Y0 + 3 * idx, y);
    if (c == 0) ptr0[g] = (int16_t)(lk < 0 ? -1 : (int)(Lt.jinfo[lk] & kJ16Seg));
  }
  pass_sync<NT>();
  float4 *cur = Y0, *nxt = Y1;
  int16_t *pc = ptr0, *pn = ptr1;
  for (int r = 0; r < b.T.rounds; ++r) {
    for (int idx = tid; idx < CS; idx += NT) {
      const int c = (int)b.divS.div(idx), g = idx - c * nseg;
      const int p = pc[g];
      Aff y = lds_aff(cur + 3 * idx);
      if (p >= 0) y = aff_mul(lds_aff(cur + 3 * (c * nseg + p)), y);
      sts_aff(nxt + 3 * idx, y);
      if (c == 0) pn[g] = (int16_t)(p >= 0 ? pc[p] : -1);
    }
    pass_sync<NT>();
    float4 *tmp = cur;
    cur = nxt;
    nxt = tmp;
    int16_t *tp = pc;
    pc = pn;
    pn = tp;
  }
  return cur;
}

// End of a persistent launch: the last CTA to finish resets the work-queue
// counter (and the finish counter) so the next launch needs no memset.  By
// then every producer warp has taken its last ticket.
__device__ __forceinline__ void last_cta_reset(int *queue_head, int *done) {
  __threadfence();
  if (atomicAdd(done, 1) == (int)gridDim.x - 1) {
    *queue_head = 0;
    *done = 0;
    __threadfence();
  }
}

// Bytes of shared memory a work item of C characters needs.
__host__ __device__ inline size_t scan_item_bytes(int n, int nseg, int C) {
  return 16ull * ((size_t)C * (3 * (size_t)n + 1) + 6ull * C * nseg) + item_table_bytes(n, nseg);
}

// ---- the same scan on rigid transforms kept as (quaternion, translation)
// pairs.  The local poses are rigid (unit scale), so the pair is an exact
// representation: (qa, ta) o (qb, tb) = (qa qb, ta + R(qa) tb), 32 bytes per
// joint in shared memory instead of a 48-byte 3x4 matrix.
struct QT {
  float4 q;  // x y z w
  float4 t;  // x y z (w unused)
};
// Pairs are stored as two planes, q at base[j] and t at base[half + j], so
// lanes on consecutive j touch consecutive 16-byte slots.
__device__ __forceinline__ QT lds_qt(const float4 *base, int j, int half) { return QT{base[j], base[half + j]}; }
__device__ __forceinline__ void sts_qt(float4 *base, int j, int half, const QT &a) {
  base[j] = a.q;
  base[half + j] = a.t;
}
// R(q) v for a unit quaternion q: v + 2 w (u x v) + 2 u x (u x v), u = q.xyz.
__device__ __forceinline__ float3 qrot(const float4 q, const float3 v) {
  const float cx = 2.f * (q.y * v.z - q.z * v.y), cy = 2.f * (q.z * v.x - q.x * v.z),
              cz = 2.f * (q.x * v.y - q.y * v.x);
  return make_float3(fmaf(q.w, cx, v.x) + (q.y * cz - q.z * cy), fmaf(q.w, cy, v.y) + (q.z * cx - q.x * cz),
                     fmaf(q.w, cz, v.z) + (q.x * cy - q.y * cx));
}
__device__ __forceinline__ QT qt_mul(const QT &a, const QT &b) {
  const float3 r = qrot(a.q, make_float3(b.t.x, b.t.y, b.t.z));
  return QT{qmul(a.q, b.q), make_float4(a.t.x + r.x, a.t.y + r.y, a.t.z + r.z, 0.f)};
}
__device__ __forceinline__ QT qt_identity() {
  return QT{make_float4(0.f, 0.f, 0.f, 1.f), make_float4(0.f, 0.f, 0.f, 0.f)};
}

// Item layout: P [C][2n + 1] float4 (per character a q plane of n, a t plane
// of n, one pad), Y0 / Y1 [2][C * nseg] float4 (q plane, t plane), then the
// type's segment tables as in the matrix layout.
__device__ __forceinline__ ItemLayout item_layout_qt(float4 *sm, int C, int n, int nseg) {
  ItemLayout L;
  L.P = sm;
  L.Y0 = L.P + C * (2 * n + 1);
  L.Y1 = L.Y0 + 2 * C * nseg;
  char *t = reinterpret_cast<char *>(L.Y1 + 2 * C * nseg);
  L.ptr0 = reinterpret_cast<int16_t *>(t);
  L.ptr1 = L.ptr0 + nseg;
  L.seg_start = reinterpret_cast<int32_t *>(t + 4 * nseg);
  L.seg_link = L.seg_start + nseg + 1;
  L.jinfo = reinterpret_cast<uint16_t *>(L.seg_link + nseg);
  L.end = reinterpret_cast<float4 *>(t + item_table_bytes(n, nseg));
  return L;
}
// Local pose of joint j of character c in the frame with layered blending:
// every clip of the type is sampled at the character's key fraction (slerp /
// lerp between keys k0 and k0 + 1); rotations are blended by incremental
// slerp (q = q_0, W = w_0, then for each further clip W += w_i and
// q = slerp(q, q_i, w_i / W) while W > 0), translations by their weighted
// mean (clip 0's when every weight is 0); an additive layer sampled the same
// way multiplies on the right, q * slerp(1, q_a, a), and adds a t_a.
__device__ __forceinline__ QT sample_layers_at(const ItemBuf &b, int j, int c) {
  const int n = b.T.n, nk = b.T.n_keys, k0 = b.k0, k1 = (k0 + 1 == nk) ? 0 : k0 + 1, nc = b.T.n_clips;
  const float4 *add = b.T.add_keys;
  const float al = b.alpha[c];
  float4 q = make_float4(0.f, 0.f, 0.f, 1.f);
  float tx = 0.f, ty = 0.f, tz = 0.f, t0x = 0.f, t0y = 0.f, t0z = 0.f, W = 0.f;
  for (int i = 0; i < nc; ++i) {
    const float4 *A0 = b.T.keys + (((size_t)i * nk + k0) * n + j) * 2;
    const float4 *A1 = b.T.keys + (((size_t)i * nk + k1) * n + j) * 2;
    const float4 qa0 = __ldg(A0), ta0 = __ldg(A0 + 1), qa1 = __ldg(A1), ta1 = __ldg(A1 + 1);
    const float4 qi = slerp_pre(qa0, qa1, ta0.w, al);
    const float ix = fmaf(al, ta1.x - ta0.x, ta0.x), iy = fmaf(al, ta1.y - ta0.y, ta0.y),
                iz = fmaf(al, ta1.z - ta0.z, ta0.z);
    const float w = b.lw[c][i];
    if (i == 0) {
      q = qi;
      t0x = ix;
      t0y = iy;
      t0z = iz;
    } else if (W + w > 0.f) {
      q = slerp_unit(q, qi, w / (W + w));
    }
    W += w;
    tx = fmaf(w, ix, tx);
    ty = fmaf(w, iy, ty);
    tz = fmaf(w, iz, tz);
  }
  if (W > 0.f) {
    const float inv = 1.f / W;
    tx *= inv;
    ty *= inv;
    tz *= inv;
  } else {
    tx = t0x;
    ty = t0y;
    tz = t0z;
  }
  if (add) {
    const float aw = b.law[c];
    const float4 *A0 = add + ((size_t)k0 * n + j) * 2, *A1 = add + ((size_t)k1 * n + j) * 2;
    const float4 qa0 = __ldg(A0), ta0 = __ldg(A0 + 1), qa1 = __ldg(A1), ta1 = __ldg(A1 + 1);
    const float4 qa = slerp_pre(qa0, qa1, ta0.w, al);
    q = qmul(q, slerp_unit(make_float4(0.f, 0.f, 0.f, 1.f), qa, aw));
    tx = fmaf(aw, fmaf(al, ta1.x - ta0.x, ta0.x), tx);
    ty = fmaf(aw, fmaf(al, ta1.y - ta0.y, ta0.y), ty);
    tz = fmaf(aw, fmaf(al, ta1.z - ta0.z, ta0.z), tz);
  }
  return QT{q, make_float4(tx, ty, tz, 0.f)};
}

__host__ __device__ inline size_t qt_item_bytes(int n, int nseg, int C) {
  return 16ull * ((size_t)C * (2 * (size_t)n + 1) + 4ull * C * nseg) + item_table_bytes(n, nseg);
}

// Pass 1b on (q, t) pairs: running products along each segment, in place
// (P's character stride cs2 in float4).
template <int NT = kComputeThreads>
__device__ __forceinline__ void pass1b_qt(const ItemBuf &b, const ItemLayout &Lt, float4 *P, int cs2, int tid) {
  const int C = b.C, NS = b.T.nseg * C;
  for (int idx = tid; idx < NS; idx += NT) {
    const int g = (int)b.divC.div(idx), c = idx - g * C;
    const int a0 = Lt.seg_start[g], a1 = Lt.seg_start[g + 1], n = b.T.n;
    float4 *Pc = P + c * cs2;
    QT acc = lds_qt(Pc, a0, n);
    if (a0 + 1 >= a1) continue;
    QT nxt = lds_qt(Pc, a0 + 1, n);
    for (int j = a0 + 1; j < a1; ++j) {
      const QT L = nxt;
      if (j + 1 < a1) nxt = lds_qt(Pc, j + 1, n);
      acc = qt_mul(acc, L);
      sts_qt(Pc, j, n, acc);
    }
  }
}

// Pass 2 on (q, t) pairs + its barriers; returns the buffer holding Y.
template <int NT = kComputeThreads>
__device__ __forceinline__ float4 *pass2_qt(const ItemBuf &b, const ItemLayout &Lt, const float4 *P, int cs2,
                                            int tid) {
  const int nseg = b.T.nseg, n = b.T.n;
  const int CS = b.C * nseg;
  float4 *Y0 = Lt.Y0, *Y1 = Lt.Y1;
  int16_t *ptr0 = Lt.ptr0, *ptr1 = Lt.ptr1;
  for (int idx = tid; idx < CS; idx += NT) {
    const int c = (int)b.divS.div(idx), g = idx - c * nseg;
    const int lk = Lt.seg_link[g];
    sts_qt(Y0, idx, CS, lk < 0 ? qt_identity() : lds_qt(P + c * cs2, lk, n));
    if (c == 0) ptr0[g] = (int16_t)(lk < 0 ? -1 : (int)(Lt.jinfo[lk] & kJ16Seg));
  }
  pass_sync<NT>();
  float4 *cur = Y0, *nxt = Y1;
  int16_t *pc = ptr0, *pn = ptr1;
  for (int r = 0; r < b.T.rounds; ++r) {
    for (int idx = tid; idx < CS; idx += NT) {
      const int c = (int)b.divS.div(idx), g = idx - c * nseg;
      const int p = pc[g];
      QT y = lds_qt(cur, idx, CS);
      if (p >= 0) y = qt_mul(lds_qt(cur, c * nseg + p, CS), y);
      sts_qt(nxt, idx, CS, y);
      if (c == 0) pn[g] = (int16_t)(p >= 0 ? pc[p] : -1);
    }
    pass_sync<NT>();
    float4 *tmp = cur;
    cur = nxt;
    nxt = tmp;
    int16_t *tp = pc;
    pc = pn;
    pn = tp;
  }
  return cur;
}

}  // namespace anim
