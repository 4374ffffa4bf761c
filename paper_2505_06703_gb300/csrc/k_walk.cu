// Chain-walk frame kernel: Simulation -> Hierarchy-Scan -> Bind MeshPose
// (Sec. 1 steps 1-3, Eq. 1) walked directly in skin space, for skeleton
// types whose natural chains can be list-scheduled on a few lanes with few
// idle steps (long pure chains stay on the segmented kernel).
//
// Skin-space walk.  With rigid inverse binds B, the skin matrix of joint j
// satisfies S_j = M_j B_j = S_p (B_p^-1 L_j B_j) = S_p L'_j (p the parent; a
// root has B_p = I).  Because slerp commutes with multiplying both of its
// ends by unit quaternions on the left and on the right, and lerp with any
// affine map, L'_j is sampled exactly like L_j from key records whose
// rotations are q' = conj(q_Bp) q q_Bj and whose translations are
// R_Bp^T (t - t_Bp); its translation then needs R' u_j with u_j = R_Bj^T t_Bj
// (minus the joint's rest position).  The host builds these records once per
// clip upload, so per joint and character the kernel samples two key pairs,
// blends them, forms L' = [R(q') | t' + R(q') u] and makes ONE 3x4 product,
// which is the skin matrix it stores -- no separate bind product, no second
// pass over the joints, no block barrier.
//
// One CTA is one warp and one work item: C = 32 / P characters of one type
// that share the key index k0; lane = (character, schedule slot).  The
// type's static schedule (host-built) names the joint each slot composes at
// each step.  A lane keeps S in registers along its natural chain; branch
// points leave S in a shared-memory slot for the lane that starts a child
// chain at a later step.
//
// Staging.  The steps are processed in chunks of K = 32 / P (at most 4)
// steps.  A chunk's key records (both clips), u vectors and schedule entries
// are contiguous in schedule order in global memory; lane 0 copies them into
// a ring of shared-memory buffers with cp.async.bulk (TMA, 1-D), each
// completing on its own mbarrier, several chunks ahead of the compute.
// Within a chunk each lane first forms its K local transforms (independent
// work, so the latency of the trigonometry overlaps), then walks the K steps.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "smem_limit.h"

namespace anim {

namespace {

constexpr int kWaitLimit = 1 << 22;  // mbarrier polls before a chunk counts as lost

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i >= 16) __nanosleep(64);
  }
  return false;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Chunk buffer layout (bytes): records of clip 0 [K][4][P] float4, records of
// clip 1, u [K][P] float4, schedule entries [K][P] uint32; K P <= 32.
constexpr uint32_t kRecBytes = 32 * 4 * 16;
constexpr uint32_t kUOff = 2 * kRecBytes;
constexpr uint32_t kTabOff = kUOff + 32 * 16;
constexpr uint32_t kChunkBytes = kTabOff + 32 * 4;
static_assert(kChunkBytes % 128 == 0, "chunk buffers stay 128-byte aligned");
// Chunk buffers per CTA: up to kStages chunks are in flight, so the copy
// latency (about a microsecond from L2 under load) overlaps several chunks'
// compute.
constexpr int kStages = 3;

// Slerp between keys from a record: cos(a theta) q0 + sin(a theta) q_perp
// (q0, q_perp orthonormal), translation t0 + a (t1 - t0).  r points at the
// slot's first field; fields are P float4 apart.
__device__ __forceinline__ void rec_sample(const float4 *r, int P, float al, float4 &q, float3 &t) {
  const float4 q0 = r[0], qp = r[P], t0 = r[2 * P], dt = r[3 * P];
  float s, c;
  __sincosf(al * t0.w, &s, &c);
  q = make_float4(fmaf(c, q0.x, s * qp.x), fmaf(c, q0.y, s * qp.y), fmaf(c, q0.z, s * qp.z), fmaf(c, q0.w, s * qp.w));
  t = make_float3(fmaf(al, dt.x, t0.x), fmaf(al, dt.y, t0.y), fmaf(al, dt.z, t0.z));
}

// L' = [R(q) | t + R(q) u] for a unit quaternion q.
__device__ __forceinline__ Aff local_skin(const float4 q, const float3 t, const float4 u) {
  Aff L = aff_from_qt(q, 0.f, 0.f, 0.f);
  L.r0.w = fmaf(L.r0.x, u.x, fmaf(L.r0.y, u.y, fmaf(L.r0.z, u.z, t.x)));
  L.r1.w = fmaf(L.r1.x, u.x, fmaf(L.r1.y, u.y, fmaf(L.r1.z, u.z, t.y)));
  L.r2.w = fmaf(L.r2.x, u.x, fmaf(L.r2.y, u.y, fmaf(L.r2.z, u.z, t.z)));
  return L;
}

struct ItemCtx {
  int P, logP, S, nk, k0, slot, c, count;
  bool act, two;
  float al, w;
  float4 *out;     // the lane's character's skin rows
  float4 *bslots;  // the lane's character's branch slots [nbs][3]
  const float4 *ra, *rb, *u;
  const uint32_t *tab;
};

// Issue chunk `ch` (steps ch K .. min(S, ch K + K) - 1) into buffer `buf`:
// the key records and u of its steps, and a whole chunk of schedule entries
// (the table is padded with idle entries to whole chunks).
template <int K>
__device__ __forceinline__ void issue_chunk(const ItemCtx &x, int ch, unsigned char *stage, uint64_t *bar) {
  const int kc = min(K, x.S - ch * K);
  const uint32_t rec = (uint32_t)(kc * 4 * x.P * 16), ub = (uint32_t)(kc * x.P * 16), tb = (uint32_t)(K * x.P * 4);
  const size_t rstep = (size_t)ch * K * 4 * x.P, ustep = (size_t)ch * K * x.P;
  // No proxy fence: the buffer is only read (ld.shared) by the generic proxy,
  // and those reads completed before the __syncwarp that precedes this
  // call.  (A fence here would also wait for the warp's outstanding global
  // stores, one round trip per chunk.)
  mbar_expect_tx(bar, (x.two ? 2u : 1u) * rec + ub + tb);
  bulk_g2s(stage, x.ra + rstep, rec, bar);
  if (x.two) bulk_g2s(stage + kRecBytes, x.rb + rstep, rec, bar);
  bulk_g2s(stage + kUOff, x.u + ustep, ub, bar);
  bulk_g2s(stage + kTabOff, x.tab + ustep, tb, bar);
}

// One staged chunk of the walk.  S carries the lane's running skin matrix.
// The local transforms of all K steps are formed first, without branches
// (steps past the end of a short last chunk compute unused values from
// whatever the buffer holds), so their latencies overlap; the walk itself is
// then one 3x4 product per step.
template <int K>
__device__ __forceinline__ void walk_chunk(const ItemCtx &x, const unsigned char *stage, Aff &S) {
  const float4 *ra = reinterpret_cast<const float4 *>(stage) + x.slot;
  const float4 *rb = reinterpret_cast<const float4 *>(stage + kRecBytes) + x.slot;
  const float4 *us = reinterpret_cast<const float4 *>(stage + kUOff) + x.slot;
  const uint32_t *ts = reinterpret_cast<const uint32_t *>(stage + kTabOff) + x.slot;
  const int P = x.P;
  Aff L[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float4 q;
    float3 t;
    rec_sample(ra + k * 4 * P, P, x.al, q, t);
    if (x.two) {
      float4 qb;
      float3 tb;
      rec_sample(rb + k * 4 * P, P, x.al, qb, tb);
      q = blend_unit(q, qb, x.w);
      t = make_float3(fmaf(x.w, tb.x - t.x, t.x), fmaf(x.w, tb.y - t.y, t.y), fmaf(x.w, tb.z - t.z, t.z));
    }
    L[k] = local_skin(q, t, us[k * P]);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t e = ts[k * P];  // idle entries past the schedule's end
    const bool valid = x.act && e != kWInvalid;
    Aff Sp = S;
    if (valid && (e & kWStart)) {
      const uint32_t ls = (e >> kWLoadShift) & 0xFFu;
      Sp = ls == kWRootSlot ? aff_identity() : lds_aff(x.bslots + 3 * ls);
    }
    const Aff Sn = aff_mul(Sp, L[k]);
    if (valid) {
      S = Sn;
      if (e & kWStore) sts_aff(x.bslots + 3 * ((e >> kWStoreShift) & 0xFFu), Sn);
      stg_aff(x.out + 3 * (e & kWJoint), Sn);
    }
    __syncwarp();  // branch slots written at this step are read at later steps
  }
}

// The whole item: the chunk sequence, up to kStages chunks staged ahead of
// the compute.  Returns false if a chunk never arrived (its wait ran out).
template <int K>
__device__ bool walk_item(const ItemCtx &x, unsigned char *stage, uint64_t *bars, uint32_t &parity,
                          uint32_t &inflight) {
  const int lane = threadIdx.x;
  const int nch = (x.S + K - 1) / K, nq = nch;
  for (int b = 0; b < kStages && b < nq; ++b) {
    if (lane == 0) issue_chunk<K>(x, b, stage + b * kChunkBytes, &bars[b]);
    inflight |= 1u << b;  // buffers with a copy issued and not yet waited for
  }
  Aff S = aff_identity();
  for (int q = 0; q < nq; ++q) {
    const int buf = q % kStages;
    if (!mbar_wait(&bars[buf], (parity >> buf) & 1u)) return false;
    parity ^= 1u << buf;
    inflight &= ~(1u << buf);
    const unsigned char *st = stage + buf * kChunkBytes;
    walk_chunk<K>(x, st, S);
    __syncwarp();
    if (q + kStages < nq) {
      if (lane == 0) issue_chunk<K>(x, q + kStages, stage + buf * kChunkBytes, &bars[buf]);
      inflight |= 1u << buf;
    }
  }
  return true;
}

__global__ void __launch_bounds__(32, 12) k_walk(const WalkArgs a) {
  extern __shared__ __align__(128) unsigned char wsm[];
  __shared__ __align__(8) uint64_t bars[kStages];
  const int lane = threadIdx.x;
  // launched with programmatic stream serialization after the work-queue
  // kernel: set up, then wait for it before reading the item
  asm volatile("griddepcontrol.launch_dependents;");
  if (lane == 0) {
    for (int b = 0; b < kStages; ++b) mbar_init(&bars[b]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const WorkItem wi = a.items[blockIdx.x];
  if (wi.count <= 0) return;
  const TypeDev &T = a.types[wi.type];
  ItemCtx x;
  x.P = T.wk_P;
  x.logP = T.wk_logP;
  x.S = T.wk_S;
  x.nk = T.n_keys;
  x.k0 = wi.k0;
  x.two = T.n_clips >= 2;
  x.c = lane >> x.logP;
  x.slot = lane & (x.P - 1);
  x.count = wi.count;
  x.act = x.c < wi.count;
  x.al = 0.f;
  x.w = 0.f;
  x.out = reinterpret_cast<float4 *>(a.skin);
  if (x.act) {
    const int cid = __ldg(a.item_chars + wi.start + x.c);
    x.out = reinterpret_cast<float4 *>(a.skin) + a.row_off[cid] * 3;
    const float tm = __ldg(a.time + cid);
    if (isfinite(tm)) {
      const float u = __fmul_rn(tm, T.rate);
      x.al = u - floorf(u);
    } else {
      atomicOr(a.status, kStatusNonfiniteTime);
    }
    x.w = x.two ? __ldg(a.blend_w + cid) : 0.f;
  }
  const size_t clip_stride = (size_t)x.nk * x.S * 4 * x.P;
  x.ra = T.wk_keys + (size_t)x.k0 * x.S * 4 * x.P;
  x.rb = x.ra + clip_stride;
  x.u = T.wk_u;
  x.tab = T.wk_tab;
  unsigned char *stage = wsm;
  x.bslots = reinterpret_cast<float4 *>(wsm + kStages * kChunkBytes) + (size_t)x.c * a.nbs_max * 3;
  uint32_t parity = 0, inflight = 0;
  bool ok;
  switch (T.wk_K) {
    case 1: ok = walk_item<1>(x, stage, bars, parity, inflight); break;
    case 2: ok = walk_item<2>(x, stage, bars, parity, inflight); break;
    default: ok = walk_item<4>(x, stage, bars, parity, inflight); break;
  }
  if (!ok) {
    // a staged chunk did not complete in time: report it, and before the CTA
    // (and its shared memory) goes away wait once more, bounded, for the
    // copies still in flight
    if (lane == 0) atomicOr(a.status, kStatusTimeout);
    for (int b = 0; b < kStages; ++b)
      if (inflight & (1u << b)) mbar_wait(&bars[b], (parity >> b) & 1u);
  }
}

}  // namespace

size_t walk_smem_bytes(int chars_per_item, int nbs) {
  return (size_t)kStages * kChunkBytes + 48ull * (size_t)chars_per_item * (size_t)nbs;
}

int walk_blocks_per_sm(size_t smem) {
  static SmemLimit lim;
  if (ensure_smem_limit((const void *)k_walk, lim, smem, 48 * 1024) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk, 32, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_walk(const WalkArgs &a, size_t smem, cudaStream_t st) {
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k_walk, lim, smem, 48 * 1024);
  if (e != cudaSuccess) return e;
  // programmatic stream serialization: the CTAs become resident and set up
  // while the work-queue kernel runs, and wait for it in griddepcontrol.wait
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)a.n_items);
  lc.blockDim = dim3(32u);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_walk, a);
}

}  // namespace anim
