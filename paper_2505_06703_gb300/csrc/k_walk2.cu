// Warp-specialized chain walk (the frame, Sec. 1 steps 1-3, Eq. 1, in skin
// space as in k_walk.cu): the same static lane schedule and bind-folded key
// records, with the work of one item split over three warps so that the
// sampling runs on more warps per SM than the walk's lanes alone provide and
// the skin matrices leave as lane-contiguous stores:
//   warps 1 and 2 (samplers)  wait for a chunk of key records staged by
//       cp.async.bulk, sample the local rotation q' and translation t' of
//       half of its steps each into the chunk's row buffer, and write the
//       previous chunk's skin matrices out: 16-byte parts of the chunk's rows
//       enumerated lane by lane, so consecutive lanes store consecutive parts
//       of one joint run (a run is a lane's chain over the chunk's steps);
//   warp 0 (walker)  takes the chunk's local transforms
//       L' = (R(q'), t' + R(q') u), composes S = S_parent L' along its chains
//       (branch points through shared memory), overwrites each transform in
//       place with its rows, and refills the record stages.
// Hand-offs are mbarriers: records staged (bulk-copy bytes), row buffer
// sampled / composed / written out.  Every wait is bounded; a wait that runs
// out sets status bit 4 and the warp stops (the others then run out too);
// the walker, which issues the bulk copies, first waits once more, bounded,
// for those in flight.
#include <cuda_runtime.h>

#include <algorithm>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "smem_limit.h"

namespace anim {

namespace {

constexpr int kW2Threads = 96;  // walker + 2 samplers
constexpr int kW2Wait = 1 << 22;               // probes per wait at most
constexpr uint64_t kW2WaitNs = 1000000000ull;  // and one second at most

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(bar)) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}
// One bounded-time probe of the phase of `parity` (the hardware suspends
// the thread until the phase completes or a time limit passes).
__device__ __forceinline__ bool mb_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(s_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of `parity` to complete (parity 1 before the
// first phase completes: a buffer that starts empty).
__device__ __forceinline__ bool mb_wait(uint64_t *bar, uint32_t parity) {
  if (mb_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (int i = 0; i < kW2Wait; ++i) {
    if (mb_try(bar, parity)) return true;
    if (global_ns() - t0 > kW2WaitNs) break;
  }
  return false;
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(s_addr(bar))
               : "memory");
}
// Slerp between keys from a record (fields P float4 apart): cos(a theta) q0
// + sin(a theta) q_perp, translation t0 + a (t1 - t0).
__device__ __forceinline__ void rec_sample_w2(const float4 *r, int P, float al, float4 &q, float3 &t) {
  rec_eval(r[0], r[P], r[2 * P], r[3 * P], al, q, t);
}
// Shared memory of one CTA (dynamic, 128-byte aligned parts):
//   rec[2]   staged key records, u and schedule entries of a chunk, the
//            layout of k_walk's chunk buffer (clip 0 records [K][4][P],
//            clip 1 records, u [K][P], entries [K][P])
//   x[2]     the chunk's row buffer, kXStride(K) float4 per lane (an odd
//            stride: lane-indexed accesses are free of bank conflicts): at
//            3k, 3k+1 the samplers' transform of step k (q', then t' with
//            the lane's schedule entry in the bits of w; kWInvalid: none),
//            which the walker overwrites with the rows r0, r1, r2 of S at
//            3k .. 3k+2; at 3K the joints of the K steps (kWInvalid: none)
//   slots    branch points [C][nbs][3] float4
constexpr uint32_t kRecBytes = 32 * 4 * 16;
constexpr uint32_t kUOff = 2 * kRecBytes;
constexpr uint32_t kTabOff = kUOff + 32 * 16;
constexpr uint32_t kRecBuf = kTabOff + 32 * 4;  // 4,736
constexpr uint32_t kXBuf = 32 * 13 * 16;        // 6,656: the K = 4 stride
constexpr uint32_t kXOff = 2 * kRecBuf;
constexpr uint32_t kSlotOff = kXOff + 2 * kXBuf;
static_assert(kRecBuf % 128 == 0 && kXBuf % 128 == 0, "128-byte aligned parts");
template <int K>
constexpr int kXStride = K == 1 ? 5 : 3 * K + 1;  // 5, 7, 13
static_assert(32 * kXStride<4> * 16 <= (int)kXBuf, "row buffer");

// Arrival counts: rec_full 1 (+ the copies' bytes), x_full 64 (sampler
// lanes), x_rows 32 (walker lanes), x_empty 64 (sampler lanes, after their
// part of the write-out).
struct Bars {
  uint64_t rec_full[2];
  uint64_t x_full[2], x_rows[2], x_empty[2];
};

struct W2Item {
  int P, logP, S, K, nch, count;
  bool two;
  const float4 *ra, *rb, *u;
  const uint32_t *tab;
};

// Chunk ch (steps ch K .. min(S, ch K + K) - 1) into a record stage: its key
// records and u, and a whole chunk of schedule entries (the table is padded
// with idle entries to whole chunks).  One thread.
template <int K>
__device__ __forceinline__ void w2_issue(const W2Item &it, int ch, unsigned char *stage, uint64_t *bar) {
  const int kc = min(K, it.S - ch * K);
  const uint32_t rec = (uint32_t)(kc * 4 * it.P * 16), ub = (uint32_t)(kc * it.P * 16),
                 tb = (uint32_t)(K * it.P * 4);
  const size_t rstep = (size_t)ch * K * 4 * it.P, ustep = (size_t)ch * K * it.P;
  mb_expect_tx(bar, (it.two ? 2u : 1u) * rec + ub + tb);
  bulk_copy(stage, it.ra + rstep, rec, bar);
  if (it.two) bulk_copy(stage + kRecBytes, it.rb + rstep, rec, bar);
  bulk_copy(stage + kUOff, it.u + ustep, ub, bar);
  bulk_copy(stage + kTabOff, it.tab + ustep, tb, bar);
}

// The write-out of a composed chunk by the two samplers: element
// e = 32 sw + lane + 64 m (m < kParts) is part r = 3 k + f of lane src's
// rows; consecutive lanes store consecutive parts of one lane's joint run.
// part[m] packs src | r << 5 | k << 9 (kNoPart: past the chunk's 96 K
// parts), the same in every chunk.
template <int K>
constexpr int kParts = (96 * K + 63) / 64;
constexpr uint32_t kNoPart = 0xFFFFFFFFu;
template <int K>
__device__ __forceinline__ void w2_parts(int sw, uint32_t (&part)[kParts<K>]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < kParts<K>; ++m) {
    const int e = 32 * sw + lane + 64 * m;
    const int src = e / (3 * K), r = e - src * (3 * K);
    part[m] = e < 96 * K ? (uint32_t)(src | r << 5 | (r / 3) << 9) : kNoPart;
  }
}
template <int K>
__device__ __forceinline__ void w2_write_out(const float4 *xb, const uint32_t (&part)[kParts<K>], float4 *const *outs,
                                             int logP) {
  constexpr int X = kXStride<K>;
  const uint32_t *xj = reinterpret_cast<const uint32_t *>(xb);
#pragma unroll
  for (int m = 0; m < kParts<K>; ++m) {
    const uint32_t d = part[m];
    if (d == kNoPart) continue;
    const int src = d & 31, r = (d >> 5) & 15, k = (d >> 9) & 3;
    const uint32_t j = xj[(src * X + 3 * K) * 4 + k];
    if (j != kWInvalid) outs[src >> logP][3 * j + (r - 3 * k)] = xb[src * X + r];
  }
}

// Sampler warp sw (0 or 1): steps k = sw, sw + 2 of every chunk into the row
// buffer, and its part of the write-out of the chunk before.  al, w: the
// lane's character's key fraction and blend weight.
template <int K>
__device__ bool w2_sampler(const W2Item &it, unsigned char *sm, Bars &B, float4 *const *outs, int sw, float al,
                           float w) {
  constexpr int X = kXStride<K>;
  const int lane = threadIdx.x & 31, P = it.P, slot = lane & (P - 1);
  const bool act = (lane >> it.logP) < it.count;
  uint32_t rpar = 0, xe = 3u, xr = 0;
  uint32_t part[kParts<K>];
  w2_parts<K>(sw, part);
  for (int q = 0; q <= it.nch; ++q) {
    if (q < it.nch) {
      const int s = q & 1;
      if (!mb_wait(&B.rec_full[s], (rpar >> s) & 1u)) return false;
      rpar ^= 1u << s;
      if (!mb_wait(&B.x_empty[s], (xe >> s) & 1u)) return false;
      xe ^= 1u << s;
      const unsigned char *rec = sm + s * kRecBuf;
      const float4 *ra = reinterpret_cast<const float4 *>(rec) + slot;
      const float4 *rb = reinterpret_cast<const float4 *>(rec + kRecBytes) + slot;
      const uint32_t *ts = reinterpret_cast<const uint32_t *>(rec + kTabOff) + slot;
      float4 *xb = reinterpret_cast<float4 *>(sm + kXOff + s * kXBuf) + lane * X;
#pragma unroll
      for (int kk = 0; kk < (K + 1) / 2; ++kk) {
        const int k = 2 * kk + sw;  // a runtime step index: no predicated copy of the other sampler's steps
        if (k >= K) break;
        float4 q4;
        float3 t;
        rec_sample_w2(ra + k * 4 * P, P, al, q4, t);
        if (it.two) {
          float4 qb;
          float3 tb;
          rec_sample_w2(rb + k * 4 * P, P, al, qb, tb);
          q4 = blend_unit(q4, qb, w);
          t = make_float3(fmaf(w, tb.x - t.x, t.x), fmaf(w, tb.y - t.y, t.y), fmaf(w, tb.z - t.z, t.z));
        }
        const uint32_t e = act ? ts[k * P] : kWInvalid;
        xb[3 * k] = q4;
        xb[3 * k + 1] = make_float4(t.x, t.y, t.z, __uint_as_float(e));
      }
      mb_arrive(&B.x_full[s]);  // also: done with the record stage
    }
    if (q >= 1) {  // write-out of chunk q - 1
      const int o = (q - 1) & 1;
      if (!mb_wait(&B.x_rows[o], (xr >> o) & 1u)) return false;
      xr ^= 1u << o;
      w2_write_out<K>(reinterpret_cast<const float4 *>(sm + kXOff + o * kXBuf), part, outs, it.logP);
      mb_arrive(&B.x_empty[o]);
    }
  }
  return true;
}

// The walker warp: compose each chunk's transforms along the chains (the
// local translation completed to t + R(q') u with the record stage's u) and
// leave the rows in place for the samplers' write-out.  Its lane 0 keeps the
// record stages filled two chunks ahead: a stage is refilled once the
// samplers have sampled it and the walker has read its u.
template <int K>
__device__ bool w2_walker(const W2Item &it, unsigned char *sm, Bars &B, float4 *bslots) {
  constexpr int X = kXStride<K>;
  const int lane = threadIdx.x & 31, slot = lane & (it.P - 1);
  Aff S = aff_identity();
  uint32_t xf = 0, rpar = 0;
  for (int q = 0; q < it.nch; ++q) {
    const int s = q & 1;
    bool ok = mb_wait(&B.x_full[s], (xf >> s) & 1u) && mb_wait(&B.rec_full[s], (rpar >> s) & 1u);
    if (!ok) {  // drain the copies in flight (chunks q and q + 1), bounded
      for (int c = q; c < q + 2 && c < it.nch; ++c) mb_wait(&B.rec_full[c & 1], (c >> 1) & 1u);
      return false;
    }
    xf ^= 1u << s;
    rpar ^= 1u << s;
    const float4 *us = reinterpret_cast<const float4 *>(sm + s * kRecBuf + kUOff) + slot;
    float3 u[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 v = us[k * it.P];
      u[k] = make_float3(v.x, v.y, v.z);
    }
    __syncwarp();  // every lane's reads of the stage before its refill
    if (lane == 0 && q + 2 < it.nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      w2_issue<K>(it, q + 2, sm + s * kRecBuf, &B.rec_full[s]);
    }
    float4 *xb = reinterpret_cast<float4 *>(sm + kXOff + s * kXBuf) + lane * X;
    uint32_t jk[4] = {kWInvalid, kWInvalid, kWInvalid, kWInvalid};
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 q4 = xb[3 * k], tt = xb[3 * k + 1];
      const uint32_t e = __float_as_uint(tt.w);
      const bool valid = e != kWInvalid;
      Aff L = aff_from_qt(q4, tt.x, tt.y, tt.z);
      L.r0.w = fmaf(L.r0.x, u[k].x, fmaf(L.r0.y, u[k].y, fmaf(L.r0.z, u[k].z, L.r0.w)));
      L.r1.w = fmaf(L.r1.x, u[k].x, fmaf(L.r1.y, u[k].y, fmaf(L.r1.z, u[k].z, L.r1.w)));
      L.r2.w = fmaf(L.r2.x, u[k].x, fmaf(L.r2.y, u[k].y, fmaf(L.r2.z, u[k].z, L.r2.w)));
      Aff Sp = S;
      if (valid && (e & kWStart)) {
        const uint32_t ls = (e >> kWLoadShift) & 0xFFu;
        Sp = ls == kWRootSlot ? aff_identity() : lds_aff(bslots + 3 * ls);
      }
      const Aff Sn = aff_mul(Sp, L);
      if (valid) {
        S = Sn;
        jk[k] = e & kWJoint;
        if (e & kWStore) sts_aff(bslots + 3 * ((e >> kWStoreShift) & 0xFFu), Sn);
      }
      xb[3 * k] = Sn.r0;
      xb[3 * k + 1] = Sn.r1;
      xb[3 * k + 2] = Sn.r2;
      __syncwarp();  // branch slots written at this step are read at later steps
    }
    xb[3 * K] = make_float4(__uint_as_float(jk[0]), __uint_as_float(jk[1]), __uint_as_float(jk[2]),
                            __uint_as_float(jk[3]));
    mb_arrive(&B.x_rows[s]);
  }
  return true;
}

__global__ void __launch_bounds__(kW2Threads, 8) k_walk2(const WalkArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) Bars B;
  __shared__ float4 *outs[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // launched with programmatic stream serialization after the work-queue
  // kernel: set up, then wait for it before reading the item (or, after
  // the segmented frame kernel, read at once and wait at the end:
  // WalkArgs::pred_waited).  Queue entries and inputs are loaded from L2
  // (.cg), never from a line an earlier frame left in L1.
  asm volatile("griddepcontrol.launch_dependents;");
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mb_init(&B.rec_full[i], 1);
      mb_init(&B.x_full[i], 64);
      mb_init(&B.x_rows[i], 32);
      mb_init(&B.x_empty[i], 64);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (!a.pred_waited) asm volatile("griddepcontrol.wait;" ::: "memory");
  WorkItem wi;
  {
    const int4 v = __ldcg(reinterpret_cast<const int4 *>(a.items) + blockIdx.x);
    wi.start = v.x;
    wi.count = v.y;
    wi.type = v.z;
    wi.k0 = v.w;
  }
  if (wi.count <= 0) {
    if (a.pred_waited && tid == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
    return;
  }
  const TypeDev &T = a.types[wi.type];
  W2Item it;
  it.P = T.wk_P;
  it.logP = T.wk_logP;
  it.S = T.wk_S;
  it.K = T.wk_K;
  it.nch = (it.S + it.K - 1) / it.K;
  it.count = wi.count;
  it.two = T.n_clips >= 2;
  it.ra = T.wk_keys + (size_t)wi.k0 * it.S * 4 * it.P;
  it.rb = it.ra + (size_t)T.n_keys * it.S * 4 * it.P;
  it.u = T.wk_u;
  it.tab = T.wk_tab;
  const int c = lane >> it.logP;
  float al = 0.f, w = 0.f;
  if (c < wi.count) {
    const int cid = __ldcg(a.item_chars + wi.start + c);
    const float tm = __ldcg(a.time + cid);
    if (isfinite(tm)) {
      const float uu = __fmul_rn(tm, T.rate);
      al = uu - floorf(uu);
    } else if (warp == 1) {
      atomicOr(a.status, kStatusNonfiniteTime);
    }
    w = it.two ? __ldcg(a.blend_w + cid) : 0.f;
  }
  if (tid < wi.count) outs[tid] = reinterpret_cast<float4 *>(a.skin) + a.row_off[__ldcg(a.item_chars + wi.start + tid)] * 3;
  __syncthreads();  // barriers initialized, outs[] filled
  if (warp == 0 && lane == 0) {
    const int K = it.K;
    for (int q = 0; q < 2 && q < it.nch; ++q) {
      if (K == 1) w2_issue<1>(it, q, sm + q * kRecBuf, &B.rec_full[q]);
      else if (K == 2) w2_issue<2>(it, q, sm + q * kRecBuf, &B.rec_full[q]);
      else w2_issue<4>(it, q, sm + q * kRecBuf, &B.rec_full[q]);
    }
  }
  float4 *bslots = reinterpret_cast<float4 *>(sm + kSlotOff) + (size_t)c * a.nbs_max * 3;
  bool ok;
  if (warp == 0) {
    ok = it.K == 1   ? w2_walker<1>(it, sm, B, bslots)
         : it.K == 2 ? w2_walker<2>(it, sm, B, bslots)
                     : w2_walker<4>(it, sm, B, bslots);
  } else {
    const int sw = warp - 1;
    ok = it.K == 1   ? w2_sampler<1>(it, sm, B, outs, sw, al, w)
         : it.K == 2 ? w2_sampler<2>(it, sm, B, outs, sw, al, w)
                     : w2_sampler<4>(it, sm, B, outs, sw, al, w);
  }
  if (!ok && lane == 0) atomicOr(a.status, kStatusTimeout);
  if (a.pred_waited && tid == 0) asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace

size_t walk2_smem_bytes(int chars_per_item, int nbs) {
  return (size_t)kSlotOff + 48ull * (size_t)chars_per_item * (size_t)nbs;
}

namespace {
SmemLimit g_walk2_lim;  // the kernel's shared-memory attribute, per device
}  // namespace

int walk2_blocks_per_sm(size_t smem) {
  if (ensure_smem_limit((const void *)k_walk2, g_walk2_lim, smem, 48 * 1024) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk2, kW2Threads, smem) != cudaSuccess) return 0;
  return nb;
}

size_t walk2_spread_smem(size_t smem, int n_items, int sm_count) {
  const int target = std::max(1, (n_items + sm_count - 1) / std::max(1, sm_count));
  if (walk2_blocks_per_sm(smem) <= target) return smem;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, k_walk2) != cudaSuccess || (size_t)optin <= fa.sharedSizeBytes + smem)
    return smem;
  size_t lo = smem, hi = (size_t)optin - fa.sharedSizeBytes;  // blocks(lo) > target
  if (walk2_blocks_per_sm(hi) > target) return smem;
  while (hi - lo > 128) {  // smallest multiple-of-128 size with blocks <= target
    const size_t mid = (lo + hi) / 2 / 128 * 128;
    if (mid <= lo) break;
    if (walk2_blocks_per_sm(mid) > target) lo = mid;
    else hi = mid;
  }
  return hi;
}

cudaError_t launch_walk2(const WalkArgs &a, size_t smem, cudaStream_t st) {
  cudaError_t e = ensure_smem_limit((const void *)k_walk2, g_walk2_lim, smem, 48 * 1024);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)a.n_items);
  lc.blockDim = dim3((unsigned)kW2Threads);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_walk2, a);
}

}  // namespace anim
