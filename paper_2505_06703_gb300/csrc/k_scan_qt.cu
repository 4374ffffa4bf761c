// The segmented Hierarchy-Scan (Eq. 1) with rigid transforms kept as
// (quaternion, translation) pairs -- 32 bytes per joint instead of a 48-byte
// 3x4 matrix -- while it runs in shared memory (scan_core.cuh):
//   MODE 0  the plain fused frame (Simulation -> Hierarchy-Scan -> Bind
//           MeshPose, Sec. 1 steps 1-3): local poses sampled from the clips;
//   MODE 1  the forward from given local poses q [total][4] (normalized
//           here), t [total][3], skin and / or model matrices out;
//   MODE 2  the frame with layered blending (up to 4 clips by per-character
//           weights and an additive layer, sample_layers_at).
// The smaller item footprint lets more characters be in flight per SM, which
// is what bounds the latency-limited scan passes.  The segment tables are
// staged by cp.async during pass 1a; one character of a pure chain longer
// than 1,024 joints takes a two-level chain scan (chain_scan_qt) instead of
// the segment walks and pointer jumping.  The bind pass normalizes
// the composed quaternion once (removing the norm drift of long products),
// forms M = [R(q) | t] and writes M and / or S = M B straight to global
// memory.  Same item pipeline as k_scan (producer warp, 8 compute warps,
// work queue); the frame with skinning keeps the matrix form there, as its
// skinning pass reads the skin matrices from shared memory.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "scan_core.cuh"
#include "smem_limit.h"

namespace anim {

namespace {

__device__ __forceinline__ QT shfl_up_qt(const QT &a, int o) {
  QT r;
  r.q.x = __shfl_up_sync(0xffffffffu, a.q.x, o);
  r.q.y = __shfl_up_sync(0xffffffffu, a.q.y, o);
  r.q.z = __shfl_up_sync(0xffffffffu, a.q.z, o);
  r.q.w = __shfl_up_sync(0xffffffffu, a.q.w, o);
  r.t.x = __shfl_up_sync(0xffffffffu, a.t.x, o);
  r.t.y = __shfl_up_sync(0xffffffffu, a.t.y, o);
  r.t.z = __shfl_up_sync(0xffffffffu, a.t.z, o);
  r.t.w = 0.f;
  return r;
}

// A pure chain, one character per item: joint j's model pose is the product
// L_0 ... L_j (Eq. 1 along the one path).  Each compute thread composes its
// run of J consecutive joints in place (J = ceil(n / 256) rounded up to
// odd); a warp-shuffle scan over the runs' products and a scan of the 8 warp
// totals give each run the product of everything before it, which the run
// then applies in place.  Two barriers instead of the segment walks and
// pointer-jumping rounds, so a 2,048-deep chain is never walked more than J
// levels by one thread.
__device__ __forceinline__ void chain_scan_qt(int n, float4 *P, QT *wtot, int tid) {
  const int lane = tid & 31, warp = tid >> 5;
  // an odd run length: the lanes' slots (J float4 apart) fall in distinct banks
  const int J = ((n + kComputeThreads - 1) / kComputeThreads) | 1;
  const int j0 = min(n, tid * J), j1 = min(n, j0 + J);
  QT acc = qt_identity();
  for (int j = j0; j < j1; ++j) {
    const QT L = lds_qt(P, j, n);
    acc = j == j0 ? L : qt_mul(acc, L);
    if (j > j0) sts_qt(P, j, n, acc);
  }
  QT x = acc;  // inclusive scan of the run products over the warp's lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const QT y = shfl_up_qt(x, o);
    if (lane >= o) x = qt_mul(y, x);
  }
  QT ex = shfl_up_qt(x, 1);
  if (lane == 0) ex = qt_identity();
  if (lane == 31) wtot[warp] = x;
  compute_sync();
  QT wp = qt_identity();
  for (int w = 0; w < warp; ++w) wp = w == 0 ? wtot[0] : qt_mul(wp, wtot[w]);
  if (tid > 0) {
    const QT E = warp == 0 ? ex : lane == 0 ? wp : qt_mul(wp, ex);
    for (int j = j0; j < j1; ++j) sts_qt(P, j, n, qt_mul(E, lds_qt(P, j, n)));
  }
  compute_sync();
}

template <int MODE, int MINB>
__global__ void __launch_bounds__(kCtaThreads, MINB) k_scan_qt(const ScanArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemBuf bufs[2];
  __shared__ QT wtot[kComputeWarps];  // chain scan: the warps' run products
  const int tid = threadIdx.x;
  // launched with programmatic stream serialization (after the work-queue
  // kernel, for the frame): wait for the preceding grid to complete before
  // reading anything it may have written.  The next launch may start now
  // (the next frame's work-queue kernel reads only plan tables before its
  // own wait) -- in the plain frame only once this grid's wait is over, as
  // the chain-walk kernel launched after it may then read the work queue
  // without a wait of its own (WalkArgs::pred_waited).
  // The forward from local poses (fixed work items) prefetches its first
  // wave's rows of q and t into L2 before the wait, and each next item's
  // while the current one runs.
  if (MODE != 0) asm volatile("griddepcontrol.launch_dependents;");
  const RowPrefetch pf = MODE == 1 ? RowPrefetch{{a.q, a.t, nullptr, nullptr}, {4, 3, 0, 0}, 0} : RowPrefetch{};
  if (MODE == 1 && tid >= kComputeThreads)
    prefetch_first_wave(bufs[1], a.n_items, a.items, a.types, a.item_chars, a.row_off, pf);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (MODE == 0) asm volatile("griddepcontrol.launch_dependents;");
  const int n_items = a.n_items;

  if (tid >= kComputeThreads) {
    producer_loop<MODE == 1 ? 1 : 0>(bufs, a.queue_head, n_items, a.items, a.types, a.item_chars, a.row_off,
                                     a.time, a.blend_w, a.status, nullptr,
                                     MODE == 2 ? LayerIn{a.layer_w, a.add_w} : LayerIn{nullptr, nullptr}, pf);
    return;
  }

  int cur = 0;
  handoff_sync();
  for (;;) {
    const ItemBuf &b = bufs[cur];
    if (b.item < 0) break;
    const int C = b.C, n = b.T.n, nseg = b.T.nseg;
    const int cs2 = 2 * n + 1;  // float4 stride between characters (16 B skew)
    const ItemLayout Lt = item_layout_qt(sm, C, n, nseg);
    float4 *P = Lt.P;

    // ---- pass 1a: local poses (q, t) from the clips or the caller's rows;
    // tables staged alongside
    stage_tables(b, Lt, tid);
    if (MODE == 1) {
      // character-major: consecutive lanes read consecutive rows
      const float4 *q4 = reinterpret_cast<const float4 *>(a.q);
      const int32_t *gat = b.T.gather;
      const int CN = C * n;
#pragma unroll 2
      for (int idx = tid; idx < CN; idx += kComputeThreads) {
        const int c = (int)b.divN.div(idx), j = idx - c * n;
        const long long row = b.off[c] + (gat ? __ldg(gat + j) : j);
        const float4 q = normalize4(__ldg(q4 + row));
        const float *tp = a.t + 3 * row;
        sts_qt(P + c * cs2, j, n, QT{q, make_float4(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2), 0.f)});
      }
    } else if (MODE == 2) {
      // character-minor: the lanes of one joint share its key records
      const int CN = C * n;
      for (int idx = tid; idx < CN; idx += kComputeThreads) {
        const int j = (int)b.divC.div(idx), c = idx - j * C;
        sts_qt(P + c * cs2, j, n, sample_layers_at(b, j, c));
      }
    } else {
      const int nk = b.T.n_keys, k0 = b.k0, k1 = (k0 + 1 == nk) ? 0 : k0 + 1;
      const float4 *KA0 = b.T.keys + (size_t)k0 * n * 2;
      const float4 *KA1 = b.T.keys + (size_t)k1 * n * 2;
      const float4 *KB0 = b.T.keys + (size_t)(nk + k0) * n * 2;
      const float4 *KB1 = b.T.keys + (size_t)(nk + k1) * n * 2;
      const bool two = b.T.n_clips >= 2;
      // joint-major: a thread loads joint j's key records once and samples
      // them for its group of characters (the pass-3 grouping)
      const int W = n * b.cgroups, cpt = b.cpt;
      for (int idx = tid; idx < W; idx += kComputeThreads) {
        const int grp = (int)b.divN.div(idx), j = idx - grp * n;
        const float4 qa0 = __ldg(KA0 + 2 * j), ta0 = __ldg(KA0 + 2 * j + 1);
        const float4 qa1 = __ldg(KA1 + 2 * j), ta1 = __ldg(KA1 + 2 * j + 1);
        float4 qb0 = qa0, tb0 = ta0, qb1 = qa1, tb1 = ta1;
        if (two) {
          qb0 = __ldg(KB0 + 2 * j);
          tb0 = __ldg(KB0 + 2 * j + 1);
          qb1 = __ldg(KB1 + 2 * j);
          tb1 = __ldg(KB1 + 2 * j + 1);
        }
        const int c1 = min(C, (grp + 1) * cpt);
        for (int c = grp * cpt; c < c1; ++c) {
          const float al = b.alpha[c];
          float4 q = slerp_pre(qa0, qa1, ta0.w, al);
          float tx = fmaf(al, ta1.x - ta0.x, ta0.x), ty = fmaf(al, ta1.y - ta0.y, ta0.y),
                tz = fmaf(al, ta1.z - ta0.z, ta0.z);
          if (two) {
            const float4 qb = slerp_pre(qb0, qb1, tb0.w, al);
            const float w = b.blend[c];
            q = slerp_unit(q, qb, w);
            tx = fmaf(w, fmaf(al, tb1.x - tb0.x, tb0.x) - tx, tx);
            ty = fmaf(w, fmaf(al, tb1.y - tb0.y, tb0.y) - ty, ty);
            tz = fmaf(w, fmaf(al, tb1.z - tb0.z, tb0.z) - tz, tz);
          }
          sts_qt(P + c * cs2, j, n, QT{q, make_float4(tx, ty, tz, 0.f)});
        }
      }
    }
    cp_async_wait_all();  // this thread's table copies (stage_tables)
    compute_sync();

    // ---- pass 1b: running products along segments; pass 2: pointer jumping
    // over segments -- or, for one character of a pure chain of more than
    // 1,024 joints, the chain scan (same-box A/B: config 3's 2,048-joint
    // chains 54.2 -> 43.8 us per frame; the forward on config 2, whose
    // 1,024-joint dragon it would also take, 50.6 -> 51.3 us)
    const bool chain = b.T.chain && C == 1 && n > 1024;
    const float4 *Y = nullptr;
    if (chain) {
      chain_scan_qt(n, P, wtot, tid);
    } else {
      pass1b_qt(b, Lt, P, cs2, tid);
      compute_sync();
      Y = pass2_qt(b, Lt, P, cs2, tid);
    }

    // ---- pass 3: model pose, normalize, matrix, (bind,) store
    {
      const int W = n * b.cgroups, cpt = b.cpt;
      float4 *skin4 = reinterpret_cast<float4 *>(a.skin);
      float4 *model4 = reinterpret_cast<float4 *>(a.model);
      const bool skin = MODE != 1 || skin4 != nullptr, model = MODE == 1 && model4 != nullptr;
      for (int idx = tid; idx < W; idx += kComputeThreads) {
        const int grp = (int)b.divN.div(idx), j = idx - grp * n;
        const uint32_t info = Lt.jinfo[j];
        const int g = (int)(info & kJ16Seg);
        Aff B;
        if (skin) B = ldg_aff(b.T.inv_bind + 3 * j);
        const int c1 = min(C, (grp + 1) * cpt);
        for (int c = grp * cpt; c < c1; ++c) {
          QT m = lds_qt(P + c * cs2, j, n);
          if (!chain && (info & kJ16Link)) m = qt_mul(lds_qt(Y, c * nseg + g, C * nseg), m);
          const Aff M = aff_from_qt(normalize4(m.q), m.t.x, m.t.y, m.t.z);
          if (model) stg_aff(model4 + (b.off[c] + j) * 3, M);
          if (skin) stg_aff(skin4 + (b.off[c] + j) * 3, aff_mul(M, B));
        }
      }
    }
    cur ^= 1;
    handoff_sync();
  }
  if (tid == 0 && a.done) last_cta_reset(a.queue_head, a.done);
}

template <int MODE, int MINB>
static cudaError_t launch_qt(const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k_scan_qt<MODE, MINB>, lim, cfg.smem);
  if (e != cudaSuccess) return e;
  // programmatic stream serialization: the CTAs become resident while the
  // preceding kernel runs and wait in griddepcontrol.wait
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)cfg.ctas);
  lc.blockDim = dim3((unsigned)cfg.threads);
  lc.dynamicSmemBytes = cfg.smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_scan_qt<MODE, MINB>, a);
}

}  // namespace

size_t scan_qt_smem_bytes(int n, int nseg, int C) { return qt_item_bytes(n, nseg, C); }

cudaError_t launch_scan_qt(int mode, const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  const bool m3 = cfg.min_blocks >= 3;
  if (mode == 0) return m3 ? launch_qt<0, 3>(a, cfg, st) : launch_qt<0, 2>(a, cfg, st);
  if (mode == 1) return m3 ? launch_qt<1, 3>(a, cfg, st) : launch_qt<1, 2>(a, cfg, st);
  return m3 ? launch_qt<2, 3>(a, cfg, st) : launch_qt<2, 2>(a, cfg, st);
}

}  // namespace anim
