// Adjoint of the Hierarchy-Scan for losses on model-space joint positions,
// and the fused IK step built on it (extensions of the paper's path).
//
// For a loss with g_j = dLoss/dp_j (p_j the translation of M_j), rigid poses:
//   F_j = sum of g over the subtree of j,   T_j = sum of p_k x g_k over it,
//   tau_j = R_p(j)^T (T_j - p_j x F_j),     dLoss/dt_j = R_p(j)^T F_j,
//   dLoss/dq_j = 2 (tau_j, 0) (x) q_hat_j / |q_j|  (Hamilton product).
// The subtree sums are the reverse (leaf-to-root) tree scan.  In depth-first
// pre-order every subtree is a contiguous range of slots, so the scan is one
// exclusive prefix sum over slots: F_j = Pre[end] - Pre[slot].  The forward
// transforms are recomputed per work item with the segmented scan in shared
// memory (nothing is stored between forward and backward).
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "scan_core.cuh"
#include "smem_limit.h"

namespace anim {

// Item layout of the adjoint: the scan's layout, then F and T [C][n+1]
// float4 each (+1 spare), then the view's subtree ends, parents and gather
// map as int16 [n] each.
size_t adjoint_smem_bytes(int n, int nseg, int C) {
  return qt_item_bytes(n, nseg, C) + 16ull * 2ull * ((size_t)C * (n + 1) + 1) + (6ull * n + 15) / 16 * 16;
}

__device__ __forceinline__ float3 cross3(const float3 a, const float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float4 shfl_up4(float4 v, int o) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, o);
  v.y = __shfl_up_sync(0xffffffffu, v.y, o);
  v.z = __shfl_up_sync(0xffffffffu, v.z, o);
  v.w = __shfl_up_sync(0xffffffffu, v.w, o);
  return v;
}
__device__ __forceinline__ void add4(float4 &a, const float4 b) {
  a.x += b.x;
  a.y += b.y;
  a.z += b.z;
  a.w += b.w;
}

// Exclusive prefix of the (F, T) float4 pairs over slots [0, n] (entry n
// receives the total).  All NT pass threads take part.
template <int NT>
__device__ void prefix_pairs(float4 *F, float4 *T, int n, float4 *wsF, float4 *wsT) {
  const int tid = threadIdx.x, nth = NT;
  const int lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  const int per = (n + nth - 1) / nth;
  const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
  float4 sf = make_float4(0.f, 0.f, 0.f, 0.f), st = sf;
  for (int i = i0; i < i1; ++i) {
    add4(sf, F[i]);
    add4(st, T[i]);
  }
  float4 xf = sf, xt = st;  // inclusive warp scan of the run sums
  for (int o = 1; o < 32; o <<= 1) {
    const float4 yf = shfl_up4(xf, o), yt = shfl_up4(xt, o);
    if (lane >= o) {
      add4(xf, yf);
      add4(xt, yt);
    }
  }
  if (lane == 31) {
    wsF[wid] = xf;
    wsT[wid] = xt;
  }
  pass_sync<NT>();
  if (wid == 0) {
    float4 wf = lane < nw ? wsF[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 wt = lane < nw ? wsT[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 1; o < 32; o <<= 1) {
      const float4 yf = shfl_up4(wf, o), yt = shfl_up4(wt, o);
      if (lane >= o) {
        add4(wf, yf);
        add4(wt, yt);
      }
    }
    if (lane < nw) {
      wsF[lane] = wf;
      wsT[lane] = wt;
    }
  }
  pass_sync<NT>();
  float4 pf = make_float4(xf.x - sf.x, xf.y - sf.y, xf.z - sf.z, xf.w - sf.w);
  float4 pt = make_float4(xt.x - st.x, xt.y - st.y, xt.z - st.z, 0.f);
  if (wid > 0) {
    add4(pf, wsF[wid - 1]);
    add4(pt, wsT[wid - 1]);
  }
  for (int i = i0; i < i1; ++i) {
    const float4 a = F[i], b = T[i];
    F[i] = pf;
    T[i] = pt;
    add4(pf, a);
    add4(pt, b);
  }
  if (tid == nth - 1) {
    F[n] = pf;
    T[n] = pt;
  }
  pass_sync<NT>();
}

// One work item: MODE 0 grad_pos given; MODE 1 loss sum |p - target|^2;
// MODE 2 IK step (effector loss, adjoint, Adam update of q, m, v), MODE 3
// the same with the moments in the IK object's own state.  NT
// threads run the passes (tid < NT); `step` is the 1-based Adam step.
// The view's tables in the item's shared memory: subtree ends, parents and
// gather map (int16), and the segment tables of the forward scan.  Plan
// data only, so the one-item kernel stages them before waiting for the
// preceding grid.
// Staged by cp.async in 4-byte words from the view's 16-bit tables when n is
// even (the three arrays then start on 4-byte boundaries), else converted
// here; every thread waits for its copies (cp_async_wait_all) before the
// barrier that follows pass 1a.
template <int NT>
__device__ __forceinline__ void adjoint_tables(const ItemBuf &b, float4 *sm, int tid) {
  const int C = b.C, n = b.T.n;
  const ItemLayout Lt = item_layout_qt(sm, C, n, b.T.nseg);
  int16_t *sub16 = reinterpret_cast<int16_t *>(Lt.end + 2 * (C * (n + 1) + 1));
  int16_t *par16 = sub16 + n, *gat16 = par16 + n;
  if ((n & 1) == 0 && b.T.sub16) {
    const int w = n / 2;
    const uint32_t *ss = reinterpret_cast<const uint32_t *>(b.T.sub16);
    const uint32_t *sp = reinterpret_cast<const uint32_t *>(b.T.par16);
    const uint32_t *sg = reinterpret_cast<const uint32_t *>(b.T.gat16);
    for (int k = tid; k < w; k += NT) {
      cp_async4(reinterpret_cast<uint32_t *>(sub16) + k, ss + k);
      cp_async4(reinterpret_cast<uint32_t *>(par16) + k, sp + k);
      cp_async4(reinterpret_cast<uint32_t *>(gat16) + k, sg + k);
    }
  } else {
    const int32_t *gat = b.T.gather;
    for (int j = tid; j < n; j += NT) {
      sub16[j] = (int16_t)__ldg(b.T.sub_end + j);
      par16[j] = (int16_t)__ldg(b.T.parent + j);
      gat16[j] = (int16_t)(gat ? __ldg(gat + j) : j);
    }
  }
  stage_tables<NT>(b, Lt, tid);  // commits this thread's copies
}

// STAGED: adjoint_tables already ran for this item (all NT threads, before
// a barrier that precedes the item).
template <int MODE, int NT, bool STAGED = false>
__device__ __forceinline__ void adjoint_item(const AdjointArgs &a, const ItemBuf &b, float4 *sm, float4 *wsF,
                                             float4 *wsT, int tid, int step) {
  const int C = b.C, n = b.T.n, nseg = b.T.nseg;
  const int cs2 = 2 * n + 1;  // the forward scan keeps (q, t) pairs
  const ItemLayout Lt = item_layout_qt(sm, C, n, nseg);
  float4 *P = Lt.P;
  float4 *PF = Lt.end;                // [C][n+1]
  float4 *PT = PF + C * (n + 1) + 1;  // [C][n+1] (+1: the scan's total)
  // The adjoint runs on views numbered in depth-first pre-order, so a
  // joint's slot is its index and its subtree is [j, sub_end[j]).
  const int16_t *sub16 = reinterpret_cast<const int16_t *>(PT + C * (n + 1) + 1);
  const int16_t *par16 = sub16 + n, *gat16 = par16 + n;
  const int32_t *gat = b.T.gather;
  const bool gath = gat != nullptr;
  const int CN = C * n;
  if (!STAGED) adjoint_tables<NT>(b, sm, tid);

  // ---- pass 1a: local poses (q normalized, t); the joint's loss input
  // (dLoss/dp or target) is fetched alongside into its depth-first slot
  // A view of every joint (the loss and backward passes) reads the rows in
  // the caller's order -- coalesced, and independent of the view table --
  // and scatters them to their view slots; the IK's partial views gather.
  const int32_t *inv = MODE < 2 ? b.T.inv_gather : nullptr;
  // backward passes: a thread's first two rows of q stay in registers for
  // the gradient pass, which visits the same (character, joint) pairs in the
  // same order (the IK step, whose kernels are larger, reads them again)
  constexpr bool kKeep = MODE < 2;
  float4 qkeep[2] = {make_float4(0.f, 0.f, 0.f, 1.f), make_float4(0.f, 0.f, 0.f, 1.f)};
  {
    const float4 *q4 = reinterpret_cast<const float4 *>(a.q);
    int it = 0;
#pragma unroll 2
    for (int idx = tid; idx < CN; idx += NT, ++it) {
      const int c = (int)b.divN.div(idx), k = idx - c * n;
      const int j = inv ? __ldg(inv + k) : k;
      const long long row = b.off[c] + (inv ? k : gath ? __ldg(gat + k) : k);
      const float4 qr = __ldg(q4 + row);
      if (kKeep && it == 0) qkeep[0] = qr;
      if (kKeep && it == 1) qkeep[1] = qr;
      const float4 q = normalize4(qr);
      const float *tp = a.t + 3 * row;
      sts_qt(P + c * cs2, j, n, QT{q, make_float4(__ldg(tp), __ldg(tp + 1), __ldg(tp + 2), 0.f)});
      if (MODE < 2) {
        const float *src = (MODE == 0 ? a.grad_pos : a.target) + 3 * row;
        PF[c * (n + 1) + j] = make_float4(__ldg(src), __ldg(src + 1), __ldg(src + 2), 0.f);
      }
    }
  }
  cp_async_wait_all();  // this thread's table copies (adjoint_tables)
  pass_sync<NT>();
  pass1b_qt<NT>(b, Lt, P, cs2, tid);
  pass_sync<NT>();
  const float4 *Y = pass2_qt<NT>(b, Lt, P, cs2, tid);

  // ---- model poses in place and the per-slot terms (g, p x g) in the same
  // pass; loss terms in F.w; slot n of each character is zero
  for (int idx = tid; idx < CN; idx += NT) {
    const int c = (int)b.divN.div(idx), j = idx - c * n;
    const uint32_t info = Lt.jinfo[j];
    float4 *Pc = P + c * cs2;
    float3 p;
    if (info & kJ16Link) {
      const QT m = qt_mul(lds_qt(Y, c * nseg + (int)(info & kJ16Seg), C * nseg), lds_qt(Pc, j, n));
      sts_qt(Pc, j, n, m);
      p = make_float3(m.t.x, m.t.y, m.t.z);
    } else {
      const float4 t = Pc[n + j];
      p = make_float3(t.x, t.y, t.z);
    }
    const int i = j;
    float3 g = make_float3(0.f, 0.f, 0.f);
    float lterm = 0.f;
    if (MODE == 0) {
      const float4 v = PF[c * (n + 1) + i];
      g = make_float3(v.x, v.y, v.z);
    } else if (MODE == 1) {
      const float4 v = PF[c * (n + 1) + i];
      const float dx = p.x - v.x, dy = p.y - v.y, dz = p.z - v.z;
      g = make_float3(2.f * dx, 2.f * dy, 2.f * dz);
      lterm = dx * dx + dy * dy + dz * dz;
    }
    const float3 pg = cross3(p, g);
    PF[c * (n + 1) + i] = make_float4(g.x, g.y, g.z, lterm);
    PT[c * (n + 1) + i] = make_float4(pg.x, pg.y, pg.z, 0.f);
    if (j == 0) {
      PF[c * (n + 1) + n] = make_float4(0.f, 0.f, 0.f, 0.f);
      PT[c * (n + 1) + n] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  pass_sync<NT>();
  if (MODE >= 2) {
    const int CE = C * a.n_eff;
    for (int idx = tid; idx < CE; idx += NT) {
      const int c = idx / a.n_eff, e = idx - c * a.n_eff;
      const int j = __ldg(a.eff_slot + b.type * a.n_eff + e);
      const int i = j;
      const float4 pt = P[c * cs2 + n + j];
      const float3 p = make_float3(pt.x, pt.y, pt.z);
      const float *tg = a.target + ((size_t)b.cid[c] * a.n_eff + e) * 3;
      const float dx = p.x - __ldg(tg), dy = p.y - __ldg(tg + 1), dz = p.z - __ldg(tg + 2);
      const float3 g = make_float3(2.f * dx, 2.f * dy, 2.f * dz);
      const float3 pg = cross3(p, g);
      PF[c * (n + 1) + i] = make_float4(g.x, g.y, g.z, dx * dx + dy * dy + dz * dz);
      PT[c * (n + 1) + i] = make_float4(pg.x, pg.y, pg.z, 0.f);
    }
    pass_sync<NT>();
  }
  // one exclusive prefix over all characters' slots; subtree sums are
  // differences inside a character
  prefix_pairs<NT>(PF, PT, C * (n + 1), wsF, wsT);
  if (MODE != 0 && a.loss != nullptr && tid < C) a.loss[b.cid[tid]] = PF[tid * (n + 1) + n].w - PF[tid * (n + 1)].w;

  // ---- per-joint gradients (and the Adam update in IK mode)
  float bc2s = 1.f, step_size = 0.f;
  if (MODE >= 2) {
    bc2s = sqrtf(1.f - powf(a.beta2, (float)step));
    step_size = a.lr / (1.f - powf(a.beta1, (float)step));
  }
  int git = 0;
  for (int idx = tid; idx < CN; idx += NT, ++git) {
    const int c = (int)b.divN.div(idx), k = idx - c * n;
    const int j = inv ? __ldg(inv + k) : k;  // in the caller's row order for full views
    const int i = j, e = sub16[j];
    const float4 f0 = PF[c * (n + 1) + i], f1 = PF[c * (n + 1) + e];
    const float4 t0 = PT[c * (n + 1) + i], t1 = PT[c * (n + 1) + e];
    const float3 F = make_float3(f1.x - f0.x, f1.y - f0.y, f1.z - f0.z);
    const float3 Tq = make_float3(t1.x - t0.x, t1.y - t0.y, t1.z - t0.z);
    const float4 pt = P[c * cs2 + n + j];
    const float3 p = make_float3(pt.x, pt.y, pt.z);
    const float3 pf = cross3(p, F);
    const float3 tw = make_float3(Tq.x - pf.x, Tq.y - pf.y, Tq.z - pf.z);
    const int par = par16[j];
    float3 tau = tw, dt = F;
    if (par >= 0) {  // into the parent's frame: R_par^T = R(conj(q_par))
      const float4 qp = normalize4(P[c * cs2 + par]);
      const float4 qc = make_float4(-qp.x, -qp.y, -qp.z, qp.w);
      tau = qrot(qc, tw);
      dt = qrot(qc, F);
    }
    const long long row = b.off[c] + (inv ? k : gat16[j]);
    const float4 q = kKeep && git == 0   ? qkeep[0]
                     : kKeep && git == 1 ? qkeep[1]
                                         : __ldg(reinterpret_cast<const float4 *>(a.q) + row);
    const float inv = rsqrtf(dot4(q, q));
    const float4 u = make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
    const float4 r = qmul(make_float4(tau.x, tau.y, tau.z, 0.f), u);
    const float k2 = 2.f * inv;
    const float4 dq = make_float4(k2 * r.x, k2 * r.y, k2 * r.z, k2 * r.w);
    if (MODE < 2) {
      reinterpret_cast<float4 *>(a.grad_q)[row] = dq;
      a.grad_t[3 * row] = dt.x;
      a.grad_t[3 * row + 1] = dt.y;
      a.grad_t[3 * row + 2] = dt.z;
    } else {
      const long long srow = MODE == 3 ? b.voff[c] + j : row;  // the Adam state's row
      float4 m = reinterpret_cast<float4 *>(a.m)[srow];
      float4 v = reinterpret_cast<float4 *>(a.v)[srow];
      float4 qn = q;
      const float b1 = a.beta1, b2 = a.beta2;
      const float gq[4] = {dq.x, dq.y, dq.z, dq.w};
      float *mm = &m.x, *vv = &v.x, *qq = &qn.x;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        mm[k] = b1 * mm[k] + (1.f - b1) * gq[k];
        vv[k] = b2 * vv[k] + (1.f - b2) * gq[k] * gq[k];
        const float denom = sqrtf(vv[k]) / bc2s + a.eps;
        qq[k] = qq[k] - step_size * (mm[k] / denom);
      }
      reinterpret_cast<float4 *>(a.m)[srow] = m;
      reinterpret_cast<float4 *>(a.v)[srow] = v;
      reinterpret_cast<float4 *>(a.q_mut)[row] = qn;
    }
  }
}

// Persistent kernel: 8 compute warps and one producer warp staging the next
// item, items from the queue (the frame kernel's CTA layout); built for 2 or
// 3 resident CTAs per SM (MINB).
template <int MODE, int MINB>
__global__ void __launch_bounds__(kCtaThreads, MINB) k_adjoint(const AdjointArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemBuf bufs[2];
  __shared__ float4 wsF[32], wsT[32];
  const int tid = threadIdx.x;
  // launched with programmatic stream serialization: the CTAs become
  // resident while the preceding kernel finishes; the queue, the IK step
  // counter and the inputs are read only after it has completed (the first
  // wave's rows are only prefetched into L2 before that: the work items and
  // views are plan data)
  asm volatile("griddepcontrol.launch_dependents;");
  const RowPrefetch pf =
      MODE == 3   ? RowPrefetch{{a.q, a.t, nullptr, nullptr}, {4, 3, 0, 0}, 0}
      : MODE == 2 ? RowPrefetch{{a.q, a.t, a.m, a.v}, {4, 3, 4, 4}, 0}
                : RowPrefetch{{a.q, a.t, MODE == 0 ? a.grad_pos : a.target, nullptr}, {4, 3, 3, 0}, 1};
  if (tid >= kComputeThreads)
    prefetch_first_wave(bufs[1], a.n_items, a.items, a.types, a.item_chars, a.row_off, pf);
  asm volatile("griddepcontrol.wait;" ::: "memory");

  if (tid >= kComputeThreads) {
    producer_loop<1>(bufs, a.queue_head, a.n_items, a.items, a.types, a.item_chars, a.row_off, nullptr, nullptr,
                     a.status, MODE == 3 ? a.state_off : nullptr, LayerIn{nullptr, nullptr}, pf);
    return;
  }
  const int step = (MODE >= 2) ? *a.step + 1 : 0;  // 1-based Adam step of this launch
  int cur = 0;
  handoff_sync();
  for (;;) {
    const ItemBuf &b = bufs[cur];
    if (b.item < 0) break;
    adjoint_item<MODE, kComputeThreads>(a, b, sm, wsF, wsT, tid, step);
    compute_sync();
    cur ^= 1;
    handoff_sync();
  }

  if (tid == 0) {  // the last CTA resets the queue (and advances the IK step)
    __threadfence();
    if (atomicAdd(a.done, 1) == (int)gridDim.x - 1) {
      if (MODE >= 2) *a.step = *a.step + 1;
      *a.queue_head = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}

static_assert(sizeof(ItemBuf) + 2 * (kAdjSmallThreads / 32) * 16 <= kAdjSmallStatic, "one-item kernel statics");

// One-item kernel: CTA b processes item b with kAdjSmallThreads threads and
// no producer warp, small enough that several CTAs share an SM; the
// hardware schedules the items in waves.  Suits many small items, where the
// persistent kernel would run each CTA's items one after another.
template <int MODE>
__global__ void __launch_bounds__(kAdjSmallThreads, 7) k_adjoint_small(const AdjointArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemBuf b;
  __shared__ float4 wsF[kAdjSmallThreads / 32], wsT[kAdjSmallThreads / 32];
  const int tid = threadIdx.x;
  // Launched with programmatic stream serialization: the next launch's CTAs
  // may become resident now and stage their items (plan data only: item
  // descriptor, type table, character rows) while this grid finishes.
  asm volatile("griddepcontrol.launch_dependents;");
  if (tid < 32) {
    const WorkItem wi = a.items[blockIdx.x];
    stage_item<1>(b, (int)blockIdx.x, wi, a.types, a.item_chars, a.row_off, nullptr, nullptr, a.status,
                  MODE == 3 ? a.state_off : nullptr);
  }
  __syncthreads();
  adjoint_tables<kAdjSmallThreads>(b, sm, tid);  // read after the item's first barrier
  if (MODE < 2) {
    // warm L2 with the item's rows of poses and loss inputs while the
    // preceding grid finishes: a prefetch loads nothing into the kernel, and
    // L2 is coherent, so the loads after the wait see that grid's writes.
    // The view's rows are a permutation of the character's n rows.
    const int n = b.T.n;
    const float *in = MODE == 0 ? a.grad_pos : a.target;
    for (int c = 0; c < b.C; ++c) {
      const char *rq = reinterpret_cast<const char *>(a.q + 4 * b.off[c]);
      const char *rt = reinterpret_cast<const char *>(a.t + 3 * b.off[c]);
      const char *rg = reinterpret_cast<const char *>(in + 3 * b.off[c]);
      for (int k = tid; k * 128 < 16 * n; k += kAdjSmallThreads) prefetch_l2(rq + k * 128);
      for (int k = tid; k * 128 < 12 * n; k += kAdjSmallThreads) {
        prefetch_l2(rt + k * 128);
        prefetch_l2(rg + k * 128);
      }
    }
  }
  // poses, targets, the IK step counter and the outputs may belong to the
  // preceding kernel in the stream: wait for it to complete
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int step = (MODE >= 2) ? *a.step + 1 : 0;
  adjoint_item<MODE, kAdjSmallThreads, true>(a, b, sm, wsF, wsT, tid, step);
  if (MODE >= 2 && tid == 0) {  // the last CTA advances the IK step
    __threadfence();
    if (atomicAdd(a.done, 1) == (int)gridDim.x - 1) {
      *a.step = *a.step + 1;
      *a.done = 0;
      __threadfence();
    }
  }
}

template <int MODE, int MINB>
static cudaError_t launch_adj_persistent(const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st);

template <int MODE>
static cudaError_t launch_adj_t(const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  if (cfg.threads == kAdjSmallThreads) {
    static SmemLimit lim_small;
    cudaError_t e = ensure_smem_limit((const void *)k_adjoint_small<MODE>, lim_small, cfg.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)a.n_items);
    lc.blockDim = dim3((unsigned)kAdjSmallThreads);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_adjoint_small<MODE>, a);
  }
  return cfg.min_blocks >= 3 ? launch_adj_persistent<MODE, 3>(a, cfg, st) : launch_adj_persistent<MODE, 2>(a, cfg, st);
}

template <int MODE, int MINB>
static cudaError_t launch_adj_persistent(const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k_adjoint<MODE, MINB>, lim, cfg.smem);
  if (e != cudaSuccess) return e;
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
  return cudaLaunchKernelEx(&lc, k_adjoint<MODE, MINB>, a);
}

cudaError_t launch_adjoint(int mode, const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  if (mode == 0) return launch_adj_t<0>(a, cfg, st);
  if (mode == 1) return launch_adj_t<1>(a, cfg, st);
  if (mode == 2) return launch_adj_t<2>(a, cfg, st);
  return launch_adj_t<3>(a, cfg, st);
}

}  // namespace anim
