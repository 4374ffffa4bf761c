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

namespace anim {

constexpr int kAdjThreads = 256;
constexpr int kAdjCMax = 64;

size_t adjoint_smem_bytes(int n, int nseg, int C) {
  return 16ull * ((size_t)C * (3 * (size_t)n + 1) + 6ull * C * nseg + 2ull * C * (n + 1));
}

__device__ __forceinline__ float3 cross3(const float3 a, const float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Exclusive prefix of the (F, T) float4 pairs over slots [0, n] of one
// character (entry n receives the total).  All threads take part.
__device__ void prefix_pairs(float4 *F, float4 *T, int n, float4 *wsF, float4 *wsT) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  const int per = (n + nth - 1) / nth;
  const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
  float4 sf = make_float4(0.f, 0.f, 0.f, 0.f), st = sf;
  for (int i = i0; i < i1; ++i) {
    const float4 a = F[i], b = T[i];
    sf.x += a.x; sf.y += a.y; sf.z += a.z; sf.w += a.w;
    st.x += b.x; st.y += b.y; st.z += b.z; st.w += b.w;
  }
  // inclusive warp scan of the run sums
  float4 xf = sf, xt = st;
  for (int o = 1; o < 32; o <<= 1) {
    float4 yf, yt;
    yf.x = __shfl_up_sync(0xffffffffu, xf.x, o); yf.y = __shfl_up_sync(0xffffffffu, xf.y, o);
    yf.z = __shfl_up_sync(0xffffffffu, xf.z, o); yf.w = __shfl_up_sync(0xffffffffu, xf.w, o);
    yt.x = __shfl_up_sync(0xffffffffu, xt.x, o); yt.y = __shfl_up_sync(0xffffffffu, xt.y, o);
    yt.z = __shfl_up_sync(0xffffffffu, xt.z, o);
    if (lane >= o) {
      xf.x += yf.x; xf.y += yf.y; xf.z += yf.z; xf.w += yf.w;
      xt.x += yt.x; xt.y += yt.y; xt.z += yt.z;
    }
  }
  if (lane == 31) {
    wsF[wid] = xf;
    wsT[wid] = xt;
  }
  __syncthreads();
  if (wid == 0) {
    float4 wf = lane < nw ? wsF[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 wt = lane < nw ? wsT[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int o = 1; o < 32; o <<= 1) {
      float4 yf, yt;
      yf.x = __shfl_up_sync(0xffffffffu, wf.x, o); yf.y = __shfl_up_sync(0xffffffffu, wf.y, o);
      yf.z = __shfl_up_sync(0xffffffffu, wf.z, o); yf.w = __shfl_up_sync(0xffffffffu, wf.w, o);
      yt.x = __shfl_up_sync(0xffffffffu, wt.x, o); yt.y = __shfl_up_sync(0xffffffffu, wt.y, o);
      yt.z = __shfl_up_sync(0xffffffffu, wt.z, o);
      if (lane >= o) {
        wf.x += yf.x; wf.y += yf.y; wf.z += yf.z; wf.w += yf.w;
        wt.x += yt.x; wt.y += yt.y; wt.z += yt.z;
      }
    }
    if (lane < nw) {
      wsF[lane] = wf;
      wsT[lane] = wt;
    }
  }
  __syncthreads();
  // exclusive prefix of this thread's run
  float4 pf, pt;
  pf.x = xf.x - sf.x; pf.y = xf.y - sf.y; pf.z = xf.z - sf.z; pf.w = xf.w - sf.w;
  pt.x = xt.x - st.x; pt.y = xt.y - st.y; pt.z = xt.z - st.z; pt.w = 0.f;
  if (wid > 0) {
    const float4 a = wsF[wid - 1], b = wsT[wid - 1];
    pf.x += a.x; pf.y += a.y; pf.z += a.z; pf.w += a.w;
    pt.x += b.x; pt.y += b.y; pt.z += b.z;
  }
  for (int i = i0; i < i1; ++i) {
    const float4 a = F[i], b = T[i];
    F[i] = pf;
    T[i] = pt;
    pf.x += a.x; pf.y += a.y; pf.z += a.z; pf.w += a.w;
    pt.x += b.x; pt.y += b.y; pt.z += b.z;
  }
  if (tid == nth - 1) {
    F[n] = pf;
    T[n] = pt;
  }
  __syncthreads();
}

// MODE 0: grad_pos given; MODE 1: loss sum |p - target|^2; MODE 2: IK step
// (effector loss, adjoint, Adam update of q, m, v).
template <int MODE>
__global__ void __launch_bounds__(kAdjThreads, 2) k_adjoint(const AdjointArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemSmem s;
  __shared__ long long sOff[kAdjCMax];
  __shared__ int sCid[kAdjCMax];
  __shared__ float4 wsF[32], wsT[32];
  __shared__ int sStep;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (MODE == 2 && tid == 0) sStep = *a.step + 1;  // 1-based Adam step of this launch

  for (;;) {
    if (tid == 0) s.item = atomicAdd(a.queue_head, 1);
    __syncthreads();
    const int item = s.item;
    if (item >= a.n_items) break;
    const WorkItem wi = a.items[item];
    const int C = wi.count;
    load_type_smem(s, a.types, wi.type, tid, nth);
    if (tid < C) {
      const int cid = __ldg(a.item_chars + wi.start + tid);
      sCid[tid] = cid;
      sOff[tid] = a.row_off[cid];
    }
    if (tid == 0) {
      const TypeDev &T = a.types[wi.type];
      s.divC.init(C);
      s.divS.init(T.nseg);
      s.divN.init(T.n);
    }
    __syncthreads();

    const int n = s.T.n, nseg = s.T.nseg;
    const int cs4 = 3 * n + 1;
    float4 *P = sm;
    float4 *Y0 = P + C * cs4;
    float4 *Y1 = Y0 + 3 * C * nseg;
    float4 *PF = Y1 + 3 * C * nseg;  // [C][n+1]
    float4 *PT = PF + C * (n + 1);   // [C][n+1]
    const int32_t *gat = s.T.gather;
    const bool gath = gat != nullptr;

    // ---- forward recompute: pass 1 from (q, t)
    {
      const int NS = nseg * C;
      for (int idx = tid; idx < NS; idx += nth) {
        const int g = (int)s.divC.div(idx), c = idx - g * C;
        const int j0 = __ldg(s.T.seg_start + g), j1 = __ldg(s.T.seg_start + g + 1);
        const long long off = sOff[c];
        float4 *Pc = P + c * cs4;
        Aff acc;
        for (int j = j0; j < j1; ++j) {
          const long long row = off + (gath ? __ldg(gat + j) : j);
          const float4 q = normalize4(__ldg(reinterpret_cast<const float4 *>(a.q) + row));
          const float *tp = a.t + 3 * row;
          const Aff L = aff_from_qt(q, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
          acc = (j == j0) ? L : aff_mul(acc, L);
          sts_aff(Pc + 3 * j, acc);
        }
      }
    }
    __syncthreads();
    const float4 *Y = scan_pass2(s, P, cs4, Y0, Y1, C, tid, nth);
    {
      // model pose in place: each thread reads only its own slot of P and Y
      const int CN = C * n;
      for (int idx = tid; idx < CN; idx += nth) {
        const int c = (int)s.divN.div(idx), j = idx - c * n;
        sts_aff(P + c * cs4 + 3 * j, scan_model(s, P, cs4, Y, c, j));
      }
    }
    __syncthreads();

    // ---- per-slot (g, p x g) in depth-first order; loss terms in F.w
    {
      const int CN = C * n;
      for (int idx = tid; idx < CN; idx += nth) {
        const int c = (int)s.divN.div(idx), i = idx - c * n;
        const int j = __ldg(s.T.dfs + i);
        float3 g = make_float3(0.f, 0.f, 0.f);
        float lterm = 0.f;
        const float3 p = make_float3(P[c * cs4 + 3 * j].w, P[c * cs4 + 3 * j + 1].w, P[c * cs4 + 3 * j + 2].w);
        if (MODE == 0) {
          const long long row = sOff[c] + j;
          g = make_float3(__ldg(a.grad_pos + 3 * row), __ldg(a.grad_pos + 3 * row + 1),
                          __ldg(a.grad_pos + 3 * row + 2));
        } else if (MODE == 1) {
          const long long row = sOff[c] + j;
          const float dx = p.x - __ldg(a.target + 3 * row), dy = p.y - __ldg(a.target + 3 * row + 1),
                      dz = p.z - __ldg(a.target + 3 * row + 2);
          g = make_float3(2.f * dx, 2.f * dy, 2.f * dz);
          lterm = dx * dx + dy * dy + dz * dz;
        }
        const float3 pg = cross3(p, g);
        PF[c * (n + 1) + i] = make_float4(g.x, g.y, g.z, lterm);
        PT[c * (n + 1) + i] = make_float4(pg.x, pg.y, pg.z, 0.f);
      }
    }
    __syncthreads();
    if (MODE == 2) {
      const int CE = C * a.n_eff;
      for (int idx = tid; idx < CE; idx += nth) {
        const int c = idx / a.n_eff, e = idx - c * a.n_eff;
        const int j = __ldg(a.eff_slot + wi.type * a.n_eff + e);
        const int i = __ldg(s.T.dfs_slot + j);
        const float3 p = make_float3(P[c * cs4 + 3 * j].w, P[c * cs4 + 3 * j + 1].w, P[c * cs4 + 3 * j + 2].w);
        const float *tg = a.target + ((size_t)sCid[c] * a.n_eff + e) * 3;
        const float dx = p.x - __ldg(tg), dy = p.y - __ldg(tg + 1), dz = p.z - __ldg(tg + 2);
        const float3 g = make_float3(2.f * dx, 2.f * dy, 2.f * dz);
        const float3 pg = cross3(p, g);
        PF[c * (n + 1) + i] = make_float4(g.x, g.y, g.z, dx * dx + dy * dy + dz * dz);
        PT[c * (n + 1) + i] = make_float4(pg.x, pg.y, pg.z, 0.f);
      }
      __syncthreads();
    }
    for (int c = 0; c < C; ++c) prefix_pairs(PF + c * (n + 1), PT + c * (n + 1), n, wsF, wsT);
    if (MODE != 0 && a.loss != nullptr && tid < C) a.loss[sCid[tid]] = PF[tid * (n + 1) + n].w;

    // ---- per-joint gradients (and the Adam update in IK mode)
    {
      const int CN = C * n;
      float bc1 = 1.f, bc2s = 1.f, step_size = 0.f;
      if (MODE == 2) {
        bc1 = 1.f - powf(a.beta1, (float)sStep);
        bc2s = sqrtf(1.f - powf(a.beta2, (float)sStep));
        step_size = a.lr / bc1;
      }
      for (int idx = tid; idx < CN; idx += nth) {
        const int c = (int)s.divN.div(idx), j = idx - c * n;
        const int i = __ldg(s.T.dfs_slot + j), e = __ldg(s.T.sub_end + i);
        const float4 f0 = PF[c * (n + 1) + i], f1 = PF[c * (n + 1) + e];
        const float4 t0 = PT[c * (n + 1) + i], t1 = PT[c * (n + 1) + e];
        const float3 F = make_float3(f1.x - f0.x, f1.y - f0.y, f1.z - f0.z);
        const float3 Tq = make_float3(t1.x - t0.x, t1.y - t0.y, t1.z - t0.z);
        const float3 p = make_float3(P[c * cs4 + 3 * j].w, P[c * cs4 + 3 * j + 1].w, P[c * cs4 + 3 * j + 2].w);
        const float3 pf = cross3(p, F);
        const float3 tw = make_float3(Tq.x - pf.x, Tq.y - pf.y, Tq.z - pf.z);
        const int par = __ldg(s.T.parent + j);
        float3 tau = tw, dt = F;
        if (par >= 0) {
          const float4 r0 = P[c * cs4 + 3 * par], r1 = P[c * cs4 + 3 * par + 1], r2 = P[c * cs4 + 3 * par + 2];
          tau = make_float3(r0.x * tw.x + r1.x * tw.y + r2.x * tw.z, r0.y * tw.x + r1.y * tw.y + r2.y * tw.z,
                            r0.z * tw.x + r1.z * tw.y + r2.z * tw.z);
          dt = make_float3(r0.x * F.x + r1.x * F.y + r2.x * F.z, r0.y * F.x + r1.y * F.y + r2.y * F.z,
                           r0.z * F.x + r1.z * F.y + r2.z * F.z);
        }
        const long long row = sOff[c] + (gath ? __ldg(gat + j) : j);
        const float4 q = __ldg(reinterpret_cast<const float4 *>(a.q) + row);
        const float inv = rsqrtf(dot4(q, q));
        const float4 u = make_float4(q.x * inv, q.y * inv, q.z * inv, q.w * inv);
        const float4 r = qmul(make_float4(tau.x, tau.y, tau.z, 0.f), u);
        const float k2 = 2.f * inv;
        const float4 dq = make_float4(k2 * r.x, k2 * r.y, k2 * r.z, k2 * r.w);
        if (MODE != 2) {
          reinterpret_cast<float4 *>(a.grad_q)[row] = dq;
          a.grad_t[3 * row] = dt.x;
          a.grad_t[3 * row + 1] = dt.y;
          a.grad_t[3 * row + 2] = dt.z;
        } else {
          float4 m = reinterpret_cast<float4 *>(a.m)[row];
          float4 v = reinterpret_cast<float4 *>(a.v)[row];
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
          reinterpret_cast<float4 *>(a.m)[row] = m;
          reinterpret_cast<float4 *>(a.v)[row] = v;
          reinterpret_cast<float4 *>(a.q_mut)[row] = qn;
        }
      }
    }
    __syncthreads();
  }

  if (MODE == 2 && tid == 0) {
    __threadfence();
    const int done = atomicAdd(a.done_ctas, 1);
    if (done == (int)gridDim.x - 1) {
      *a.step = *a.step + 1;
      *a.done_ctas = 0;
      __threadfence();
    }
  }
}

template <int MODE>
static cudaError_t launch_adj_t(const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  static size_t set_smem = 0;
  if (cfg.smem > set_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_adjoint<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    set_smem = cfg.smem;
  }
  k_adjoint<MODE><<<cfg.ctas, cfg.threads, cfg.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(int mode, const AdjointArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  if (mode == 0) return launch_adj_t<0>(a, cfg, st);
  if (mode == 1) return launch_adj_t<1>(a, cfg, st);
  return launch_adj_t<2>(a, cfg, st);
}

}  // namespace anim
