// Fused frame kernel (Simulation -> Hierarchy-Scan -> Bind MeshPose, Sec. 1
// steps 1-3 and Eq. 1), the per-frame work queue, and setup kernels.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "scan_core.cuh"

namespace anim {

constexpr int kCMax = 64;          // characters per work item
constexpr int kScanThreads = 256;  // CTA size of the persistent scan

size_t scan_smem_bytes(int n, int nseg, int C) {
  return 16ull * ((size_t)C * (3 * (size_t)n + 1) + 6ull * C * nseg);
}

// Persistent kernel: each CTA pulls work items (C characters of one type)
// from a global counter, runs the three scan passes in shared memory and
// streams the finished character blocks to global memory with bulk copies.
//   MODE 0: local poses sampled from the type's clips at each character's
//           time (slerp/lerp between keys, then slerp/lerp between clip 0
//           and clip 1 with the character's blend weight);
//   MODE 1: local poses read from q [total][4] (normalized here), t [total][3].
template <int MODE, bool SKIN, bool MODEL>
__global__ void __launch_bounds__(kScanThreads, 2) k_scan(const ScanArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemSmem s;
  __shared__ long long sOff[kCMax];
  __shared__ float sAlpha[kCMax];
  __shared__ float sBlend[kCMax];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int n_items = a.n_items_dev ? *a.n_items_dev : a.n_items;
  bool pending = false;  // thread 0: bulk stores in flight

  for (;;) {
    if (tid == 0) {
      if (pending) {
        bulk_wait_read_all();  // the staging buffer may be overwritten again
        pending = false;
      }
      s.item = atomicAdd(a.queue_head, 1);
    }
    __syncthreads();
    const int item = s.item;
    if (item >= n_items) break;
    const WorkItem wi = a.items[item];
    const int C = wi.count;
    load_type_smem(s, a.types, wi.type, tid, nth);
    if (tid < C) {
      const int cid = __ldg(a.item_chars + wi.start + tid);
      sOff[tid] = a.row_off[cid];
      if (MODE == 0) {
        const float tm = __ldg(a.time + cid);
        const float rate = a.types[wi.type].rate;
        float alpha = 0.f;
        if (isfinite(tm)) {
          const float u = __fmul_rn(tm, rate);
          alpha = u - floorf(u);
        } else {
          atomicOr(a.status, 1);
        }
        sAlpha[tid] = alpha;
        sBlend[tid] = __ldg(a.blend_w + cid);
      }
    }
    if (tid == 0) {
      const TypeDev &T = a.types[wi.type];
      s.wi = wi;
      s.divC.init(C);
      s.divS.init(T.nseg);
      s.divN.init(T.n);
    }
    __syncthreads();

    const int n = s.T.n, nseg = s.T.nseg;
    const int cs4 = 3 * n + 1;  // float4 stride between characters (16 B skew against bank conflicts)
    float4 *P = sm;
    float4 *Y0 = P + C * cs4;
    float4 *Y1 = Y0 + 3 * C * nseg;

    // ---- pass 1: per (segment, character) running products
    {
      const int NS = nseg * C;
      if (MODE == 0) {
        const int nk = s.T.n_keys, k0 = wi.k0, k1 = (k0 + 1 == nk) ? 0 : k0 + 1;
        const float4 *KA0 = s.T.keys + (size_t)k0 * n * 2;
        const float4 *KA1 = s.T.keys + (size_t)k1 * n * 2;
        const float4 *KB0 = s.T.keys + (size_t)(nk + k0) * n * 2;
        const float4 *KB1 = s.T.keys + (size_t)(nk + k1) * n * 2;
        const bool two = s.T.n_clips >= 2;
        for (int idx = tid; idx < NS; idx += nth) {
          const int g = (int)s.divC.div(idx), c = idx - g * C;
          const int j0 = __ldg(s.T.seg_start + g), j1 = __ldg(s.T.seg_start + g + 1);
          const float al = sAlpha[c], w = sBlend[c];
          float4 *Pc = P + c * cs4;
          Aff acc;
          for (int j = j0; j < j1; ++j) {
            const float4 qa0 = __ldg(KA0 + 2 * j), ta0 = __ldg(KA0 + 2 * j + 1);
            const float4 qa1 = __ldg(KA1 + 2 * j), ta1 = __ldg(KA1 + 2 * j + 1);
            float4 q = slerp_pre(qa0, qa1, ta0.w, al);
            float tx = fmaf(al, ta1.x - ta0.x, ta0.x);
            float ty = fmaf(al, ta1.y - ta0.y, ta0.y);
            float tz = fmaf(al, ta1.z - ta0.z, ta0.z);
            if (two) {
              const float4 qb0 = __ldg(KB0 + 2 * j), tb0 = __ldg(KB0 + 2 * j + 1);
              const float4 qb1 = __ldg(KB1 + 2 * j), tb1 = __ldg(KB1 + 2 * j + 1);
              const float4 qb = slerp_pre(qb0, qb1, tb0.w, al);
              const float bx = fmaf(al, tb1.x - tb0.x, tb0.x);
              const float by = fmaf(al, tb1.y - tb0.y, tb0.y);
              const float bz = fmaf(al, tb1.z - tb0.z, tb0.z);
              q = slerp_unit(q, qb, w);
              tx = fmaf(w, bx - tx, tx);
              ty = fmaf(w, by - ty, ty);
              tz = fmaf(w, bz - tz, tz);
            }
            const Aff L = aff_from_qt(q, tx, ty, tz);
            acc = (j == j0) ? L : aff_mul(acc, L);
            sts_aff(Pc + 3 * j, acc);
          }
        }
      } else {
        const bool gath = s.T.gather != nullptr;
        for (int idx = tid; idx < NS; idx += nth) {
          const int g = (int)s.divC.div(idx), c = idx - g * C;
          const int j0 = __ldg(s.T.seg_start + g), j1 = __ldg(s.T.seg_start + g + 1);
          const long long off = sOff[c];
          float4 *Pc = P + c * cs4;
          Aff acc;
          for (int j = j0; j < j1; ++j) {
            const long long row = off + (gath ? __ldg(s.T.gather + j) : j);
            const float4 q = normalize4(__ldg(reinterpret_cast<const float4 *>(a.q) + row));
            const float *tp = a.t + 3 * row;
            const Aff L = aff_from_qt(q, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
            acc = (j == j0) ? L : aff_mul(acc, L);
            sts_aff(Pc + 3 * j, acc);
          }
        }
      }
    }
    __syncthreads();

    // ---- pass 2: pointer jumping over segments
    const float4 *Y = scan_pass2(s, P, cs4, Y0, Y1, C, tid, nth);

    // ---- pass 3: model pose, bind, stage in place
    {
      const int CN = C * n;
      for (int idx = tid; idx < CN; idx += nth) {
        const int c = (int)s.divN.div(idx), j = idx - c * n;
        Aff m = scan_model(s, P, cs4, Y, c, j);
        if (MODEL && SKIN) stg_aff(reinterpret_cast<float4 *>(a.model) + (sOff[c] + j) * 3, m);
        if (SKIN) m = aff_mul(m, ldg_aff(s.T.inv_bind + 3 * j));
        sts_aff(P + c * cs4 + 3 * j, m);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      float *dst = SKIN ? a.skin : a.model;
      const uint32_t bytes = (uint32_t)n * 48u;
      for (int c = 0; c < C; ++c) bulk_store(dst + sOff[c] * 12, P + c * cs4, bytes);
      bulk_commit();
      pending = true;
    }
  }
  if (tid == 0 && pending) bulk_wait_all();
}

template <int MODE, bool SKIN, bool MODEL>
static cudaError_t launch_scan_t(const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  auto k = k_scan<MODE, SKIN, MODEL>;
  static size_t set_smem = 0;  // attribute calls stay out of graph captures after the first launch
  if (cfg.smem > set_smem) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    set_smem = cfg.smem;
  }
  k<<<cfg.ctas, cfg.threads, cfg.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scan(int mode, const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  const bool skin = a.skin != nullptr, model = a.model != nullptr;
  if (mode == 0) return launch_scan_t<0, true, false>(a, cfg, st);
  if (skin && model) return launch_scan_t<1, true, true>(a, cfg, st);
  if (skin) return launch_scan_t<1, true, false>(a, cfg, st);
  return launch_scan_t<1, false, true>(a, cfg, st);
}

// ------------------------------------------------------------ work queue
// One CTA: counting sort of the characters by (type rank, key index k0),
// then the items (at most cap[type] characters sharing type and k0) in
// that order, so the most costly types come first.
constexpr int kBucketThreads = 1024;

__device__ __forceinline__ int key_index(float tm, float rate, int nk, int *status) {
  if (!isfinite(tm)) {
    atomicOr(status, 1);
    return 0;
  }
  const float u = __fmul_rn(tm, rate);
  const int k = (int)floorf(u);
  int m = k % nk;
  return m < 0 ? m + nk : m;
}

// Block-wide exclusive scan of one int per thread; returns the prefix and
// writes the total to *total.
__device__ int block_excl_scan(int v, int *warp_sums, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  const int before = (wid ? warp_sums[wid - 1] : 0) + x - v;
  if (threadIdx.x == blockDim.x - 1) *total = before + v;
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kBucketThreads) k_bucket(const BucketArgs a) {
  __shared__ int s_hist[kMaxBins];
  __shared__ int s_start[kMaxBins];
  __shared__ int s_cursor[kMaxBins];
  __shared__ int s_tbase[kMaxTypes];
  __shared__ int s_warp[32];
  __shared__ int s_nbins, s_total;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int t = tid; t < a.n_types; t += nth) s_tbase[t] = -1;
  __syncthreads();
  if (tid == 0) {
    int base = 0;
    for (int r = 0; r < a.n_used; ++r) {
      const int t = a.used[r];
      s_tbase[t] = base;
      base += a.types[t].n_keys;
    }
    s_nbins = base;
  }
  __syncthreads();
  const int nb = s_nbins;
  for (int b = tid; b < nb; b += nth) {
    s_hist[b] = 0;
    s_cursor[b] = 0;
  }
  __syncthreads();
  for (int64_t c = tid; c < a.n_chars; c += nth) {
    const int t = a.char_type[c];
    const int b = s_tbase[t] + key_index(a.time[c], a.types[t].rate, a.types[t].n_keys, a.status);
    atomicAdd(&s_hist[b], 1);
  }
  __syncthreads();
  // exclusive scan of the histogram: each thread owns a run of bins
  const int per = (nb + nth - 1) / nth;
  const int b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
  int run = 0;
  for (int b = b0; b < b1; ++b) run += s_hist[b];
  int pre = block_excl_scan(run, s_warp, &s_total);
  for (int b = b0; b < b1; ++b) {
    s_start[b] = pre;
    pre += s_hist[b];
  }
  __syncthreads();
  // scatter character ids into their bins
  for (int64_t c = tid; c < a.n_chars; c += nth) {
    const int t = a.char_type[c];
    const int b = s_tbase[t] + key_index(a.time[c], a.types[t].rate, a.types[t].n_keys, a.status);
    const int pos = atomicAdd(&s_cursor[b], 1);
    a.sorted[s_start[b] + pos] = (int32_t)c;
  }
  __syncthreads();  // every scatter is done before s_cursor is reused below
  // items: bin b holds ceil(hist/cap) of them; type of a bin found by rank
  int nit = 0;
  for (int b = b0; b < b1; ++b) {
    int r = 0;
    while (r + 1 < a.n_used && s_tbase[a.used[r + 1]] <= b) ++r;
    const int cap = a.cap[a.used[r]];
    s_cursor[b] = (s_hist[b] + cap - 1) / cap;  // reuse: items of the bin
    nit += s_cursor[b];
  }
  int ipre = block_excl_scan(nit, s_warp, &s_total);
  for (int b = b0; b < b1; ++b) {
    int r = 0;
    while (r + 1 < a.n_used && s_tbase[a.used[r + 1]] <= b) ++r;
    const int t = a.used[r];
    const int cap = a.cap[t];
    const int cnt = s_hist[b];
    for (int k = 0; k < s_cursor[b]; ++k) {
      WorkItem w;
      w.start = s_start[b] + k * cap;
      w.count = min(cap, cnt - k * cap);
      w.type = t;
      w.k0 = b - s_tbase[t];
      a.items[ipre + k] = w;
    }
    ipre += s_cursor[b];
  }
  if (tid == 0) {
    *a.n_items = s_total;
    *a.queue_head = 0;
  }
}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st) {
  k_bucket<<<1, kBucketThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------ setup kernels
// Arc angle between consecutive keys (shorter arc), stored in the pad slot
// of the first key of each pair: theta = 2 atan2(|a - b'|, |a + b'|) with
// b' = +-b on a's hemisphere.  Keys loop, so key n_keys-1 pairs with key 0.
__global__ void k_prepare_keys(float4 *keys, int n_clips, int n_keys, int n) {
  const long long total = (long long)n_clips * n_keys * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i % n);
    const long long ck = i / n;
    const int k = (int)(ck % n_keys), c = (int)(ck / n_keys);
    const int k1 = (k + 1 == n_keys) ? 0 : k + 1;
    const float4 a = keys[2 * i];
    const float4 b = keys[2 * (((long long)c * n_keys + k1) * n + j)];
    const float sg = dot4(a, b) < 0.f ? -1.f : 1.f;
    float dm = 0.f, dp = 0.f, d;
    d = a.x - sg * b.x; dm += d * d; d = a.x + sg * b.x; dp += d * d;
    d = a.y - sg * b.y; dm += d * d; d = a.y + sg * b.y; dp += d * d;
    d = a.z - sg * b.z; dm += d * d; d = a.z + sg * b.z; dp += d * d;
    d = a.w - sg * b.w; dm += d * d; d = a.w + sg * b.w; dp += d * d;
    keys[2 * i + 1].w = 2.f * atan2f(sqrtf(dm), sqrtf(dp));
  }
}

cudaError_t launch_prepare_keys(float4 *keys, int n_clips, int n_keys, int n, cudaStream_t st) {
  const long long total = (long long)n_clips * n_keys * n;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_prepare_keys<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(keys, n_clips, n_keys, n);
  return cudaGetLastError();
}

// Inverse bind poses from a rest pose: thread 0 composes the rest pose down
// the joint list (parent before child) into inv_bind, then every thread
// replaces its model pose [R | t] by the rigid inverse [R^T | -R^T t].
__global__ void k_bind_from_rest(const int32_t *parent, const float *rest_q, const float *rest_t, int n,
                                 float4 *out) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) {
      const float4 q = normalize4(make_float4(rest_q[4 * i], rest_q[4 * i + 1], rest_q[4 * i + 2], rest_q[4 * i + 3]));
      Aff L = aff_from_qt(q, rest_t[3 * i], rest_t[3 * i + 1], rest_t[3 * i + 2]);
      const int p = parent[i];
      if (p >= 0) {
        Aff M;
        M.r0 = out[3 * p];
        M.r1 = out[3 * p + 1];
        M.r2 = out[3 * p + 2];
        L = aff_mul(M, L);
      }
      out[3 * i] = L.r0;
      out[3 * i + 1] = L.r1;
      out[3 * i + 2] = L.r2;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float4 a = out[3 * i], b = out[3 * i + 1], c = out[3 * i + 2];
    // R^T rows are the columns of R
    const float tx = -(a.x * a.w + b.x * b.w + c.x * c.w);
    const float ty = -(a.y * a.w + b.y * b.w + c.y * c.w);
    const float tz = -(a.z * a.w + b.z * b.w + c.z * c.w);
    out[3 * i] = make_float4(a.x, b.x, c.x, tx);
    out[3 * i + 1] = make_float4(a.y, b.y, c.y, ty);
    out[3 * i + 2] = make_float4(a.z, b.z, c.z, tz);
  }
}

cudaError_t launch_bind_from_rest(const int32_t *parent, const float *rest_q, const float *rest_t, int n,
                                  float4 *inv_bind, cudaStream_t st) {
  k_bind_from_rest<<<1, 256, 0, st>>>(parent, rest_q, rest_t, n, inv_bind);
  return cudaGetLastError();
}

}  // namespace anim
