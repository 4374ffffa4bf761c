// Fused frame kernel (Simulation -> Hierarchy-Scan -> Bind MeshPose, Sec. 1
// steps 1-3 and Eq. 1), the per-frame work queue, and setup kernels.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "scan_core.cuh"
#include "smem_limit.h"

#define ANIM_MAX_KEYS_DEV 1024  // keys per clip (ANIM_MAX_KEYS in the ABI)

namespace anim {

size_t scan_smem_bytes(int n, int nseg, int C) { return scan_item_bytes(n, nseg, C); }

// The four key records (keys k0 and k1 of clip 0 and clip 1) of one joint.
struct KeyRecs {
  float4 qa0, ta0, qa1, ta1, qb0, tb0, qb1, tb1;
};

// Simulation stage for one joint: slerp/lerp between the keys of each clip at
// fraction al, then slerp/lerp from clip 0 to clip 1 by w; the local matrix.
__device__ __forceinline__ Aff sample_local(const KeyRecs &r, float al, float w, bool two) {
  float4 q = slerp_pre(r.qa0, r.qa1, r.ta0.w, al);
  float tx = fmaf(al, r.ta1.x - r.ta0.x, r.ta0.x);
  float ty = fmaf(al, r.ta1.y - r.ta0.y, r.ta0.y);
  float tz = fmaf(al, r.ta1.z - r.ta0.z, r.ta0.z);
  if (two) {
    const float4 qb = slerp_pre(r.qb0, r.qb1, r.tb0.w, al);
    const float bx = fmaf(al, r.tb1.x - r.tb0.x, r.tb0.x);
    const float by = fmaf(al, r.tb1.y - r.tb0.y, r.tb0.y);
    const float bz = fmaf(al, r.tb1.z - r.tb0.z, r.tb0.z);
    q = slerp_unit(q, qb, w);
    tx = fmaf(w, bx - tx, tx);
    ty = fmaf(w, by - ty, ty);
    tz = fmaf(w, bz - tz, tz);
  }
  return aff_from_qt(q, tx, ty, tz);
}

// Linear blend skinning of the item's characters: vertex v of character c
// goes to sum_k w_k S_{b_k} [p; 1] with normal normalize(sum_k w_k R_{b_k} n)
// (rigid skin matrices; zero weights skipped), written as 6 floats at the
// character's vertex offset.  Consecutive threads take consecutive vertices.
__device__ __forceinline__ void skin_mesh(const ItemBuf &b, const float4 *P, int cs4, float *verts, int tid) {
  const int nv = b.T.n_verts;
  const float4 *mesh = b.T.mesh;
  for (int c = 0; c < b.C; ++c) {
    const float4 *Sc = P + c * cs4;
    float2 *out = reinterpret_cast<float2 *>(verts + b.voff[c] * 6);
    for (int v = tid; v < nv; v += kComputeThreads) {
      const float4 r0 = __ldg(mesh + 3 * v), r1 = __ldg(mesh + 3 * v + 1), r2 = __ldg(mesh + 3 * v + 2);
      const float w[4] = {r1.z, r1.w, r2.x, r2.y};
      const uint32_t b01 = __float_as_uint(r2.z), b23 = __float_as_uint(r2.w);
      const int bone[4] = {(int)(b01 & 0xFFFFu), (int)(b01 >> 16), (int)(b23 & 0xFFFFu), (int)(b23 >> 16)};
      float px = 0.f, py = 0.f, pz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (w[k] == 0.f) continue;
        const Aff S = lds_aff(Sc + 3 * bone[k]);
        px = fmaf(w[k], fmaf(S.r0.x, r0.x, fmaf(S.r0.y, r0.y, fmaf(S.r0.z, r0.z, S.r0.w))), px);
        py = fmaf(w[k], fmaf(S.r1.x, r0.x, fmaf(S.r1.y, r0.y, fmaf(S.r1.z, r0.z, S.r1.w))), py);
        pz = fmaf(w[k], fmaf(S.r2.x, r0.x, fmaf(S.r2.y, r0.y, fmaf(S.r2.z, r0.z, S.r2.w))), pz);
        nx = fmaf(w[k], fmaf(S.r0.x, r0.w, fmaf(S.r0.y, r1.x, S.r0.z * r1.y)), nx);
        ny = fmaf(w[k], fmaf(S.r1.x, r0.w, fmaf(S.r1.y, r1.x, S.r1.z * r1.y)), ny);
        nz = fmaf(w[k], fmaf(S.r2.x, r0.w, fmaf(S.r2.y, r1.x, S.r2.z * r1.y)), nz);
      }
      const float l2 = nx * nx + ny * ny + nz * nz;
      const float inv = l2 > 0.f ? rsqrtf(l2) : 0.f;
      out[3 * v] = make_float2(px, py);
      out[3 * v + 1] = make_float2(pz, nx * inv);
      out[3 * v + 2] = make_float2(ny * inv, nz * inv);
    }
  }
}

// Persistent frame kernel on 3x4 matrices for the frame with linear blend
// skinning, whose last pass reads the skin matrices from shared memory (the
// other frames and the forward from local poses run on (q, t) items,
// k_scan_qt.cu).  Work item = C characters of one type sharing the key index
// k0, so they read the same key records.  Compute warps run passes 1a/1b/2/3
// and the skinning pass in shared memory and thread 0 streams the finished
// skin-matrix blocks out with bulk copies (when the caller wants them); the
// producer warp stages the next item meanwhile.
template <int MINB>
__global__ void __launch_bounds__(kCtaThreads, MINB) k_scan(const ScanArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemBuf bufs[2];
  const int tid = threadIdx.x;
  const int n_items = a.n_items;

  if (tid >= kComputeThreads) {
    producer_loop<0>(bufs, a.queue_head, n_items, a.items, a.types, a.item_chars, a.row_off, a.time, a.blend_w,
                     a.status, a.vert_off);
    return;
  }

  bool pending = false;  // thread 0: bulk stores in flight
  int cur = 0;
  handoff_sync();
  for (;;) {
    const ItemBuf &b = bufs[cur];
    if (b.item < 0) break;
    const int C = b.C, n = b.T.n, nseg = b.T.nseg;
    const int cs4 = 3 * n + 1;  // float4 stride between characters (16 B skew against bank conflicts)
    const ItemLayout Lt = item_layout(sm, C, n, nseg);
    float4 *P = Lt.P;
    if (tid == 0 && pending) {
      bulk_wait_read_all();  // the staging buffer of the previous item has been read out
      pending = false;
    }
    compute_sync();

    // ---- pass 1a: local matrices of every (joint, character); the type's
    // tables are staged into shared memory alongside
    stage_tables(b, Lt, tid);
    {
      const int nk = b.T.n_keys, k0 = b.k0, k1 = (k0 + 1 == nk) ? 0 : k0 + 1;
      const float4 *KA0 = b.T.keys + (size_t)k0 * n * 2;
      const float4 *KA1 = b.T.keys + (size_t)k1 * n * 2;
      const float4 *KB0 = b.T.keys + (size_t)(nk + k0) * n * 2;
      const float4 *KB1 = b.T.keys + (size_t)(nk + k1) * n * 2;
      const bool two = b.T.n_clips >= 2;
      const int CN = C * n;
#pragma unroll 2
      for (int idx = tid; idx < CN; idx += kComputeThreads) {
        const int j = (int)b.divC.div(idx), c = idx - j * C;  // character-minor: lanes share key records
        KeyRecs r;
        r.qa0 = __ldg(KA0 + 2 * j);
        r.ta0 = __ldg(KA0 + 2 * j + 1);
        r.qa1 = __ldg(KA1 + 2 * j);
        r.ta1 = __ldg(KA1 + 2 * j + 1);
        if (two) {
          r.qb0 = __ldg(KB0 + 2 * j);
          r.tb0 = __ldg(KB0 + 2 * j + 1);
          r.qb1 = __ldg(KB1 + 2 * j);
          r.tb1 = __ldg(KB1 + 2 * j + 1);
        }
        sts_aff(P + c * cs4 + 3 * j, sample_local(r, b.alpha[c], b.blend[c], two));
      }
    }
    cp_async_wait_all();  // this thread's table copies (stage_tables)
    compute_sync();

    // ---- pass 1b: running products along segments
    pass1b(b, Lt, P, cs4, tid);
    compute_sync();
    // ---- pass 2: pointer jumping over segments
    const float4 *Y = pass2(b, Lt, P, cs4, tid);

    // ---- pass 3: model pose, bind, stage in place
    {
      const int W = n * b.cgroups, cpt = b.cpt;
      for (int idx = tid; idx < W; idx += kComputeThreads) {
        const int grp = (int)b.divN.div(idx), j = idx - grp * n;
        const uint32_t info = Lt.jinfo[j];
        const int g = (int)(info & kJ16Seg);
        const Aff B = ldg_aff(b.T.inv_bind + 3 * j);
        const int c1 = min(C, (grp + 1) * cpt);
        for (int c = grp * cpt; c < c1; ++c) {
          float4 *slot = P + c * cs4 + 3 * j;
          Aff m = lds_aff(slot);
          if (info & kJ16Link) m = aff_mul(lds_aff(Y + 3 * (c * nseg + g)), m);
          sts_aff(slot, aff_mul(m, B));
        }
      }
    }
    fence_proxy_async_smem();
    compute_sync();
    float *dst = a.skin;  // NULL: the skinned frame keeps the skin matrices on chip
    if (tid == 0 && dst) {
      const uint32_t bytes = (uint32_t)n * 48u;
      for (int c = 0; c < C; ++c) bulk_store(dst + b.off[c] * 12, P + c * cs4, bytes);
      bulk_commit();
      pending = true;
    }
    // ---- pass 4 (frame with skinning): linear blend skinning of the
    // characters' meshes from the skin matrices still in shared memory
    skin_mesh(b, P, cs4, a.verts, tid);
    cur ^= 1;
    handoff_sync();
  }
  if (tid == 0 && pending) bulk_wait_all();
  if (tid == 0 && a.done) last_cta_reset(a.queue_head, a.done);
}

template <int MINB>
static cudaError_t launch_scan_t(const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  auto k = k_scan<MINB>;
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k, lim, cfg.smem);
  if (e != cudaSuccess) return e;
  k<<<cfg.ctas, cfg.threads, cfg.smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scan(const ScanArgs &a, const LaunchCfg &cfg, cudaStream_t st) {
  if (!a.verts) return cudaErrorInvalidValue;  // the other frames run on k_scan_qt
  return cfg.min_blocks >= 3 ? launch_scan_t<3>(a, cfg, st) : launch_scan_t<2>(a, cfg, st);
}

// ------------------------------------------------------------ work queue
constexpr int kBucketThreads = 256;
constexpr int kBucketPer = kRangeCharsMax / kBucketThreads;  // characters per thread
static_assert(kBucketPer * kBucketThreads == kRangeCharsMax, "range size");

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

// One CTA per range of <= kRangeCharsMax characters of one type: counting sort
// by key index k0 in shared memory, items of <= cap characters per (k0) bin
// written to the range's slot region, and empty items (count 0) in the
// region's remaining slots.  Regions are laid out in range order (types most
// costly first); the persistent kernel's producer warp skips empty slots.
__global__ void __launch_bounds__(kBucketThreads) k_bucket(const BucketArgs a) {
  __shared__ int s_hist[ANIM_MAX_KEYS_DEV];
  __shared__ int s_start[ANIM_MAX_KEYS_DEV];
  __shared__ int s_istart[ANIM_MAX_KEYS_DEV];
  __shared__ int s_warp[32];
  __shared__ int s_total, s_itotal;
  const int tid = threadIdx.x, nth = blockDim.x;
  // a frame kernel launched after this one with programmatic stream
  // serialization may start now; it waits for this grid's completion (and
  // its memory) in griddepcontrol.wait before reading the queue
  asm volatile("griddepcontrol.launch_dependents;");
  // launched the same way after the previous frame's kernel: the plan's
  // tables are read before waiting for it, the times (which the preceding
  // kernel may have written) and every write of this grid after
  const RangeDev R = a.ranges[blockIdx.x];
  const int nk = a.types[R.type].n_keys;
  const float rate = a.types[R.type].rate;
  const int cap = a.cap[R.type];
  const int region_end = (blockIdx.x + 1 < a.n_ranges) ? a.ranges[blockIdx.x + 1].region : a.n_slots;
  for (int b = tid; b < nk; b += nth) s_hist[b] = 0;
  int cid[kBucketPer], k[kBucketPer], pos[kBucketPer];
#pragma unroll
  for (int m = 0; m < kBucketPer; ++m) {
    const int i = tid + m * nth;
    cid[m] = i < R.count ? __ldg(a.type_chars + R.start + i) : -1;
    k[m] = 0;
    pos[m] = 0;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (blockIdx.x == 0 && tid == 0) *a.queue_head = 0;  // consumed by the next launch in stream order
  __syncthreads();
#pragma unroll
  for (int m = 0; m < kBucketPer; ++m)
    if (cid[m] >= 0) {
      k[m] = key_index(a.time[cid[m]], rate, nk, a.status);
      pos[m] = atomicAdd(&s_hist[k[m]], 1);  // rank inside the bin
    }
  __syncthreads();
  // exclusive scans over the bins: character starts and item starts (one
  // warp's shuffles when the bins fit in a warp, else block-wide)
  const int per = (nk + nth - 1) / nth;
  const int b0 = min(nk, tid * per), b1 = min(nk, b0 + per);
  if (nk <= 32) {
    if (tid < 32) {
      const int h = tid < nk ? s_hist[tid] : 0, ih = (h + cap - 1) / cap;
      int x = h, ix = ih;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o), iy = __shfl_up_sync(0xffffffffu, ix, o);
        if (tid >= o) {
          x += y;
          ix += iy;
        }
      }
      if (tid < nk) {
        s_start[tid] = x - h;
        s_istart[tid] = ix - ih;
      }
      if (tid == 31) s_itotal = ix;
    }
  } else {
    int run = 0, irun = 0;
    for (int b = b0; b < b1; ++b) {
      run += s_hist[b];
      irun += (s_hist[b] + cap - 1) / cap;
    }
    int pre = block_excl_scan(run, s_warp, &s_total);
    int ipre = block_excl_scan(irun, s_warp, &s_itotal);
    for (int b = b0; b < b1; ++b) {
      s_start[b] = pre;
      s_istart[b] = ipre;
      pre += s_hist[b];
      ipre += (s_hist[b] + cap - 1) / cap;
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < kBucketPer; ++m)
    if (cid[m] >= 0) a.sorted[R.start + s_start[k[m]] + pos[m]] = cid[m];
  for (int b = b0; b < b1; ++b) {
    const int cnt = s_hist[b];
    for (int m = 0; m * cap < cnt; ++m) {
      WorkItem w;
      w.start = R.start + s_start[b] + m * cap;
      w.count = min(cap, cnt - m * cap);
      w.type = R.type;
      w.k0 = b;
      a.items[R.region + s_istart[b] + m] = w;
    }
  }
  const WorkItem empty = {0, 0, R.type, 0};
  for (int sl = R.region + s_itotal + tid; sl < region_end; sl += nth) a.items[sl] = empty;
}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t st) {
  if (a.n_ranges == 0) return cudaSuccess;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)a.n_ranges);
  lc.blockDim = dim3((unsigned)kBucketThreads);
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, k_bucket, a);
}

// ------------------------------------------------------------ setup kernels
// Arc angle between consecutive keys (shorter arc), stored in the pad slot
// of the first key of each pair: theta = 2 atan2(|a - b'|, |a + b'|) with
// b' = +-b on a's hemisphere, carrying the sign of that choice (slerp_pre).
// Keys loop, so key n_keys-1 pairs with key 0.
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
    keys[2 * i + 1].w = copysignf(2.f * atan2f(sqrtf(dm), sqrtf(dp)), sg);  // the sign: b's hemisphere
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
