// The plain comparator: the level-synchronous schedule.  One CTA per
// character, one launch per skeleton type, one thread per joint (strided when
// the type has more joints than threads):
//   phase A  each thread builds its joints' local matrices L_j (sampled from
//            the clips, or from given q, t) in shared memory;
//   phase B  for depth d = 2 .. max depth: a barrier, then the joints at depth
//            d form M_j = M_parent(j) L_j in place (Eq. 1 one tree level at a
//            time; parents are final because they sit one level up);
//   phase C  S_j = M_j B_j (Sec. 1 step 3), stored straight to global memory.
// It does the same Simulation and Bind work as the fused kernel; only the
// schedule of the Hierarchy-Scan differs.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "smem_limit.h"

namespace anim {

constexpr int kLevelMaxPerThread = 2;  // joints per thread (n <= 2048 with 1024 threads)

template <int MODE>
__global__ void __launch_bounds__(1024) k_levelsync(const LevelArgs a) {
  extern __shared__ __align__(16) float4 sm[];
  const TypeDev &T = a.type;
  const int n = T.n;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int cid = a.chars[blockIdx.x];
  const long long off = a.row_off[cid];

  float alpha = 0.f, w = 0.f;
  int k0 = 0, k1 = 0;
  if (MODE == 0) {
    const float tm = a.time[cid];
    if (isfinite(tm)) {
      const float u = __fmul_rn(tm, T.rate);
      const float kf = floorf(u);
      alpha = u - kf;
      int m = ((int)kf) % T.n_keys;
      k0 = m < 0 ? m + T.n_keys : m;
    } else if (tid == 0) {
      atomicOr(a.status, 1);
    }
    k1 = (k0 + 1 == T.n_keys) ? 0 : k0 + 1;
    w = a.blend_w[cid];
  }

  int my_depth[kLevelMaxPerThread], my_parent[kLevelMaxPerThread];
#pragma unroll
  for (int r = 0; r < kLevelMaxPerThread; ++r) {
    const int j = tid + r * nth;
    my_depth[r] = 0;
    my_parent[r] = -1;
    if (j >= n) continue;
    my_depth[r] = __ldg(T.depth + j);
    my_parent[r] = __ldg(T.parent + j);
    float4 q;
    float tx, ty, tz;
    if (MODE == 0) {
      const float4 *KA0 = T.keys + ((size_t)k0 * n + j) * 2;
      const float4 *KA1 = T.keys + ((size_t)k1 * n + j) * 2;
      const float4 qa0 = __ldg(KA0), ta0 = __ldg(KA0 + 1), qa1 = __ldg(KA1), ta1 = __ldg(KA1 + 1);
      q = slerp_pre(qa0, qa1, ta0.w, alpha);
      tx = fmaf(alpha, ta1.x - ta0.x, ta0.x);
      ty = fmaf(alpha, ta1.y - ta0.y, ta0.y);
      tz = fmaf(alpha, ta1.z - ta0.z, ta0.z);
      if (T.n_clips >= 2) {
        const float4 *KB0 = T.keys + ((size_t)(T.n_keys + k0) * n + j) * 2;
        const float4 *KB1 = T.keys + ((size_t)(T.n_keys + k1) * n + j) * 2;
        const float4 qb0 = __ldg(KB0), tb0 = __ldg(KB0 + 1), qb1 = __ldg(KB1), tb1 = __ldg(KB1 + 1);
        const float4 qb = slerp_pre(qb0, qb1, tb0.w, alpha);
        q = slerp_unit(q, qb, w);
        tx = fmaf(w, fmaf(alpha, tb1.x - tb0.x, tb0.x) - tx, tx);
        ty = fmaf(w, fmaf(alpha, tb1.y - tb0.y, tb0.y) - ty, ty);
        tz = fmaf(w, fmaf(alpha, tb1.z - tb0.z, tb0.z) - tz, tz);
      }
    } else {
      const long long row = off + j;
      q = normalize4(__ldg(reinterpret_cast<const float4 *>(a.q) + row));
      tx = __ldg(a.t + 3 * row);
      ty = __ldg(a.t + 3 * row + 1);
      tz = __ldg(a.t + 3 * row + 2);
    }
    sts_aff(sm + 3 * j, aff_from_qt(q, tx, ty, tz));
  }

  for (int d = 2; d <= T.max_depth; ++d) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kLevelMaxPerThread; ++r) {
      if (my_depth[r] == d) {
        const int j = tid + r * nth;
        sts_aff(sm + 3 * j, aff_mul(lds_aff(sm + 3 * my_parent[r]), lds_aff(sm + 3 * j)));
      }
    }
  }
  __syncthreads();

  float4 *out = reinterpret_cast<float4 *>(a.skin) + off * 3;
#pragma unroll
  for (int r = 0; r < kLevelMaxPerThread; ++r) {
    const int j = tid + r * nth;
    if (j < n) stg_aff(out + 3 * j, aff_mul(lds_aff(sm + 3 * j), ldg_aff(T.inv_bind + 3 * j)));
  }
}

cudaError_t launch_levelsync(int mode, const LevelArgs &a, int threads, cudaStream_t st) {
  if (a.n_chars == 0) return cudaSuccess;
  const size_t smem = (size_t)a.type.n * 48;
  static SmemLimit lim[2];
  cudaError_t e =
      ensure_smem_limit(mode == 0 ? (const void *)k_levelsync<0> : (const void *)k_levelsync<1>, lim[mode], smem);
  if (e != cudaSuccess) return e;
  if (mode == 0)
    k_levelsync<0><<<a.n_chars, threads, smem, st>>>(a);
  else
    k_levelsync<1><<<a.n_chars, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace anim
