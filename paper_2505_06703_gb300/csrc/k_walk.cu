// Chain-walk frame kernel: Simulation -> Hierarchy-Scan -> Bind MeshPose
// (Sec. 1 steps 1-3, Eq. 1) for skeleton types whose natural chains can be
// walked parent-first with few idle lanes, and for pure chains.
//
// One CTA is one warp and a persistent worker.  A work item is C = 32 / P
// characters of one type that share the key index k0; lane = (character
// c, schedule slot).  The type's static schedule (built on the host) tells
// each lane which joint it composes at each step, so every lane keeps its
// model pose M in registers while it walks a natural chain:
//   sample L_j from the key records (one 64-byte record per clip: q0, the
//   unit tangent q_perp, t0 with the arc angle, t1 - t0), M = M * L_j (or
//   slot[link] * L_j at a chain start), S_j = M * B_j, stage S_j.
// Branch points (joints that other chains hang from) leave M in a shared
// memory slot for the lane that starts the child chain at a later step.
// The key records and inverse binds are stored in schedule order, so at
// step s the P lanes of a character read P consecutive float4 (one or two
// cache lines per load instruction), and the C characters of an item read
// the same addresses.  Skin rows go out from registers.
//
// Pure chains (mode 2, e.g. a 1,024-joint tail) cannot be walked this way
// without a 1,024-step dependency; they are cut into P pieces: pass A forms
// each piece's product, a warp-shuffle Hillis-Steele scan over the pieces
// gives each piece's parent transform, and pass B walks the piece again
// from it (sampling twice instead of storing every local matrix).
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "smem_limit.h"

namespace anim {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ Rec ld_rec(const float4 *p, int P) {
  Rec r;
  r.q0 = __ldg(p);
  r.qp = __ldg(p + P);
  r.t0 = __ldg(p + 2 * P);
  r.dt = __ldg(p + 3 * P);
  return r;
}

__device__ __forceinline__ Aff ld_bind(const float4 *p, int P) {
  Aff b;
  b.r0 = __ldg(p);
  b.r1 = __ldg(p + P);
  b.r2 = __ldg(p + 2 * P);
  return b;
}


__device__ __forceinline__ Aff shfl_up_aff(const Aff &a, int d, int width) {
  Aff r;
  r.r0 = make_float4(__shfl_up_sync(kFull, a.r0.x, d, width), __shfl_up_sync(kFull, a.r0.y, d, width),
                     __shfl_up_sync(kFull, a.r0.z, d, width), __shfl_up_sync(kFull, a.r0.w, d, width));
  r.r1 = make_float4(__shfl_up_sync(kFull, a.r1.x, d, width), __shfl_up_sync(kFull, a.r1.y, d, width),
                     __shfl_up_sync(kFull, a.r1.z, d, width), __shfl_up_sync(kFull, a.r1.w, d, width));
  r.r2 = make_float4(__shfl_up_sync(kFull, a.r2.x, d, width), __shfl_up_sync(kFull, a.r2.y, d, width),
                     __shfl_up_sync(kFull, a.r2.z, d, width), __shfl_up_sync(kFull, a.r2.w, d, width));
  return r;
}

// The step loop shared by the tree walk (KIND 0) and the two passes of a
// chain split (KIND 1: piece product only, KIND 2: walk from the piece's
// parent transform M0).  Loads of step s + 1 are issued before step s is
// composed.  KIND 0 and 2 store S_j = M_j B_j straight from registers (three
// 16-byte stores; the three land in the same or adjacent sectors, which L2
// merges before write-back).
template <int KIND>
__device__ __forceinline__ Aff walk_steps(const uint32_t *tab, const float4 *ka, const float4 *kb,
                                          const float4 *bb, int P, int S, bool act, bool two, float al,
                                          float w, Aff M, float4 *bsl, float *skin_c) {
  uint32_t e_n = __ldg(tab);
  Rec ra_n = ld_rec(ka, P), rb_n = two ? ld_rec(kb, P) : ra_n;
  Aff b_n;
  if (KIND != 1) b_n = ld_bind(bb, P);
  for (int s = 0; s < S; ++s) {
    const uint32_t e = e_n;
    const Rec ra = ra_n, rb = rb_n;
    const Aff B = b_n;
    if (s + 1 < S) {
      tab += P;
      ka += 4 * P;
      kb += 4 * P;
      e_n = __ldg(tab);
      ra_n = ld_rec(ka, P);
      if (two) rb_n = ld_rec(kb, P);
      if (KIND != 1) {
        bb += 3 * P;
        b_n = ld_bind(bb, P);
      }
    }
    if (act && !(e & 0x80000000u)) {
      const Aff L = sample_rec(ra, rb, al, w, two);
      Aff Mp = M;
      if (KIND == 0 && (e & kWStart)) {
        const uint32_t ls = (e >> kWLoadShift) & 0xFFu;
        Mp = ls == kWRootSlot ? aff_identity() : lds_aff(bsl + ls * 3);
      }
      M = aff_mul(Mp, L);
      if (KIND == 0 && (e & kWStore)) sts_aff(bsl + ((e >> kWStoreShift) & 0xFFu) * 3, M);
      if (KIND != 1) stg_aff(reinterpret_cast<float4 *>(skin_c) + (e & kWJoint) * 3, aff_mul(M, B));
    }
    if (KIND == 0) __syncwarp();  // branch slots written this step are read at later steps
  }
  return M;
}

__global__ void __launch_bounds__(32, 8) k_walk(const WalkArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  const int lane = threadIdx.x;

  int ticket = 0;
  if (lane == 0) ticket = atomicAdd(a.queue_head, 1);
  int it = __shfl_sync(kFull, ticket, 0);
  while (it < a.n_items) {
    if (lane == 0) ticket = atomicAdd(a.queue_head, 1);  // next item, consumed at the end of this one
    const WorkItem wi = a.items[it];
    if (wi.count > 0) {
      const TypeDev &T = a.types[wi.type];
      const int P = T.wk_P, logP = T.wk_logP, S = T.wk_S, nk = T.n_keys;
      const bool two = T.n_clips >= 2;
      const int c = lane >> logP, slot = lane & (P - 1);
      const bool act = c < wi.count;
      float al = 0.f, w = 0.f;
      float *skin_c = a.skin;
      if (act) {
        const int cid = __ldg(a.item_chars + wi.start + c);
        skin_c = a.skin + a.row_off[cid] * 12;
        const float tm = __ldg(a.time + cid);
        if (isfinite(tm)) {
          const float u = __fmul_rn(tm, T.rate);
          al = u - floorf(u);
        } else {
          atomicOr(a.status, 1);
        }
        w = __ldg(a.blend_w + cid);
      }
      const uint32_t *tab = T.wk_tab + slot;
      const float4 *ka = T.wk_keys + (size_t)wi.k0 * S * 4 * P + slot;
      const float4 *kb = two ? ka + (size_t)nk * S * 4 * P : ka;
      const float4 *bb = T.wk_bind + slot;
      float4 *bsl = sm + (size_t)c * a.nbs_max * 3;
      if (T.wk_mode == 1) {
        walk_steps<0>(tab, ka, kb, bb, P, S, act, two, al, w, aff_identity(), bsl, skin_c);
      } else {
        // pass A: product of this lane's piece
        Aff Tp = walk_steps<1>(tab, ka, kb, bb, P, S, act, two, al, w, aff_identity(), bsl, skin_c);
        // inclusive scan over the character's P pieces, then shift by one
        for (int d = 1; d < P; d <<= 1) {
          const Aff X = shfl_up_aff(Tp, d, P);
          if (slot >= d) Tp = aff_mul(X, Tp);
        }
        Aff M0 = shfl_up_aff(Tp, 1, P);
        if (slot == 0) M0 = aff_identity();
        // pass B: walk the piece again from its parent transform
        walk_steps<2>(tab, ka, kb, bb, P, S, act, two, al, w, M0, bsl, skin_c);
      }
      __syncwarp();
    }
    it = __shfl_sync(kFull, ticket, 0);
  }
  if (lane == 0 && a.done) {
    __threadfence();
    if (atomicAdd(a.done, 1) == (int)gridDim.x - 1) {
      *a.queue_head = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}

// Schedule-ordered tables.  Record of (clip, key k, step s, slot): the joint
// j of entry [s][slot]; keys k and k1 = (k + 1) mod n_keys of the clip,
// normalized, b on a's hemisphere; theta = 2 atan2(|a - b|, |a + b|);
// q_perp = (b - (a.b) a) / |b - (a.b) a| (0 when b == a).
__global__ void k_build_walk_keys(const TypeDev T, const float4 *keys, float4 *out) {
  const int P = T.wk_P, S = T.wk_S, n = T.n, nk = T.n_keys;
  const long long total = (long long)T.n_clips * nk * S * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(i % P);
    const long long r = i / P;
    const int s = (int)(r % S);
    const long long ck = r / S;
    const int k = (int)(ck % nk), clip = (int)(ck / nk);
    float4 *o = out + (ck * S + s) * 4 * P + slot;
    const uint32_t e = T.wk_tab[s * P + slot];
    if (e & 0x80000000u) {
      for (int f = 0; f < 4; ++f) o[f * P] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    float4 rec[4];
    make_rec(keys, clip, k, nk, n, (int)(e & kWJoint), rec);
    for (int f = 0; f < 4; ++f) o[f * P] = rec[f];
  }
}

__global__ void k_build_walk_bind(const TypeDev T, float4 *out) {
  const int P = T.wk_P, S = T.wk_S;
  const int total = S * P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int slot = i % P, s = i / P;
    const uint32_t e = T.wk_tab[i];
    float4 *o = out + (size_t)s * 3 * P + slot;
    for (int r = 0; r < 3; ++r)
      o[r * P] = (e & 0x80000000u) ? make_float4(0.f, 0.f, 0.f, 0.f) : T.inv_bind[(e & kWJoint) * 3 + r];
  }
}

}  // namespace

size_t walk_smem_bytes(int chars_per_item, int nbs) {
  const size_t b = 48ull * (size_t)chars_per_item * (size_t)nbs;
  return b > 16 ? b : 16;
}

int walk_blocks_per_sm(size_t smem) {
  int nb = 0;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                              cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk, 32, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_walk(const WalkArgs &a, int ctas, size_t smem, cudaStream_t st) {
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k_walk, lim, smem, 48 * 1024);
  if (e != cudaSuccess) return e;
  k_walk<<<ctas, 32, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_build_walk(const TypeDev &T, const float4 *keys, float4 *wk_keys, float4 *wk_bind,
                              cudaStream_t st) {
  if (T.wk_mode == 0) return cudaSuccess;
  if (wk_bind && T.inv_bind) {
    k_build_walk_bind<<<(T.wk_S * T.wk_P + 255) / 256, 256, 0, st>>>(T, wk_bind);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (wk_keys && keys && T.n_clips > 0) {
    const long long total = (long long)T.n_clips * T.n_keys * T.wk_S * T.wk_P;
    const long long nb = (total + 255) / 256;
    const int blocks = (int)(nb < 4096 ? nb : 4096);
    k_build_walk_keys<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(T, keys, wk_keys);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace anim
