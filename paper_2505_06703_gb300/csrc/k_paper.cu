// The paper's own Hierarchy-Scan schedules as GPU kernels, kept as
// comparators for the segmented scan: one CTA per character, one thread per
// joint (looping when the CTA is smaller), local and partial matrices in
// shared memory, a block barrier between phases.  Readings of the printed
// listings (the same ones the CPU emulations in the tests follow):
//   Alg. 1 (Sec. 2, the per-joint walk of earlier GPU skinning work): each
//     joint's thread walks to the root multiplying the ancestors' local
//     matrices; no barrier after the local matrices.
//   Alg. 2 (Sec. 3.1, Eq. 2): pointer doubling over joints; round d
//     multiplies by the 2^(d-1)-th ancestor's running product, double
//     buffered, ceil(log2 depth) rounds with a barrier each.
//   Alg. 3 (Sec. 3.2.1): joints cut into 64-node blocks by index; 6 rounds of
//     doubling over in-block parents, then each thread walks the chain of
//     nearest out-of-block ancestors multiplying their in-block partials.
//   Alg. 4 (Sec. 3.2.2): a joint and up to 7 in-block ancestors serially,
//     barrier, up to 7 jumps of stride 8 over those partials, barrier, then
//     the out-of-block walk of Alg. 3.
//   KIYA's scheme (Sec. 2, described in words only; numbered 5 here): threads
//     for the leaf joints only; each leaf's thread records its root path,
//     then composes down it, writing the model pose of every joint on the
//     path (ancestors shared by several leaves are written with equal
//     values by each of them).
// Then the Bind MeshPose product S_j = M_j B_j, stored from registers.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"
#include "smem_limit.h"

namespace anim {

namespace {

constexpr int kBlock = 64;  // the paper's node-block size (Algs. 3, 4)
constexpr int kComp = 8;    // Alg. 4 compression stride

__device__ __forceinline__ int inblock_parent(const int32_t *par, int j) {
  const int p = __ldg(par + j);
  return (p >= 0 && p / kBlock == j / kBlock) ? p : -1;
}

__global__ void k_paper(const PaperArgs a) {
  extern __shared__ __align__(16) float4 sm[];
  const int c = blockIdx.x;
  const TypeDev &T = a.types[a.char_type[c]];
  const int n = T.n;
  const long long off = a.row_off[c];
  const int tid = threadIdx.x, nt = blockDim.x;
  float4 *Lm = sm;              // [n][3] local matrices
  float4 *M0 = Lm + 3 * n;      // [n][3] buffer 0
  float4 *M1 = M0 + 3 * n;      // [n][3] buffer 1
  int16_t *p0 = reinterpret_cast<int16_t *>(M1 + 3 * n), *p1 = p0 + n;
  const int32_t *par = T.parent;

  const float4 *q4 = reinterpret_cast<const float4 *>(a.q);
  for (int j = tid; j < n; j += nt) {
    const float4 q = normalize4(__ldg(q4 + off + j));
    const float *tp = a.t + 3 * (off + j);
    sts_aff(Lm + 3 * j, aff_from_qt(q, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2)));
  }
  __syncthreads();

  const float4 *R = M0;  // the buffer holding the model poses at the end
  if (a.algo == 5) {
    // leaves: joints no other joint names as parent (flags in p0)
    for (int j = tid; j < n; j += nt) p0[j] = 0;
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      const int p = __ldg(par + j);
      if (p >= 0) p0[p] = 1;
    }
    __syncthreads();
    int16_t path[kPaperMaxJoints];  // root path of the leaf (local memory)
    for (int j = tid; j < n; j += nt) {
      if (p0[j]) continue;
      int d = 0;
      for (int u = j; u >= 0; u = __ldg(par + u)) path[d++] = (int16_t)u;
      Aff m = lds_aff(Lm + 3 * path[d - 1]);
      sts_aff(M0 + 3 * path[d - 1], m);
      for (int k = d - 2; k >= 0; --k) {
        m = aff_mul(m, lds_aff(Lm + 3 * path[k]));
        sts_aff(M0 + 3 * path[k], m);
      }
    }
  } else if (a.algo == 1) {
    for (int j = tid; j < n; j += nt) {
      Aff m = lds_aff(Lm + 3 * j);
      for (int p = __ldg(par + j); p >= 0; p = __ldg(par + p)) m = aff_mul(lds_aff(Lm + 3 * p), m);
      sts_aff(M0 + 3 * j, m);
    }
  } else if (a.algo == 2) {
    for (int j = tid; j < n; j += nt) {
      sts_aff(M0 + 3 * j, lds_aff(Lm + 3 * j));
      p0[j] = (int16_t)__ldg(par + j);
    }
    __syncthreads();
    int rounds = 0;
    while ((1 << rounds) < T.max_depth) ++rounds;
    float4 *cur = M0, *nxt = M1;
    int16_t *pc = p0, *pn = p1;
    for (int r = 0; r < rounds; ++r) {
      for (int j = tid; j < n; j += nt) {
        const int p = pc[j];
        Aff m = lds_aff(cur + 3 * j);
        if (p >= 0) m = aff_mul(lds_aff(cur + 3 * p), m);
        sts_aff(nxt + 3 * j, m);
        pn[j] = (int16_t)(p >= 0 ? pc[p] : -1);
      }
      __syncthreads();
      float4 *tm = cur;
      cur = nxt;
      nxt = tm;
      int16_t *tp = pc;
      pc = pn;
      pn = tp;
    }
    R = cur;
  } else {
    // in-block partial products into M0 (Alg. 3: doubling; Alg. 4: compressed)
    float4 *part = M0, *other = M1;
    if (a.algo == 3) {
      for (int j = tid; j < n; j += nt) {
        sts_aff(M0 + 3 * j, lds_aff(Lm + 3 * j));
        p0[j] = (int16_t)inblock_parent(par, j);
      }
      __syncthreads();
      float4 *cur = M0, *nxt = M1;
      int16_t *pc = p0, *pn = p1;
      for (int r = 0; (1 << r) < kBlock; ++r) {
        for (int j = tid; j < n; j += nt) {
          const int p = pc[j];
          Aff m = lds_aff(cur + 3 * j);
          if (p >= 0) m = aff_mul(lds_aff(cur + 3 * p), m);
          sts_aff(nxt + 3 * j, m);
          pn[j] = (int16_t)(p >= 0 ? pc[p] : -1);
        }
        __syncthreads();
        float4 *tm = cur;
        cur = nxt;
        nxt = tm;
        int16_t *tp = pc;
        pc = pn;
        pn = tp;
      }
      part = cur;
      other = nxt;
    } else {
      for (int j = tid; j < n; j += nt) {
        Aff m = lds_aff(Lm + 3 * j);
        int p = inblock_parent(par, j);
        for (int k = 0; p >= 0 && k < kComp - 1; ++k) {
          m = aff_mul(lds_aff(Lm + 3 * p), m);
          p = inblock_parent(par, p);
        }
        sts_aff(M1 + 3 * j, m);
        p0[j] = (int16_t)p;  // the in-block ancestor kComp levels up
      }
      __syncthreads();
      for (int j = tid; j < n; j += nt) {
        Aff m = lds_aff(M1 + 3 * j);
        int p = p0[j];
        for (int k = 0; p >= 0 && k < kComp - 1; ++k) {
          m = aff_mul(lds_aff(M1 + 3 * p), m);
          p = p0[p];
        }
        sts_aff(M0 + 3 * j, m);
      }
      part = M0;
      other = M1;
    }
    __syncthreads();
    // out-of-block walk over the nearest out-of-block ancestors' partials
    for (int j = tid; j < n; j += nt) {
      Aff m = lds_aff(part + 3 * j);
      for (int p = __ldg(T.blk_out + j); p >= 0; p = __ldg(T.blk_out + p)) m = aff_mul(lds_aff(part + 3 * p), m);
      sts_aff(other + 3 * j, m);
    }
    R = other;
  }
  __syncthreads();

  // Bind MeshPose, stored from registers
  float4 *dst = reinterpret_cast<float4 *>(a.skin) + off * 3;
  for (int j = tid; j < n; j += nt) stg_aff(dst + 3 * j, aff_mul(lds_aff(R + 3 * j), ldg_aff(T.inv_bind + 3 * j)));
}

}  // namespace

size_t paper_smem_bytes(int n) { return 3ull * 48ull * n + 4ull * n + 16; }

cudaError_t launch_paper(const PaperArgs &a, int n_chars, int threads, size_t smem, cudaStream_t st) {
  static SmemLimit lim;
  cudaError_t e = ensure_smem_limit((const void *)k_paper, lim, smem, 48 * 1024);
  if (e != cudaSuccess) return e;
  k_paper<<<n_chars, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace anim
