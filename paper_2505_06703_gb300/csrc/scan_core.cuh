// The segmented Hierarchy-Scan shared by the forward and adjoint kernels.
//
// Eq. 1 defines the model pose of joint i as the product of the local
// matrices on the root-to-i path.  The paper evaluates it with one thread per
// joint, pointer jumping and block barriers (Sec. 3, Algs. 2-4).  Here the
// tree is cut into segments (runs of consecutive joints where each joint is
// the parent of the next, at most seg_len long) and the product is formed in
// three passes over a work item of C characters staged in shared memory:
//   pass 1  one lane per (segment, character) walks its segment and writes
//           the running product P_j = L_first ... L_j (work-efficient: one
//           3x4 product per joint);
//   pass 2  pointer jumping over the segment tree (the paper's doubling idea
//           applied to segments instead of joints): Y_g starts as the
//           partial product at the joint the segment hangs from and, after
//           ceil(log2(segment depth)) rounds, is the model pose of that joint;
//   pass 3  one thread per (character, joint): M_j = Y_seg(j) P_j, then the
//           Bind MeshPose product S_j = M_j B_j, written back in place.
#pragma once
#include "anim_internal.h"
#include "dev_math.cuh"

namespace anim {

// Per-item constants staged in shared memory by the kernels.
struct ItemSmem {
  TypeDev T;
  WorkItem wi;
  FastDiv divC, divS, divN;  // by C, by nseg, by n
  int item;
};

__device__ __forceinline__ void load_type_smem(ItemSmem &s, const TypeDev *types, int type, int tid, int nth) {
  const int *src = reinterpret_cast<const int *>(types + type);
  int *dst = reinterpret_cast<int *>(&s.T);
  for (int k = tid; k < (int)(sizeof(TypeDev) / 4); k += nth) dst[k] = src[k];
}

// Pass 2 + its barriers.  Returns the buffer holding the final Y.
__device__ __forceinline__ float4 *scan_pass2(const ItemSmem &s, float4 *P, int cs4, float4 *Y0, float4 *Y1,
                                              int C, int tid, int nth) {
  const int nseg = s.T.nseg;
  const int CS = C * nseg;
  for (int idx = tid; idx < CS; idx += nth) {
    const int c = (int)s.divS.div(idx), g = idx - c * nseg;
    const int lk = __ldg(s.T.seg_link + g);
    const Aff y = lk < 0 ? aff_identity() : lds_aff(P + c * cs4 + 3 * lk);
    sts_aff(Y0 + 3 * idx, y);
  }
  __syncthreads();
  float4 *cur = Y0, *nxt = Y1;
  for (int r = 0; r < s.T.rounds; ++r) {
    const int16_t *jr = s.T.jump + (size_t)r * nseg;
    for (int idx = tid; idx < CS; idx += nth) {
      const int c = (int)s.divS.div(idx), g = idx - c * nseg;
      const int p = __ldg(jr + g);
      Aff y = lds_aff(cur + 3 * idx);
      if (p >= 0) y = aff_mul(lds_aff(cur + 3 * (c * nseg + p)), y);
      sts_aff(nxt + 3 * idx, y);
    }
    __syncthreads();
    float4 *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  return cur;
}

// Model pose of joint j of character c after pass 2 (P holds P_j).
__device__ __forceinline__ Aff scan_model(const ItemSmem &s, const float4 *P, int cs4, const float4 *Y, int c,
                                          int j) {
  Aff m = lds_aff(P + c * cs4 + 3 * j);
  const int g = __ldg(s.T.seg_of + j);
  if (__ldg(s.T.seg_link + g) >= 0) m = aff_mul(lds_aff(Y + 3 * (c * s.T.nseg + g)), m);
  return m;
}

}  // namespace anim
