// Device helpers: 3x4 affine transforms, quaternions, slerp, fast integer
// division, and the bulk-copy (TMA, non-tensor) PTX used to stream skin
// matrices out of shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace anim {

// A 3x4 row-major affine [R | t] held as three float4 rows.
struct Aff {
  float4 r0, r1, r2;
};

__device__ __forceinline__ Aff aff_identity() {
  Aff a;
  a.r0 = make_float4(1.f, 0.f, 0.f, 0.f);
  a.r1 = make_float4(0.f, 1.f, 0.f, 0.f);
  a.r2 = make_float4(0.f, 0.f, 1.f, 0.f);
  return a;
}

// One output row of A*B: row = a.x*B.r0 + a.y*B.r1 + a.z*B.r2 + (0,0,0,a.w).
__device__ __forceinline__ float4 aff_row(const float4 a, const Aff &B) {
  float4 r;
  r.x = fmaf(a.x, B.r0.x, fmaf(a.y, B.r1.x, a.z * B.r2.x));
  r.y = fmaf(a.x, B.r0.y, fmaf(a.y, B.r1.y, a.z * B.r2.y));
  r.z = fmaf(a.x, B.r0.z, fmaf(a.y, B.r1.z, a.z * B.r2.z));
  r.w = fmaf(a.x, B.r0.w, fmaf(a.y, B.r1.w, fmaf(a.z, B.r2.w, a.w)));
  return r;
}

// Product of 3x4 affines (as 4x4 with last row 0 0 0 1): C = A B.
__device__ __forceinline__ Aff aff_mul(const Aff &A, const Aff &B) {
  Aff C;
  C.r0 = aff_row(A.r0, B);
  C.r1 = aff_row(A.r1, B);
  C.r2 = aff_row(A.r2, B);
  return C;
}

// L = [R(q) | t] for a unit quaternion q = (x, y, z, w).
__device__ __forceinline__ Aff aff_from_qt(const float4 q, const float tx, const float ty, const float tz) {
  const float x2 = q.x + q.x, y2 = q.y + q.y, z2 = q.z + q.z;
  const float xx = q.x * x2, yy = q.y * y2, zz = q.z * z2;
  const float xy = q.x * y2, xz = q.x * z2, yz = q.y * z2;
  const float wx = q.w * x2, wy = q.w * y2, wz = q.w * z2;
  Aff a;
  a.r0 = make_float4(1.f - (yy + zz), xy - wz, xz + wy, tx);
  a.r1 = make_float4(xy + wz, 1.f - (xx + zz), yz - wx, ty);
  a.r2 = make_float4(xz - wy, yz + wx, 1.f - (xx + yy), tz);
  return a;
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

__device__ __forceinline__ float4 normalize4(const float4 a) {
  const float s = rsqrtf(dot4(a, a));
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}

// Weighted sum w0*a + w1*b followed by normalization.
__device__ __forceinline__ float4 combine_norm(const float4 a, const float4 b, const float w0, const float w1) {
  float4 r;
  r.x = fmaf(w0, a.x, w1 * b.x);
  r.y = fmaf(w0, a.y, w1 * b.y);
  r.z = fmaf(w0, a.z, w1 * b.z);
  r.w = fmaf(w0, a.w, w1 * b.w);
  return normalize4(r);
}

// Slerp between adjacent keys whose signed arc angle was computed once at
// upload: |theta_s| is the angle of the shorter arc (in [0, pi/2]) and its
// sign bit is set when b lies on the other hemisphere (dot(a, b) < 0), so b
// enters negated.  The 1/sin(theta) factor of the slerp weights is dropped
// because the result is normalized; below theta = 1e-6 the weights fall
// back to (1 - alpha, alpha).
__device__ __forceinline__ float4 slerp_pre(const float4 a, const float4 b, const float theta_s, const float alpha) {
  const float theta = fabsf(theta_s), sgn = copysignf(1.f, theta_s);
  float w0, w1;
  if (theta > 1e-6f) {
    w0 = __sinf((1.f - alpha) * theta);
    w1 = __sinf(alpha * theta);
  } else {
    w0 = 1.f - alpha;
    w1 = alpha;
  }
  return combine_norm(a, b, w0, w1 * sgn);
}

// Slerp between two unit quaternions (shorter arc); angle from acos of the
// clamped |dot|.
__device__ __forceinline__ float4 slerp_unit(const float4 a, const float4 b, const float alpha) {
  const float d = dot4(a, b);
  const float sgn = d < 0.f ? -1.f : 1.f;
  const float ad = fminf(fabsf(d), 1.f);
  const float theta = acosf(ad);
  float w0, w1;
  if (theta > 1e-6f) {
    w0 = __sinf((1.f - alpha) * theta);
    w1 = __sinf(alpha * theta);
  } else {
    w0 = 1.f - alpha;
    w1 = alpha;
  }
  return combine_norm(a, b, w0, w1 * sgn);
}

// atan2(y, x) for y, x >= 0 (the first quadrant), branch-free: with
// t = min / max in [0, 1], atan(t) = t P(t^2) for a degree-7 polynomial P
// fitted here to minimize the maximum error on [0, 1] (Lawson's iteratively
// reweighted least squares on Chebyshev points; approximation error 4e-8,
// about 1.3e-7 rad with float evaluation), then pi/2 - atan(t) when y > x.
// Straight-line code, so the compiler can interleave several samples.
__device__ __forceinline__ float atan2_q1(const float y, const float x) {
  const float lo = fminf(x, y), hi = fmaxf(fmaxf(x, y), 1e-30f);
  const float t = __fdividef(lo, hi), u = t * t;
  float p = -0.004054560791701078f;
  p = fmaf(p, u, 0.0218629352748394f);
  p = fmaf(p, u, -0.05591229721903801f);
  p = fmaf(p, u, 0.09642194956541061f);
  p = fmaf(p, u, -0.1390862911939621f);
  p = fmaf(p, u, 0.19946566224098206f);
  p = fmaf(p, u, -0.33329859375953674f);
  p = fmaf(p, u, 0.9999993443489075f);
  const float a = t * p;
  return y > x ? 1.5707963267948966f - a : a;
}

// Slerp on the shorter arc between unit quaternions a and b at weight w:
// with d = a.b, v = sign(d) b - |d| a (orthogonal to a, |v| = sin(theta)),
// theta = atan2(|v|, |d|), the result is cos(w theta) a + sin(w theta) v/|v|.
// For v = 0 (equal rotations) theta = 0 and the result is a.
__device__ __forceinline__ float4 blend_unit(const float4 a, const float4 b, const float w) {
  const float d = dot4(a, b);
  const float sg = d < 0.f ? -1.f : 1.f, x = fabsf(d);
  const float4 v = make_float4(fmaf(sg, b.x, -x * a.x), fmaf(sg, b.y, -x * a.y), fmaf(sg, b.z, -x * a.z),
                               fmaf(sg, b.w, -x * a.w));
  const float vv = fmaxf(dot4(v, v), 1e-36f);
  const float rs = rsqrtf(vv);
  const float th = atan2_q1(vv * rs, x);
  float s, c;
  __sincosf(w * th, &s, &c);
  const float k = s * rs;
  return make_float4(fmaf(c, a.x, k * v.x), fmaf(c, a.y, k * v.y), fmaf(c, a.z, k * v.z), fmaf(c, a.w, k * v.w));
}

// Key slerp from a key-pair record held in registers: cos(a theta) q0 +
// sin(a theta) q_perp (q0, q_perp orthonormal; theta in t0.w), translation
// t0 + a dt.
__device__ __forceinline__ void rec_eval(const float4 q0, const float4 qp, const float4 t0, const float4 dt,
                                         const float al, float4 &q, float3 &t) {
  float s, c;
  __sincosf(al * t0.w, &s, &c);
  q = make_float4(fmaf(c, q0.x, s * qp.x), fmaf(c, q0.y, s * qp.y), fmaf(c, q0.z, s * qp.z), fmaf(c, q0.w, s * qp.w));
  t = make_float3(fmaf(al, dt.x, t0.x), fmaf(al, dt.y, t0.y), fmaf(al, dt.z, t0.z));
}

// Hamilton product a (x) b, quaternions stored (x, y, z, w).
__device__ __forceinline__ float4 qmul(const float4 a, const float4 b) {
  float4 r;
  r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  return r;
}

// Shared-memory float4 row access of an Aff stored as 3 consecutive float4.
__device__ __forceinline__ Aff lds_aff(const float4 *p) {
  Aff a;
  a.r0 = p[0];
  a.r1 = p[1];
  a.r2 = p[2];
  return a;
}
__device__ __forceinline__ void sts_aff(float4 *p, const Aff &a) {
  p[0] = a.r0;
  p[1] = a.r1;
  p[2] = a.r2;
}
__device__ __forceinline__ Aff ldg_aff(const float4 *p) {
  Aff a;
  a.r0 = __ldg(p);
  a.r1 = __ldg(p + 1);
  a.r2 = __ldg(p + 2);
  return a;
}
__device__ __forceinline__ void stg_aff(float4 *p, const Aff &a) {
  p[0] = a.r0;
  p[1] = a.r1;
  p[2] = a.r2;
}

// Division by a runtime divisor d >= 1 for numerators below 2^31
// (multiply-high method: q = (umulhi(x, m) + x) >> s).
struct FastDiv {
  uint32_t d, m, s;
  __host__ __device__ void init(uint32_t dd) {
    d = dd;
    s = 0;
    while ((1u << s) < dd) ++s;
    const uint64_t two32 = 1ull << 32;
    m = (uint32_t)((two32 * ((1ull << s) - dd)) / dd + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t x) const { return (__umulhi(x, m) + x) >> s; }
};

// ---- key-pair records (built once per clip upload from the raw keys)
// Record of (clip, key k, joint j): keys k and k1 = (k + 1) mod n_keys of
// the clip, normalized, b on a's hemisphere; theta = 2 atan2(|a - b|,
// |a + b|); q_perp = (b - (a.b) a) / |b - (a.b) a| (0 when b == a); so the
// slerp at fraction al is cos(al theta) a + sin(al theta) q_perp.
//   r[0] = a, r[1] = q_perp, r[2] = (t_k, theta), r[3] = (t_k1 - t_k, 0).
// keys: [clip][key][n][2] float4 (q xyzw, t xyz + pad).
__device__ __forceinline__ void make_rec(const float4 *keys, int clip, int k, int nk, int n, int j, float4 *r) {
  const int k1 = (k + 1 == nk) ? 0 : k + 1;
  const float4 *ra = keys + (((size_t)clip * nk + k) * n + j) * 2;
  const float4 *rb = keys + (((size_t)clip * nk + k1) * n + j) * 2;
  const float4 qa = normalize4(ra[0]);
  float4 qb = normalize4(rb[0]);
  const float d = dot4(qa, qb);
  if (d < 0.f) qb = make_float4(-qb.x, -qb.y, -qb.z, -qb.w);
  const float ad = fabsf(d);
  float dm = 0.f, dp = 0.f, t;
  t = qa.x - qb.x; dm += t * t; t = qa.x + qb.x; dp += t * t;
  t = qa.y - qb.y; dm += t * t; t = qa.y + qb.y; dp += t * t;
  t = qa.z - qb.z; dm += t * t; t = qa.z + qb.z; dp += t * t;
  t = qa.w - qb.w; dm += t * t; t = qa.w + qb.w; dp += t * t;
  const float theta = 2.f * atan2f(sqrtf(dm), sqrtf(dp));
  float4 v = make_float4(qb.x - ad * qa.x, qb.y - ad * qa.y, qb.z - ad * qa.z, qb.w - ad * qa.w);
  const float nv = sqrtf(dot4(v, v));
  v = nv > 0.f ? make_float4(v.x / nv, v.y / nv, v.z / nv, v.w / nv) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 ta = ra[1], tb = rb[1];
  r[0] = qa;
  r[1] = v;
  r[2] = make_float4(ta.x, ta.y, ta.z, theta);
  r[3] = make_float4(tb.x - ta.x, tb.y - ta.y, tb.z - ta.z, 0.f);
}

struct Rec {
  float4 q0, qp, t0, dt;
};

// Key slerp from a precomputed record: cos(a theta) q0 + sin(a theta) q_perp,
// which equals the normalized slerp between the two unit keys; lerp for t.
__device__ __forceinline__ float4 rec_q(const Rec &r, float al) {
  float s, c;
  __sincosf(al * r.t0.w, &s, &c);
  return make_float4(fmaf(c, r.q0.x, s * r.qp.x), fmaf(c, r.q0.y, s * r.qp.y), fmaf(c, r.q0.z, s * r.qp.z),
                     fmaf(c, r.q0.w, s * r.qp.w));
}

__device__ __forceinline__ Aff sample_rec(const Rec &a, const Rec &b, float al, float w, bool two) {
  float4 q = rec_q(a, al);
  float tx = fmaf(al, a.dt.x, a.t0.x), ty = fmaf(al, a.dt.y, a.t0.y), tz = fmaf(al, a.dt.z, a.t0.z);
  if (two) {
    const float4 qb = rec_q(b, al);
    const float bx = fmaf(al, b.dt.x, b.t0.x), by = fmaf(al, b.dt.y, b.t0.y), bz = fmaf(al, b.dt.z, b.t0.z);
    q = slerp_unit(q, qb, w);
    tx = fmaf(w, bx - tx, tx);
    ty = fmaf(w, by - ty, ty);
    tz = fmaf(w, bz - tz, tz);
  }
  return aff_from_qt(q, tx, ty, tz);
}

// ---- bulk copy shared -> global (cp.async.bulk, bulk-group completion)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(s), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace anim
