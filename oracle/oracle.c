/*
 * FP64 CPU oracle for the skeletal-animation hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is written from the
 * paper's definitions in the plainest form: sequential loops, fp64
 * arithmetic, no blocking, fusion or reordering.
 *
 * Stages (Section 1 of the paper lists them as Simulation, Hierarchy-Scan and
 * Bind MeshPose):
 *   1. Simulation (Sec. 1 step 1, Sec. 2): per joint, sample two keyframes
 *      of each clip, interpolate (slerp for rotations, lerp for
 *      translations), then blend the two clips the same way.
 *   2. Hierarchy-Scan (Sec. 1 step 2, Eq. 1): the model pose of joint i is
 *      the product of local matrices along the root-to-i path.  Because the
 *      joint list is topologically ordered (parent index < child index,
 *      Sec. 3.2.1), one pass in index order computes it: M_i = M_parent(i) L_i.
 *   3. Bind MeshPose (Sec. 1 step 3): S_i = M_i B_i with B_i the inverse bind
 *      pose.
 *
 * Conventions (the paper fixes none of them): column vectors, quaternions
 * stored (x, y, z, w), 3x4 row-major affine matrices [R | t] standing for the
 * 4x4 matrix with last row (0 0 0 1).
 *
 * Beyond the paper (its stated extensions of the path):
 *   * the gradient of a loss on model-space joint positions with respect to
 *     the local quaternions (unnormalized 4-vectors) and translations,
 *     computed by a generic reverse pass over 4x4 matrix products
 *     (oracle_grad) and, independently, by subtree force/moment sums
 *     (oracle_grad_force_moment);
 *   * Adam as PyTorch defines it, and batched IK built from the two.
 *
 * Where the paper is silent the readings are: slerp with the shortest-arc
 * sign flip and the angle from 2*atan2(|a-b|, |a+b|); 30 Hz looping keys with
 * key index floor(time*rate) taken in float32 exactly as the GPU takes it
 * (the one place floating point decides an integer); translations lerped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small fp64 helpers                                                  */
/* ------------------------------------------------------------------ */

/* Rotation matrix of a unit quaternion (x, y, z, w), column-vector form. */
static void quat_to_rot(const double q[4], double R[9]) {
  double x = q[0], y = q[1], z = q[2], w = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
  R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
  R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

/* C = A B for 3x4 affine matrices (as 4x4 with last row 0 0 0 1). */
static void affine_mul(const double *A, const double *B, double *C) {
  double T[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += A[r * 4 + k] * B[k * 4 + c];
      if (c == 3) s += A[r * 4 + 3];
      T[r * 4 + c] = s;
    }
  }
  memcpy(C, T, sizeof T);
}

/* 4x4 product of full matrices. */
static void mat4_mul(const double *A, const double *B, double *C) {
  double T[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += A[r * 4 + k] * B[k * 4 + c];
      T[r * 4 + c] = s;
    }
  memcpy(C, T, sizeof T);
}

static void to4x4(const double *A, double *H) {
  for (int i = 0; i < 12; ++i) H[i] = A[i];
  H[12] = 0; H[13] = 0; H[14] = 0; H[15] = 1;
}

static void transpose4(const double *A, double *T) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) T[c * 4 + r] = A[r * 4 + c];
}

/* Local matrix L = [R(q/|q|) | t]. */
static void local_matrix(const double q[4], const double t[3], double L[12]) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double u[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
  double R[9];
  quat_to_rot(u, R);
  for (int r = 0; r < 3; ++r) {
    L[r * 4 + 0] = R[r * 3 + 0];
    L[r * 4 + 1] = R[r * 3 + 1];
    L[r * 4 + 2] = R[r * 3 + 2];
    L[r * 4 + 3] = t[r];
  }
}

/* ------------------------------------------------------------------ */
/* Simulation: slerp, sampling, blending (Sec. 1 step 1; Sec. 2 keeps  */
/* interpolation and blending as the feature the method must retain)   */
/* ------------------------------------------------------------------ */

/* Spherical linear interpolation from a (alpha = 0) to b (alpha = 1) along
 * the shorter arc; result normalized. */
void oracle_slerp(const double *a, const double *b_in, double alpha, double *out) {
  double b[4] = {b_in[0], b_in[1], b_in[2], b_in[3]};
  double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
  if (d < 0) {
    for (int k = 0; k < 4; ++k) b[k] = -b[k];
  }
  double dm = 0, dp = 0;
  for (int k = 0; k < 4; ++k) {
    dm += (a[k] - b[k]) * (a[k] - b[k]);
    dp += (a[k] + b[k]) * (a[k] + b[k]);
  }
  double theta = 2.0 * atan2(sqrt(dm), sqrt(dp));
  double s = sin(theta);
  double r[4];
  if (s < 1e-12) {
    for (int k = 0; k < 4; ++k) r[k] = (1.0 - alpha) * a[k] + alpha * b[k];
  } else {
    double wa = sin((1.0 - alpha) * theta) / s, wb = sin(alpha * theta) / s;
    for (int k = 0; k < 4; ++k) r[k] = wa * a[k] + wb * b[k];
  }
  double n = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
  for (int k = 0; k < 4; ++k) out[k] = r[k] / n;
}

/* Key indices and fraction for a looping clip of n_keys keys at rate Hz.
 * The product time*rate, its floor and the fraction are taken in float32,
 * as the GPU takes them, so both sides pick the same pair of keys. */
static void key_pos(float time, float rate, int n_keys, int *k0, int *k1, double *alpha) {
  volatile float u = time * rate;
  float kf = floorf(u);
  float a = u - kf;
  long long k = (long long)kf;
  long long m = k % n_keys;
  if (m < 0) m += n_keys;
  *k0 = (int)m;
  *k1 = (int)((m + 1) % n_keys);
  *alpha = (double)a;
}

/* Local pose (q, t) of every joint of one character at `time`, blending
 * clip 0 and clip 1 with `weight` (0 -> clip 0).  keys: [clip][key][joint][8]
 * = qx qy qz qw tx ty tz pad.  With one clip the weight is ignored. */
void oracle_sample_local(int n, int n_clips, int n_keys, float rate, const float *keys,
                         float time, float weight, double *q_out, double *t_out) {
  int k0, k1;
  double alpha;
  key_pos(time, rate, n_keys, &k0, &k1, &alpha);
  for (int j = 0; j < n; ++j) {
    double qc[2][4], tc[2][3];
    for (int c = 0; c < n_clips && c < 2; ++c) {
      const float *r0 = keys + (((size_t)c * n_keys + k0) * n + j) * 8;
      const float *r1 = keys + (((size_t)c * n_keys + k1) * n + j) * 8;
      double a[4] = {r0[0], r0[1], r0[2], r0[3]}, b[4] = {r1[0], r1[1], r1[2], r1[3]};
      oracle_slerp(a, b, alpha, qc[c]);
      for (int k = 0; k < 3; ++k) tc[c][k] = (1.0 - alpha) * (double)r0[4 + k] + alpha * (double)r1[4 + k];
    }
    if (n_clips >= 2) {
      double w = weight;
      oracle_slerp(qc[0], qc[1], w, q_out + 4 * (size_t)j);
      for (int k = 0; k < 3; ++k) t_out[3 * (size_t)j + k] = (1.0 - w) * tc[0][k] + w * tc[1][k];
    } else {
      for (int k = 0; k < 4; ++k) q_out[4 * (size_t)j + k] = qc[0][k];
      for (int k = 0; k < 3; ++k) t_out[3 * (size_t)j + k] = tc[0][k];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Hierarchy-Scan (Eq. 1) and Bind MeshPose                            */
/* ------------------------------------------------------------------ */

/* Sequential parent-before-child traversal: M_i = M_parent(i) L_i, roots
 * (parent -1) take M_i = L_i.  Valid because parent(i) < i (Sec. 3.2.1). */
void oracle_forward(int n, const int32_t *parents, const double *L, double *M) {
  for (int i = 0; i < n; ++i) {
    if (parents[i] < 0)
      memcpy(M + 12 * (size_t)i, L + 12 * (size_t)i, 12 * sizeof(double));
    else
      affine_mul(M + 12 * (size_t)parents[i], L + 12 * (size_t)i, M + 12 * (size_t)i);
  }
}

/* S_i = M_i B_i (Sec. 1 step 3). */
void oracle_bind(int n, const double *M, const double *B, double *S) {
  for (int i = 0; i < n; ++i) affine_mul(M + 12 * (size_t)i, B + 12 * (size_t)i, S + 12 * (size_t)i);
}

/* General inverse of a 3x4 affine matrix: [A|b]^-1 = [A^-1 | -A^-1 b],
 * A^-1 from the adjugate and the determinant.  Returns 0 if singular. */
static int affine_inverse(const double *M, double *Inv) {
  double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9], k = M[10];
  double A = e * k - f * h, B = -(d * k - f * g), C = d * h - e * g;
  double det = a * A + b * B + c * C;
  if (det == 0.0) return 0;
  double I[9];
  I[0] = A / det; I[1] = -(b * k - c * h) / det; I[2] = (b * f - c * e) / det;
  I[3] = B / det; I[4] = (a * k - c * g) / det;  I[5] = -(a * f - c * d) / det;
  I[6] = C / det; I[7] = -(a * h - b * g) / det; I[8] = (a * e - b * d) / det;
  for (int r = 0; r < 3; ++r) {
    Inv[r * 4 + 0] = I[r * 3 + 0];
    Inv[r * 4 + 1] = I[r * 3 + 1];
    Inv[r * 4 + 2] = I[r * 3 + 2];
    Inv[r * 4 + 3] = -(I[r * 3 + 0] * M[3] + I[r * 3 + 1] * M[7] + I[r * 3 + 2] * M[11]);
  }
  return 1;
}

/* Inverse bind poses of one skeleton: B_i = (model pose of the rest pose)^-1. */
int oracle_inverse_bind(int n, const int32_t *parents, const float *rest_q, const float *rest_t, double *B) {
  if (n <= 0) return 0;
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)n);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)n);
  if (!L || !M) { free(L); free(M); return -2; }
  for (int i = 0; i < n; ++i) {
    double q[4] = {rest_q[4 * i], rest_q[4 * i + 1], rest_q[4 * i + 2], rest_q[4 * i + 3]};
    double t[3] = {rest_t[3 * i], rest_t[3 * i + 1], rest_t[3 * i + 2]};
    local_matrix(q, t, L + 12 * (size_t)i);
  }
  oracle_forward(n, parents, L, M);
  int ok = 1;
  for (int i = 0; i < n; ++i) ok &= affine_inverse(M + 12 * (size_t)i, B + 12 * (size_t)i);
  free(L);
  free(M);
  return ok ? 0 : -1;
}

/* ------------------------------------------------------------------ */
/* Batched drivers over characters of several skeleton types           */
/* ------------------------------------------------------------------ */

/* type_off[t] = first joint of type t in the concatenated per-type arrays. */
static int64_t *type_offsets(int n_types, const int32_t *counts) {
  int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n_types + 1));
  if (!off) return NULL;
  off[0] = 0;
  for (int t = 0; t < n_types; ++t) off[t + 1] = off[t] + counts[t];
  return off;
}

/* Full frame: Simulation -> Hierarchy-Scan -> Bind MeshPose for every
 * character.  invbind_cat: [sum counts][12]; keys of type t start at
 * keys_cat + key_off[t] with layout [clip][key][joint][8].  Outputs (fp64,
 * rows out_off[c] .. out_off[c]+n-1): skin (required), model (nullable). */
int oracle_frame(int n_types, const int32_t *counts, const int32_t *parents_cat, const double *invbind_cat,
                 const float *keys_cat, const int64_t *key_off, const int32_t *n_clips, const int32_t *n_keys,
                 const float *rate, int64_t n_chars, const int32_t *char_type, const float *time,
                 const float *weight, const int64_t *out_off, double *skin, double *model) {
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *q = (double *)malloc(sizeof(double) * 4 * (size_t)maxn);
  double *tr = (double *)malloc(sizeof(double) * 3 * (size_t)maxn);
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  if (!toff || !q || !tr || !L || !M) { free(toff); free(q); free(tr); free(L); free(M); return -2; }
  for (int64_t c = 0; c < n_chars; ++c) {
    int ty = char_type[c];
    int n = counts[ty];
    const int32_t *par = parents_cat + toff[ty];
    oracle_sample_local(n, n_clips[ty], n_keys[ty], rate[ty], keys_cat + key_off[ty], time[c], weight[c], q, tr);
    for (int j = 0; j < n; ++j) local_matrix(q + 4 * (size_t)j, tr + 3 * (size_t)j, L + 12 * (size_t)j);
    oracle_forward(n, par, L, M);
    oracle_bind(n, M, invbind_cat + 12 * toff[ty], skin + 12 * out_off[c]);
    if (model) memcpy(model + 12 * out_off[c], M, sizeof(double) * 12 * (size_t)n);
  }
  free(toff); free(q); free(tr); free(L); free(M);
  return 0;
}

/* Hierarchy-Scan + Bind from given local poses q (unnormalized, [sum][4]) and
 * t ([sum][3]).  invbind_cat may be NULL (then skin is not written). */
int oracle_forward_qt(int n_types, const int32_t *counts, const int32_t *parents_cat, const double *invbind_cat,
                      int64_t n_chars, const int32_t *char_type, const double *qin, const double *tin,
                      const int64_t *out_off, double *skin, double *model) {
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  if (!toff || !L || !M) { free(toff); free(L); free(M); return -2; }
  for (int64_t c = 0; c < n_chars; ++c) {
    int ty = char_type[c];
    int n = counts[ty];
    int64_t o = out_off[c];
    for (int j = 0; j < n; ++j) {
      double q[4] = {qin[4 * (o + j)], qin[4 * (o + j) + 1], qin[4 * (o + j) + 2], qin[4 * (o + j) + 3]};
      double t[3] = {tin[3 * (o + j)], tin[3 * (o + j) + 1], tin[3 * (o + j) + 2]};
      local_matrix(q, t, L + 12 * (size_t)j);
    }
    oracle_forward(n, parents_cat + toff[ty], L, M);
    if (skin && invbind_cat) oracle_bind(n, M, invbind_cat + 12 * toff[ty], skin + 12 * o);
    if (model) memcpy(model + 12 * o, M, sizeof(double) * 12 * (size_t)n);
  }
  free(toff); free(L); free(M);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Gradients of a loss on model-space joint positions                  */
/* ------------------------------------------------------------------ */

/* d R_ab / d q_k for the polynomial rotation formula, written out entry by
 * entry; qbar_k = sum_ab Rbar_ab dR_ab/dq_k. */
static void rot_grad_to_quat(const double q[4], const double Rb[9], double qb[4]) {
  double x = q[0], y = q[1], z = q[2], w = q[3];
  double gx = 0, gy = 0, gz = 0, gw = 0;
  /* R00 = 1-2(y^2+z^2) */ gy += Rb[0] * (-4 * y); gz += Rb[0] * (-4 * z);
  /* R01 = 2(xy - zw)   */ gx += Rb[1] * (2 * y); gy += Rb[1] * (2 * x); gz += Rb[1] * (-2 * w); gw += Rb[1] * (-2 * z);
  /* R02 = 2(xz + yw)   */ gx += Rb[2] * (2 * z); gy += Rb[2] * (2 * w); gz += Rb[2] * (2 * x); gw += Rb[2] * (2 * y);
  /* R10 = 2(xy + zw)   */ gx += Rb[3] * (2 * y); gy += Rb[3] * (2 * x); gz += Rb[3] * (2 * w); gw += Rb[3] * (2 * z);
  /* R11 = 1-2(x^2+z^2) */ gx += Rb[4] * (-4 * x); gz += Rb[4] * (-4 * z);
  /* R12 = 2(yz - xw)   */ gx += Rb[5] * (-2 * w); gy += Rb[5] * (2 * z); gz += Rb[5] * (2 * y); gw += Rb[5] * (-2 * x);
  /* R20 = 2(xz - yw)   */ gx += Rb[6] * (2 * z); gy += Rb[6] * (-2 * w); gz += Rb[6] * (2 * x); gw += Rb[6] * (-2 * y);
  /* R21 = 2(yz + xw)   */ gx += Rb[7] * (2 * w); gy += Rb[7] * (2 * z); gz += Rb[7] * (2 * y); gw += Rb[7] * (2 * x);
  /* R22 = 1-2(x^2+y^2) */ gx += Rb[8] * (-4 * x); gy += Rb[8] * (-4 * y);
  qb[0] = gx; qb[1] = gy; qb[2] = gz; qb[3] = gw;
}

/* Chain rule through q_hat = q/|q|: dq = (I - q_hat q_hat^T) qbar_hat / |q|. */
static void unnormalize_grad(const double q[4], const double qb_hat[4], double dq[4]) {
  double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double u[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
  double dot = u[0] * qb_hat[0] + u[1] * qb_hat[1] + u[2] * qb_hat[2] + u[3] * qb_hat[3];
  for (int k = 0; k < 4; ++k) dq[k] = (qb_hat[k] - dot * u[k]) / nq;
}

/* Generic reverse pass.  g_pos: dLoss/dp_j (p_j = translation of M_j),
 * [sum][3].  Outputs dq [sum][4] (w.r.t. the unnormalized q) and dt [sum][3].
 * For M_i = M_p L_i as 4x4 products: Gbar_p += Gbar_i L_i^T and
 * Lbar_i = M_p^T Gbar_i, visiting joints from the last index to the first
 * so that every child is done before its parent. */
int oracle_grad(int n_types, const int32_t *counts, const int32_t *parents_cat, int64_t n_chars,
                const int32_t *char_type, const double *qin, const double *tin, const double *g_pos,
                const int64_t *out_off, double *dq, double *dt) {
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *G = (double *)malloc(sizeof(double) * 16 * (size_t)maxn);
  if (!toff || !L || !M || !G) { free(toff); free(L); free(M); free(G); return -2; }
  for (int64_t c = 0; c < n_chars; ++c) {
    int ty = char_type[c];
    int n = counts[ty];
    int64_t o = out_off[c];
    const int32_t *par = parents_cat + toff[ty];
    for (int j = 0; j < n; ++j) {
      double q[4] = {qin[4 * (o + j)], qin[4 * (o + j) + 1], qin[4 * (o + j) + 2], qin[4 * (o + j) + 3]};
      double t[3] = {tin[3 * (o + j)], tin[3 * (o + j) + 1], tin[3 * (o + j) + 2]};
      local_matrix(q, t, L + 12 * (size_t)j);
    }
    oracle_forward(n, par, L, M);
    memset(G, 0, sizeof(double) * 16 * (size_t)n);
    for (int j = 0; j < n; ++j)
      for (int r = 0; r < 3; ++r) G[16 * (size_t)j + r * 4 + 3] = g_pos[3 * (o + j) + r];
    for (int i = n - 1; i >= 0; --i) {
      double *Gi = G + 16 * (size_t)i;
      double Lb[16];
      int p = par[i];
      if (p >= 0) {
        double Lh[16], Lt[16], Mh[16], Mt[16], tmp[16];
        to4x4(L + 12 * (size_t)i, Lh);
        transpose4(Lh, Lt);
        mat4_mul(Gi, Lt, tmp);
        for (int k = 0; k < 12; ++k) G[16 * (size_t)p + k] += tmp[k];
        to4x4(M + 12 * (size_t)p, Mh);
        transpose4(Mh, Mt);
        mat4_mul(Mt, Gi, Lb);
      } else {
        memcpy(Lb, Gi, sizeof Lb);
      }
      double Rb[9] = {Lb[0], Lb[1], Lb[2], Lb[4], Lb[5], Lb[6], Lb[8], Lb[9], Lb[10]};
      double q[4] = {qin[4 * (o + i)], qin[4 * (o + i) + 1], qin[4 * (o + i) + 2], qin[4 * (o + i) + 3]};
      double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      double u[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
      double qbh[4];
      rot_grad_to_quat(u, Rb, qbh);
      unnormalize_grad(q, qbh, dq + 4 * (o + i));
      dt[3 * (o + i) + 0] = Lb[3];
      dt[3 * (o + i) + 1] = Lb[7];
      dt[3 * (o + i) + 2] = Lb[11];
    }
  }
  free(toff); free(L); free(M); free(G);
  return 0;
}

static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Second, independent derivation of the same gradient (rigid poses only).
 * F_j = sum of g over the subtree of j, T_j = sum of p_k x g_k over it;
 * the world-frame torque about p_j is T_j - p_j x F_j; expressed in the
 * parent frame (R_p^T) it is tau_j.  dt_j = R_p^T F_j and
 * dq_j = 2 (tau_j, 0) (x) q_hat_j / |q_j| (Hamilton product, (x,y,z,w)). */
int oracle_grad_force_moment(int n_types, const int32_t *counts, const int32_t *parents_cat, int64_t n_chars,
                             const int32_t *char_type, const double *qin, const double *tin, const double *g_pos,
                             const int64_t *out_off, double *dq, double *dt) {
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *F = (double *)malloc(sizeof(double) * 3 * (size_t)maxn);
  double *T = (double *)malloc(sizeof(double) * 3 * (size_t)maxn);
  if (!toff || !L || !M || !F || !T) { free(toff); free(L); free(M); free(F); free(T); return -2; }
  for (int64_t c = 0; c < n_chars; ++c) {
    int ty = char_type[c];
    int n = counts[ty];
    int64_t o = out_off[c];
    const int32_t *par = parents_cat + toff[ty];
    for (int j = 0; j < n; ++j) {
      double q[4] = {qin[4 * (o + j)], qin[4 * (o + j) + 1], qin[4 * (o + j) + 2], qin[4 * (o + j) + 3]};
      double t[3] = {tin[3 * (o + j)], tin[3 * (o + j) + 1], tin[3 * (o + j) + 2]};
      local_matrix(q, t, L + 12 * (size_t)j);
    }
    oracle_forward(n, par, L, M);
    for (int j = 0; j < n; ++j) {
      const double *g = g_pos + 3 * (o + j);
      double p[3] = {M[12 * j + 3], M[12 * j + 7], M[12 * j + 11]}, pg[3];
      cross3(p, g, pg);
      for (int k = 0; k < 3; ++k) { F[3 * j + k] = g[k]; T[3 * j + k] = pg[k]; }
    }
    for (int i = n - 1; i >= 1; --i) {
      int p = par[i];
      if (p < 0) continue;
      for (int k = 0; k < 3; ++k) { F[3 * p + k] += F[3 * i + k]; T[3 * p + k] += T[3 * i + k]; }
    }
    for (int j = 0; j < n; ++j) {
      double Rp[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
      int p = par[j];
      if (p >= 0)
        for (int r = 0; r < 3; ++r)
          for (int k = 0; k < 3; ++k) Rp[r * 3 + k] = M[12 * (size_t)p + r * 4 + k];
      double pj[3] = {M[12 * j + 3], M[12 * j + 7], M[12 * j + 11]}, pf[3], tw[3], tau[3], ft[3];
      cross3(pj, F + 3 * j, pf);
      for (int k = 0; k < 3; ++k) tw[k] = T[3 * j + k] - pf[k];
      for (int k = 0; k < 3; ++k) {
        tau[k] = Rp[0 * 3 + k] * tw[0] + Rp[1 * 3 + k] * tw[1] + Rp[2 * 3 + k] * tw[2];
        ft[k] = Rp[0 * 3 + k] * F[3 * j + 0] + Rp[1 * 3 + k] * F[3 * j + 1] + Rp[2 * 3 + k] * F[3 * j + 2];
      }
      double q[4] = {qin[4 * (o + j)], qin[4 * (o + j) + 1], qin[4 * (o + j) + 2], qin[4 * (o + j) + 3]};
      double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      double u[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
      /* (a (x) b) with a = (tau, 0), b = u: */
      double ax = tau[0], ay = tau[1], az = tau[2];
      double rx = ax * u[3] + ay * u[2] - az * u[1];
      double ry = -ax * u[2] + ay * u[3] + az * u[0];
      double rz = ax * u[1] - ay * u[0] + az * u[3];
      double rw = -ax * u[0] - ay * u[1] - az * u[2];
      dq[4 * (o + j) + 0] = 2 * rx / nq;
      dq[4 * (o + j) + 1] = 2 * ry / nq;
      dq[4 * (o + j) + 2] = 2 * rz / nq;
      dq[4 * (o + j) + 3] = 2 * rw / nq;
      for (int k = 0; k < 3; ++k) dt[3 * (o + j) + k] = ft[k];
    }
  }
  free(toff); free(L); free(M); free(F); free(T);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Adam (PyTorch's definition) and batched IK                          */
/* ------------------------------------------------------------------ */

/* One Adam step at step number `step` (1-based): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps). */
void oracle_adam(int64_t n, double *p, const double *g, double *m, double *v, int step, double lr, double b1,
                 double b2, double eps) {
  double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / bc1, vh = v[i] / bc2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* Batched IK: n_steps Adam steps on the local quaternions (translations
 * fixed) minimizing sum_e |p_e - target_e|^2 over the n_eff effectors of each
 * character.  effectors: [n_types][n_eff] joint ids; targets: [n_chars][n_eff][3].
 * q_io: [sum][4] fp64 in/out (Adam state m, v start at zero); loss_hist[s] is
 * the total loss at the start of step s. */
int oracle_ik(int n_types, const int32_t *counts, const int32_t *parents_cat, const int32_t *effectors, int n_eff,
              int64_t n_chars, const int32_t *char_type, const double *tin, const double *targets,
              const int64_t *out_off, int n_steps, double lr, double b1, double b2, double eps, double *q_io,
              double *loss_hist) {
  int64_t total = out_off[n_chars];
  double *m = (double *)calloc((size_t)total * 4, sizeof(double));
  double *v = (double *)calloc((size_t)total * 4, sizeof(double));
  double *g = (double *)calloc((size_t)total * 4, sizeof(double));
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *G = (double *)malloc(sizeof(double) * 16 * (size_t)maxn);
  if (!m || !v || !g || !toff || !L || !M || !G) {
    free(m); free(v); free(g); free(toff); free(L); free(M); free(G);
    return -2;
  }
  for (int s = 1; s <= n_steps; ++s) {
    double loss = 0;
    for (int64_t c = 0; c < n_chars; ++c) {
      int ty = char_type[c];
      int n = counts[ty];
      int64_t o = out_off[c];
      const int32_t *par = parents_cat + toff[ty];
      for (int j = 0; j < n; ++j) {
        double t[3] = {tin[3 * (o + j)], tin[3 * (o + j) + 1], tin[3 * (o + j) + 2]};
        local_matrix(q_io + 4 * (o + j), t, L + 12 * (size_t)j);
      }
      oracle_forward(n, par, L, M);
      memset(G, 0, sizeof(double) * 16 * (size_t)n);
      for (int e = 0; e < n_eff; ++e) {
        int j = effectors[ty * n_eff + e];
        for (int r = 0; r < 3; ++r) {
          double d = M[12 * (size_t)j + r * 4 + 3] - targets[(c * n_eff + e) * 3 + r];
          loss += d * d;
          G[16 * (size_t)j + r * 4 + 3] += 2 * d;
        }
      }
      for (int i = n - 1; i >= 0; --i) {
        double *Gi = G + 16 * (size_t)i;
        double Lb[16];
        int p = par[i];
        if (p >= 0) {
          double Lh[16], Lt[16], Mh[16], Mt[16], tmp[16];
          to4x4(L + 12 * (size_t)i, Lh);
          transpose4(Lh, Lt);
          mat4_mul(Gi, Lt, tmp);
          for (int k = 0; k < 12; ++k) G[16 * (size_t)p + k] += tmp[k];
          to4x4(M + 12 * (size_t)p, Mh);
          transpose4(Mh, Mt);
          mat4_mul(Mt, Gi, Lb);
        } else {
          memcpy(Lb, Gi, sizeof Lb);
        }
        double Rb[9] = {Lb[0], Lb[1], Lb[2], Lb[4], Lb[5], Lb[6], Lb[8], Lb[9], Lb[10]};
        double *q = q_io + 4 * (o + i);
        double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double u[4] = {q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq};
        double qbh[4];
        rot_grad_to_quat(u, Rb, qbh);
        unnormalize_grad(q, qbh, g + 4 * (o + i));
      }
    }
    if (loss_hist) loss_hist[s - 1] = loss;
    oracle_adam(total * 4, q_io, g, m, v, s, lr, b1, b2, eps);
  }
  free(m); free(v); free(g); free(toff); free(L); free(M); free(G);
  return 0;
}

/*
 * Linear blend skinning: the skinning step that follows Bind MeshPose in the
 * paper's pipeline (Sec. 1; Table 1 lists meshes of 1,000-3,000 faces).  The
 * paper does not spell it out, so this is the textbook form.  Vertex v with
 * rest position p, rest normal nrm, bones b_k and weights w_k (k < 4, weights
 * summing to 1, zero weights ignored):
 *     p' = sum_k w_k S_{b_k} [p; 1]
 *     n' = normalize(sum_k w_k R_{b_k} nrm)      (S = [R | t], rigid)
 * S: the character's skin matrices [n][12]; out [n_verts][6] = p', n'.
 */
void oracle_lbs(int n_verts, const float *pos, const float *nrm, const int32_t *bones, const float *weights,
                const double *S, double *out) {
  for (int v = 0; v < n_verts; ++v) {
    const double p[3] = {pos[3 * v], pos[3 * v + 1], pos[3 * v + 2]};
    const double q[3] = {nrm[3 * v], nrm[3 * v + 1], nrm[3 * v + 2]};
    double pp[3] = {0.0, 0.0, 0.0}, nn[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
      const double w = weights[4 * v + k];
      if (w == 0.0) continue;
      const double *M = S + 12 * (int64_t)bones[4 * v + k];
      for (int r = 0; r < 3; ++r) {
        pp[r] += w * (M[4 * r] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3]);
        nn[r] += w * (M[4 * r] * q[0] + M[4 * r + 1] * q[1] + M[4 * r + 2] * q[2]);
      }
    }
    const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
    for (int r = 0; r < 3; ++r) {
      out[6 * (int64_t)v + r] = pp[r];
      out[6 * (int64_t)v + 3 + r] = len > 0.0 ? nn[r] / len : 0.0;
    }
  }
}

/* Hamilton product a b of quaternions stored (x, y, z, w). */
static void quat_mul(const double *a, const double *b, double *r) {
  r[0] = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  r[1] = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  r[2] = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  r[3] = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
}

/*
 * Layered blend (the paper asks the method to keep the state-machine
 * blending of clips, Sec. 2, without giving one; this is the reading used):
 * up to 4 clips sampled at the character's time as in oracle_sample_local,
 * rotations blended by incremental slerp -- q = q_0, W = w_0, then for each
 * further clip i: W += w_i and, if W > 0, q = slerp(q, q_i, w_i / W) -- and
 * translations by their weighted mean (t_0 when every weight is 0); two
 * clips with weights (1 - w, w) give the two-clip blend.  An optional
 * additive layer (add_keys [key][joint][8], same key count and rate) sampled
 * at the same time is applied on top with weight a:
 *     q <- q * slerp(identity, q_a, a),   t <- t + a t_a.
 */
void oracle_sample_layers(int n, int n_clips, int n_keys, float rate, const float *keys, const float *add_keys,
                          float time, const float *weights, float add_w, double *q_out, double *t_out) {
  int k0, k1;
  double alpha;
  key_pos(time, rate, n_keys, &k0, &k1, &alpha);
  for (int j = 0; j < n; ++j) {
    double q[4], t[3] = {0.0, 0.0, 0.0}, W = 0.0;
    for (int c = 0; c < n_clips; ++c) {
      const float *r0 = keys + (((size_t)c * n_keys + k0) * n + j) * 8;
      const float *r1 = keys + (((size_t)c * n_keys + k1) * n + j) * 8;
      double a[4] = {r0[0], r0[1], r0[2], r0[3]}, b[4] = {r1[0], r1[1], r1[2], r1[3]}, qc[4];
      oracle_slerp(a, b, alpha, qc);
      const double w = weights[c];
      if (c == 0) {
        for (int k = 0; k < 4; ++k) q[k] = qc[k];
      } else if (W + w > 0.0) {
        double r[4];
        oracle_slerp(q, qc, w / (W + w), r);
        for (int k = 0; k < 4; ++k) q[k] = r[k];
      }
      W += w;
      for (int k = 0; k < 3; ++k) t[k] += w * ((1.0 - alpha) * (double)r0[4 + k] + alpha * (double)r1[4 + k]);
      if (c == 0 && W == 0.0)
        for (int k = 0; k < 3; ++k) t[k] = 0.0;
    }
    if (W > 0.0) {
      for (int k = 0; k < 3; ++k) t[k] /= W;
    } else {
      const float *r0 = keys + ((size_t)k0 * n + j) * 8, *r1 = keys + ((size_t)k1 * n + j) * 8;
      for (int k = 0; k < 3; ++k) t[k] = (1.0 - alpha) * (double)r0[4 + k] + alpha * (double)r1[4 + k];
    }
    if (add_keys) {
      const float *r0 = add_keys + ((size_t)k0 * n + j) * 8, *r1 = add_keys + ((size_t)k1 * n + j) * 8;
      double a[4] = {r0[0], r0[1], r0[2], r0[3]}, b[4] = {r1[0], r1[1], r1[2], r1[3]}, qa[4], qs[4], r[4];
      const double id[4] = {0.0, 0.0, 0.0, 1.0};
      oracle_slerp(a, b, alpha, qa);
      oracle_slerp(id, qa, add_w, qs);
      quat_mul(q, qs, r);
      for (int k = 0; k < 4; ++k) q[k] = r[k];
      for (int k = 0; k < 3; ++k) t[k] += add_w * ((1.0 - alpha) * (double)r0[4 + k] + alpha * (double)r1[4 + k]);
    }
    for (int k = 0; k < 4; ++k) q_out[4 * (size_t)j + k] = q[k];
    for (int k = 0; k < 3; ++k) t_out[3 * (size_t)j + k] = t[k];
  }
}

/* The frame with layered blending: per character its clip weights
 * weights[c][4] and additive weight add_w[c]; add_off[type] < 0: no
 * additive layer. */
int oracle_frame_layers(int n_types, const int32_t *counts, const int32_t *parents_cat, const double *invbind_cat,
                        const float *keys_cat, const int64_t *key_off, const int32_t *n_clips,
                        const int32_t *n_keys, const float *rate, const float *add_cat, const int64_t *add_off,
                        int64_t n_chars, const int32_t *char_type, const float *time, const float *weights,
                        const float *add_w, const int64_t *out_off, double *skin) {
  int64_t *toff = type_offsets(n_types, counts);
  int maxn = 0;
  for (int t = 0; t < n_types; ++t) maxn = counts[t] > maxn ? counts[t] : maxn;
  double *q = (double *)malloc(sizeof(double) * 4 * (size_t)maxn);
  double *tr = (double *)malloc(sizeof(double) * 3 * (size_t)maxn);
  double *L = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  double *M = (double *)malloc(sizeof(double) * 12 * (size_t)maxn);
  if (!toff || !q || !tr || !L || !M) { free(toff); free(q); free(tr); free(L); free(M); return -2; }
  for (int64_t c = 0; c < n_chars; ++c) {
    int ty = char_type[c];
    int n = counts[ty];
    const int32_t *par = parents_cat + toff[ty];
    oracle_sample_layers(n, n_clips[ty], n_keys[ty], rate[ty], keys_cat + key_off[ty],
                         add_off[ty] >= 0 ? add_cat + add_off[ty] : NULL, time[c], weights + 4 * c, add_w[c], q, tr);
    for (int j = 0; j < n; ++j) local_matrix(q + 4 * (size_t)j, tr + 3 * (size_t)j, L + 12 * (size_t)j);
    oracle_forward(n, par, L, M);
    oracle_bind(n, M, invbind_cat + 12 * toff[ty], skin + 12 * out_off[c]);
  }
  free(toff); free(q); free(tr); free(L); free(M);
  return 0;
}

/*
 * Headless rasterization of the skinned crowd (the paper renders its crowd,
 * Sec. 4 and Fig. 6, through a graphics API; this is the same picture as a
 * plain software rasterizer with fixed rules).  Character c stands at world
 * offset (col * spacing, -row * spacing, 0), col = c % cols, row = c / cols;
 * orthographic camera looking down -Z: a world point (X, Y, Z) lands at
 * screen (ox + scale X, oy - scale Y), depth d = (2 - Z) / 4 (smaller is
 * nearer).  Screen positions are snapped to 1/256 pixel (round to nearest,
 * halves away from zero); coverage of pixel (x, y) -- centre (x + 0.5,
 * y + 0.5) -- uses 64-bit integer edge functions of the snapped positions
 * with the triangle oriented to positive area and the tie rule: a centre on
 * an edge a->b belongs to the triangle if b - a points down (dy > 0), or
 * horizontally left (dy == 0, dx < 0), so two triangles sharing an edge never
 * both take (or both miss) a centre on it; zero-area triangles cover
 * nothing.  Visibility: the smallest (depth, id) with depth interpolated
 * barycentrically at the centre; id = c * 4096 + face index.
 *   ids [height][width] receives the winning id or 0xFFFFFFFF; cover
 *   (nullable) the number of triangles covering each pixel.
 */
static int64_t snap256(double v) { return (int64_t)llround(v * 256.0); }

void oracle_raster(int n_chars, const int32_t *n_faces, const int32_t *const *faces, const int64_t *vert_off,
                   const double *verts, int cols, double spacing, double ox, double oy, double scale, int width,
                   int height, uint32_t *ids, int32_t *cover) {
  double *depth = (double *)malloc(sizeof(double) * (size_t)width * height);
  for (size_t i = 0; i < (size_t)width * height; ++i) {
    ids[i] = 0xFFFFFFFFu;
    depth[i] = INFINITY;
    if (cover) cover[i] = 0;
  }
  for (int c = 0; c < n_chars; ++c) {
    const double wx = (c % cols) * spacing, wy = -(c / cols) * spacing;
    for (int f = 0; f < n_faces[c]; ++f) {
      int64_t X[3], Y[3];
      double D[3];
      for (int k = 0; k < 3; ++k) {
        const double *v = verts + 6 * (vert_off[c] + faces[c][3 * f + k]);
        X[k] = snap256(ox + scale * (v[0] + wx));
        Y[k] = snap256(oy - scale * (v[1] + wy));
        D[k] = (2.0 - v[2]) / 4.0;
      }
      int64_t area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
      if (area == 0) continue;
      if (area < 0) {  // orient to positive area
        int64_t tx = X[1], ty = Y[1];
        double td = D[1];
        X[1] = X[2]; Y[1] = Y[2]; D[1] = D[2];
        X[2] = tx; Y[2] = ty; D[2] = td;
        area = -area;
      }
      int64_t xmin = X[0], xmax = X[0], ymin = Y[0], ymax = Y[0];
      for (int k = 1; k < 3; ++k) {
        xmin = X[k] < xmin ? X[k] : xmin; xmax = X[k] > xmax ? X[k] : xmax;
        ymin = Y[k] < ymin ? Y[k] : ymin; ymax = Y[k] > ymax ? Y[k] : ymax;
      }
      /* pixels whose centre x*256+128 lies in [xmin, xmax] */
      int px0 = (int)((xmin - 128 + 255) >> 8), px1 = (int)((xmax - 128) >> 8);
      int py0 = (int)((ymin - 128 + 255) >> 8), py1 = (int)((ymax - 128) >> 8);
      if (px0 < 0) px0 = 0;
      if (py0 < 0) py0 = 0;
      if (px1 > width - 1) px1 = width - 1;
      if (py1 > height - 1) py1 = height - 1;
      for (int py = py0; py <= py1; ++py) {
        for (int px = px0; px <= px1; ++px) {
          const int64_t cx = (int64_t)px * 256 + 128, cy = (int64_t)py * 256 + 128;
          int64_t e[3];
          int inside = 1;
          for (int k = 0; k < 3 && inside; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;  /* edge opposite vertex k */
            const int64_t dx = X[b] - X[a], dy = Y[b] - Y[a];
            e[k] = dx * (cy - Y[a]) - dy * (cx - X[a]);
            if (e[k] < 0 || (e[k] == 0 && !(dy > 0 || (dy == 0 && dx < 0)))) inside = 0;
          }
          if (!inside) continue;
          if (cover) ++cover[(size_t)py * width + px];
          const double d = ((double)e[0] * D[0] + (double)e[1] * D[1] + (double)e[2] * D[2]) / (double)area;
          const uint32_t id = (uint32_t)c * 4096u + (uint32_t)f;
          const size_t pi = (size_t)py * width + px;
          if (d < depth[pi] || (d == depth[pi] && id < ids[pi])) {
            depth[pi] = d;
            ids[pi] = id;
          }
        }
      }
    }
  }
  free(depth);
}
