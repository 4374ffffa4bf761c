// Headless rasterization of the skinned crowd (the picture the paper draws
// through a graphics API, Sec. 4 and Fig. 6), as plain CUDA: no graphics
// stack, a visibility buffer of 64-bit keys in device memory.
//
// Rules (fixed so that results are reproducible): character c stands at
// world offset (col * spacing, -row * spacing, 0), col = c % cols,
// row = c / cols; an orthographic camera looking down -Z maps a world point
// to screen (ox + scale X, oy - scale Y) with depth d = (2 - Z) / 4 (smaller
// is nearer).  Screen positions are snapped to 1/256 pixel (round to
// nearest, halves away from zero); pixel (x, y) is covered when its centre
// (x + 0.5, y + 0.5) is inside the triangle by 64-bit integer edge
// functions of the snapped positions, the triangle oriented to positive
// area, with the tie rule that a centre on an edge a->b belongs to it when
// b - a points down (dy > 0) or horizontally left (dy == 0, dx < 0); zero-
// area triangles cover nothing.  Visibility: the smallest key
// (depth bits << 32 | id), id = c * 4096 + face, by atomicMin.
#include <cuda_runtime.h>

#include "anim_internal.h"
#include "dev_math.cuh"

namespace anim {

namespace {

__global__ void k_raster_clear(unsigned long long *vis, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    vis[i] = ~0ull;
}

__device__ __forceinline__ long long snap256(float v) { return llroundf(v * 256.f); }

__global__ void k_raster_tris(const RasterArgs a) {
  const int c = blockIdx.x;
  const TypeDev &T = a.types[a.char_type[c]];
  const int nf = T.n_faces;
  if (nf == 0) return;
  const float wx = (float)(c % a.cols) * a.spacing, wy = -(float)(c / a.cols) * a.spacing;
  const float *vb = a.verts + a.vert_off[c] * 6;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    long long X[3], Y[3];
    float D[3];
    for (int k = 0; k < 3; ++k) {
      const float *v = vb + 6 * (long long)__ldg(T.faces + 3 * f + k);
      X[k] = snap256(a.ox + a.scale * (__ldg(v) + wx));
      Y[k] = snap256(a.oy - a.scale * (__ldg(v + 1) + wy));
      D[k] = (2.f - __ldg(v + 2)) * 0.25f;
    }
    long long area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    if (area == 0) continue;
    if (area < 0) {
      long long t = X[1];
      X[1] = X[2];
      X[2] = t;
      t = Y[1];
      Y[1] = Y[2];
      Y[2] = t;
      const float td = D[1];
      D[1] = D[2];
      D[2] = td;
      area = -area;
    }
    long long xmin = min(X[0], min(X[1], X[2])), xmax = max(X[0], max(X[1], X[2]));
    long long ymin = min(Y[0], min(Y[1], Y[2])), ymax = max(Y[0], max(Y[1], Y[2]));
    const long long px0 = max(0ll, (xmin - 128 + 255) >> 8), px1 = min((long long)a.width - 1, (xmax - 128) >> 8);
    const long long py0 = max(0ll, (ymin - 128 + 255) >> 8), py1 = min((long long)a.height - 1, (ymax - 128) >> 8);
    const float inv_area = 1.f / (float)area;
    const unsigned int id = (unsigned int)c * 4096u + (unsigned int)f;
    for (long long py = py0; py <= py1; ++py) {
      for (long long px = px0; px <= px1; ++px) {
        const long long cx = px * 256 + 128, cy = py * 256 + 128;
        long long e[3];
        bool inside = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int ia = (k + 1) % 3, ib = (k + 2) % 3;
          const long long dx = X[ib] - X[ia], dy = Y[ib] - Y[ia];
          e[k] = dx * (cy - Y[ia]) - dy * (cx - X[ia]);
          inside = inside && (e[k] > 0 || (e[k] == 0 && (dy > 0 || (dy == 0 && dx < 0))));
        }
        if (!inside) continue;
        float d = ((float)e[0] * D[0] + (float)e[1] * D[1] + (float)e[2] * D[2]) * inv_area;
        d = fmaxf(d, 0.f);
        const unsigned long long key = ((unsigned long long)__float_as_uint(d) << 32) | id;
        atomicMin(a.vis + py * a.width + px, key);
      }
    }
  }
}

__global__ void k_raster_resolve(const RasterArgs a) {
  const long long n = (long long)a.width * a.height;
  const float lx = 0.3f, ly = 0.5f, lz = 0.8f, ln = rsqrtf(lx * lx + ly * ly + lz * lz);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = a.vis[i];
    const unsigned int id = key == ~0ull ? 0xFFFFFFFFu : (unsigned int)(key & 0xFFFFFFFFull);
    if (a.ids) a.ids[i] = id;
    if (!a.rgba) continue;
    if (id == 0xFFFFFFFFu) {
      a.rgba[i] = 0xFF201810u;  // background (A B G R bytes)
      continue;
    }
    const int c = (int)(id >> 12), f = (int)(id & 4095u);
    const TypeDev &T = a.types[a.char_type[c]];
    const float *vb = a.verts + a.vert_off[c] * 6;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    for (int k = 0; k < 3; ++k) {
      const float *v = vb + 6 * (long long)__ldg(T.faces + 3 * f + k);
      nx += __ldg(v + 3);
      ny += __ldg(v + 4);
      nz += __ldg(v + 5);
    }
    const float nn = nx * nx + ny * ny + nz * nz;
    const float lam = nn > 0.f ? fabsf(nx * lx + ny * ly + nz * lz) * ln * rsqrtf(nn) : 0.f;
    const float g = 0.25f + 0.75f * lam;
    const unsigned int h = (unsigned int)c * 2654435761u;  // per-character tint
    const float r = g * (0.6f + 0.4f * ((h >> 8) & 255u) / 255.f), gg = g * (0.6f + 0.4f * ((h >> 16) & 255u) / 255.f),
                b = g * (0.6f + 0.4f * ((h >> 24) & 255u) / 255.f);
    a.rgba[i] = 0xFF000000u | ((unsigned int)(b * 255.f) << 16) | ((unsigned int)(gg * 255.f) << 8) |
                (unsigned int)(r * 255.f);
  }
}

}  // namespace

cudaError_t launch_raster(const RasterArgs &a, int n_chars, cudaStream_t st) {
  const long long n = (long long)a.width * a.height;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_raster_clear<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(a.vis, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (n_chars > 0) {
    k_raster_tris<<<n_chars, 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_raster_resolve<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace anim
