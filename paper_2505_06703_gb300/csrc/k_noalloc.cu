// anim_forward_local_noalloc: the forward scan + bind for a batch of
// characters of one skeleton type, for callers that may not allocate device
// memory (see include/anim.h).  Its scratch -- the skeleton's segment tables,
// the type record the kernel reads and the work-queue counter -- lives in
// the file-scope array below instead of cudaMalloc'd buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/anim.h"
#include "anim_internal.h"
#include "dev_math.cuh"
#include "scan_core.cuh"
#include "smem_limit.h"

namespace anim {

// Shared by every call on a device; holds whatever the last call put there.
constexpr size_t kNoAllocScratchBytes = 96 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
constexpr int kNoAllocSegLen = 16;

// Scratch layout (byte offsets inside g_noalloc_scratch).
constexpr size_t kOffType = 0;  // TypeDev
constexpr size_t kOffQueue = 256;
constexpr size_t kOffParent = 512;
constexpr size_t kOffSegStart = kOffParent + 4 * ANIM_MAX_JOINTS;
constexpr size_t kOffSegLink = kOffSegStart + 4 * (ANIM_MAX_JOINTS + 64);
constexpr size_t kOffJinfo = kOffSegLink + 4 * ANIM_MAX_JOINTS;
constexpr size_t kScratchUsed = kOffJinfo + 4 * ANIM_MAX_JOINTS;
static_assert(kScratchUsed <= kNoAllocScratchBytes, "scratch layout exceeds the static array");
static_assert(sizeof(TypeDev) <= kOffQueue, "type record overlaps the queue counter");

// Device address of the scratch array per device (set up once per device).
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Host staging of the tables (no heap allocation).
struct HostTables {
  unsigned char bytes[kScratchUsed];
};
thread_local HostTables g_host;

int set_msg(int code, const char *) { return code; }  // the code is the whole report

}  // namespace

// Implicit work items: item i is characters [i*C, min(n_chars, (i+1)*C)),
// character c's rows start at c*n.  The producer warp stages them as the
// persistent scan kernel's producer does for explicit items.
__device__ __forceinline__ void fetch_implicit(ItemBuf &b, int *queue_head, int n_items, int C, int n_chars,
                                               const TypeDev *type) {
  const int lane = threadIdx.x & 31;
  int it = 0;
  if (lane == 0) it = atomicAdd(queue_head, 1);
  it = __shfl_sync(0xffffffffu, it, 0);
  if (it >= n_items) {
    if (lane == 0) b.item = -1;
    __syncwarp();
    return;
  }
  const int first = it * C, count = min(C, n_chars - first);
  const int *src = reinterpret_cast<const int *>(type);
  int *dst = reinterpret_cast<int *>(&b.T);
  for (int k = lane; k < (int)(sizeof(TypeDev) / 4); k += 32) dst[k] = src[k];
  const int n = type->n;
  for (int c = lane; c < count; c += 32) {
    b.cid[c] = first + c;
    b.off[c] = (long long)(first + c) * n;
  }
  if (lane == 0) {
    b.item = it;
    b.C = count;
    b.k0 = 0;
    b.type = 0;
    b.divC.init(count);
    b.divS.init(type->nseg);
    b.divN.init(n);
    int g = (kComputeThreads + n - 1) / n;
    g = g < 1 ? 1 : (g > count ? count : g);
    b.cpt = (count + g - 1) / g;
    b.cgroups = (count + b.cpt - 1) / b.cpt;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kCtaThreads, 2)
    k_scan_noalloc(unsigned char *scratch, int n_chars, int C, const float *q, const float *t, const float4 *inv_bind,
                   float *skin) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ ItemBuf bufs[2];
  const int tid = threadIdx.x;
  const TypeDev *type = reinterpret_cast<const TypeDev *>(scratch + kOffType);
  int *queue = reinterpret_cast<int *>(scratch + kOffQueue);
  const int n_items = (n_chars + C - 1) / C;

  if (tid >= kComputeThreads) {
    int cur = 0;
    fetch_implicit(bufs[0], queue, n_items, C, n_chars, type);
    handoff_sync();
    while (bufs[cur].item >= 0) {
      cur ^= 1;
      fetch_implicit(bufs[cur], queue, n_items, C, n_chars, type);
      handoff_sync();
    }
    return;
  }
  bool pending = false;
  int cur = 0;
  handoff_sync();
  for (;;) {
    const ItemBuf &b = bufs[cur];
    if (b.item < 0) break;
    const int Cn = b.C, n = b.T.n, nseg = b.T.nseg;
    const int cs4 = 3 * n + 1;
    const ItemLayout Lt = item_layout(sm, Cn, n, nseg);
    float4 *P = Lt.P;
    if (tid == 0 && pending) {
      bulk_wait_read_all();
      pending = false;
    }
    compute_sync();
    stage_tables<kComputeThreads, false>(b, Lt, tid);
    pass1a_qt(b, P, cs4, q, t, tid);
    compute_sync();
    pass1b(b, Lt, P, cs4, tid);
    compute_sync();
    const float4 *Y = pass2(b, Lt, P, cs4, tid);
    const int W = n * b.cgroups, cpt = b.cpt;
    for (int idx = tid; idx < W; idx += kComputeThreads) {
      const int grp = (int)b.divN.div(idx), j = idx - grp * n;
      const uint32_t info = Lt.jinfo[j];
      const Aff B = ldg_aff(inv_bind + 3 * j);
      const int c1 = min(Cn, (grp + 1) * cpt);
      for (int c = grp * cpt; c < c1; ++c) {
        float4 *slot = P + c * cs4 + 3 * j;
        Aff m = lds_aff(slot);
        if (info & kJ16Link) m = aff_mul(lds_aff(Y + 3 * (c * nseg + (int)(info & kJ16Seg))), m);
        sts_aff(slot, aff_mul(m, B));
      }
    }
    fence_proxy_async_smem();
    compute_sync();
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)n * 48u;
      for (int c = 0; c < Cn; ++c) bulk_store(skin + b.off[c] * 12, P + c * cs4, bytes);
      bulk_commit();
      pending = true;
    }
    cur ^= 1;
    handoff_sync();
  }
  if (tid == 0 && pending) bulk_wait_all();
}

}  // namespace anim

using namespace anim;

extern "C" ANIM_API int anim_forward_local_noalloc(int n_joints, const int32_t *parents, int64_t n_chars,
                                                   const float *d_q, const float *d_t, const float *d_inv_bind,
                                                   float *d_skin, void *stream) {
  if (n_joints < 1 || n_joints > ANIM_MAX_JOINTS) return set_msg(ANIM_EUNSUPPORTED, "n_joints must be in [1, 2048]");
  if (n_chars < 0 || n_chars > (1 << 24)) return set_msg(ANIM_EUNSUPPORTED, "n_chars must be in [0, 16777216]");
  if (!parents || !d_q || !d_t || !d_inv_bind || !d_skin) return set_msg(ANIM_EINVAL, "NULL pointer");
  if (((uintptr_t)d_q | (uintptr_t)d_inv_bind | (uintptr_t)d_skin) & 15u)
    return set_msg(ANIM_EINVAL, "d_q, d_inv_bind and d_skin must be 16-byte aligned");
  for (int i = 0; i < n_joints; ++i)
    if (parents[i] < -1 || parents[i] >= i) return set_msg(ANIM_EINVAL, "parents[i] must be in [-1, i-1]");
  if (n_chars == 0) return ANIM_OK;
  // The tables below reach the device by a copy from this thread's host
  // staging buffer, which the next call overwrites: a graph node recorded
  // from that copy would replay whatever skeleton was staged last.  So a
  // stream that is capturing is refused before anything is enqueued.
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (ce != cudaSuccess) return set_msg(ANIM_ECUDA, cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone) return set_msg(ANIM_EUNSUPPORTED, "stream is capturing");
  }

  // ---- once per device: the device address of the scratch array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return set_msg(ANIM_ECUDA, "cudaGetDevice failed");
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_msg(ANIM_ECUDA, cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  unsigned char *scratch = g_scratch_ptr[dev];

  // ---- segment tables on the host (fixed-size staging, no heap)
  unsigned char *h = g_host.bytes;
  memset(h, 0, kScratchUsed);
  int32_t *par = reinterpret_cast<int32_t *>(h + kOffParent);
  int32_t *start = reinterpret_cast<int32_t *>(h + kOffSegStart);
  int32_t *link = reinterpret_cast<int32_t *>(h + kOffSegLink);
  uint32_t *jinfo = reinterpret_cast<uint32_t *>(h + kOffJinfo);
  memcpy(par, parents, sizeof(int32_t) * n_joints);
  int nseg = 0;
  for (int a = 0; a < n_joints;) {  // natural chains cut into near-equal pieces of <= 16
    int b = a + 1;
    while (b < n_joints && parents[b] == b - 1) ++b;
    const int m = b - a, pieces = (m + kNoAllocSegLen - 1) / kNoAllocSegLen;
    for (int k = 0; k < pieces; ++k) start[nseg++] = a + (int)((long long)m * k / pieces);
    a = b;
  }
  start[nseg] = n_joints;
  static thread_local int16_t seg_of[ANIM_MAX_JOINTS];
  static thread_local int16_t ptr[ANIM_MAX_JOINTS], nxt[ANIM_MAX_JOINTS];
  for (int g = 0; g < nseg; ++g)
    for (int j = start[g]; j < start[g + 1]; ++j) seg_of[j] = (int16_t)g;
  for (int g = 0; g < nseg; ++g) {
    link[g] = parents[start[g]];
    ptr[g] = link[g] < 0 ? -1 : seg_of[link[g]];
  }
  int rounds = 0;
  for (;;) {
    bool any = false;
    for (int g = 0; g < nseg; ++g) any |= ptr[g] >= 0;
    if (!any) break;
    for (int g = 0; g < nseg; ++g) nxt[g] = ptr[g] < 0 ? -1 : ptr[ptr[g]];
    memcpy(ptr, nxt, sizeof(int16_t) * nseg);
    ++rounds;
  }
  for (int j = 0; j < n_joints; ++j) {
    const int g = seg_of[j];
    jinfo[j] = (uint32_t)g | (j == start[g] ? kJStart : 0u) | (link[g] >= 0 ? kJLink : 0u);
  }
  TypeDev T{};
  T.n = n_joints;
  T.nseg = nseg;
  T.rounds = rounds;
  T.parent = reinterpret_cast<const int32_t *>(scratch + kOffParent);
  T.seg_start = reinterpret_cast<const int32_t *>(scratch + kOffSegStart);
  T.seg_link = reinterpret_cast<const int32_t *>(scratch + kOffSegLink);
  T.jinfo = reinterpret_cast<const uint32_t *>(scratch + kOffJinfo);
  T.inv_bind = reinterpret_cast<const float4 *>(d_inv_bind);
  memcpy(h + kOffType, &T, sizeof T);  // queue counter at kOffQueue stays 0 (memset above)

  // ---- launch shape: two resident CTAs per SM, C characters per item
  int sms = 0, smem_sm = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return set_msg(ANIM_ECUDA, "device attribute query failed");
  const size_t budget = std::min((size_t)optin - kStaticSmemAllowance, (size_t)smem_sm / 2 - 1024 - kStaticSmemAllowance);
  int C = std::max(1, std::min(kCMax, 2048 / n_joints));
  while (C > 1 && scan_item_bytes(n_joints, nseg, C) > budget) --C;
  const size_t smem = scan_item_bytes(n_joints, nseg, C);
  if (smem > (size_t)optin - kStaticSmemAllowance) return set_msg(ANIM_EUNSUPPORTED, "skeleton does not fit in shared memory");
  static SmemLimit lim;
  e = ensure_smem_limit((const void *)k_scan_noalloc, lim, smem);
  if (e != cudaSuccess) return set_msg(ANIM_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemcpyAsync(scratch, h, kScratchUsed, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return set_msg(ANIM_ECUDA, cudaGetErrorString(e));
  const long long n_items = ((long long)n_chars + C - 1) / C;
  const int grid = (int)std::min<long long>(n_items, (long long)sms * 2);
  k_scan_noalloc<<<grid, kCtaThreads, smem, st>>>(scratch, (int)n_chars, C, d_q, d_t,
                                                  reinterpret_cast<const float4 *>(d_inv_bind), d_skin);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_msg(ANIM_ECUDA, cudaGetErrorString(e));
  return ANIM_OK;
}
