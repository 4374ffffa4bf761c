// Host runtime behind the C ABI (include/anim.h): context, skeleton analysis
// (segments for the scan, depth-first order for the adjoint), device tables,
// plans and work items, kernel launches, IK state, autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "../../include/anim.h"
#include "anim_internal.h"

using namespace anim;

namespace {

constexpr int kScanThreads = kPersistentThreads;
constexpr int kAdjThreads = kPersistentThreads;
constexpr int kCMax = 64;
constexpr int kTargetJointsPerItem = 2048;
thread_local std::string g_create_error;

// ------------------------------------------------------------ analysis
struct Segments {
  int nseg = 0, rounds = 0;
  std::vector<int32_t> start, link;
  std::vector<uint16_t> seg_of;
  std::vector<uint32_t> jinfo;     // per joint: segment | kJStart | kJLink
};

// Segments: maximal runs of consecutive joints where each joint's parent is
// the previous joint (natural chains), each cut into ceil(m / seg_len)
// pieces of nearly equal length.  Then the number of pointer-jumping rounds
// over the segment tree: ptr[g] = segment the segment g hangs from, doubled
// (ptr[g] = ptr[ptr[g]]) until every pointer is -1.
Segments analyze_segments(const std::vector<int32_t> &par, int seg_len) {
  Segments S;
  const int n = (int)par.size();
  std::vector<int> chain_starts;
  for (int i = 0; i < n; ++i)
    if (i == 0 || par[i] != i - 1) chain_starts.push_back(i);
  chain_starts.push_back(n);
  for (size_t c = 0; c + 1 < chain_starts.size(); ++c) {
    const int a = chain_starts[c], b = chain_starts[c + 1], m = b - a;
    const int pieces = (m + seg_len - 1) / seg_len;
    for (int p = 0; p < pieces; ++p) S.start.push_back(a + (int)((long long)m * p / pieces));
  }
  S.nseg = (int)S.start.size();
  S.start.push_back(n);
  S.seg_of.resize(n);
  for (int g = 0; g < S.nseg; ++g)
    for (int j = S.start[g]; j < S.start[g + 1]; ++j) S.seg_of[j] = (uint16_t)g;
  S.link.resize(S.nseg);
  std::vector<int> ptr(S.nseg);
  for (int g = 0; g < S.nseg; ++g) {
    S.link[g] = par[S.start[g]];
    ptr[g] = S.link[g] < 0 ? -1 : S.seg_of[S.link[g]];
  }
  for (;;) {
    bool any = false;
    for (int g = 0; g < S.nseg; ++g) any |= ptr[g] >= 0;
    if (!any) break;
    std::vector<int> nxt(S.nseg);
    for (int g = 0; g < S.nseg; ++g) nxt[g] = ptr[g] < 0 ? -1 : ptr[ptr[g]];
    ptr.swap(nxt);
    ++S.rounds;
  }
  S.jinfo.resize(n);
  for (int j = 0; j < n; ++j) {
    const int g = S.seg_of[j];
    S.jinfo[j] = (uint32_t)g | (j == S.start[g] ? kJStart : 0u) | (S.link[g] >= 0 ? kJLink : 0u);
  }
  return S;
}

struct DfsOrder {
  std::vector<int32_t> dfs, slot, sub_end;
};

// Depth-first pre-order (children in index order): every subtree occupies
// the contiguous slot range [slot(j), sub_end[slot(j)]).
DfsOrder analyze_dfs(const std::vector<int32_t> &par) {
  const int n = (int)par.size();
  std::vector<std::vector<int>> kids(n);
  std::vector<int> roots;
  for (int i = 0; i < n; ++i) (par[i] < 0 ? roots : kids[par[i]]).push_back(i);
  DfsOrder D;
  D.dfs.reserve(n);
  std::vector<int> st(roots.rbegin(), roots.rend());
  while (!st.empty()) {
    const int u = st.back();
    st.pop_back();
    D.dfs.push_back(u);
    for (auto it = kids[u].rbegin(); it != kids[u].rend(); ++it) st.push_back(*it);
  }
  D.slot.resize(n);
  for (int i = 0; i < n; ++i) D.slot[D.dfs[i]] = i;
  std::vector<int> size(n, 1);
  for (int j = n - 1; j >= 0; --j)
    if (par[j] >= 0) size[par[j]] += size[j];
  D.sub_end.resize(n);
  for (int i = 0; i < n; ++i) D.sub_end[i] = i + size[D.dfs[i]];
  return D;
}

int validate_parents(const int32_t *p, int n) {
  for (int i = 0; i < n; ++i)
    if (p[i] < -1 || p[i] >= i) return i;
  return -1;
}

std::vector<int32_t> depths_of(const std::vector<int32_t> &par) {
  std::vector<int32_t> d(par.size());
  for (size_t i = 0; i < par.size(); ++i) d[i] = par[i] < 0 ? 1 : d[par[i]] + 1;
  return d;
}

int default_seg_len(int) { return 16; }

// ------------------------------------------------------------ walk schedules
// Static lane schedule of the chain-walk frame kernel for one character on
// P lanes.  mode 1: natural chains (consecutive joints, parent[i+1] == i),
// list-scheduled on P lanes: a free lane takes the ready chain with the
// longest path to a leaf; a chain is ready one step after its link joint
// was composed.  Joints that chains hang from keep their model pose in a
// branch slot from their step to the last start that reads it (slots reused
// by interval colouring).  A pure chain longer than kWalkMaxSteps is not
// walked (its one dependent path would take that many steps); the segmented
// kernel's pointer jumping serves it.
struct WalkSched {
  int mode = 0, P = 0, logP = 0, S = 0, nbs = 0;
  int K = 1;                  // steps per staged chunk
  std::vector<uint32_t> tab;  // [S][P], then idle entries up to a multiple of K steps
};

// Steps per staged chunk: K P <= 32 lane-steps (one chunk buffer), K <= 4.
int walk_chunk_steps(int P) { return std::max(1, std::min(4, 32 / P)); }

// Chunk length of a checked schedule; its table gets idle entries up to a
// whole chunk (the kernel copies whole chunks of entries, 16-byte multiples,
// and only the steps < S of key records).
void walk_pad(WalkSched &W) {
  W.K = walk_chunk_steps(W.P);
  const int S = (W.S + W.K - 1) / W.K * W.K;
  W.tab.resize((size_t)S * W.P, kWInvalid);
}

static int ilog2(int p) {
  int l = 0;
  while ((1 << l) < p) ++l;
  return l;
}

WalkSched walk_tree(const std::vector<int32_t> &par, int P) {
  WalkSched W;
  const int n = (int)par.size();
  std::vector<int> cs;
  for (int i = 0; i < n; ++i)
    if (i == 0 || par[i] != i - 1) cs.push_back(i);
  const int nc = (int)cs.size();
  cs.push_back(n);
  std::vector<int> h(n, 1);  // joints on the longest downward path
  for (int j = n - 1; j > 0; --j)
    if (par[j] >= 0) h[par[j]] = std::max(h[par[j]], h[j] + 1);
  std::vector<std::vector<int>> kids(n);  // chains hanging from each joint
  const int kNever = 1 << 30;
  std::vector<int> ready(nc, kNever), start(nc, -1), lane_of(nc, -1), step(n, -1);
  for (int c = 0; c < nc; ++c) {
    const int lk = par[cs[c]];
    if (lk < 0)
      ready[c] = 0;
    else
      kids[lk].push_back(c);
  }
  std::vector<int> lane_free(P, 0);
  for (int it = 0; it < nc; ++it) {
    const int l = (int)(std::min_element(lane_free.begin(), lane_free.end()) - lane_free.begin());
    const int f = lane_free[l];
    int best = -1;
    for (int c = 0; c < nc; ++c)
      if (start[c] < 0 && ready[c] <= f && (best < 0 || h[cs[c]] > h[cs[best]])) best = c;
    if (best < 0)
      for (int c = 0; c < nc; ++c)
        if (start[c] < 0 && ready[c] < kNever &&
            (best < 0 || ready[c] < ready[best] || (ready[c] == ready[best] && h[cs[c]] > h[cs[best]])))
          best = c;
    if (best < 0) return W;  // unreachable for a forest with parent[i] < i
    const int st = std::max(f, ready[best]);
    start[best] = st;
    lane_of[best] = l;
    for (int j = cs[best]; j < cs[best + 1]; ++j) {
      step[j] = st + (j - cs[best]);
      for (int k : kids[j]) ready[k] = step[j] + 1;
    }
    lane_free[l] = st + (cs[best + 1] - cs[best]);
  }
  const int S = *std::max_element(lane_free.begin(), lane_free.end());
  // branch slots: store at step[j], free after the last child chain start
  std::vector<int> bps;
  for (int j = 0; j < n; ++j)
    if (!kids[j].empty()) bps.push_back(j);
  std::sort(bps.begin(), bps.end(), [&](int x, int y) { return step[x] < step[y]; });
  std::vector<int> slot_of(n, -1), slot_free;  // slot_free[s]: last step the slot is read
  for (int j : bps) {
    int last = 0;
    for (int k : kids[j]) last = std::max(last, start[k]);
    int sl = -1;
    for (size_t q = 0; q < slot_free.size(); ++q)
      if (slot_free[q] < step[j]) {
        sl = (int)q;
        break;
      }
    if (sl < 0) {
      sl = (int)slot_free.size();
      slot_free.push_back(0);
    }
    slot_free[sl] = last;
    slot_of[j] = sl;
  }
  if ((int)slot_free.size() > (int)kWRootSlot - 1) return W;
  W.mode = 1;
  W.P = P;
  W.logP = ilog2(P);
  W.S = S;
  W.nbs = (int)slot_free.size();
  W.tab.assign((size_t)S * P, kWInvalid);
  for (int c = 0; c < nc; ++c) {
    const int len = cs[c + 1] - cs[c], lk = par[cs[c]];
    for (int i = 0; i < len; ++i) {
      const int j = cs[c] + i;
      uint32_t e = (uint32_t)j;
      if (i == 0) e |= kWStart | ((lk < 0 ? kWRootSlot : (uint32_t)slot_of[lk]) << kWLoadShift);
      if (slot_of[j] >= 0) e |= kWStore | ((uint32_t)slot_of[j] << kWStoreShift);
      W.tab[(size_t)(start[c] + i) * P + lane_of[c]] = e;
    }
  }
  return W;
}

// Replays a schedule on the host: every joint exactly once, a chain start
// reads the slot its link joint wrote at an earlier step and nobody
// overwrote since, no slot is written and read in the same step, a chain
// continues on its lane at the next step.  Returns false on any violation.
bool walk_check(const WalkSched &W, const std::vector<int32_t> &par) {
  const int n = (int)par.size();
  if (W.mode == 0 || W.P < 1 || W.P > 32 || (W.P & (W.P - 1)) || W.S < 1) return false;
  std::vector<int> seen(n, 0), done_step(n, -1), lane_at(n, -1), owner(std::max(W.nbs, 1), -1);
  for (int s = 0; s < W.S; ++s) {
    std::vector<int> read_slot, write_slot;
    for (int l = 0; l < W.P; ++l) {
      const uint32_t e = W.tab[(size_t)s * W.P + l];
      if (e == kWInvalid) continue;
      const int j = (int)(e & kWJoint);
      if (j >= n || seen[j]++) return false;
      done_step[j] = s;
      lane_at[j] = l;
      if (e & kWStart) {
        const uint32_t ls = (e >> kWLoadShift) & 0xFFu;
        if (par[j] < 0) {
          if (ls != kWRootSlot) return false;
        } else {
          if (ls >= (uint32_t)W.nbs || owner[ls] != par[j] || done_step[par[j]] < 0 || done_step[par[j]] >= s)
            return false;
          read_slot.push_back((int)ls);
        }
      } else if (j == 0 || par[j] != j - 1 || done_step[j - 1] != s - 1 || lane_at[j - 1] != l) {
        return false;
      }
      if (e & kWStore) write_slot.push_back((int)((e >> kWStoreShift) & 0xFFu));
    }
    for (int w : write_slot) {
      if (w >= W.nbs || std::count(read_slot.begin(), read_slot.end(), w)) return false;
    }
    for (int l = 0; l < W.P; ++l) {
      const uint32_t e = W.tab[(size_t)s * W.P + l];
      if (e != kWInvalid && (e & kWStore)) owner[(e >> kWStoreShift) & 0xFFu] = (int)(e & kWJoint);
    }
  }
  for (int j = 0; j < n; ++j)
    if (seen[j] != 1) return false;
  return true;
}

// Pick the type's walk schedule: mode 1 on the lane count whose schedule
// keeps lanes busiest, preferring fewer steps among counts within 15 % of
// the best lane utilization.  A type whose best utilization is below 60 %,
// or whose schedule is longer than kWalkMaxSteps (a pure chain longer than
// that among them), stays off the walk kernel.
WalkSched choose_walk(const std::vector<int32_t> &par) {
  const int n = (int)par.size();
  std::vector<WalkSched> cand;
  double best = 0.0;
  for (int P = 1; P <= 32; P *= 2) {
    WalkSched W = walk_tree(par, P);
    if (W.mode == 0 || W.S > kWalkMaxSteps) continue;
    if (walk_smem_bytes(32 / P, W.nbs) > kWalkMaxSmem) continue;
    if (!walk_check(W, par)) continue;
    best = std::max(best, (double)n / ((double)W.S * P));
    cand.push_back(std::move(W));
  }
  if (best < 0.6) return WalkSched{};
  WalkSched *pick = nullptr;
  for (auto &W : cand)
    if ((double)n / ((double)W.S * W.P) >= 0.85 * best && (!pick || W.S < pick->S)) pick = &W;
  if (!pick) return WalkSched{};
  walk_pad(*pick);
  return std::move(*pick);
}

// ------------------------------------------------------------ rigid transforms
// Host-side double-precision quaternion algebra for the walk kernel's tables
// (quaternions stored x y z w, Hamilton product, R(q) for unit q).
void dq_mul(const double *a, const double *b, double *r) {
  const double x = a[3] * b[0] + a[0] * b[3] + a[1] * b[2] - a[2] * b[1];
  const double y = a[3] * b[1] - a[0] * b[2] + a[1] * b[3] + a[2] * b[0];
  const double z = a[3] * b[2] + a[0] * b[1] - a[1] * b[0] + a[2] * b[3];
  const double w = a[3] * b[3] - a[0] * b[0] - a[1] * b[1] - a[2] * b[2];
  r[0] = x;
  r[1] = y;
  r[2] = z;
  r[3] = w;
}
void dq_conj(const double *a, double *r) {
  r[0] = -a[0];
  r[1] = -a[1];
  r[2] = -a[2];
  r[3] = a[3];
}
void dq_normalize(double *q) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] = n > 0.0 ? q[k] / n : (k == 3 ? 1.0 : 0.0);
}
// r = R(q) v: v + 2 w (u x v) + 2 u x (u x v), u = q.xyz
void dq_rot(const double *q, const double *v, double *r) {
  const double cx = 2.0 * (q[1] * v[2] - q[2] * v[1]), cy = 2.0 * (q[2] * v[0] - q[0] * v[2]),
               cz = 2.0 * (q[0] * v[1] - q[1] * v[0]);
  r[0] = v[0] + q[3] * cx + (q[1] * cz - q[2] * cy);
  r[1] = v[1] + q[3] * cy + (q[2] * cx - q[0] * cz);
  r[2] = v[2] + q[3] * cz + (q[0] * cy - q[1] * cx);
}
// Unit quaternion of a rotation matrix (Shepperd's method: the largest of
// 4w^2, 4x^2, 4y^2, 4z^2 is taken from the diagonal, the others from the
// off-diagonal sums and differences).
void dq_from_rot(const double R[3][3], double *q) {
  const double tr = R[0][0] + R[1][1] + R[2][2];
  if (tr > 0.0) {
    const double s = 2.0 * std::sqrt(tr + 1.0);
    q[3] = 0.25 * s;
    q[0] = (R[2][1] - R[1][2]) / s;
    q[1] = (R[0][2] - R[2][0]) / s;
    q[2] = (R[1][0] - R[0][1]) / s;
  } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
    const double s = 2.0 * std::sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
    q[3] = (R[2][1] - R[1][2]) / s;
    q[0] = 0.25 * s;
    q[1] = (R[0][1] + R[1][0]) / s;
    q[2] = (R[0][2] + R[2][0]) / s;
  } else if (R[1][1] > R[2][2]) {
    const double s = 2.0 * std::sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]);
    q[3] = (R[0][2] - R[2][0]) / s;
    q[0] = (R[0][1] + R[1][0]) / s;
    q[1] = 0.25 * s;
    q[2] = (R[1][2] + R[2][1]) / s;
  } else {
    const double s = 2.0 * std::sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]);
    q[3] = (R[1][0] - R[0][1]) / s;
    q[0] = (R[0][2] + R[2][0]) / s;
    q[1] = (R[1][2] + R[2][1]) / s;
    q[2] = 0.25 * s;
  }
  dq_normalize(q);
}

// ------------------------------------------------------------ device blocks
struct DevBlock {
  void *ptr = nullptr;
  size_t used = 0, cap = 0;
  ~DevBlock() {
    if (ptr) cudaFree(ptr);
  }
};

// One device allocation holding several host vectors, each 256-byte aligned.
struct BlockBuilder {
  std::vector<std::pair<const void *, size_t>> parts;
  size_t total = 0;
  std::vector<size_t> offs;
  size_t add(const void *p, size_t bytes) {
    total = (total + 255) & ~(size_t)255;
    offs.push_back(total);
    parts.push_back({p, bytes});
    total += bytes;
    return offs.back();
  }
  cudaError_t upload(void **dev) {
    std::vector<char> host(std::max<size_t>(total, 1));
    for (size_t k = 0; k < parts.size(); ++k)
      if (parts[k].second) memcpy(host.data() + offs[k], parts[k].first, parts[k].second);
    cudaError_t e = cudaMalloc(dev, std::max<size_t>(total, 16));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dev, host.data(), total, cudaMemcpyHostToDevice);
  }
};

// A skeleton type (or an IK view of one): host analysis + device tables.
struct TypeHost {
  int n = 0, max_depth = 0, seg_len = 8;
  bool is_view = false;             // an internal relabelling of (part of) another type
  std::unique_ptr<TypeHost> adj;    // the adjoint's view of this type (longest path first)
  std::vector<int32_t> parent, depth;
  Segments seg;
  DfsOrder dfsord;
  void *d_tables = nullptr;  // parent, depth, segments, dfs, gather
  float4 *d_inv_bind = nullptr;
  float4 *d_keys = nullptr;
  int n_clips = 0, n_keys = 0;
  float rate = 0.f;
  std::vector<int32_t> gather;  // views only
  std::vector<int32_t> inv_gather;  // views of every joint: type joint -> view joint
  WalkSched ws;                 // chain-walk schedule (mode 0: not walkable)
  bool ws_done = false;
  float4 *d_add = nullptr;      // additive layer keys [n_keys][n][2]
  float4 *d_mesh = nullptr;     // skinned mesh, 3 float4 per vertex
  int n_verts = 0;
  int32_t *d_faces = nullptr;   // [n_faces][3]
  int n_faces = 0;
  float4 *d_wkeys = nullptr;    // schedule-ordered key records, inverse binds folded in
  float4 *d_wu = nullptr;       // schedule-ordered u = R_B^T t_B
  // the inverse binds as rigid transforms (q x y z w, t), when they are
  // rigid: from the rest pose in double precision, or from the given
  // matrices (rotation block orthonormal to 1e-5, determinant > 0)
  bool bind_rigid = false;
  std::vector<double> bind_q, bind_t;  // [n][4], [n][3]
  std::vector<float> keys_h;           // host copy of clips 0 and 1: [clip][key][n][8]
  TypeDev dev{};
  ~TypeHost() {
    for (void *p : {(void *)d_tables, (void *)d_inv_bind, (void *)d_keys, (void *)d_wkeys, (void *)d_wu,
                    (void *)d_mesh, (void *)d_add, (void *)d_faces})
      if (p) cudaFree(p);
  }
  cudaError_t build_tables() {
    seg = analyze_segments(parent, seg_len);
    dfsord = analyze_dfs(parent);
    if (!ws_done) {
      if (!is_view) ws = choose_walk(parent);
      ws_done = true;
    }
    if (!is_view) {
      cudaError_t ev = build_adjoint_view();
      if (ev != cudaSuccess) return ev;
    }
    if (d_tables) {
      cudaFree(d_tables);
      d_tables = nullptr;
    }
    BlockBuilder B;
    const size_t o_par = B.add(parent.data(), parent.size() * 4);
    const size_t o_dep = B.add(depth.data(), depth.size() * 4);
    const size_t o_ss = B.add(seg.start.data(), seg.start.size() * 4);
    const size_t o_sl = B.add(seg.link.data(), seg.link.size() * 4);
    const size_t o_se = B.add(dfsord.sub_end.data(), dfsord.sub_end.size() * 4);
    const size_t o_g = B.add(gather.data(), gather.size() * 4);
    const size_t o_ig = B.add(inv_gather.data(), inv_gather.size() * 4);
    const size_t o_ji = B.add(seg.jinfo.data(), seg.jinfo.size() * 4);
    // 16-bit forms staged by cp.async (jinfo16 padded to an even count)
    std::vector<uint16_t> j16((size_t)(n + (n & 1)), 0);
    std::vector<int16_t> s16(n), p16(n), g16(n);
    for (int j = 0; j < n; ++j) {
      const uint32_t i = seg.jinfo[j];
      j16[j] = (uint16_t)((i & kJ16Seg) | ((i & kJStart) ? kJ16Start : 0u) | ((i & kJLink) ? kJ16Link : 0u));
      s16[j] = (int16_t)dfsord.sub_end[j];
      p16[j] = (int16_t)parent[j];
      g16[j] = (int16_t)(gather.empty() ? j : gather[j]);
    }
    const size_t o_j16 = B.add(j16.data(), j16.size() * 2);
    const size_t o_s16 = B.add(s16.data(), s16.size() * 2);
    const size_t o_p16 = B.add(p16.data(), p16.size() * 2);
    const size_t o_g16 = B.add(g16.data(), g16.size() * 2);
    const size_t o_wt = B.add(ws.tab.data(), ws.tab.size() * 4);
    std::vector<int32_t> blk_out(n);
    for (int j = 0; j < n; ++j) {  // parent of the block-local root of j
      int r = j;
      while (parent[r] >= 0 && parent[r] / 64 == r / 64) r = parent[r];
      blk_out[j] = parent[r];
    }
    const size_t o_bo = B.add(blk_out.data(), blk_out.size() * 4);
    void *d = nullptr;
    cudaError_t e = B.upload(&d);
    if (e != cudaSuccess) {
      if (d) cudaFree(d);
      return e;
    }
    d_tables = d;
    char *base = (char *)d;
    dev.n = n;
    dev.nseg = seg.nseg;
    dev.rounds = seg.rounds;
    dev.max_depth = max_depth;
    dev.chain = n >= 2 && max_depth == n ? 1 : 0;  // depth n with parent[i] < i: parent[i] = i - 1
    dev.parent = (const int32_t *)(base + o_par);
    dev.depth = (const int32_t *)(base + o_dep);
    dev.seg_start = (const int32_t *)(base + o_ss);
    dev.seg_link = (const int32_t *)(base + o_sl);
    dev.sub_end = (const int32_t *)(base + o_se);
    dev.gather = gather.empty() ? nullptr : (const int32_t *)(base + o_g);
    dev.inv_gather = inv_gather.empty() ? nullptr : (const int32_t *)(base + o_ig);
    dev.jinfo = (const uint32_t *)(base + o_ji);
    dev.jinfo16 = (const uint16_t *)(base + o_j16);
    dev.sub16 = (const int16_t *)(base + o_s16);
    dev.par16 = (const int16_t *)(base + o_p16);
    dev.gat16 = (const int16_t *)(base + o_g16);
    dev.wk_mode = ws.mode;
    dev.wk_P = ws.P;
    dev.wk_logP = ws.logP;
    dev.wk_S = ws.S;
    dev.wk_nbs = ws.nbs;
    dev.wk_K = ws.K;
    dev.wk_tab = ws.mode ? (const uint32_t *)(base + o_wt) : nullptr;
    dev.blk_out = (const int32_t *)(base + o_bo);
    sync_dev();
    return cudaSuccess;
  }
  cudaError_t build_adjoint_view();
  void sync_dev() {
    dev.n_clips = n_clips;
    dev.n_keys = n_keys;
    dev.rate = rate;
    dev.inv_bind = d_inv_bind;
    dev.keys = d_keys;
    dev.add_keys = d_add;
    dev.wk_keys = d_wkeys;
    dev.wk_u = d_wu;
    dev.n_verts = n_verts;
    dev.mesh = d_mesh;
    dev.n_faces = n_faces;
    dev.faces = d_faces;
  }
  bool walk_ready() const { return ws.mode != 0 && d_wkeys != nullptr; }
  // Key-pair records with the inverse binds folded in (skin-space walk), for
  // a walkable type with rigid inverse binds and clips (synchronous; without
  // them the tables stay empty and the type runs on the segmented kernel).
  // Record of (clip c, key k, joint j), parent pj, keys a = key k and b = key
  // k + 1 (mod n_keys) of joint j, normalized, b on a's hemisphere:
  //   theta = 2 atan2(|a - b|, |a + b|),  q_perp = (b - (a.b) a) / |...| (0 if
  //   b == a),  and with the parent's inverse bind (q_Bp, t_Bp) (identity at
  //   a root) and the joint's q_Bj folded in:
  //   q0' = conj(q_Bp) a q_Bj,  q_perp' = conj(q_Bp) q_perp q_Bj,
  //   t0' = R(conj(q_Bp)) (t_a - t_Bp),  dt' = R(conj(q_Bp)) (t_b - t_a),
  // stored as 4 float4 (q0', q_perp', (t0', theta), (dt', 0)); u of joint j is
  // R(conj(q_Bj)) t_Bj.  Built per joint, then laid out in the walk
  // schedule's order [clip][key][S][4][P] (d_wkeys) and [S][P] (d_wu).
  // Computed in double, stored as float.
  cudaError_t build_walk_data() {
    for (float4 **p : {&d_wkeys, &d_wu}) {
      if (*p) cudaFree(*p);
      *p = nullptr;
    }
    if (ws.mode == 0 || !bind_rigid || n_clips == 0 || keys_h.empty()) {
      sync_dev();
      return cudaSuccess;
    }
    const int nc = std::min(n_clips, 2), nk = n_keys;
    const double ident[4] = {0.0, 0.0, 0.0, 1.0}, zero[3] = {0.0, 0.0, 0.0};
    std::vector<float4> frec((size_t)nc * nk * n * 4), fu((size_t)n);
    for (int j = 0; j < n; ++j) {
      const int pj = parent[j];
      const double *qBj = &bind_q[4 * j], *tBj = &bind_t[3 * j];
      const double *qBp = pj >= 0 ? &bind_q[4 * pj] : ident, *tBp = pj >= 0 ? &bind_t[3 * pj] : zero;
      double cBp[4], cBj[4], uj[3];
      dq_conj(qBp, cBp);
      dq_conj(qBj, cBj);
      dq_rot(cBj, tBj, uj);
      fu[j] = make_float4((float)uj[0], (float)uj[1], (float)uj[2], 0.f);
      for (int c = 0; c < nc; ++c)
        for (int k = 0; k < nk; ++k) {
          const int k1 = k + 1 == nk ? 0 : k + 1;
          const float *ka = &keys_h[(((size_t)c * nk + k) * n + j) * 8];
          const float *kb = &keys_h[(((size_t)c * nk + k1) * n + j) * 8];
          double a[4], b[4];
          for (int m = 0; m < 4; ++m) {
            a[m] = ka[m];
            b[m] = kb[m];
          }
          dq_normalize(a);
          dq_normalize(b);
          double d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
          if (d < 0.0) {
            for (int m = 0; m < 4; ++m) b[m] = -b[m];
            d = -d;
          }
          double dm = 0.0, dp = 0.0, v[4], nv = 0.0;
          for (int m = 0; m < 4; ++m) {
            dm += (a[m] - b[m]) * (a[m] - b[m]);
            dp += (a[m] + b[m]) * (a[m] + b[m]);
            v[m] = b[m] - d * a[m];
            nv += v[m] * v[m];
          }
          const double theta = 2.0 * std::atan2(std::sqrt(dm), std::sqrt(dp));
          nv = std::sqrt(nv);
          for (int m = 0; m < 4; ++m) v[m] = nv > 0.0 ? v[m] / nv : 0.0;
          double q0[4], qp[4], tmp[4], ta[3], dt[3], t0f[3], dtf[3];
          dq_mul(cBp, a, tmp);
          dq_mul(tmp, qBj, q0);
          dq_mul(cBp, v, tmp);
          dq_mul(tmp, qBj, qp);
          for (int m = 0; m < 3; ++m) {
            ta[m] = (double)ka[4 + m] - tBp[m];
            dt[m] = (double)kb[4 + m] - (double)ka[4 + m];
          }
          dq_rot(cBp, ta, t0f);
          dq_rot(cBp, dt, dtf);
          float4 *r = &frec[(((size_t)c * nk + k) * n + j) * 4];
          r[0] = make_float4((float)q0[0], (float)q0[1], (float)q0[2], (float)q0[3]);
          r[1] = make_float4((float)qp[0], (float)qp[1], (float)qp[2], (float)qp[3]);
          r[2] = make_float4((float)t0f[0], (float)t0f[1], (float)t0f[2], (float)theta);
          r[3] = make_float4((float)dtf[0], (float)dtf[1], (float)dtf[2], 0.f);
        }
    }
    std::vector<std::pair<float4 **, const std::vector<float4> *>> up;
    std::vector<float4> wrec, wu;
    {  // the records in the walk schedule's order
      const int P = ws.P, S = ws.S;
      wrec.assign((size_t)nc * nk * S * 4 * P, make_float4(0.f, 0.f, 0.f, 0.f));
      wu.assign((size_t)S * P, make_float4(0.f, 0.f, 0.f, 0.f));
      for (int st = 0; st < S; ++st)
        for (int p = 0; p < P; ++p) {
          const uint32_t e = ws.tab[(size_t)st * P + p];
          if (e == kWInvalid) continue;
          const int j = (int)(e & kWJoint);
          wu[(size_t)st * P + p] = fu[j];
          for (int c = 0; c < nc; ++c)
            for (int k = 0; k < nk; ++k)
              for (int f = 0; f < 4; ++f)
                wrec[((((size_t)c * nk + k) * S + st) * 4 + f) * P + p] = frec[(((size_t)c * nk + k) * n + j) * 4 + f];
        }
      up.push_back({&d_wkeys, &wrec});
      up.push_back({&d_wu, &wu});
    }
    cudaError_t e = cudaSuccess;
    for (auto &u : up) {
      if (e == cudaSuccess) e = cudaMalloc(u.first, u.second->size() * sizeof(float4));
      if (e == cudaSuccess)
        e = cudaMemcpy(*u.first, u.second->data(), u.second->size() * sizeof(float4), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess)
      for (float4 **p : {&d_wkeys, &d_wu}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
      }
    sync_dev();
    return e;
  }
  // Inverse binds as rigid transforms: from the rest pose (composed down
  // the joint list in double, then inverted), or from 3x4 matrices when
  // their rotation blocks are rotations to 1e-5.
  void set_bind_from_rest(const float *rq, const float *rt) {
    bind_q.assign(4 * (size_t)n, 0.0);
    bind_t.assign(3 * (size_t)n, 0.0);
    std::vector<double> gq(4 * (size_t)n), gt(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
      double q[4] = {rq[4 * i], rq[4 * i + 1], rq[4 * i + 2], rq[4 * i + 3]}, t[3] = {rt[3 * i], rt[3 * i + 1],
                                                                                  rt[3 * i + 2]};
      dq_normalize(q);
      const int p = parent[i];
      if (p < 0) {
        std::copy(q, q + 4, &gq[4 * i]);
        std::copy(t, t + 3, &gt[3 * i]);
      } else {
        double r[3];
        dq_mul(&gq[4 * p], q, &gq[4 * i]);
        dq_rot(&gq[4 * p], t, r);
        for (int m = 0; m < 3; ++m) gt[3 * i + m] = gt[3 * p + m] + r[m];
      }
      double cq[4], r[3];
      dq_conj(&gq[4 * i], cq);
      dq_rot(cq, &gt[3 * i], r);
      std::copy(cq, cq + 4, &bind_q[4 * i]);
      for (int m = 0; m < 3; ++m) bind_t[3 * i + m] = -r[m];
    }
    bind_rigid = true;
  }
  void set_bind_from_matrices(const float *B) {
    bind_q.assign(4 * (size_t)n, 0.0);
    bind_t.assign(3 * (size_t)n, 0.0);
    bind_rigid = true;
    for (int i = 0; i < n && bind_rigid; ++i) {
      const float *m = B + 12 * (size_t)i;
      double R[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[r][c] = m[4 * r + c];
      double worst = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double d = 0.0;
          for (int r = 0; r < 3; ++r) d += R[r][a] * R[r][b];
          worst = std::max(worst, std::fabs(d - (a == b ? 1.0 : 0.0)));
        }
      const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                         R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                         R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
      if (!(worst <= 1e-5) || !(det > 0.0)) {
        bind_rigid = false;
        break;
      }
      dq_from_rot(R, &bind_q[4 * i]);
      for (int r = 0; r < 3; ++r) bind_t[3 * i + r] = m[4 * r + 3];
    }
    if (!bind_rigid) {
      bind_q.clear();
      bind_t.clear();
    }
  }
};

// A view of the joints j with keep[j] (closed under parent) of type T,
// numbered in depth-first pre-order that visits the child with the longest
// path to a leaf first: natural chains then follow the longest paths, which
// shortens the segment tree (fewer pointer-jumping rounds).  gather maps a
// view joint to T's joint; vid (if given) receives T's joint -> view joint.
std::unique_ptr<TypeHost> make_view(const TypeHost &T, const std::vector<char> &keep, std::vector<int> *vid_out,
                                    cudaError_t *err) {
  const int n = T.n;
  std::vector<std::vector<int>> kids(n);
  std::vector<int> roots, h(n, 1);
  for (int j = n - 1; j >= 0; --j) {
    if (!keep[j]) continue;
    const int p = T.parent[j];
    if (p < 0)
      roots.push_back(j);
    else {
      kids[p].push_back(j);
      h[p] = std::max(h[p], h[j] + 1);
    }
  }
  std::reverse(roots.begin(), roots.end());
  auto V = std::make_unique<TypeHost>();
  V->is_view = true;
  std::vector<int> vid(n, -1), st(roots.rbegin(), roots.rend());
  while (!st.empty()) {
    const int u = st.back();
    st.pop_back();
    vid[u] = (int)V->gather.size();
    V->gather.push_back(u);
    auto &k = kids[u];
    std::stable_sort(k.begin(), k.end(), [&](int a, int b) { return h[a] != h[b] ? h[a] > h[b] : a < b; });
    for (auto it = k.rbegin(); it != k.rend(); ++it) st.push_back(*it);
  }
  V->n = (int)V->gather.size();
  if (V->n == n) V->inv_gather.assign(vid.begin(), vid.end());
  for (int j : V->gather) V->parent.push_back(T.parent[j] < 0 ? -1 : vid[T.parent[j]]);
  V->depth = depths_of(V->parent);
  V->max_depth = *std::max_element(V->depth.begin(), V->depth.end());
  V->seg_len = T.seg_len;
  *err = V->build_tables();
  // the adjoint kernel relies on the view's depth-first slots being its
  // joint indices
  for (int i = 0; i < V->n && *err == cudaSuccess; ++i)
    if (V->dfsord.dfs[i] != i) *err = cudaErrorInvalidValue;
  if (vid_out) *vid_out = std::move(vid);
  return V;
}

cudaError_t TypeHost::build_adjoint_view() {
  cudaError_t e = cudaSuccess;
  adj = make_view(*this, std::vector<char>(n, 1), nullptr, &e);
  return e;
}

struct Sched {
  int C = 1;  // characters per item
};

}  // namespace

// ------------------------------------------------------------ ABI objects
struct anim_plan {
  anim_ctx *ctx = nullptr;
  int64_t n_chars = 0;
  std::vector<int32_t> char_type;
  std::vector<int64_t> row_off;
  std::vector<int> used;                      // type ids, most costly first
  std::vector<std::vector<int32_t>> by_type;  // characters of each used type (indexed like used)
  std::vector<int> C_scan, C_adj;             // per ctx type id
  std::vector<int> C_frame;                   // plain frame: characters per (q, t) item
  int64_t total = 0;
  int version = -1;  // schedule version the items were built for
  // device
  int32_t *d_char_type = nullptr;
  int64_t *d_row_off = nullptr;
  int32_t *d_type_chars = nullptr;  // characters grouped by type in `used` order
  std::vector<int> type_chars_start;
  WorkItem *d_items_scan = nullptr, *d_items_adj = nullptr;
  int n_items_scan = 0, n_items_adj = 0;
  int32_t *d_sorted = nullptr;
  WorkItem *d_items_frame = nullptr;
  RangeDev *d_ranges = nullptr;
  int n_ranges = 0, n_slots = 0;
  int *d_queue = nullptr;  // work-queue heads and finished-CTA counters, back to 0 after each launch:
                           // [2], [3] the plain frame's CTA kernel; [0], [1] every other persistent launch
  int32_t *d_used = nullptr, *d_cap = nullptr;
  LaunchCfg cfg_scan{}, cfg_adj{};
  size_t smem_frame = 0;     // plain frame, (q, t) items
  size_t smem_frame_mat = 0; // frame with skinning or layers, matrix items
  int adj_unfit = -1;
  // frame: item slots [0, n_slots_walk) belong to the chain-walk kernel
  // (queue counters d_queue[0..1]), the rest to the segmented CTA kernel
  // (d_queue[2..3])
  int n_slots_walk = 0;
  int walk_nbs = 0;
  size_t walk_smem = 0;
  // frame with skinning: every type on the segmented CTA kernel (its own
  // range layout when the frame's layout gives some types to the walk kernel)
  RangeDev *d_ranges_cta = nullptr;
  int32_t *d_cap_cta = nullptr;
  int n_ranges_cta = 0, n_slots_cta = 0;
  RangeDev *d_ranges_qa = nullptr;  // (q, t) items of every type: the frame with layered blending
  int32_t *d_cap_qa = nullptr;
  int n_ranges_qa = 0, n_slots_qa = 0;
  std::vector<int64_t> vert_off;  // [n_chars + 1]
  int64_t *d_vert_off = nullptr;
  float *d_host_in = nullptr, *d_host_skin = nullptr;  // staging of the host-buffer frame
  // host-buffer frame: the characters in contiguous ranges, each a plan of its
  // own (registered with the context, destroyed with this plan), so that a
  // range's copy-out on copy_stream overlaps the next range's frame
  std::vector<anim_plan *> host_parts;
  std::vector<int64_t> part_char0;  // first character of each range, then n_chars
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> part_ev;  // range i's frame done (on the call's stream)
  cudaEvent_t copy_ev = nullptr;     // every copy-out issued so far done (on copy_stream)
  ~anim_plan() {
    for (cudaEvent_t e : part_ev)
      if (e) cudaEventDestroy(e);
    if (copy_ev) cudaEventDestroy(copy_ev);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (void *p : {(void *)d_char_type, (void *)d_row_off, (void *)d_type_chars, (void *)d_items_scan,
                    (void *)d_items_adj, (void *)d_sorted, (void *)d_items_frame, (void *)d_ranges,
                    (void *)d_queue, (void *)d_used,
                    (void *)d_cap, (void *)d_ranges_cta, (void *)d_cap_cta, (void *)d_vert_off,
                    (void *)d_ranges_qa, (void *)d_cap_qa,
                    (void *)d_host_in, (void *)d_host_skin})
      if (p) cudaFree(p);
  }
};

struct anim_ik {
  anim_ctx *ctx = nullptr;
  const anim_plan *plan = nullptr;
  int n_eff = 0;
  std::vector<std::unique_ptr<TypeHost>> views;  // indexed by ctx type id (null if unused)
  TypeDev *d_views = nullptr;
  int32_t *d_eff = nullptr;
  WorkItem *d_items = nullptr;
  int n_items = 0;
  int *d_counters = nullptr;  // [0] queue, [1] step, [2] done
  // the object's own Adam state (m rows, then v rows): one row per view
  // joint of each character, character c's rows from d_state_off[c]
  float *d_state = nullptr;
  int64_t *d_state_off = nullptr;
  int64_t state_rows = 0;
  LaunchCfg cfg{};
  ~anim_ik() {
    for (void *p : {(void *)d_views, (void *)d_eff, (void *)d_items, (void *)d_counters, (void *)d_state,
                    (void *)d_state_off})
      if (p) cudaFree(p);
  }
};

struct anim_ctx {
  int device = 0;
  int sm_count = 0;
  size_t smem_optin = 0, smem_per_sm = 0;
  std::string err;
  std::vector<std::unique_ptr<TypeHost>> types;
  TypeDev *d_types = nullptr;
  TypeDev *d_adj_types = nullptr;  // the types' adjoint views, same ids
  int *d_status = nullptr;
  int version = 0;  // bumps when types/schedules change
  int ctas_per_sm = 2;            // resident persistent CTAs per SM the schedule is sized for
  int use_walk = 1;               // frame: walkable types run on the chain-walk kernel (2: its
                                  // warp-specialized variant)
  int adj_ctas = 0;               // adjoint: 0 = persistent kernel, k = one-item kernel sized for k CTAs per SM
  cudaStream_t side = nullptr;    // frame: the CTA kernel's stream when both kernels have work
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int joints_per_item = kTargetJointsPerItem;  // target work-item size (characters x joints)
  std::set<anim_plan *> plans;
  std::set<anim_ik *> iks;
  struct TuneChoice {
    int seg_len, ctas_per_sm, joints_per_item, walk, adj_ctas;
    float ms;
  };
  std::map<uint64_t, TuneChoice> tune_cache;  // (which, types, counts) hash -> best schedule
  ~anim_ctx() {
    for (auto *p : plans) delete p;
    for (auto *k : iks) delete k;
    if (d_types) cudaFree(d_types);
    if (d_adj_types) cudaFree(d_adj_types);
    if (d_status) cudaFree(d_status);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
  }
};

namespace {

int fail(anim_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_create_error = buf;
  return code;
}

#define CK(call)                                                                                       \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return fail(ctx, ANIM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned4(const void *p) { return ((uintptr_t)p & 3u) == 0; }

cudaError_t upload_types(anim_ctx *ctx) {
  std::vector<TypeDev> host(ctx->types.size()), hadj(ctx->types.size());
  for (size_t t = 0; t < ctx->types.size(); ++t) {
    ctx->types[t]->sync_dev();
    host[t] = ctx->types[t]->dev;
    hadj[t] = ctx->types[t]->adj->dev;
  }
  for (TypeDev **d : {&ctx->d_types, &ctx->d_adj_types}) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    cudaError_t e = cudaMalloc(d, std::max<size_t>(1, host.size()) * sizeof(TypeDev));
    if (e != cudaSuccess) return e;
  }
  ++ctx->version;
  cudaError_t e = cudaMemcpy(ctx->d_types, host.data(), host.size() * sizeof(TypeDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(ctx->d_adj_types, hadj.data(), hadj.size() * sizeof(TypeDev), cudaMemcpyHostToDevice);
}

size_t smem_budget(const anim_ctx *ctx) {
  // ctas_per_sm resident CTAs per SM: each also takes 1 KB of system shared
  // memory and the kernels' static shared memory (staged work items)
  const size_t per = ctx->smem_per_sm / (size_t)ctx->ctas_per_sm;
  return std::min(ctx->smem_optin - kStaticSmemAllowance, per - 1024 - kStaticSmemAllowance);
}

// Shared memory one work item of the adjoint may use: the persistent
// kernel's budget, or a 1/adj_ctas share of the SM for the one-item kernel.
size_t adj_budget(const anim_ctx *ctx) {
  if (ctx->adj_ctas <= 0) return smem_budget(ctx);
  return ctx->smem_per_sm / (size_t)ctx->adj_ctas - 1024 - kAdjSmallStatic;
}

// Characters per work item: kind 0 the matrix scan, 1 the adjoint, 2 the
// plain frame's (q, t) items.
int choose_C(const anim_ctx *ctx, const TypeHost &T, int kind) {
  const bool adjoint = kind == 1;
  const size_t budget = adjoint ? adj_budget(ctx) : smem_budget(ctx);
  int C = std::max(1, std::min(kCMax, ctx->joints_per_item / std::max(1, T.n)));
  auto bytes = [&](int c) {
    return kind == 1 ? adjoint_smem_bytes(T.n, T.seg.nseg, c)
                     : kind == 2 ? scan_qt_smem_bytes(T.n, T.seg.nseg, c) : scan_smem_bytes(T.n, T.seg.nseg, c);
  };
  while (C > 1 && bytes(C) > budget) --C;
  if (bytes(C) > ctx->smem_optin - kStaticSmemAllowance) return 0;
  return C;
}

template <class T>
cudaError_t upload_vec(T **dev, const std::vector<T> &v) {
  if (*dev) cudaFree(*dev);
  *dev = nullptr;
  cudaError_t e = cudaMalloc((void **)dev, std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*dev, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Work items (C characters of one type) in `used` order; start indexes the
// type-grouped character list.
std::vector<WorkItem> make_items(const anim_plan *P, const std::vector<int> &Cv) {
  std::vector<WorkItem> items;
  for (size_t u = 0; u < P->used.size(); ++u) {
    const int t = P->used[u];
    const int cnt = (int)P->by_type[u].size(), C = Cv[t];
    for (int k = 0; k < cnt; k += C) {
      WorkItem w;
      w.start = P->type_chars_start[u] + k;
      w.count = std::min(C, cnt - k);
      w.type = t;
      w.k0 = 0;
      items.push_back(w);
    }
  }
  return items;
}

// (Re)build the schedule-dependent parts of a plan: characters per item,
// static items, launch configurations.
int plan_schedule(anim_ctx *ctx, anim_plan *P) {
  if (P->version == ctx->version) return ANIM_OK;
  const int nt = (int)ctx->types.size();
  P->C_scan.assign(nt, 1);
  P->C_adj.assign(nt, 1);
  P->C_frame.assign(nt, 1);
  P->adj_unfit = -1;
  size_t smem_s = 0, smem_a = 0, smem_q = 0;
  for (int t : P->used) {
    const TypeHost &T = *ctx->types[t];
    const int cs = choose_C(ctx, T, 0), ca = choose_C(ctx, *T.adj, 1);
    if (cs == 0)
      return fail(ctx, ANIM_EUNSUPPORTED,
                  "type %d (%d joints, %d segments) does not fit in shared memory with one character", t, T.n,
                  T.seg.nseg);
    P->C_scan[t] = cs;
    P->C_frame[t] = std::max(cs, choose_C(ctx, T, 2));  // (q, t) items are smaller
    smem_s = std::max(smem_s, scan_smem_bytes(T.n, T.seg.nseg, cs));
    smem_q = std::max(smem_q, scan_qt_smem_bytes(T.n, T.seg.nseg, P->C_frame[t]));
    // the adjoint keeps two more vectors per joint: a schedule may fit the
    // forward kernels and not the adjoint, which then refuses to run
    if (ca == 0) {
      if (P->adj_unfit < 0) P->adj_unfit = t;
      continue;
    }
    P->C_adj[t] = ca;
    smem_a = std::max(smem_a, adjoint_smem_bytes(T.adj->n, T.adj->seg.nseg, ca));
  }
  // static items: (q, t) items for the forward from local poses, adjoint items
  auto is = make_items(P, P->C_frame), ia = make_items(P, P->C_adj);
  P->n_items_scan = (int)is.size();
  P->n_items_adj = (int)ia.size();
  CK(upload_vec(&P->d_items_scan, is));
  CK(upload_vec(&P->d_items_adj, ia));
  // plain frame: walkable types (chain-walk kernel, 32 / P characters per
  // item) take the first item regions, the others ((q, t) items) follow
  std::vector<int32_t> cap(P->C_frame);
  std::vector<char> walk_t(nt, 0);
  int wcmax = 0;
  size_t smem_f = 0;
  P->walk_nbs = 0;
  for (int t : P->used) {
    const TypeHost &T = *ctx->types[t];
    if (!ctx->use_walk || !T.walk_ready()) {
      smem_f = std::max(smem_f, scan_qt_smem_bytes(T.n, T.seg.nseg, P->C_frame[t]));
      continue;
    }
    walk_t[t] = 1;
    cap[t] = 32 / T.ws.P;
    wcmax = std::max(wcmax, cap[t]);
    P->walk_nbs = std::max(P->walk_nbs, T.ws.nbs);
  }
  CK(upload_vec(&P->d_cap, cap));
  // frame work queue: ranges of <= kRangeChars characters of one type, each
  // with an item slot region large enough for any key distribution
  std::vector<RangeDev> ranges;
  int slots = 0;
  P->n_slots_walk = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (size_t u = 0; u < P->used.size(); ++u) {
      const int t = P->used[u];
      if (walk_t[t] != (pass == 0)) continue;
      const int cnt = (int)P->by_type[u].size(), C = cap[t], nk = ctx->types[t]->n_keys;
      const int rc = pass == 0 ? kRangeCharsMax : kRangeChars;
      for (int k = 0; k < cnt; k += rc) {
        RangeDev r;
        r.type = t;
        r.start = P->type_chars_start[u] + k;
        r.count = std::min(rc, cnt - k);
        r.region = slots;
        slots += (r.count + C - 1) / C + std::min(r.count, std::max(nk, 1));
        ranges.push_back(r);
      }
    }
    if (pass == 0) P->n_slots_walk = slots;
  }
  const bool walk2 = ctx->use_walk == 2;
  P->walk_smem = P->n_slots_walk == 0 ? 0 : walk2 ? walk2_smem_bytes(wcmax, P->walk_nbs)
                                                   : walk_smem_bytes(wcmax, P->walk_nbs);
  if (walk2 && P->n_slots_walk > 0) P->walk_smem = walk2_spread_smem(P->walk_smem, P->n_slots_walk, ctx->sm_count);
  if (P->n_slots_walk > 0 &&
      (walk2 ? walk2_blocks_per_sm(P->walk_smem) : walk_blocks_per_sm(P->walk_smem)) < 1)
    return fail(ctx, ANIM_EUNSUPPORTED, "chain-walk kernel: no resident CTA at %zu bytes of shared memory",
                P->walk_smem);
  P->n_ranges = (int)ranges.size();
  P->n_slots = slots;
  CK(upload_vec(&P->d_ranges, ranges));
  // layouts of every type on one kernel: matrix items (the frame with
  // skinning) and (q, t) items (the frame with layered blending)
  auto all_types = [&](const std::vector<int> &Cv, std::vector<RangeDev> &out) {
    int sl = 0;
    for (size_t u = 0; u < P->used.size(); ++u) {
      const int t = P->used[u];
      const int cnt = (int)P->by_type[u].size(), C = Cv[t], nk = ctx->types[t]->n_keys;
      for (int k = 0; k < cnt; k += kRangeChars) {
        RangeDev r;
        r.type = t;
        r.start = P->type_chars_start[u] + k;
        r.count = std::min(kRangeChars, cnt - k);
        r.region = sl;
        sl += (r.count + C - 1) / C + std::min(r.count, std::max(nk, 1));
        out.push_back(r);
      }
    }
    return sl;
  };
  std::vector<RangeDev> ranges_cta, ranges_qa;
  const int slots_cta = all_types(P->C_scan, ranges_cta), slots_qa = all_types(P->C_frame, ranges_qa);
  P->n_ranges_cta = (int)ranges_cta.size();
  P->n_slots_cta = slots_cta;
  CK(upload_vec(&P->d_ranges_cta, ranges_cta));
  CK(upload_vec(&P->d_cap_cta, P->C_scan));
  P->n_ranges_qa = (int)ranges_qa.size();
  P->n_slots_qa = slots_qa;
  CK(upload_vec(&P->d_ranges_qa, ranges_qa));
  CK(upload_vec(&P->d_cap_qa, P->C_frame));
  P->vert_off.assign(P->n_chars + 1, 0);
  for (int64_t c = 0; c < P->n_chars; ++c)
    P->vert_off[c + 1] = P->vert_off[c] + ctx->types[P->char_type[c]]->n_verts;
  CK(upload_vec(&P->d_vert_off, P->vert_off));
  if (P->d_items_frame) cudaFree(P->d_items_frame);
  P->d_items_frame = nullptr;
  CK(cudaMalloc(&P->d_items_frame, std::max({1, slots, slots_cta, slots_qa}) * sizeof(WorkItem)));
  const int grid = ctx->sm_count * ctx->ctas_per_sm;
  P->cfg_scan = {kScanThreads, std::max(1, std::min(grid, P->n_items_scan)), std::max<size_t>(smem_q, 16),
                 ctx->ctas_per_sm >= 3 ? 3 : 2};
  if (ctx->adj_ctas > 0)
    P->cfg_adj = {kAdjSmallThreads, std::max(1, P->n_items_adj), std::max<size_t>(smem_a, 16)};
  else
    P->cfg_adj = {kAdjThreads, std::max(1, std::min(grid, P->n_items_adj)), std::max<size_t>(smem_a, 16),
                  ctx->ctas_per_sm >= 3 ? 3 : 2};
  P->smem_frame = std::max<size_t>(smem_f, 16);
  P->smem_frame_mat = std::max<size_t>(smem_s, 16);
  P->version = ctx->version;
  return ANIM_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int anim_version(void) { return 10000; }

const char *anim_last_error(const anim_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int anim_create(anim_ctx **out, int device) {
  anim_ctx *ctx = nullptr;
  if (!out) return fail(nullptr, ANIM_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(nullptr, ANIM_EDEVICE, "no CUDA device");
  if (device < 0 || device >= ndev) return fail(nullptr, ANIM_EINVAL, "device %d out of range", device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return fail(nullptr, ANIM_ECUDA, "device query failed");
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, ANIM_EDEVICE, "device %d is sm_%d%d; this library is built for sm_103a", device, prop.major,
                prop.minor);
  if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, ANIM_ECUDA, "cudaSetDevice failed");
  ctx = new (std::nothrow) anim_ctx();
  if (!ctx) return fail(nullptr, ANIM_ENOMEM, "out of host memory");
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  ctx->smem_per_sm = prop.sharedMemPerMultiprocessor;
  if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return fail(nullptr, ANIM_ENOMEM, "device allocation failed");
  }
  *out = ctx;
  return ANIM_OK;
}

int anim_destroy(anim_ctx *ctx) {
  if (!ctx) return ANIM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  delete ctx;
  return ANIM_OK;
}

int anim_create_skeletons(anim_ctx *ctx, int n_types, const int32_t *joint_counts, const int32_t *parents,
                          const float *inv_bind, const float *rest_q, const float *rest_t, int32_t *out_type_ids) {
  if (!ctx) return ANIM_EINVAL;
  if (n_types <= 0 || !joint_counts || !parents || !out_type_ids)
    return fail(ctx, ANIM_EINVAL, "n_types must be > 0 and joint_counts, parents, out_type_ids non-NULL");
  if (!inv_bind && (!rest_q || !rest_t)) return fail(ctx, ANIM_EINVAL, "inv_bind is NULL: rest_q and rest_t are required");
  if ((int)ctx->types.size() + n_types > kMaxTypes) return fail(ctx, ANIM_EUNSUPPORTED, "more than %d types", kMaxTypes);
  CK(cudaSetDevice(ctx->device));
  int64_t off = 0;
  for (int t = 0; t < n_types; ++t) {
    const int n = joint_counts[t];
    if (n < 1 || n > ANIM_MAX_JOINTS) return fail(ctx, ANIM_EINVAL, "type %d: joint count %d not in [1, %d]", t, n, ANIM_MAX_JOINTS);
    const int bad = validate_parents(parents + off, n);
    if (bad >= 0)
      return fail(ctx, ANIM_EINVAL, "type %d: parent[%d] = %d violates -1 <= parent[i] < i", t, bad, parents[off + bad]);
    off += n;
  }
  off = 0;
  const int first = (int)ctx->types.size();
  for (int t = 0; t < n_types; ++t) {
    const int n = joint_counts[t];
    auto T = std::make_unique<TypeHost>();
    T->n = n;
    T->parent.assign(parents + off, parents + off + n);
    T->depth = depths_of(T->parent);
    T->max_depth = *std::max_element(T->depth.begin(), T->depth.end());
    T->seg_len = default_seg_len(n);
    CK(T->build_tables());
    CK(cudaMalloc(&T->d_inv_bind, (size_t)n * 48));
    if (inv_bind) {
      CK(cudaMemcpy(T->d_inv_bind, inv_bind + off * 12, (size_t)n * 48, cudaMemcpyHostToDevice));
    } else {
      float *dq = nullptr, *dt = nullptr;
      CK(cudaMalloc(&dq, (size_t)n * 16));
      if (cudaMalloc(&dt, (size_t)n * 12) != cudaSuccess) {
        cudaFree(dq);
        return fail(ctx, ANIM_ENOMEM, "device allocation failed");
      }
      cudaError_t e = cudaMemcpy(dq, rest_q + off * 4, (size_t)n * 16, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(dt, rest_t + off * 3, (size_t)n * 12, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = launch_bind_from_rest(T->dev.parent, dq, dt, n, T->d_inv_bind, 0);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      cudaFree(dq);
      cudaFree(dt);
      if (e != cudaSuccess) return fail(ctx, ANIM_ECUDA, "inverse bind from rest pose: %s", cudaGetErrorString(e));
    }
    if (inv_bind)
      T->set_bind_from_matrices(inv_bind + off * 12);
    else
      T->set_bind_from_rest(rest_q + off * 4, rest_t + off * 3);
    T->sync_dev();
    CK(T->build_walk_data());
    ctx->types.push_back(std::move(T));
    off += n;
  }
  CK(upload_types(ctx));
  for (int t = 0; t < n_types; ++t) out_type_ids[t] = first + t;
  return ANIM_OK;
}

int anim_upload_clips(anim_ctx *ctx, int32_t type_id, int n_clips, int n_keys, float rate_hz, const float *keys) {
  if (!ctx) return ANIM_EINVAL;
  if (type_id < 0 || type_id >= (int)ctx->types.size()) return fail(ctx, ANIM_EINVAL, "type id %d unknown", type_id);
  if (n_clips < 1 || n_clips > ANIM_MAX_CLIPS) return fail(ctx, ANIM_EINVAL, "n_clips must be in [1, %d]", ANIM_MAX_CLIPS);
  if (n_keys < 2 || n_keys > ANIM_MAX_KEYS) return fail(ctx, ANIM_EINVAL, "n_keys must be in [2, %d]", ANIM_MAX_KEYS);
  if (!(rate_hz > 0.f) || !std::isfinite(rate_hz)) return fail(ctx, ANIM_EINVAL, "rate_hz must be finite and > 0");
  if (!keys) return fail(ctx, ANIM_EINVAL, "keys is NULL");
  CK(cudaSetDevice(ctx->device));
  TypeHost &T = *ctx->types[type_id];
  const size_t bytes = (size_t)n_clips * n_keys * T.n * 32;
  if (T.d_keys) cudaFree(T.d_keys);
  T.d_keys = nullptr;
  CK(cudaMalloc(&T.d_keys, bytes));
  CK(cudaMemcpy(T.d_keys, keys, bytes, cudaMemcpyHostToDevice));
  CK(launch_prepare_keys(T.d_keys, n_clips, n_keys, T.n, 0));
  CK(cudaDeviceSynchronize());
  if (T.d_add && (T.n_keys != n_keys || T.rate != rate_hz)) {  // the additive layer no longer matches
    cudaFree(T.d_add);
    T.d_add = nullptr;
  }
  T.n_clips = n_clips;
  T.n_keys = n_keys;
  T.rate = rate_hz;
  T.keys_h.assign(keys, keys + (size_t)std::min(n_clips, 2) * n_keys * T.n * 8);
  CK(T.build_walk_data());
  CK(upload_types(ctx));
  return ANIM_OK;
}

int anim_upload_additive(anim_ctx *ctx, int32_t type_id, int n_keys, float rate_hz, const float *keys) {
  if (!ctx) return ANIM_EINVAL;
  if (type_id < 0 || type_id >= (int)ctx->types.size()) return fail(ctx, ANIM_EINVAL, "type id %d unknown", type_id);
  TypeHost &T = *ctx->types[type_id];
  if (T.n_clips == 0) return fail(ctx, ANIM_ESTATE, "type %d has no clips: upload them first", type_id);
  if (n_keys != T.n_keys || !(rate_hz == T.rate))
    return fail(ctx, ANIM_EINVAL, "the additive layer must have the clips' key count (%d) and rate", T.n_keys);
  if (!keys) return fail(ctx, ANIM_EINVAL, "keys is NULL");
  CK(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)n_keys * T.n * 32;
  if (T.d_add) cudaFree(T.d_add);
  T.d_add = nullptr;
  CK(cudaMalloc(&T.d_add, bytes));
  CK(cudaMemcpy(T.d_add, keys, bytes, cudaMemcpyHostToDevice));
  CK(launch_prepare_keys(T.d_add, 1, n_keys, T.n, 0));
  CK(cudaDeviceSynchronize());
  CK(upload_types(ctx));
  return ANIM_OK;
}

static int check_plan(anim_ctx *ctx, const anim_plan *plan);

int anim_upload_mesh(anim_ctx *ctx, int32_t type_id, int n_verts, const float *rest_pos, const float *rest_nrm,
                     const int32_t *bones, const float *weights) {
  if (!ctx) return ANIM_EINVAL;
  if (type_id < 0 || type_id >= (int)ctx->types.size()) return fail(ctx, ANIM_EINVAL, "type id %d unknown", type_id);
  if (n_verts < 1 || n_verts > ANIM_MAX_VERTS) return fail(ctx, ANIM_EINVAL, "n_verts must be in [1, %d]", ANIM_MAX_VERTS);
  if (!rest_pos || !rest_nrm || !bones || !weights) return fail(ctx, ANIM_EINVAL, "NULL mesh array");
  TypeHost &T = *ctx->types[type_id];
  std::vector<float4> rec((size_t)n_verts * 3);
  for (int v = 0; v < n_verts; ++v) {
    for (int k = 0; k < 4; ++k) {
      const int b = bones[4 * v + k];
      const float w = weights[4 * v + k];
      if (b < 0 || b >= T.n) return fail(ctx, ANIM_EINVAL, "vertex %d: bone %d out of range", v, b);
      if (!std::isfinite(w)) return fail(ctx, ANIM_EINVAL, "vertex %d: non-finite weight", v);
    }
    const float *p = rest_pos + 3 * v, *q = rest_nrm + 3 * v, *w = weights + 4 * v;
    const int32_t *b = bones + 4 * v;
    const uint32_t b01 = (uint32_t)b[0] | ((uint32_t)b[1] << 16), b23 = (uint32_t)b[2] | ((uint32_t)b[3] << 16);
    float f01, f23;
    memcpy(&f01, &b01, 4);
    memcpy(&f23, &b23, 4);
    rec[3 * v] = make_float4(p[0], p[1], p[2], q[0]);
    rec[3 * v + 1] = make_float4(q[1], q[2], w[0], w[1]);
    rec[3 * v + 2] = make_float4(w[2], w[3], f01, f23);
  }
  CK(cudaSetDevice(ctx->device));
  if (T.d_mesh) cudaFree(T.d_mesh);
  T.d_mesh = nullptr;
  T.n_verts = 0;
  CK(cudaMalloc(&T.d_mesh, rec.size() * sizeof(float4)));
  CK(cudaMemcpy(T.d_mesh, rec.data(), rec.size() * sizeof(float4), cudaMemcpyHostToDevice));
  T.n_verts = n_verts;
  if (T.d_faces) {  // faces index the mesh they were uploaded for
    cudaFree(T.d_faces);
    T.d_faces = nullptr;
    T.n_faces = 0;
  }
  CK(upload_types(ctx));  // bumps the version: plans rebuild their vertex offsets
  return ANIM_OK;
}

int anim_upload_faces(anim_ctx *ctx, int32_t type_id, int n_faces, const int32_t *faces) {
  if (!ctx) return ANIM_EINVAL;
  if (type_id < 0 || type_id >= (int)ctx->types.size()) return fail(ctx, ANIM_EINVAL, "type id %d unknown", type_id);
  TypeHost &T = *ctx->types[type_id];
  if (T.n_verts == 0) return fail(ctx, ANIM_ESTATE, "type %d has no mesh: upload it first", type_id);
  if (n_faces < 1 || n_faces > 4096) return fail(ctx, ANIM_EINVAL, "n_faces must be in [1, 4096]");
  if (!faces) return fail(ctx, ANIM_EINVAL, "faces is NULL");
  for (int i = 0; i < 3 * n_faces; ++i)
    if (faces[i] < 0 || faces[i] >= T.n_verts)
      return fail(ctx, ANIM_EINVAL, "face %d: vertex %d out of range", i / 3, faces[i]);
  CK(cudaSetDevice(ctx->device));
  if (T.d_faces) cudaFree(T.d_faces);
  T.d_faces = nullptr;
  T.n_faces = 0;
  CK(cudaMalloc(&T.d_faces, (size_t)n_faces * 12));
  CK(cudaMemcpy(T.d_faces, faces, (size_t)n_faces * 12, cudaMemcpyHostToDevice));
  T.n_faces = n_faces;
  CK(upload_types(ctx));
  return ANIM_OK;
}

int anim_raster(anim_ctx *ctx, const anim_plan *plan, const float *d_verts, const anim_raster_params *params,
                uint64_t *d_vis, uint32_t *d_ids, uint32_t *d_rgba, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (!params || params->width < 1 || params->height < 1 || params->cols < 1 ||
      (int64_t)params->width * params->height > (1ll << 28) || !std::isfinite(params->spacing) ||
      !std::isfinite(params->ox) || !std::isfinite(params->oy) || !std::isfinite(params->scale))
    return fail(ctx, ANIM_EINVAL, "bad raster parameters");
  if (plan->n_chars >= (1 << 20)) return fail(ctx, ANIM_EUNSUPPORTED, "at most 1,048,575 characters");
  if (!d_vis || ((uintptr_t)d_vis & 7u)) return fail(ctx, ANIM_EINVAL, "d_vis must be an 8-byte aligned device pointer");
  if (plan->n_chars > 0 && (!d_verts || !aligned4(d_verts)))
    return fail(ctx, ANIM_EINVAL, "d_verts must be a 4-byte aligned device pointer");
  RasterArgs a{};
  a.types = ctx->d_types;
  a.char_type = plan->d_char_type;
  a.vert_off = plan->d_vert_off;
  a.verts = d_verts;
  a.vis = reinterpret_cast<unsigned long long *>(d_vis);
  a.ids = d_ids;
  a.rgba = d_rgba;
  a.width = params->width;
  a.height = params->height;
  a.cols = params->cols;
  a.spacing = params->spacing;
  a.ox = params->ox;
  a.oy = params->oy;
  a.scale = params->scale;
  CK(launch_raster(a, (int)plan->n_chars, (cudaStream_t)stream));
  return ANIM_OK;
}

int anim_plan_vertex_offsets(anim_ctx *ctx, const anim_plan *plan, int64_t *out) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (!out) return fail(ctx, ANIM_EINVAL, "out is NULL");
  memcpy(out, plan->vert_off.data(), plan->vert_off.size() * sizeof(int64_t));
  return ANIM_OK;
}

int anim_plan_create(anim_ctx *ctx, int64_t n_chars, const int32_t *char_type, anim_plan **out) {
  if (!ctx) return ANIM_EINVAL;
  if (!out || n_chars < 0 || (n_chars > 0 && !char_type)) return fail(ctx, ANIM_EINVAL, "bad plan arguments");
  if (n_chars > (int64_t)kRangeChars * (kMaxRanges - kMaxTypes))
    return fail(ctx, ANIM_EUNSUPPORTED, "more than %lld characters in one plan",
                (long long)kRangeChars * (kMaxRanges - kMaxTypes));
  *out = nullptr;
  const int nt = (int)ctx->types.size();
  for (int64_t c = 0; c < n_chars; ++c)
    if (char_type[c] < 0 || char_type[c] >= nt)
      return fail(ctx, ANIM_EINVAL, "char_type[%lld] = %d is not a type id", (long long)c, char_type[c]);
  CK(cudaSetDevice(ctx->device));
  std::unique_ptr<anim_plan> P(new anim_plan());
  P->ctx = ctx;
  P->n_chars = n_chars;
  P->char_type.assign(char_type, char_type + n_chars);
  P->row_off.resize(n_chars + 1);
  P->row_off[0] = 0;
  std::vector<int64_t> count(nt, 0);
  for (int64_t c = 0; c < n_chars; ++c) {
    P->row_off[c + 1] = P->row_off[c] + ctx->types[char_type[c]]->n;
    ++count[char_type[c]];
  }
  P->total = P->row_off[n_chars];
  for (int t = 0; t < nt; ++t)
    if (count[t]) P->used.push_back(t);
  std::stable_sort(P->used.begin(), P->used.end(), [&](int a, int b) {
    const TypeHost &A = *ctx->types[a], &B = *ctx->types[b];
    return A.n != B.n ? A.n > B.n : A.max_depth > B.max_depth;
  });
  std::vector<int> rank(nt, -1);
  for (size_t u = 0; u < P->used.size(); ++u) rank[P->used[u]] = (int)u;
  P->by_type.assign(P->used.size(), {});
  for (int64_t c = 0; c < n_chars; ++c) P->by_type[rank[char_type[c]]].push_back((int32_t)c);
  std::vector<int32_t> grouped;
  for (auto &v : P->by_type) {
    P->type_chars_start.push_back((int)grouped.size());
    grouped.insert(grouped.end(), v.begin(), v.end());
  }
  CK(upload_vec(&P->d_char_type, P->char_type));
  CK(upload_vec(&P->d_row_off, P->row_off));
  CK(upload_vec(&P->d_type_chars, grouped));
  std::vector<int32_t> used32(P->used.begin(), P->used.end());
  CK(upload_vec(&P->d_used, used32));
  CK(cudaMalloc(&P->d_sorted, std::max<int64_t>(1, n_chars) * sizeof(int32_t)));
  CK(cudaMalloc(&P->d_queue, 4 * sizeof(int)));
  CK(cudaMemset(P->d_queue, 0, 4 * sizeof(int)));
  const int rc = plan_schedule(ctx, P.get());
  if (rc != ANIM_OK) return rc;
  ctx->plans.insert(P.get());
  *out = P.release();
  return ANIM_OK;
}

int anim_plan_destroy(anim_ctx *ctx, anim_plan *plan) {
  if (!ctx || !plan || !ctx->plans.count(plan)) return ctx ? fail(ctx, ANIM_EINVAL, "unknown plan") : ANIM_EINVAL;
  for (anim_plan *part : plan->host_parts) anim_plan_destroy(ctx, part);
  plan->host_parts.clear();
  for (auto it = ctx->iks.begin(); it != ctx->iks.end();) {
    if ((*it)->plan == plan) {
      delete *it;
      it = ctx->iks.erase(it);
    } else {
      ++it;
    }
  }
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->plans.erase(plan);
  delete plan;
  return ANIM_OK;
}

int anim_plan_total_joints(const anim_plan *plan, int64_t *out_total) {
  if (!plan || !out_total) return ANIM_EINVAL;
  *out_total = plan->total;
  return ANIM_OK;
}

int anim_plan_row_offsets(const anim_plan *plan, int64_t *out) {
  if (!plan || !out) return ANIM_EINVAL;
  memcpy(out, plan->row_off.data(), plan->row_off.size() * sizeof(int64_t));
  return ANIM_OK;
}

static int check_plan(anim_ctx *ctx, const anim_plan *plan) {
  if (!ctx) return ANIM_EINVAL;
  if (!plan || !ctx->plans.count(const_cast<anim_plan *>(plan))) return fail(ctx, ANIM_EINVAL, "unknown plan");
  if (plan->version != ctx->version) {
    const int rc = plan_schedule(ctx, const_cast<anim_plan *>(plan));
    if (rc != ANIM_OK) return rc;
  }
  return ANIM_OK;
}

static int frame_checks(anim_ctx *ctx, const anim_plan *plan, const float *d_time) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_time || !aligned4(d_time)) return fail(ctx, ANIM_EINVAL, "d_time must be a 4-byte aligned device pointer");
  for (int t : plan->used)
    if (ctx->types[t]->n_clips == 0) return fail(ctx, ANIM_ESTATE, "type %d has no clips uploaded", t);
  return ANIM_OK;
}

int anim_frame_build_queue(anim_ctx *ctx, const anim_plan *plan, const float *d_time, void *stream) {
  int rc = frame_checks(ctx, plan, d_time);
  if (rc || plan->n_chars == 0) return rc;
  BucketArgs b{};
  b.ranges = plan->d_ranges;
  b.n_ranges = plan->n_ranges;
  b.n_slots = plan->n_slots;
  b.type_chars = plan->d_type_chars;
  b.time = d_time;
  b.types = ctx->d_types;
  b.cap = plan->d_cap;
  b.sorted = plan->d_sorted;
  b.items = plan->d_items_frame;
  b.queue_head = plan->d_queue;
  b.status = ctx->d_status;
  CK(launch_bucket(b, (cudaStream_t)stream));
  return ANIM_OK;
}

// Item slots of the segmented kernel up to which a frame runs it on the
// same stream before the warp-specialized walk kernel (anim_frame_run_queue).
constexpr int kChainSlots = 16;

int anim_frame_run_queue(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_blend_w,
                         float *d_skin, void *stream) {
  int rc = frame_checks(ctx, plan, d_time);
  if (rc || plan->n_chars == 0) return rc;
  if (!d_blend_w || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_skin) || !aligned4(d_blend_w))
    return fail(ctx, ANIM_EINVAL, "d_skin must be 16-byte aligned, d_blend_w 4-byte aligned");
  cudaStream_t st = (cudaStream_t)stream, cta_st = st;
  const bool has_walk = plan->n_slots_walk > 0, has_cta = plan->n_slots > plan->n_slots_walk;
  // A segmented part of a few items beside the warp-specialized walk (a
  // dragon chain among bipeds) runs first on the same stream: the two
  // kernels overlap through programmatic dependent launch (the walk kernel
  // starts once the segmented kernel has seen the work queue, and finishes
  // after it), and the next launch in the stream keeps a single kernel
  // predecessor -- a fork onto the side stream and back ends that chain and
  // costs the next frame its early start.
  const bool chain = has_walk && has_cta && ctx->use_walk == 2 && plan->n_slots - plan->n_slots_walk <= kChainSlots;
  if (has_walk && has_cta && !chain) {
    // the two kernels run side by side: fork onto the context's side stream
    if (!ctx->side) {
      CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(ctx->ev_fork, st));
    CK(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
    cta_st = ctx->side;
  }
  if (has_cta) {
    ScanArgs a{};
    a.types = ctx->d_types;
    a.items = plan->d_items_frame + plan->n_slots_walk;
    a.n_items = plan->n_slots - plan->n_slots_walk;
    a.item_chars = plan->d_sorted;
    a.row_off = plan->d_row_off;
    a.queue_head = plan->d_queue + 2;
    a.done = plan->d_queue + 3;  // the last CTA resets the head
    a.status = ctx->d_status;
    a.time = d_time;
    a.blend_w = d_blend_w;
    a.skin = d_skin;
    LaunchCfg cfg = plan->cfg_scan;
    // persistent CTAs, but no more than the queue region has item slots: a
    // frame whose segmented part is one long chain beside the chain-walk
    // kernel (a dragon among bipeds) then takes one or two SMs' shared
    // memory instead of a slice of every SM's
    cfg.ctas = std::max(1, std::min(ctx->sm_count * ctx->ctas_per_sm, a.n_items));
    cfg.smem = plan->smem_frame;
    CK(launch_scan_qt(0, a, cfg, cta_st));
  }
  if (has_walk) {
    WalkArgs w{};
    w.types = ctx->d_types;
    w.items = plan->d_items_frame;
    w.n_items = plan->n_slots_walk;
    w.nbs_max = plan->walk_nbs;
    w.item_chars = plan->d_sorted;
    w.row_off = plan->d_row_off;
    w.status = ctx->d_status;
    w.time = d_time;
    w.blend_w = d_blend_w;
    w.skin = d_skin;
    w.pred_waited = chain ? 1 : 0;
    if (ctx->use_walk == 2)
      CK(launch_walk2(w, plan->walk_smem, st));
    else
      CK(launch_walk(w, plan->walk_smem, st));
  }
  if (has_walk && has_cta && !chain) {
    CK(cudaEventRecord(ctx->ev_join, ctx->side));
    CK(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  }
  return ANIM_OK;
}

int anim_evaluate_frame(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_blend_w,
                        float *d_skin, void *stream) {
  int rc = frame_checks(ctx, plan, d_time);
  if (rc || plan->n_chars == 0) return rc;
  if (!d_blend_w || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_skin) || !aligned4(d_blend_w))
    return fail(ctx, ANIM_EINVAL, "d_skin must be 16-byte aligned, d_blend_w 4-byte aligned");
  rc = anim_frame_build_queue(ctx, plan, d_time, stream);
  if (rc) return rc;
  return anim_frame_run_queue(ctx, plan, d_time, d_blend_w, d_skin, stream);
}

// Ranges of the host-buffer frame: up to kHostParts of nearly equal joint
// counts, for plans of at least kHostPartMinChars characters.
constexpr int kHostParts = 4;
constexpr int64_t kHostPartMinChars = 1024;

static int make_host_parts(anim_ctx *ctx, anim_plan *plan) {
  const int64_t N = plan->n_chars, total = plan->total;
  std::vector<int64_t> cut = {0};
  for (int k = 1; k < kHostParts; ++k) {
    const int64_t target = total * k / kHostParts;
    int64_t c = cut.back();
    while (c < N && plan->row_off[c] < target) ++c;
    if (c > cut.back() && c < N) cut.push_back(c);
  }
  cut.push_back(N);
  std::vector<anim_plan *> parts;
  for (size_t i = 0; i + 1 < cut.size(); ++i) {
    anim_plan *p = nullptr;
    const int rc = anim_plan_create(ctx, cut[i + 1] - cut[i], plan->char_type.data() + cut[i], &p);
    if (rc != ANIM_OK) {
      for (anim_plan *q : parts) anim_plan_destroy(ctx, q);
      return rc;
    }
    parts.push_back(p);
  }
  CK(cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&plan->copy_ev, cudaEventDisableTiming));
  plan->part_ev.assign(parts.size(), nullptr);
  for (auto &e : plan->part_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  plan->host_parts = std::move(parts);
  plan->part_char0 = std::move(cut);
  return ANIM_OK;
}

int anim_evaluate_frame_host(anim_ctx *ctx, anim_plan *plan, const float *h_time, const float *h_blend_w,
                             float *h_skin, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc || plan->n_chars == 0) return rc;
  if (!h_time || !h_blend_w || !h_skin) return fail(ctx, ANIM_EINVAL, "NULL host pointer");
  CK(cudaSetDevice(ctx->device));
  const size_t n = (size_t)plan->n_chars, n_pad = (n + 3) / 4 * 4;
  if (!plan->d_host_in) {
    CK(cudaMalloc(&plan->d_host_in, 2 * n_pad * sizeof(float)));
    cudaError_t e = cudaMalloc(&plan->d_host_skin, (size_t)plan->total * 48);
    if (e != cudaSuccess) {
      cudaFree(plan->d_host_in);
      plan->d_host_in = nullptr;
      plan->d_host_skin = nullptr;
      return fail(ctx, ANIM_ECUDA, "%s", cudaGetErrorString(e));
    }
    if (plan->n_chars >= kHostPartMinChars) {
      rc = make_host_parts(ctx, plan);
      if (rc) return rc;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  float *d_time = plan->d_host_in, *d_blend = plan->d_host_in + n_pad;
  CK(cudaMemcpyAsync(d_time, h_time, n * sizeof(float), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_blend, h_blend_w, n * sizeof(float), cudaMemcpyHostToDevice, st));
  if (plan->host_parts.empty()) {
    rc = anim_evaluate_frame(ctx, plan, d_time, d_blend, plan->d_host_skin, stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h_skin, plan->d_host_skin, (size_t)plan->total * 48, cudaMemcpyDeviceToHost, st));
    return ANIM_OK;
  }
  // range by range: range i's frame on `stream`, then its copy-out on the
  // copy stream while range i + 1's frame runs; `stream` finally waits for
  // the copies, so the output is complete when `stream` is
  for (size_t i = 0; i < plan->host_parts.size(); ++i) {
    const int64_t c0 = plan->part_char0[i], c1 = plan->part_char0[i + 1];
    const int64_t r0 = plan->row_off[c0], r1 = plan->row_off[c1];
    rc = anim_evaluate_frame(ctx, plan->host_parts[i], d_time + c0, d_blend + c0, plan->d_host_skin + r0 * 12,
                             stream);
    if (rc) return rc;
    CK(cudaEventRecord(plan->part_ev[i], st));
    CK(cudaStreamWaitEvent(plan->copy_stream, plan->part_ev[i], 0));
    CK(cudaMemcpyAsync(h_skin + r0 * 12, plan->d_host_skin + r0 * 12, (size_t)(r1 - r0) * 48,
                       cudaMemcpyDeviceToHost, plan->copy_stream));
  }
  CK(cudaEventRecord(plan->copy_ev, plan->copy_stream));
  CK(cudaStreamWaitEvent(st, plan->copy_ev, 0));
  return ANIM_OK;
}

int anim_evaluate_frame_skinned(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_blend_w,
                                float *d_skin, float *d_verts, void *stream) {
  int rc = frame_checks(ctx, plan, d_time);
  if (rc || plan->n_chars == 0) return rc;
  if (!d_blend_w || !d_verts) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_verts) || (d_skin && !aligned16(d_skin)) || !aligned4(d_blend_w))
    return fail(ctx, ANIM_EINVAL, "d_verts, d_skin must be 16-byte aligned, d_blend_w 4-byte aligned");
  BucketArgs bk{};  // matrix items of every type
  bk.ranges = plan->d_ranges_cta;
  bk.n_ranges = plan->n_ranges_cta;
  bk.n_slots = plan->n_slots_cta;
  bk.type_chars = plan->d_type_chars;
  bk.time = d_time;
  bk.types = ctx->d_types;
  bk.cap = plan->d_cap_cta;
  bk.sorted = plan->d_sorted;
  bk.items = plan->d_items_frame;
  bk.queue_head = plan->d_queue;
  bk.status = ctx->d_status;
  CK(launch_bucket(bk, (cudaStream_t)stream));
  ScanArgs a{};
  a.types = ctx->d_types;
  a.items = plan->d_items_frame;
  a.n_items = bk.n_slots;
  a.item_chars = plan->d_sorted;
  a.row_off = plan->d_row_off;
  a.queue_head = plan->d_queue;
  a.done = plan->d_queue + 1;
  a.status = ctx->d_status;
  a.time = d_time;
  a.blend_w = d_blend_w;
  a.skin = d_skin;
  a.verts = d_verts;
  a.vert_off = plan->d_vert_off;
  LaunchCfg cfg = plan->cfg_scan;
  cfg.ctas = ctx->sm_count * ctx->ctas_per_sm;
  cfg.smem = plan->smem_frame_mat;
  CK(launch_scan(a, cfg, (cudaStream_t)stream));
  return ANIM_OK;
}

int anim_evaluate_frame_layers(anim_ctx *ctx, const anim_plan *plan, const float *d_time, const float *d_weights,
                               const float *d_add_w, float *d_skin, void *stream) {
  int rc = frame_checks(ctx, plan, d_time);
  if (rc || plan->n_chars == 0) return rc;
  if (!d_weights || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_skin) || !aligned4(d_weights) || (d_add_w && !aligned4(d_add_w)))
    return fail(ctx, ANIM_EINVAL, "d_skin must be 16-byte aligned, d_weights and d_add_w 4-byte aligned");
  BucketArgs bk{};  // (q, t) items of every type (the plain frame gives some to the walk kernel)
  bk.ranges = plan->d_ranges_qa;
  bk.n_ranges = plan->n_ranges_qa;
  bk.n_slots = plan->n_slots_qa;
  bk.type_chars = plan->d_type_chars;
  bk.time = d_time;
  bk.types = ctx->d_types;
  bk.cap = plan->d_cap_qa;
  bk.sorted = plan->d_sorted;
  bk.items = plan->d_items_frame;
  bk.queue_head = plan->d_queue;
  bk.status = ctx->d_status;
  CK(launch_bucket(bk, (cudaStream_t)stream));
  ScanArgs a{};
  a.types = ctx->d_types;
  a.items = plan->d_items_frame;
  a.n_items = bk.n_slots;
  a.item_chars = plan->d_sorted;
  a.row_off = plan->d_row_off;
  a.queue_head = plan->d_queue;
  a.done = plan->d_queue + 1;
  a.status = ctx->d_status;
  a.time = d_time;
  a.skin = d_skin;
  a.layer_w = d_weights;
  a.add_w = d_add_w;
  LaunchCfg cfg = plan->cfg_scan;  // its shared memory covers every type's (q, t) item
  cfg.ctas = ctx->sm_count * ctx->ctas_per_sm;
  CK(launch_scan_qt(2, a, cfg, (cudaStream_t)stream));
  return ANIM_OK;
}

int anim_evaluate_frame_levelsync(anim_ctx *ctx, const anim_plan *plan, const float *d_time,
                                  const float *d_blend_w, float *d_skin, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_time || !d_blend_w || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_skin)) return fail(ctx, ANIM_EINVAL, "d_skin must be 16-byte aligned");
  for (size_t u = 0; u < plan->used.size(); ++u) {
    const TypeHost &T = *ctx->types[plan->used[u]];
    if (T.n_clips == 0) return fail(ctx, ANIM_ESTATE, "type %d has no clips uploaded", plan->used[u]);
    LevelArgs a{};
    a.type = T.dev;
    a.chars = plan->d_type_chars + plan->type_chars_start[u];
    a.n_chars = (int)plan->by_type[u].size();
    a.row_off = plan->d_row_off;
    a.time = d_time;
    a.blend_w = d_blend_w;
    a.skin = d_skin;
    a.status = ctx->d_status;
    const int threads = T.n <= 1024 ? std::max(32, (T.n + 31) / 32 * 32) : 1024;
    CK(launch_levelsync(0, a, threads,
                        (cudaStream_t)stream));
  }
  return ANIM_OK;
}

int anim_forward_local(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t, float *d_skin,
                       float *d_model, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_q || !d_t || (!d_skin && !d_model)) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_q) || (d_skin && !aligned16(d_skin)) || (d_model && !aligned16(d_model)) || !aligned4(d_t))
    return fail(ctx, ANIM_EINVAL, "d_q, d_skin, d_model must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  ScanArgs a{};
  a.types = ctx->d_types;
  a.done = plan->d_queue + 1;
  a.items = plan->d_items_scan;
  a.n_items = plan->n_items_scan;
  a.item_chars = plan->d_type_chars;
  a.row_off = plan->d_row_off;
  a.queue_head = plan->d_queue;
  a.status = ctx->d_status;
  a.q = d_q;
  a.t = d_t;
  a.skin = d_skin;
  a.model = d_model;
  CK(launch_scan_qt(1, a, plan->cfg_scan, st));
  return ANIM_OK;
}

int anim_forward_local_levelsync(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t,
                                 float *d_skin, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_q || !d_t || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_q) || !aligned16(d_skin)) return fail(ctx, ANIM_EINVAL, "d_q, d_skin must be 16-byte aligned");
  for (size_t u = 0; u < plan->used.size(); ++u) {
    const TypeHost &T = *ctx->types[plan->used[u]];
    LevelArgs a{};
    a.type = T.dev;
    a.chars = plan->d_type_chars + plan->type_chars_start[u];
    a.n_chars = (int)plan->by_type[u].size();
    a.row_off = plan->d_row_off;
    a.q = d_q;
    a.t = d_t;
    a.skin = d_skin;
    a.status = ctx->d_status;
    const int threads = T.n <= 1024 ? std::max(32, (T.n + 31) / 32 * 32) : 1024;
    CK(launch_levelsync(1, a, threads, (cudaStream_t)stream));
  }
  return ANIM_OK;
}

int anim_forward_local_paper(anim_ctx *ctx, const anim_plan *plan, int algorithm, const float *d_q,
                             const float *d_t, float *d_skin, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (algorithm < 1 || algorithm > 5) return fail(ctx, ANIM_EINVAL, "algorithm must be in 1..5");
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_q || !d_t || !d_skin) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!aligned16(d_q) || !aligned16(d_skin) || !aligned4(d_t))
    return fail(ctx, ANIM_EINVAL, "d_q, d_skin must be 16-byte aligned");
  int nmax = 0;
  for (int t : plan->used) nmax = std::max(nmax, ctx->types[t]->n);
  if (nmax > kPaperMaxJoints)
    return fail(ctx, ANIM_EUNSUPPORTED, "the paper's schedules run one thread per joint: at most %d joints",
                kPaperMaxJoints);
  PaperArgs a{};
  a.types = ctx->d_types;
  a.char_type = plan->d_char_type;
  a.row_off = plan->d_row_off;
  a.algo = algorithm;
  a.q = d_q;
  a.t = d_t;
  a.skin = d_skin;
  const int threads = std::min(kPaperMaxJoints, (nmax + 31) / 32 * 32);
  CK(launch_paper(a, (int)plan->n_chars, threads, paper_smem_bytes(nmax), (cudaStream_t)stream));
  return ANIM_OK;
}

static int run_adjoint(anim_ctx *ctx, const anim_plan *plan, int mode, const float *d_q, const float *d_t,
                       const float *d_in, float *d_grad_q, float *d_grad_t, float *d_loss, void *stream) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_q || !d_t || !d_in || !d_grad_q || !d_grad_t) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (plan->adj_unfit >= 0)
    return fail(ctx, ANIM_EUNSUPPORTED,
                "the adjoint of type %d does not fit in shared memory under this schedule (segment length %d)",
                plan->adj_unfit, ctx->types[plan->adj_unfit]->seg_len);
  if (!aligned16(d_q) || !aligned16(d_grad_q)) return fail(ctx, ANIM_EINVAL, "d_q, d_grad_q must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  AdjointArgs a{};
  a.done = plan->d_queue + 1;
  a.types = ctx->d_adj_types;
  a.items = plan->d_items_adj;
  a.n_items = plan->n_items_adj;
  a.item_chars = plan->d_type_chars;
  a.row_off = plan->d_row_off;
  a.queue_head = plan->d_queue;
  a.status = ctx->d_status;
  a.q = d_q;
  a.t = d_t;
  if (mode == 0)
    a.grad_pos = d_in;
  else
    a.target = d_in;
  a.grad_q = d_grad_q;
  a.grad_t = d_grad_t;
  a.loss = d_loss;
  CK(launch_adjoint(mode, a, plan->cfg_adj, st));
  return ANIM_OK;
}

int anim_backward(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t, const float *d_grad_pos,
                  float *d_grad_q, float *d_grad_t, void *stream) {
  return run_adjoint(ctx, plan, 0, d_q, d_t, d_grad_pos, d_grad_q, d_grad_t, nullptr, stream);
}

int anim_loss_backward(anim_ctx *ctx, const anim_plan *plan, const float *d_q, const float *d_t,
                       const float *d_target, float *d_grad_q, float *d_grad_t, float *d_loss, void *stream) {
  return run_adjoint(ctx, plan, 1, d_q, d_t, d_target, d_grad_q, d_grad_t, d_loss, stream);
}

int anim_ik_create(anim_ctx *ctx, const anim_plan *plan, int n_eff, const int32_t *effectors, anim_ik **out) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (!out || n_eff < 1 || n_eff > 64 || !effectors) return fail(ctx, ANIM_EINVAL, "bad IK arguments");
  *out = nullptr;
  CK(cudaSetDevice(ctx->device));
  const int nt = (int)ctx->types.size();
  std::unique_ptr<anim_ik> K(new anim_ik());
  K->ctx = ctx;
  K->plan = plan;
  K->n_eff = n_eff;
  K->views.resize(nt);
  std::vector<int32_t> eff_slot((size_t)nt * n_eff, 0);
  std::vector<TypeDev> vdev(nt);
  std::vector<int> Cv(nt, 1);
  size_t smem = 16;
  for (int t : plan->used) {
    const TypeHost &T = *ctx->types[t];
    std::vector<char> act(T.n, 0);
    for (int e = 0; e < n_eff; ++e) {
      const int j = effectors[(size_t)t * n_eff + e];
      if (j < 0 || j >= T.n) return fail(ctx, ANIM_EINVAL, "effector %d of type %d out of range", j, t);
      for (int a = j; a >= 0 && !act[a]; a = T.parent[a]) act[a] = 1;
    }
    std::vector<int> vid;
    cudaError_t ev = cudaSuccess;
    auto V = make_view(T, act, &vid, &ev);
    CK(ev);
    for (int e = 0; e < n_eff; ++e) eff_slot[(size_t)t * n_eff + e] = vid[effectors[(size_t)t * n_eff + e]];
    vdev[t] = V->dev;
    const int C = choose_C(ctx, *V, 1);
    if (C == 0) return fail(ctx, ANIM_EUNSUPPORTED, "IK view of type %d does not fit in shared memory", t);
    Cv[t] = C;
    smem = std::max(smem, adjoint_smem_bytes(V->n, V->seg.nseg, C));
    K->views[t] = std::move(V);
  }
  CK(upload_vec(&K->d_views, vdev));
  CK(upload_vec(&K->d_eff, eff_slot));
  auto items = make_items(plan, Cv);
  K->n_items = (int)items.size();
  CK(upload_vec(&K->d_items, items));
  CK(cudaMalloc(&K->d_counters, 4 * sizeof(int)));
  CK(cudaMemset(K->d_counters, 0, 4 * sizeof(int)));
  std::vector<int64_t> state_off(plan->n_chars);
  for (int64_t c = 0; c < plan->n_chars; ++c) {
    state_off[c] = K->state_rows;
    K->state_rows += K->views[plan->char_type[c]]->n;
  }
  CK(upload_vec(&K->d_state_off, state_off));
  CK(cudaMalloc(&K->d_state, std::max<int64_t>(1, 2 * K->state_rows) * 16));
  CK(cudaMemset(K->d_state, 0, std::max<int64_t>(1, 2 * K->state_rows) * 16));
  if (ctx->adj_ctas > 0)
    K->cfg = {kAdjSmallThreads, std::max(1, K->n_items), smem};
  else
    K->cfg = {kAdjThreads, std::max(1, std::min(ctx->sm_count * ctx->ctas_per_sm, K->n_items)), smem,
              ctx->ctas_per_sm >= 3 ? 3 : 2};
  ctx->iks.insert(K.get());
  *out = K.release();
  return ANIM_OK;
}

int anim_ik_destroy(anim_ctx *ctx, anim_ik *ik) {
  if (!ctx || !ik || !ctx->iks.count(ik)) return ctx ? fail(ctx, ANIM_EINVAL, "unknown IK object") : ANIM_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->iks.erase(ik);
  delete ik;
  return ANIM_OK;
}

int anim_ik_reset(anim_ctx *ctx, anim_ik *ik, void *stream) {
  if (!ctx || !ik || !ctx->iks.count(ik)) return ctx ? fail(ctx, ANIM_EINVAL, "unknown IK object") : ANIM_EINVAL;
  CK(cudaMemsetAsync(ik->d_counters, 0, 4 * sizeof(int), (cudaStream_t)stream));
  CK(cudaMemsetAsync(ik->d_state, 0, std::max<int64_t>(1, 2 * ik->state_rows) * 16, (cudaStream_t)stream));
  return ANIM_OK;
}

int anim_ik_step(anim_ctx *ctx, anim_ik *ik, float *d_q, float *d_m, float *d_v, const float *d_t,
                 const float *d_targets, float lr, float beta1, float beta2, float eps, float *d_loss, void *stream) {
  if (!ctx || !ik || !ctx->iks.count(ik)) return ctx ? fail(ctx, ANIM_EINVAL, "unknown IK object") : ANIM_EINVAL;
  const anim_plan *plan = ik->plan;
  if (plan->n_chars == 0) return ANIM_OK;
  if (!d_q || !d_t || !d_targets) return fail(ctx, ANIM_EINVAL, "NULL device pointer");
  if (!d_m != !d_v) return fail(ctx, ANIM_EINVAL, "d_m and d_v must both be given or both be NULL");
  if (!aligned16(d_q) || (d_m && (!aligned16(d_m) || !aligned16(d_v))))
    return fail(ctx, ANIM_EINVAL, "d_q, d_m, d_v must be 16-byte aligned");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(ctx, ANIM_EINVAL, "bad Adam hyper-parameters");
  cudaStream_t st = (cudaStream_t)stream;
  AdjointArgs a{};
  a.types = ik->d_views;
  a.items = ik->d_items;
  a.n_items = ik->n_items;
  a.item_chars = plan->d_type_chars;
  a.row_off = plan->d_row_off;
  a.queue_head = ik->d_counters;
  a.status = ctx->d_status;
  a.q = d_q;
  a.t = d_t;
  a.target = d_targets;
  a.loss = d_loss;
  a.eff_slot = ik->d_eff;
  a.n_eff = ik->n_eff;
  if (d_m) {
    a.m = d_m;
    a.v = d_v;
  } else {  // the object's own state
    a.m = ik->d_state;
    a.v = ik->d_state + 4 * ik->state_rows;
    a.state_off = ik->d_state_off;
  }
  a.q_mut = d_q;
  a.step = ik->d_counters + 1;
  a.done = ik->d_counters + 2;
  a.lr = lr;
  a.beta1 = beta1;
  a.beta2 = beta2;
  a.eps = eps;
  CK(launch_adjoint(d_m ? 2 : 3, a, ik->cfg, st));
  return ANIM_OK;
}

int anim_get_status(anim_ctx *ctx, void *stream, int *out_status) {
  if (!ctx || !out_status) return ANIM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int v = 0;
  CK(cudaMemcpyAsync(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  CK(cudaStreamSynchronize(st));
  *out_status = v;
  return ANIM_OK;
}

static uint64_t mix_hash(const anim_ctx *ctx, const anim_plan *P, int which) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)which;
  auto add = [&](uint64_t v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  for (size_t u = 0; u < P->used.size(); ++u) {
    const TypeHost &T = *ctx->types[P->used[u]];
    add((uint64_t)P->used[u]);
    add((uint64_t)T.n);
    add((uint64_t)T.max_depth);
    add((uint64_t)P->by_type[u].size());
  }
  return h;
}

static int apply_choice(anim_ctx *ctx, const anim_plan *P, int seg_len, int cps, int jpi, int walk,
                        int adj_ctas) {
  ctx->ctas_per_sm = cps;
  ctx->joints_per_item = jpi;
  ctx->use_walk = walk;
  ctx->adj_ctas = adj_ctas;
  for (int t : P->used) {
    TypeHost &T = *ctx->types[t];
    if (T.seg_len != seg_len) {
      T.seg_len = seg_len;
      CK(T.build_tables());
    }
  }
  CK(upload_types(ctx));  // bumps the version: every plan rebuilds its schedule
  return plan_schedule(ctx, const_cast<anim_plan *>(P));
}

// Autotuner: time every candidate schedule (segment length, resident CTAs per
// SM, work-item size) on scratch inputs with CUDA events and keep the best;
// the result is cached by a hash of (which, type ids, joint counts, depths,
// character counts) and re-applied by anim_plan_create for the same mix.
// The autotuner's candidate schedules for a search (which: 0 frame, 1
// forward_local, 2 loss_backward and the IK step, 3 the skinned frame, 4 the
// layered frame).  The chain-walk kernel serves the plain frame only, the
// adjoint kernel choice the adjoint only: the other searches keep the
// context's settings.
extern "C++" {  // a template inside the ABI's extern "C" block
template <class F>
static void for_each_candidate(const anim_ctx *ctx, int which, F &&f) {
  const int segs[] = {4, 8, 16, 32}, cpss[] = {1, 2, 3}, jpis[] = {256, 512, 1024, 2048, 4096};
  const int adjs[] = {0, 4, 6, 7, 8};
  const int walk_lo = which == 0 ? 0 : ctx->use_walk, walk_hi = which == 0 ? 2 : ctx->use_walk;
  const int adj_keep = ctx->adj_ctas;
  for (int walk = walk_lo; walk <= walk_hi; ++walk)
    for (int adj : adjs)
      for (int seg : segs)
        for (int cps : cpss)
          for (int jpi : jpis) {
            if (which != 2 && adj != adjs[0]) continue;
            const int adj_c = which == 2 ? adj : adj_keep;
            if (which != 2 && jpi < 1024) continue;  // small items only pay off in the one-item adjoint
            if (which == 2 && adj_c == 0 && jpi < 1024) continue;
            if (which == 2 && adj_c > 0 && cps != 2) continue;  // CTAs per SM of the persistent kernels: unused
            f(seg, cps, jpi, walk, adj_c);
          }
}
}  // extern "C++"

int anim_tune(anim_ctx *ctx, anim_plan *plan, int which) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (which < 0 || which > 4) return fail(ctx, ANIM_EINVAL, "which must be 0 to 4");
  if (plan->n_chars == 0) return ANIM_OK;
  if (which == 0 || which >= 3)
    for (int t : plan->used)
      if (ctx->types[t]->n_clips == 0) return fail(ctx, ANIM_ESTATE, "type %d has no clips uploaded", t);
  CK(cudaSetDevice(ctx->device));
  const uint64_t key = mix_hash(ctx, plan, which);
  auto hit = ctx->tune_cache.find(key);
  if (hit != ctx->tune_cache.end())
    return apply_choice(ctx, plan, hit->second.seg_len, hit->second.ctas_per_sm, hit->second.joints_per_item,
                        hit->second.walk, hit->second.adj_ctas);

  // scratch inputs (tuning may allocate; evaluation calls never do)
  const int64_t N = plan->n_chars, J = plan->total;
  std::vector<void *> bufs;
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void *p : bufs) cudaFree(p);
  };
  const int64_t V = plan->vert_off.empty() ? 0 : plan->vert_off.back();
  // The matrix outputs rotate over enough buffers to exceed L2 (at most 4),
  // as frames do in use: a single buffer that mostly fits in L2 times the
  // stores of a store-heavy candidate as cheaper than they are.
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device);
  const int n_buf = (int)std::max<int64_t>(1, std::min<int64_t>(4, (5ll * l2 / 2 + J * 48 - 1) / std::max<int64_t>(1, J * 48)));
  float *d_time = (float *)dalloc(N * 4), *d_w = (float *)dalloc(N * 16);  // [N] blend or [N][4] layer weights
  float *d_q = (float *)dalloc(J * 16), *d_t = (float *)dalloc(J * 12), *d_tg = (float *)dalloc(J * 12);
  float *d_out = (float *)dalloc(J * 48 * n_buf), *d_gq = (float *)dalloc(J * 16), *d_gt = (float *)dalloc(J * 12);
  float *d_verts = which == 3 ? (float *)dalloc(V * 24) : nullptr;
  if (bufs.size() != (which == 3 ? 9u : 8u) || std::count(bufs.begin(), bufs.end(), nullptr)) {
    release();
    return fail(ctx, ANIM_ENOMEM, "tuning buffers");
  }
  {
    std::vector<float> h(std::max<int64_t>(N, 1)), hw(std::max<int64_t>(4 * N, 1));
    for (int64_t c = 0; c < N; ++c) h[c] = (float)std::fmod(0.6180339887 * (double)c, 1.0);
    for (int64_t c = 0; c < 4 * N; ++c) hw[c] = (float)std::fmod(0.4142135623 * (double)c, 1.0);
    std::vector<float> q(J * 4, 0.f), t(J * 3, 0.05f);
    for (int64_t j = 0; j < J; ++j) q[4 * j + 3] = 1.f;
    cudaError_t e = cudaMemcpy(d_time, h.data(), N * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_w, hw.data(), N * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_q, q.data(), J * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_t, t.data(), J * 12, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_tg, t.data(), J * 12, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      release();
      return fail(ctx, ANIM_ECUDA, "tuning inputs: %s", cudaGetErrorString(e));
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Candidates are timed the way frames usually run: one call captured in a
  // CUDA graph on a private stream and the graph launched five times back to
  // back (a frame whose two kernels fork onto the side stream pays for that
  // in every graph launch); direct launches if the capture fails.
  cudaStream_t ts = nullptr;
  if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    return fail(ctx, ANIM_ECUDA, "tuning stream");
  }
  auto run_one = [&](cudaStream_t s, int k) -> int {
    float *out = d_out + (size_t)k * (size_t)J * 12;
    if (which == 0) return anim_evaluate_frame(ctx, plan, d_time, d_w, out, s);
    if (which == 1) return anim_forward_local(ctx, plan, d_q, d_t, out, nullptr, s);
    if (which == 3) return anim_evaluate_frame_skinned(ctx, plan, d_time, d_w, nullptr, d_verts, s);
    if (which == 4) return anim_evaluate_frame_layers(ctx, plan, d_time, d_w, d_w, out, s);
    return anim_loss_backward(ctx, plan, d_q, d_t, d_tg, d_gq, d_gt, nullptr, s);
  };
  // one call per output buffer: the unit that is captured and timed
  auto run_once = [&](cudaStream_t s) -> int {
    for (int k = 0; k < n_buf; ++k) {
      const int r = run_one(s, k);
      if (r != ANIM_OK) return r;
    }
    return ANIM_OK;
  };
  auto time_graph = [&](float *ms) -> bool {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    bool ok = run_once(ts) == ANIM_OK;
    const cudaError_t ce = cudaStreamEndCapture(ts, &g);
    ok = ok && ce == cudaSuccess && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    for (int r = 0; r < 2 && ok; ++r) ok = cudaGraphLaunch(ge, ts) == cudaSuccess;
    // the best of three batches of five launches: one batch is easily
    // disturbed by a few microseconds, as much as candidates differ
    float best = 1e30f;
    for (int b = 0; b < 3 && ok; ++b) {
      cudaEventRecord(e0, ts);
      for (int r = 0; r < 5 && ok; ++r) ok = cudaGraphLaunch(ge, ts) == cudaSuccess;
      cudaEventRecord(e1, ts);
      ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
      float t = 0.f;
      if (ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) best = std::min(best, t / (5.f * n_buf));
    }
    if (ok) *ms = best;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();  // a failed capture leaves its error here: do not report it later
    return ok;
  };
  anim_ctx::TuneChoice best{0, 0, 0, 0, 0, 1e30f};
  for_each_candidate(ctx, which, [&](int seg, int cps, int jpi, int walk, int adj_c) {
    if (apply_choice(ctx, plan, seg, cps, jpi, walk, adj_c) != ANIM_OK) return;  // e.g. does not fit
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w) ok = run_once(ts) == ANIM_OK;  // outside capture: attributes, side stream
    if (!ok || cudaStreamSynchronize(ts) != cudaSuccess) return;
    float ms = 0.f;
    if (!time_graph(&ms)) {
      cudaEventRecord(e0, ts);
      for (int r = 0; r < 5 && ok; ++r) ok = run_once(ts) == ANIM_OK;
      cudaEventRecord(e1, ts);
      if (!ok || cudaEventSynchronize(e1) != cudaSuccess) return;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= 5.f * n_buf;
    }
    if (ms < best.ms) best = {seg, cps, jpi, walk, adj_c, ms};
  });
  cudaStreamSynchronize(ts);
  cudaStreamDestroy(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (best.seg_len == 0) return fail(ctx, ANIM_ECUDA, "no candidate schedule ran");
  ctx->tune_cache[key] = best;
  ctx->err.clear();
  return apply_choice(ctx, plan, best.seg_len, best.ctas_per_sm, best.joints_per_item, best.walk,
                      best.adj_ctas);
}

int anim_tune_ik(anim_ctx *ctx, anim_plan *plan, int n_eff, const int32_t *effectors) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (n_eff < 1 || !effectors) return fail(ctx, ANIM_EINVAL, "need n_eff >= 1 effectors per type");
  if (plan->n_chars == 0) return ANIM_OK;
  CK(cudaSetDevice(ctx->device));
  uint64_t key = mix_hash(ctx, plan, 3);  // and the used types' effectors
  for (int t : plan->used)
    for (int e = 0; e < n_eff; ++e)
      key = (key ^ (uint64_t)(uint32_t)effectors[(size_t)t * n_eff + e]) * 1099511628211ull;
  auto hit = ctx->tune_cache.find(key);
  if (hit != ctx->tune_cache.end())
    return apply_choice(ctx, plan, hit->second.seg_len, hit->second.ctas_per_sm, hit->second.joints_per_item,
                        hit->second.walk, hit->second.adj_ctas);
  // scratch state (tuning may allocate; steps never do): identity poses,
  // targets near the origin; the candidates' IK objects keep their own
  // (zeroed) Adam state
  const int64_t N = plan->n_chars, J = plan->total;
  float *d_q = nullptr, *d_t = nullptr, *d_tg = nullptr;
  auto release = [&]() {
    for (float *p : {d_q, d_t, d_tg})
      if (p) cudaFree(p);
  };
  bool ok = cudaMalloc(&d_q, J * 16) == cudaSuccess && cudaMalloc(&d_t, J * 12) == cudaSuccess &&
            cudaMalloc(&d_tg, std::max<int64_t>(N * n_eff * 12, 16)) == cudaSuccess;
  if (!ok) {
    release();
    return fail(ctx, ANIM_ENOMEM, "IK tuning buffers");
  }
  {
    std::vector<float> q(J * 4, 0.f), t(J * 3, 0.05f), tg(N * n_eff * 3, 0.1f);
    for (int64_t j = 0; j < J; ++j) q[4 * j + 3] = 1.f;
    cudaError_t e = cudaMemcpy(d_q, q.data(), J * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_t, t.data(), J * 12, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && N > 0) e = cudaMemcpy(d_tg, tg.data(), N * n_eff * 12, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      release();
      return fail(ctx, ANIM_ECUDA, "IK tuning inputs: %s", cudaGetErrorString(e));
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  anim_ctx::TuneChoice best{0, 0, 0, 0, 0, 1e30f};
  for_each_candidate(ctx, 2, [&](int seg, int cps, int jpi, int walk, int adj_c) {
    if (apply_choice(ctx, plan, seg, cps, jpi, walk, adj_c) != ANIM_OK) return;  // e.g. does not fit
    anim_ik *ik = nullptr;
    if (anim_ik_create(ctx, plan, n_eff, effectors, &ik) != ANIM_OK) return;  // a view does not fit
    auto step = [&]() {
      return anim_ik_step(ctx, ik, d_q, nullptr, nullptr, d_t, d_tg, 1e-2f, 0.9f, 0.999f, 1e-8f, nullptr, nullptr);
    };
    bool good = anim_ik_reset(ctx, ik, nullptr) == ANIM_OK;
    for (int w = 0; w < 2 && good; ++w) good = step() == ANIM_OK;
    cudaEventRecord(e0, nullptr);
    for (int r = 0; r < 5 && good; ++r) good = step() == ANIM_OK;
    cudaEventRecord(e1, nullptr);
    good = good && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (good) cudaEventElapsedTime(&ms, e0, e1);
    anim_ik_destroy(ctx, ik);
    if (good && ms / 5.f < best.ms) best = {seg, cps, jpi, walk, adj_c, ms / 5.f};
  });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (best.seg_len == 0) return fail(ctx, ANIM_ECUDA, "no candidate schedule ran");
  ctx->tune_cache[key] = best;
  ctx->err.clear();
  return apply_choice(ctx, plan, best.seg_len, best.ctas_per_sm, best.joints_per_item, best.walk,
                      best.adj_ctas);
}

int anim_get_schedule(anim_ctx *ctx, const anim_plan *plan, int32_t *out5) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (!out5) return fail(ctx, ANIM_EINVAL, "out5 is NULL");
  const TypeHost *T = plan->used.empty() ? nullptr : ctx->types[plan->used[0]].get();
  out5[0] = T ? T->seg_len : 16;
  out5[1] = ctx->ctas_per_sm;
  out5[2] = ctx->joints_per_item;
  out5[3] = ctx->use_walk;
  out5[4] = ctx->adj_ctas;
  return ANIM_OK;
}

int anim_set_schedule(anim_ctx *ctx, anim_plan *plan, const int32_t *in5) {
  int rc = check_plan(ctx, plan);
  if (rc) return rc;
  if (!in5 || in5[0] < 1 || in5[0] > ANIM_MAX_JOINTS || in5[1] < 1 || in5[1] > 3 || in5[2] < 1 ||
      in5[3] < 0 || in5[3] > 2 || in5[4] < 0 || in5[4] > 8)
    return fail(ctx, ANIM_EINVAL, "schedule out of range");
  CK(cudaSetDevice(ctx->device));
  int32_t prev[5];
  anim_get_schedule(ctx, plan, prev);
  rc = apply_choice(ctx, plan, in5[0], in5[1], in5[2], in5[3], in5[4]);
  if (rc != ANIM_OK) {
    // keep the failure's message and put the previous schedule back
    const std::string msg = ctx->err;
    apply_choice(ctx, plan, prev[0], prev[1], prev[2], prev[3], prev[4]);
    ctx->err = msg;
  }
  return rc;
}

int anim_analyze_skeleton(int n, const int32_t *parents, int seg_len, int32_t *out_nseg, int32_t *out_seg_start,
                          int32_t *out_rounds, int32_t *out_depth) {
  if (n < 1 || n > ANIM_MAX_JOINTS || !parents || seg_len < 1 || !out_nseg || !out_seg_start || !out_rounds ||
      !out_depth)
    return ANIM_EINVAL;
  if (validate_parents(parents, n) >= 0) return ANIM_EINVAL;
  std::vector<int32_t> par(parents, parents + n);
  Segments S = analyze_segments(par, seg_len);
  *out_nseg = S.nseg;
  *out_rounds = S.rounds;
  std::copy(S.start.begin(), S.start.end(), out_seg_start);
  const auto d = depths_of(par);
  *out_depth = *std::max_element(d.begin(), d.end());
  return ANIM_OK;
}

}  // extern "C"
