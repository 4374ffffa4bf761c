"""Seeded synthetic inputs for the skeletal-animation hot path.

This module draws skeleton trees, rest poses, keyframe clips, per-character
sample times and blend weights, local poses and targets.  It serves both the
FP64 oracle and the CUDA library, so it holds none of the method's arithmetic:
no transform is composed, no pose is sampled or blended, no forward or
inverse kinematics is evaluated here.  Quantities that need the method (the
inverse bind pose of a rest pose, IK targets as effector positions of a
target pose) are derived independently on each side from the raw draws
returned here.

Conventions shared by both sides:
  * quaternions are stored (x, y, z, w);
  * a skeleton is a parent array with parent[i] < i (parent[i] = -1 marks a
    root); depth counts levels with a root at depth 1;
  * a keyframe record is 8 float32: qx qy qz qw tx ty tz pad (pad = 0).

The workload shapes mirror the paper's experiment (Table 1: 10,000
characters of about 300 joints, hierarchy depths 15-120) and the five
configurations of the benchmark; everything is synthetic (no dataset is
named by the paper).
"""
from __future__ import annotations

import numpy as np

KEY_RATE_HZ = 30.0
N_KEYS = 30
N_CLIPS = 2


# --------------------------------------------------------------------------
# random rotations (input construction only)
# --------------------------------------------------------------------------
def random_unit_quats(rng: np.random.Generator, n: int, max_angle_deg: float) -> np.ndarray:
    """Unit quaternions (x,y,z,w) with axis uniform on S^2 and rotation angle
    uniform in [0, max_angle_deg]; returned in float64."""
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(0.0, max_angle_deg, size=n))
    q = np.empty((n, 4))
    q[:, :3] = axis * np.sin(ang / 2)[:, None]
    q[:, 3] = np.cos(ang / 2)
    return q


# --------------------------------------------------------------------------
# trees
# --------------------------------------------------------------------------
def depths_of(parents: np.ndarray) -> np.ndarray:
    """Depth of each joint, root = 1 (parent[i] < i is assumed)."""
    d = np.zeros(len(parents), dtype=np.int64)
    for i, p in enumerate(parents):
        d[i] = 1 if p < 0 else d[p] + 1
    return d


def random_tree(n: int, max_depth: int, rng: np.random.Generator, spine: int = 0) -> np.ndarray:
    """Random tree with parent[i] < i and depth <= max_depth.

    Joints 0..spine-1 form a chain (so the maximum depth is reached when
    spine == max_depth); every other joint picks its parent uniformly among
    the earlier joints whose depth is below max_depth."""
    assert n >= 1 and max_depth >= 1 and spine <= min(n, max_depth)
    parents = np.full(n, -1, dtype=np.int32)
    depth = np.zeros(n, dtype=np.int64)
    depth[0] = 1
    cand = [0] if max_depth > 1 else []
    for i in range(1, n):
        if i < spine:
            p = i - 1
        else:
            assert cand, "no joint can take a child under this depth limit"
            p = cand[rng.integers(len(cand))]
        parents[i] = p
        depth[i] = depth[p] + 1
        if depth[i] < max_depth:
            cand.append(i)
    return parents


def chain(n: int) -> np.ndarray:
    """A pure chain of n joints (depth n)."""
    return np.arange(-1, n - 1, dtype=np.int32)


def relabel_dfs(parents: np.ndarray, rng: np.random.Generator | None):
    """Renumber joints in depth-first pre-order, children visited in random
    order (or in index order when rng is None).  Returns (new_parents, perm)
    with perm[new] = old."""
    n = len(parents)
    kids = [[] for _ in range(n)]
    roots = []
    for i, p in enumerate(parents):
        (roots if p < 0 else kids[p]).append(i)
    order = []
    stack = list(reversed(roots))
    while stack:
        u = stack.pop()
        order.append(u)
        ch = list(kids[u])
        if rng is not None:
            rng.shuffle(ch)
        stack.extend(reversed(ch))
    perm = np.array(order, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    newp = np.array([-1 if parents[o] < 0 else inv[parents[o]] for o in perm], dtype=np.int32)
    return newp, perm


def relabel_random_topological(parents: np.ndarray, rng: np.random.Generator):
    """Renumber joints in a random topological order (parent before child),
    which is generally not depth-first.  Returns (new_parents, perm)."""
    n = len(parents)
    kids = [[] for _ in range(n)]
    ready = []
    for i, p in enumerate(parents):
        (ready if p < 0 else kids[p]).append(i)
    order = []
    while ready:
        k = rng.integers(len(ready))
        u = ready.pop(k)
        order.append(u)
        ready.extend(kids[u])
    perm = np.array(order, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    newp = np.array([-1 if parents[o] < 0 else inv[parents[o]] for o in perm], dtype=np.int32)
    return newp, perm


def biped_with_chains(rng: np.random.Generator, body: int = 40, body_depth: int = 11,
                      n_chains: int = 8, chain_len: int = 59) -> np.ndarray:
    """A 40-joint body (depth 11) with 8 cloth/tail chains of 59 joints hung
    from 8 distinct body joints, one of them at the body's deepest joint, so
    the maximum depth is 11 + 59 = 70 and the joint count 40 + 8*59 = 512."""
    bp = random_tree(body, body_depth, rng, spine=body_depth)
    others = np.array([j for j in range(body) if j != body_depth - 1])
    attach = [body_depth - 1] + list(rng.choice(others, size=n_chains - 1, replace=False))
    parents = list(bp)
    for a in attach:
        start = len(parents)
        parents.append(int(a))
        for k in range(1, chain_len):
            parents.append(start + k - 1)
    return np.array(parents, dtype=np.int32)


def path_length_bound(parents: np.ndarray, seg_len: np.ndarray) -> float:
    """Largest sum of per-joint lengths along any root-to-joint path: an upper
    bound of the skeleton's extent by the triangle inequality."""
    acc = np.zeros(len(parents))
    for i, p in enumerate(parents):
        acc[i] = seg_len[i] + (acc[p] if p >= 0 else 0.0)
    return float(acc.max())


# --------------------------------------------------------------------------
# skeleton types with rest pose and clips
# --------------------------------------------------------------------------
def make_type(parents: np.ndarray, rng: np.random.Generator, *, with_clips: bool,
              unit_extent: bool = True, rest_angle: float = 30.0, key_angle: float = 30.0,
              t_half: float = 0.1, key_noise: float = 0.01) -> dict:
    """Rest pose (rotation within rest_angle of identity, translation uniform
    in [-t_half, t_half]^3) and, optionally, 2 clips x 30 keys at 30 Hz with
    rotations within key_angle of identity and translations equal to the rest
    translation plus uniform noise of +-key_noise (relative to the bone scale).

    With unit_extent, all translations are scaled so that the largest
    root-to-joint path length over every key and the rest pose is at most 1,
    so every sampled or blended pose has extent <= 1."""
    n = len(parents)
    rest_q = random_unit_quats(rng, n, rest_angle)
    rest_t = rng.uniform(-t_half, t_half, size=(n, 3))
    typ = {"parents": parents.astype(np.int32), "rest_q": rest_q}
    keys = None
    if with_clips:
        keys = np.zeros((N_CLIPS, N_KEYS, n, 8))
        for c in range(N_CLIPS):
            for k in range(N_KEYS):
                keys[c, k, :, 0:4] = random_unit_quats(rng, n, key_angle)
                keys[c, k, :, 4:7] = rest_t + rng.uniform(-key_noise, key_noise, size=(n, 3)) * (t_half / 0.1)
    scale = 1.0
    if unit_extent:
        seg = np.linalg.norm(rest_t, axis=1)
        if keys is not None:
            seg = np.maximum(seg, np.linalg.norm(keys[..., 4:7], axis=-1).max(axis=(0, 1)))
        scale = 1.0 / max(path_length_bound(parents, seg), 1e-30)
    typ["rest_t"] = rest_t * scale
    typ["scale"] = scale
    if keys is not None:
        keys[..., 4:7] *= scale
        typ["keys"] = keys.astype(np.float32)
        typ["rate_hz"] = KEY_RATE_HZ
    typ["rest_q"] = typ["rest_q"].astype(np.float32)
    typ["rest_t"] = typ["rest_t"].astype(np.float32)
    typ["depth"] = int(depths_of(parents).max())
    return typ


def make_mesh(parents: np.ndarray, n_verts: int, rng: np.random.Generator, max_influences: int = 4) -> dict:
    """A synthetic skinned mesh in bind space, laid out the way exporters
    write one: vertices grouped by a home joint in joint order, each
    weighted to the home joint and its nearest relatives (parent,
    grandparent, first child), weights positive, decreasing away from the
    home joint and summing to 1 (a quarter of the vertices use fewer
    influences; unused slots have weight 0).  Positions: a random centre in
    [-0.5, 0.5]^3 per home joint plus uniform offsets of +-0.03, so a
    joint's vertices form a small patch; unit normals uniform on the sphere.
    Faces: a triangle strip over the vertex sequence (n_verts - 2 faces,
    alternating orientation), i.e. small triangles within a patch."""
    parents = np.asarray(parents)
    n = len(parents)
    first_child = np.full(n, -1)
    for j in range(n - 1, 0, -1):
        if parents[j] >= 0:
            first_child[parents[j]] = j
    centre = rng.uniform(-0.5, 0.5, size=(n, 3))
    home_of = np.arange(n_verts) * n // n_verts
    pos = centre[home_of] + rng.uniform(-0.03, 0.03, size=(n_verts, 3))
    nrm = rng.normal(size=(n_verts, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    bones = np.zeros((n_verts, 4), np.int32)
    wts = np.zeros((n_verts, 4))
    for v in range(n_verts):
        home = v * n // n_verts
        cand = [home]
        p = int(parents[home])
        for r in (p, int(parents[p]) if p >= 0 else -1, int(first_child[home])):
            if r >= 0 and r not in cand:
                cand.append(r)
        k = min(max_influences, len(cand))
        m = int(rng.integers(1, k + 1)) if rng.uniform() < 0.25 else k
        bones[v, :m] = cand[:m]
        w = np.sort(rng.uniform(0.05, 1.0, size=m))[::-1]
        wts[v, :m] = w / w.sum()
    faces = np.array([(v, v + 1, v + 2) if v % 2 == 0 else (v, v + 2, v + 1) for v in range(max(0, n_verts - 2))],
                     np.int32).reshape(-1, 3)
    return {"pos": pos.astype(np.float32), "nrm": nrm.astype(np.float32), "bones": bones,
            "weights": wts.astype(np.float32), "faces": faces}


def with_meshes(w: dict, n_verts: int = 1500, seed: int = 11) -> dict:
    """The workload with a mesh attached to every type (1,500 vertices by
    default: about 3,000 faces, the top of the paper's Table 1 range)."""
    rng = np.random.default_rng(seed)
    w = dict(w)
    w["types"] = [dict(t, mesh=make_mesh(t["parents"], n_verts, rng)) for t in w["types"]]
    return w


def with_layers(w: dict, n_clips: int = 4, additive: bool = True, seed: int = 31) -> dict:
    """The workload with up to 4 clips per type (extra clips drawn like the
    first ones: rotations within 30 degrees of identity, translations those
    of clip 0 plus noise of 1 % of the bone scale), an optional additive
    layer per type (rotations within 15 degrees of identity, translations
    within 5 % of clip 0's), per-character clip weights [n_chars][4]
    (uniform, a third of them zeroed, never all) and additive weights
    uniform in [0, 1]."""
    rng = np.random.default_rng(seed)
    w = dict(w)
    types = []
    for t in w["types"]:
        t = dict(t)
        k = t["keys"]
        nc, nk, n = k.shape[:3]
        if n_clips > nc:
            extra = np.zeros((n_clips - nc, nk, n, 8), np.float32)
            for c in range(n_clips - nc):
                for kk in range(nk):
                    extra[c, kk, :, 0:4] = random_unit_quats(rng, n, 30.0)
                    extra[c, kk, :, 4:7] = k[0, kk, :, 4:7] + rng.uniform(-0.01, 0.01, (n, 3)) * t["scale"]
            t["keys"] = np.concatenate([k, extra]).astype(np.float32)
        if additive:
            add = np.zeros((nk, n, 8), np.float32)
            for kk in range(nk):
                add[kk, :, 0:4] = random_unit_quats(rng, n, 15.0)
                add[kk, :, 4:7] = 0.05 * k[0, kk, :, 4:7] * rng.uniform(-1, 1, (n, 1))
            t["add_keys"] = add
        types.append(t)
    w["types"] = types
    m = len(w["char_type"])
    wts = rng.uniform(0.0, 1.0, size=(m, 4))
    wts[rng.uniform(size=(m, 4)) < 1 / 3] = 0.0
    wts[np.arange(m), rng.integers(0, n_clips, size=m)] += 0.1
    wts[:, n_clips:] = 0.0
    w["weights"] = wts.astype(np.float32)
    w["add_w"] = rng.uniform(0.0, 1.0, size=m).astype(np.float32)
    return w


def char_offsets(char_type: np.ndarray, types: list) -> np.ndarray:
    """Exclusive prefix of joint counts in character order (row offsets of
    each character's joints in the [sum n][...] arrays)."""
    n = np.array([len(types[t]["parents"]) for t in char_type], dtype=np.int64)
    off = np.zeros(len(n) + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


def local_poses(rng: np.random.Generator, n_joints: int, max_angle: float = 30.0,
                t_half: float = 0.1, t_scale=1.0, unnormalized: bool = False):
    """Local rotations within max_angle of identity (optionally scaled by a
    factor uniform in [0.8, 1.2], i.e. unnormalized) and translations uniform
    in [-t_half, t_half]^3 times t_scale (scalar or per-joint array)."""
    q = random_unit_quats(rng, n_joints, max_angle)
    if unnormalized:
        q *= rng.uniform(0.8, 1.2, size=(n_joints, 1))
    t = rng.uniform(-t_half, t_half, size=(n_joints, 3))
    t = t * np.asarray(t_scale).reshape(-1, 1) if np.ndim(t_scale) else t * t_scale
    return q.astype(np.float32), t.astype(np.float32)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def config1(seed: int = 1, n_chars: int = 64) -> dict:
    """64 characters sharing one random 64-joint tree (max depth 12); local
    poses within 30 degrees of identity, translations in [-0.1,0.1]^3, unit
    scale; inverse bind = inverse of the model pose of a separate rest pose."""
    rng = np.random.default_rng(seed)
    parents = random_tree(64, 12, rng, spine=12)
    parents, _ = relabel_dfs(parents, rng)
    typ = make_type(parents, rng, with_clips=False, unit_extent=False)
    char_type = np.zeros(n_chars, dtype=np.int32)
    q, t = local_poses(rng, n_chars * 64)
    return {"name": "config1", "types": [typ], "char_type": char_type, "q": q, "t": t}


def config2_types(rng: np.random.Generator):
    body, _ = relabel_dfs(biped_with_chains(rng), rng)
    t512 = make_type(body, rng, with_clips=True)
    t_dragon = make_type(chain(1024), rng, with_clips=True)
    return t512, t_dragon


def config2(seed: int = 2, n_chars: int = 4096, n_dragons: int = 1) -> dict:
    """4,096 characters of the 512-joint type plus one 1,024-joint dragon
    chain, 2 clips x 30 keys at 30 Hz, time ~ U[0,1), blend weight ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    t512, t_dragon = config2_types(rng)
    char_type = np.concatenate([np.zeros(n_chars, np.int32), np.ones(n_dragons, np.int32)])
    nc = len(char_type)
    return {"name": "config2", "types": [t512, t_dragon], "char_type": char_type,
            "time": rng.uniform(0.0, 1.0, nc).astype(np.float32),
            "weight": rng.uniform(0.0, 1.0, nc).astype(np.float32)}


CONFIG3_MIX = ((32, 8), (128, 16), (512, 70), (1024, 256), (2048, 2048))
CONFIG3_FRACTIONS = (0.40, 0.30, 0.15, 0.10, 0.05)


def config3_types(rng: np.random.Generator):
    types = []
    for n, d in CONFIG3_MIX:
        if n == 512:
            p, _ = relabel_dfs(biped_with_chains(rng), rng)
        elif n == d:
            p = chain(n)
        else:
            p, _ = relabel_dfs(random_tree(n, d, rng, spine=d), rng)
        types.append(make_type(p, rng, with_clips=True))
    return types


def config3(seed: int = 3, n_chars: int = 10000) -> dict:
    """10,000 characters of 5 types (32/128/512/1024/2048 joints, depths
    8/16/70/256/2048) mixed 40/30/15/10/5 %, shuffled; clips as config 2."""
    rng = np.random.default_rng(seed)
    types = config3_types(rng)
    counts = [int(round(f * n_chars)) for f in CONFIG3_FRACTIONS]
    counts[0] += n_chars - sum(counts)
    char_type = np.concatenate([np.full(c, i, np.int32) for i, c in enumerate(counts)])
    rng.shuffle(char_type)
    return {"name": "config3", "types": types, "char_type": char_type,
            "time": rng.uniform(0.0, 1.0, n_chars).astype(np.float32),
            "weight": rng.uniform(0.0, 1.0, n_chars).astype(np.float32)}


def config4(seed: int = 4, n_chars: int = 1024) -> dict:
    """1,024 characters of one 256-joint tree (spine depth 96); local
    rotations unnormalized (unit within 30 degrees times U[0.8,1.2]);
    translations U[-0.1,0.1]^3 scaled to unit extent; targets drawn directly
    as points uniform in [-0.5,0.5]^3."""
    rng = np.random.default_rng(seed)
    p, _ = relabel_dfs(random_tree(256, 96, rng, spine=96), rng)
    typ = make_type(p, rng, with_clips=False)
    char_type = np.zeros(n_chars, dtype=np.int32)
    q, t = local_poses(rng, n_chars * 256, unnormalized=True, t_scale=typ["scale"])
    target = rng.uniform(-0.5, 0.5, size=(n_chars * 256, 3)).astype(np.float32)
    return {"name": "config4", "types": [typ], "char_type": char_type, "q": q, "t": t, "target": target}


def pick_effectors(parents: np.ndarray, rng: np.random.Generator, k: int = 8) -> np.ndarray:
    """k distinct leaves, deepest first (ties broken by a seeded shuffle)."""
    n = len(parents)
    has_kid = np.zeros(n, bool)
    has_kid[parents[parents >= 0]] = True
    leaves = np.nonzero(~has_kid)[0]
    d = depths_of(parents)
    rng.shuffle(leaves)
    leaves = leaves[np.argsort(-d[leaves], kind="stable")]
    assert len(leaves) >= k
    return np.sort(leaves[:k]).astype(np.int32)


def config5(seed: int = 5, n_chars: int = 8192, n_steps: int = 200) -> dict:
    """8,192 characters alternating a 128-joint (depth 16) and a 1,024-joint
    (depth 256) type; 8 effectors per type; IK starts from identity local
    rotations with the rest translations (fixed); the target pose draws
    rotations within 45 degrees of identity; Adam lr 1e-2, PyTorch betas/eps."""
    rng = np.random.default_rng(seed)
    types = []
    for n, d in ((128, 16), (1024, 256)):
        p, _ = relabel_dfs(random_tree(n, d, rng, spine=d), rng)
        types.append(make_type(p, rng, with_clips=False))
    effectors = np.stack([pick_effectors(ty["parents"], rng) for ty in types])
    char_type = (np.arange(n_chars) % 2).astype(np.int32)
    off = char_offsets(char_type, types)
    nt = int(off[-1])
    t = np.concatenate([types[c]["rest_t"] for c in char_type]).astype(np.float32)
    q0 = np.zeros((nt, 4), np.float32)
    q0[:, 3] = 1.0
    q_target = random_unit_quats(rng, nt, 45.0).astype(np.float32)
    return {"name": "config5", "types": types, "char_type": char_type, "t": t, "q0": q0,
            "q_target": q_target, "effectors": effectors, "n_steps": n_steps,
            "lr": 1e-2, "betas": (0.9, 0.999), "eps": 1e-8}


def subset(w: dict, chars) -> dict:
    """The same workload restricted to the listed characters (per-joint arrays
    re-sliced by character offsets), for bounded samples and parity checks."""
    chars = np.asarray(chars, dtype=np.int64)
    off = char_offsets(w["char_type"], w["types"])
    out = dict(w)
    out["char_type"] = w["char_type"][chars]
    for k in ("time", "weight"):
        if k in w:
            out[k] = w[k][chars]
    for k in ("q", "t", "target", "q0", "q_target"):
        if k in w:
            out[k] = np.concatenate([w[k][off[c]:off[c + 1]] for c in chars]) if len(chars) else w[k][:0]
    return out
