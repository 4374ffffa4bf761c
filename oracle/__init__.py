"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or calls it.  The oracle shares
no code with the CUDA path: it is ``oracle.c`` (plain sequential C in fp64)
plus this ctypes wrapper, which only marshals numpy arrays.

Functions and the passages they follow (paper section, equation):
  * slerp / sample_local  -- Simulation stage, Sec. 1 step 1 and Sec. 2
    (interpolation and blending kept).  Parity pinned by the slerp
    special cases (endpoints, same-axis closed form, constant angular
    velocity, near-parallel branch) and the sampling special cases (exact
    key times, wrap, blend weights 0 and 1).  The combination of the two
    for general inputs (the reading stated in the header of oracle.c) is
    pinned against scipy's Slerp composed stage by stage -- each clip's
    bracketing keys at the key fraction, then the two clip poses at the
    blend weight -- on random keys, signs, times and weights.
  * forward / forward_qt  -- Hierarchy-Scan, Eq. 1, by the sequential
    parent-before-child traversal (Sec. 3.2.1 ordering).  Pinned by a
    brute-force root-to-joint product over every tree of up to 7 joints,
    the paper's own schedules (Algorithms 2-4, emulated with barriers as
    phases), same-axis closed forms, rest/bind special cases and rigidity.
  * bind / inverse_bind   -- Bind MeshPose, Sec. 1 step 3.  Pinned by the
    identity case (local = rest pose gives S = I).
  * frame                 -- the three stages together.
  * grad / grad_force_moment -- two independent derivations of the
    gradient of a position loss, pinned against central finite
    differences and a single-joint closed form.
  * adam / ik             -- Adam as PyTorch defines it (pinned against
    torch.optim.Adam in fp64) and batched IK; ik_all_cores runs ik on
    shares of the characters in parallel processes (same arithmetic).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (plain C11,
    -O2, no floating-point contraction so x86 and Arm give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        d, f, i32, i64 = POINTER(c_double), POINTER(c_float), POINTER(c_int32), POINTER(c_int64)
        _lib.oracle_slerp.argtypes = [d, d, c_double, d]
        _lib.oracle_sample_local.argtypes = [c_int, c_int, c_int, c_float, f, c_float, c_float, d, d]
        _lib.oracle_forward.argtypes = [c_int, i32, d, d]
        _lib.oracle_bind.argtypes = [c_int, d, d, d]
        _lib.oracle_inverse_bind.argtypes = [c_int, i32, f, f, d]
        _lib.oracle_inverse_bind.restype = c_int
        _lib.oracle_frame.argtypes = [c_int, i32, i32, d, f, i64, i32, i32, f, c_int64, i32, f, f, i64, d, c_void_p]
        _lib.oracle_frame.restype = c_int
        _lib.oracle_forward_qt.argtypes = [c_int, i32, i32, c_void_p, c_int64, i32, d, d, i64, c_void_p, c_void_p]
        _lib.oracle_forward_qt.restype = c_int
        for fn in (_lib.oracle_grad, _lib.oracle_grad_force_moment):
            fn.argtypes = [c_int, i32, i32, c_int64, i32, d, d, d, i64, d, d]
            fn.restype = c_int
        _lib.oracle_adam.argtypes = [c_int64, d, d, d, d, c_int, c_double, c_double, c_double, c_double]
        _lib.oracle_ik.argtypes = [c_int, i32, i32, i32, c_int, c_int64, i32, d, d, i64, c_int, c_double,
                                   c_double, c_double, c_double, d, d]
        _lib.oracle_ik.restype = c_int
        _lib.oracle_lbs.argtypes = [c_int, f, f, i32, f, d, d]
        _lib.oracle_sample_layers.argtypes = [c_int, c_int, c_int, c_float, f, c_void_p, c_float, f, c_float, d, d]
        _lib.oracle_frame_layers.argtypes = [c_int, i32, i32, d, f, i64, i32, i32, f, f, i64, c_int64, i32, f, f, f,
                                             i64, d]
        _lib.oracle_frame_layers.restype = c_int
        _lib.oracle_raster.argtypes = [c_int, i32, POINTER(POINTER(c_int32)), i64, d, c_int, c_double, c_double,
                                       c_double, c_double, c_int, c_int, POINTER(ctypes.c_uint32), c_void_p]
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(POINTER(ct))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ---------------------------------------------------------------- singles
def slerp(a, b, alpha: float) -> np.ndarray:
    lib = _load()
    a, b = _f64(a), _f64(b)
    out = np.empty(4)
    lib.oracle_slerp(_p(a, c_double), _p(b, c_double), float(alpha), _p(out, c_double))
    return out


def sample_local(keys: np.ndarray, rate: float, time: float, weight: float):
    """keys: [n_clips][n_keys][n][8] float32 -> (q [n][4], t [n][3]) fp64."""
    lib = _load()
    keys = _f32(keys)
    nc, nk, n, _ = keys.shape
    q, t = np.empty((n, 4)), np.empty((n, 3))
    lib.oracle_sample_local(n, nc, nk, float(rate), _p(keys, c_float), float(time), float(weight),
                            _p(q, c_double), _p(t, c_double))
    return q, t


def forward(parents, L) -> np.ndarray:
    """Sequential Hierarchy-Scan of local 3x4 matrices L [n][3][4] (fp64)."""
    lib = _load()
    parents, L = _i32(parents), _f64(L).reshape(-1, 12)
    M = np.empty_like(L)
    lib.oracle_forward(len(parents), _p(parents, c_int32), _p(L, c_double), _p(M, c_double))
    return M.reshape(-1, 3, 4)


def bind(M, B) -> np.ndarray:
    lib = _load()
    M, B = _f64(M).reshape(-1, 12), _f64(B).reshape(-1, 12)
    S = np.empty_like(M)
    lib.oracle_bind(len(M), _p(M, c_double), _p(B, c_double), _p(S, c_double))
    return S.reshape(-1, 3, 4)


def inverse_bind(parents, rest_q, rest_t) -> np.ndarray:
    lib = _load()
    parents, rq, rt = _i32(parents), _f32(rest_q), _f32(rest_t)
    B = np.empty((len(parents), 12))
    _check(lib.oracle_inverse_bind(len(parents), _p(parents, c_int32), _p(rq, c_float), _p(rt, c_float),
                                   _p(B, c_double)), "inverse_bind")
    return B.reshape(-1, 3, 4)


# ---------------------------------------------------------------- batched
class _Types:
    def __init__(self, types):
        self.counts = _i32([len(t["parents"]) for t in types])
        self.parents = _i32(np.concatenate([t["parents"] for t in types]))
        self.n = len(types)


def offsets(char_type, types) -> np.ndarray:
    n = np.array([len(types[t]["parents"]) for t in char_type], dtype=np.int64)
    off = np.zeros(len(n) + 1, dtype=np.int64)
    np.cumsum(n, out=off[1:])
    return off


def inverse_binds(types) -> np.ndarray:
    """Concatenated inverse bind poses [sum n_type][12] of every type."""
    return np.concatenate([inverse_bind(t["parents"], t["rest_q"], t["rest_t"]).reshape(-1, 12) for t in types])


def frame(w: dict, want_model: bool = False):
    """Skin matrices [sum][3][4] (fp64) of a clip-driven workload dict."""
    lib = _load()
    types = w["types"]
    T = _Types(types)
    B = inverse_binds(types)
    keys = [_f32(t["keys"]).ravel() for t in types]
    key_off = _i64(np.concatenate([[0], np.cumsum([k.size for k in keys])[:-1]]))
    keys_cat = _f32(np.concatenate(keys))
    n_clips = _i32([t["keys"].shape[0] for t in types])
    n_keys = _i32([t["keys"].shape[1] for t in types])
    rate = _f32([t["rate_hz"] for t in types])
    ct, tm, wt = _i32(w["char_type"]), _f32(w["time"]), _f32(w["weight"])
    off = offsets(ct, types)
    skin = np.empty((int(off[-1]), 12))
    model = np.empty((int(off[-1]), 12)) if want_model else None
    _check(lib.oracle_frame(T.n, _p(T.counts, c_int32), _p(T.parents, c_int32), _p(B, c_double),
                            _p(keys_cat, c_float), _p(key_off, c_int64), _p(n_clips, c_int32), _p(n_keys, c_int32),
                            _p(rate, c_float), len(ct), _p(ct, c_int32), _p(tm, c_float), _p(wt, c_float),
                            _p(off, c_int64), _p(skin, c_double),
                            model.ctypes.data_as(c_void_p) if model is not None else None), "frame")
    skin = skin.reshape(-1, 3, 4)
    return (skin, model.reshape(-1, 3, 4)) if want_model else skin


def forward_qt(types, char_type, q, t, with_skin: bool = True):
    """(skin or None, model) [sum][3][4] fp64 from local poses q [sum][4], t [sum][3]."""
    lib = _load()
    T = _Types(types)
    B = inverse_binds(types) if with_skin else None
    ct, q, t = _i32(char_type), _f64(q), _f64(t)
    off = offsets(ct, types)
    nt = int(off[-1])
    model = np.empty((nt, 12))
    skin = np.empty((nt, 12)) if with_skin else None
    _check(lib.oracle_forward_qt(T.n, _p(T.counts, c_int32), _p(T.parents, c_int32),
                                 B.ctypes.data_as(c_void_p) if B is not None else None, len(ct), _p(ct, c_int32),
                                 _p(q, c_double), _p(t, c_double), _p(off, c_int64),
                                 skin.ctypes.data_as(c_void_p) if skin is not None else None,
                                 model.ctypes.data_as(c_void_p)), "forward_qt")
    return (skin.reshape(-1, 3, 4) if skin is not None else None), model.reshape(-1, 3, 4)


def _grad(fn, types, char_type, q, t, g_pos):
    T = _Types(types)
    ct, q, t, g = _i32(char_type), _f64(q), _f64(t), _f64(g_pos)
    off = offsets(ct, types)
    nt = int(off[-1])
    dq, dt = np.empty((nt, 4)), np.empty((nt, 3))
    _check(fn(T.n, _p(T.counts, c_int32), _p(T.parents, c_int32), len(ct), _p(ct, c_int32), _p(q, c_double),
              _p(t, c_double), _p(g, c_double), _p(off, c_int64), _p(dq, c_double), _p(dt, c_double)), "grad")
    return dq, dt


def grad(types, char_type, q, t, g_pos):
    """(dq [sum][4], dt [sum][3]) of a loss with dLoss/dp = g_pos, by the
    generic reverse pass over 4x4 products."""
    return _grad(_load().oracle_grad, types, char_type, q, t, g_pos)


def grad_force_moment(types, char_type, q, t, g_pos):
    """The same gradient by subtree force/moment sums (independent derivation)."""
    return _grad(_load().oracle_grad_force_moment, types, char_type, q, t, g_pos)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on fp64 arrays p, m, v."""
    lib = _load()
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.oracle_adam(p.size, _p(p, c_double), _p(g, c_double), _p(m, c_double), _p(v, c_double), int(step),
                    float(lr), float(b1), float(b2), float(eps))


def ik(types, char_type, t, q0, effectors, targets, n_steps, lr=1e-2, betas=(0.9, 0.999), eps=1e-8):
    """Batched IK.  Returns (q_final [sum][4] fp64, loss history [n_steps])."""
    lib = _load()
    T = _Types(types)
    ct, t = _i32(char_type), _f64(t)
    eff = _i32(effectors)
    n_eff = eff.shape[1]
    tg = _f64(targets).reshape(len(ct), n_eff, 3)
    off = offsets(ct, types)
    q = _f64(q0).copy()
    hist = np.empty(n_steps)
    _check(lib.oracle_ik(T.n, _p(T.counts, c_int32), _p(T.parents, c_int32), _p(eff, c_int32), n_eff, len(ct),
                         _p(ct, c_int32), _p(t, c_double), _p(tg, c_double), _p(off, c_int64), int(n_steps),
                         float(lr), float(betas[0]), float(betas[1]), float(eps), _p(q, c_double),
                         _p(hist, c_double)), "ik")
    return q, hist


def _ik_share(task):
    """One process of ik_all_cores: oracle.ik on a contiguous share of the
    characters (the characters are independent problems)."""
    types, ct, t, q0, eff, tg, n_steps, lr, betas, eps = task
    return ik(types, ct, t, q0, eff, tg, n_steps, lr, betas, eps)


def ik_all_cores(types, char_type, t, q0, effectors, targets, n_steps, lr=1e-2, betas=(0.9, 0.999), eps=1e-8,
                 workers: int | None = None):
    """oracle.ik with the characters split into contiguous shares, one per
    process (started with spawn, so none forks after CUDA has started).
    Returns (q_final [sum][4] fp64, loss history [n_steps] summed over the
    shares, processes used)."""
    import multiprocessing as mp
    ct = _i32(char_type)
    if workers is None:
        try:
            workers = len(os.sched_getaffinity(0))
        except (AttributeError, OSError):
            workers = os.cpu_count() or 1
    workers = max(1, min(workers, len(ct)))
    off = offsets(ct, types)
    t, q0, tg = _f64(t), _f64(q0), _f64(targets).reshape(len(ct), -1, 3)
    tasks = []
    for idx in np.array_split(np.arange(len(ct)), workers):
        if len(idx) == 0:
            continue
        r0, r1 = int(off[idx[0]]), int(off[idx[-1] + 1])
        tasks.append((types, ct[idx], t[r0:r1], q0[r0:r1], effectors, tg[idx], n_steps, lr, betas, eps))
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        res = pool.map(_ik_share, tasks)
    return np.concatenate([r[0] for r in res]), np.sum([r[1] for r in res], axis=0), len(tasks)


def ik_targets(w: dict) -> np.ndarray:
    """Effector positions of the workload's target pose, [n_chars][n_eff][3]
    fp64 (the oracle's own derivation of the IK targets)."""
    types = w["types"]
    _, model = forward_qt(types, w["char_type"], w["q_target"], w["t"], with_skin=False)
    off = offsets(w["char_type"], types)
    eff = w["effectors"]
    out = np.empty((len(w["char_type"]), eff.shape[1], 3))
    for c, ty in enumerate(w["char_type"]):
        out[c] = model[off[c] + eff[ty], :, 3]
    return out


def lbs(mesh: dict, skin) -> np.ndarray:
    """Linear blend skinning of one character's mesh with its skin matrices
    skin [n][3][4]: [n_verts][6] fp64 (skinned position, unit normal)."""
    lib = _load()
    pos, nrm = _f32(mesh["pos"]), _f32(mesh["nrm"])
    bones, wts = _i32(mesh["bones"]), _f32(mesh["weights"])
    S = _f64(np.asarray(skin).reshape(-1, 12))
    out = np.empty((len(pos), 6))
    lib.oracle_lbs(len(pos), _p(pos, c_float), _p(nrm, c_float), _p(bones, c_int32), _p(wts, c_float),
                   _p(S, c_double), _p(out, c_double))
    return out


def vertex_offsets(char_type, types) -> np.ndarray:
    """Exclusive prefix of the characters' vertex counts (n_chars + 1); a
    type without a mesh has none."""
    nv = np.array([len(types[int(t)]["mesh"]["pos"]) if "mesh" in types[int(t)] else 0 for t in char_type], np.int64)
    return np.concatenate([[0], np.cumsum(nv)]).astype(np.int64)


def skin_vertices(w: dict, skin) -> np.ndarray:
    """Skinned vertices [sum of vertex counts][6] of a workload whose types
    carry meshes, from the skin matrices [sum][3][4] of its characters."""
    types, ct = w["types"], w["char_type"]
    off, voff = offsets(ct, types), vertex_offsets(ct, types)
    out = np.empty((int(voff[-1]), 6))
    for c, ty in enumerate(ct):
        if voff[c + 1] > voff[c]:
            out[voff[c]:voff[c + 1]] = lbs(types[int(ty)]["mesh"], skin[off[c]:off[c + 1]])
    return out


def sample_layers(keys: np.ndarray, rate: float, time: float, weights, add_keys=None, add_w: float = 0.0):
    """Layered blend of one character's joints: (q [n][4], t [n][3]) fp64.
    keys [n_clips][n_keys][n][8] (n_clips <= 4), weights [n_clips], optional
    additive layer add_keys [n_keys][n][8] applied with weight add_w."""
    lib = _load()
    k = _f32(keys)
    nc, nk, n = k.shape[:3]
    wts = _f32(np.resize(np.asarray(weights, np.float32), 4))
    ak = _f32(add_keys) if add_keys is not None else None
    q, t = np.empty((n, 4)), np.empty((n, 3))
    lib.oracle_sample_layers(n, nc, nk, float(rate), _p(k, c_float),
                             ak.ctypes.data_as(c_void_p) if ak is not None else None, float(time), _p(wts, c_float),
                             float(add_w), _p(q, c_double), _p(t, c_double))
    return q, t


def frame_layers(w: dict):
    """Skin matrices [sum][3][4] of a workload with per-character clip
    weights w["weights"] [n_chars][4] and additive weights w["add_w"];
    types may carry "add_keys" [n_keys][n][8]."""
    lib = _load()
    types = w["types"]
    T = _Types(types)
    B = inverse_binds(types)
    keys = [_f32(t["keys"]).ravel() for t in types]
    key_off = _i64(np.concatenate([[0], np.cumsum([k.size for k in keys])[:-1]]))
    keys_cat = _f32(np.concatenate(keys))
    adds = [_f32(t["add_keys"]).ravel() if "add_keys" in t else np.zeros(0, np.float32) for t in types]
    add_cat = _f32(np.concatenate(adds)) if sum(a.size for a in adds) else _f32(np.zeros(1))
    pos = np.concatenate([[0], np.cumsum([a.size for a in adds])[:-1]])
    add_off = _i64([pos[i] if "add_keys" in t else -1 for i, t in enumerate(types)])
    n_clips = _i32([t["keys"].shape[0] for t in types])
    n_keys = _i32([t["keys"].shape[1] for t in types])
    rate = _f32([t["rate_hz"] for t in types])
    ct, tm = _i32(w["char_type"]), _f32(w["time"])
    wts, aw = _f32(w["weights"]).reshape(-1, 4), _f32(w["add_w"])
    off = offsets(ct, types)
    skin = np.empty((int(off[-1]), 12))
    _check(lib.oracle_frame_layers(T.n, _p(T.counts, c_int32), _p(T.parents, c_int32), _p(B, c_double),
                                   _p(keys_cat, c_float), _p(key_off, c_int64), _p(n_clips, c_int32),
                                   _p(n_keys, c_int32), _p(rate, c_float), _p(add_cat, c_float), _p(add_off, c_int64),
                                   len(ct), _p(ct, c_int32), _p(tm, c_float), _p(wts, c_float), _p(aw, c_float),
                                   _p(off, c_int64), _p(skin, c_double)), "frame_layers")
    return skin.reshape(-1, 3, 4)


RASTER_EMPTY = 0xFFFFFFFF


def raster(faces_per_char, verts, vert_off, cols: int, spacing: float, ox: float, oy: float, scale: float,
           width: int, height: int, with_cover: bool = False):
    """Software rasterization of skinned characters (fixed rules, see
    oracle_raster): faces_per_char[c] [n_faces][3] vertex indices of
    character c, verts [sum][6] positions + normals, vert_off [n_chars + 1].
    Returns ids [height][width] uint32 (and per-pixel coverage counts)."""
    lib = _load()
    n = len(faces_per_char)
    fs = [np.ascontiguousarray(f, dtype=np.int32).reshape(-1) for f in faces_per_char]
    nf = _i32([len(f) // 3 for f in fs])
    arr = (POINTER(c_int32) * max(n, 1))(*[f.ctypes.data_as(POINTER(c_int32)) for f in fs])
    v = _f64(verts)
    vo = _i64(vert_off)
    ids = np.empty((height, width), np.uint32)
    cover = np.empty((height, width), np.int32) if with_cover else None
    lib.oracle_raster(n, _p(nf, c_int32), arr, _p(vo, c_int64), _p(v, c_double), int(cols), float(spacing), float(ox),
                      float(oy), float(scale), int(width), int(height), ids.ctypes.data_as(POINTER(ctypes.c_uint32)),
                      cover.ctypes.data_as(c_void_p) if cover is not None else None)
    return (ids, cover) if with_cover else ids
