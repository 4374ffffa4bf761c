"""Thin Python binding of the C ABI in include/anim.h.

Argument marshalling only: every computation runs in the CUDA library's
kernels.  PyTorch supplies device memory (tensors) and streams.  There is no
CPU fallback: loading fails loudly if the library is missing or cannot be
built, and every call raises on a non-zero return code.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_float, c_int, c_int32, c_int64, c_void_p

import numpy as np

from . import _build

ANIM_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EDEVICE", -6: "ESTATE", -7: "EUNSUPPORTED"}

# name -> (restype, argtypes), mirroring include/anim.h
_P = c_void_p
SIGNATURES = {
    "anim_version": (c_int, []),
    "anim_last_error": (ctypes.c_char_p, [_P]),
    "anim_create": (c_int, [POINTER(_P), c_int]),
    "anim_destroy": (c_int, [_P]),
    "anim_create_skeletons": (c_int, [_P, c_int, _P, _P, _P, _P, _P, _P]),
    "anim_upload_clips": (c_int, [_P, c_int32, c_int, c_int, c_float, _P]),
    "anim_plan_create": (c_int, [_P, c_int64, _P, POINTER(_P)]),
    "anim_plan_destroy": (c_int, [_P, _P]),
    "anim_plan_total_joints": (c_int, [_P, POINTER(c_int64)]),
    "anim_plan_row_offsets": (c_int, [_P, _P]),
    "anim_upload_mesh": (c_int, [_P, c_int32, c_int, _P, _P, _P, _P]),
    "anim_plan_vertex_offsets": (c_int, [_P, _P, _P]),
    "anim_evaluate_frame_skinned": (c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "anim_upload_additive": (c_int, [_P, c_int32, c_int, c_float, _P]),
    "anim_upload_faces": (c_int, [_P, c_int32, c_int, _P]),
    "anim_raster": (c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "anim_evaluate_frame_layers": (c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "anim_evaluate_frame": (c_int, [_P, _P, _P, _P, _P, _P]),
    "anim_evaluate_frame_host": (c_int, [_P, _P, _P, _P, _P, _P]),
    "anim_evaluate_frame_levelsync": (c_int, [_P, _P, _P, _P, _P, _P]),
    "anim_frame_build_queue": (c_int, [_P, _P, _P, _P]),
    "anim_frame_run_queue": (c_int, [_P, _P, _P, _P, _P, _P]),
    "anim_forward_local": (c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "anim_forward_local_levelsync": (c_int, [_P, _P, _P, _P, _P, _P]),
    "anim_forward_local_paper": (c_int, [_P, _P, c_int, _P, _P, _P, _P]),
    "anim_backward": (c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "anim_loss_backward": (c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "anim_ik_create": (c_int, [_P, _P, c_int, _P, POINTER(_P)]),
    "anim_ik_destroy": (c_int, [_P, _P]),
    "anim_ik_reset": (c_int, [_P, _P, _P]),
    "anim_ik_step": (c_int, [_P, _P, _P, _P, _P, _P, _P, c_float, c_float, c_float, c_float, _P, _P]),
    "anim_tune": (c_int, [_P, _P, c_int]),
    "anim_tune_ik": (c_int, [_P, _P, c_int, _P]),
    "anim_get_status": (c_int, [_P, _P, POINTER(c_int)]),
    "anim_analyze_skeleton": (c_int, [c_int, _P, c_int, POINTER(c_int32), _P, POINTER(c_int32), POINTER(c_int32)]),
    "anim_forward_local_noalloc": (c_int, [c_int, _P, c_int64, _P, _P, _P, _P, _P]),
    "anim_get_schedule": (c_int, [_P, _P, _P]),
    "anim_set_schedule": (c_int, [_P, _P, _P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libanim.so (building it in-tree first if needed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class AnimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _np_ptr(a):
    return c_void_p(a.ctypes.data) if a is not None else None


def _dptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def analyze_skeleton(parents, seg_len: int = 8):
    """Host-only: (seg_start, rounds, depth) of the scan's segment decomposition."""
    lib = load()
    p = np.ascontiguousarray(parents, dtype=np.int32)
    starts = np.zeros(len(p) + 1, dtype=np.int32)
    nseg, rounds, depth = c_int32(), c_int32(), c_int32()
    rc = lib.anim_analyze_skeleton(len(p), _np_ptr(p), int(seg_len), ctypes.byref(nseg), _np_ptr(starts),
                                   ctypes.byref(rounds), ctypes.byref(depth))
    if rc != ANIM_OK:
        raise AnimError(rc, "anim_analyze_skeleton rejected the parent array")
    return starts[: nseg.value + 1].copy(), rounds.value, depth.value


class Context:
    """An anim_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        self.lib = load()
        self.device = device
        torch.cuda.init()
        h = c_void_p()
        rc = self.lib.anim_create(ctypes.byref(h), int(device))
        if rc != ANIM_OK:
            raise AnimError(rc, self.lib.anim_last_error(None).decode())
        self.h = h
        self.type_sizes = []

    def _ck(self, rc):
        if rc != ANIM_OK:
            raise AnimError(rc, self.lib.anim_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.anim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- setup
    def create_skeletons(self, parents_list, inv_bind=None, rest_q=None, rest_t=None):
        """Register skeleton types; returns their type ids."""
        counts = np.array([len(p) for p in parents_list], dtype=np.int32)
        par = np.ascontiguousarray(np.concatenate(parents_list), dtype=np.int32)
        cat = lambda xs: None if xs is None else np.ascontiguousarray(np.concatenate(
            [np.asarray(x, np.float32).reshape(len(p), -1) for x, p in zip(xs, parents_list)]), dtype=np.float32)
        ib, rq, rt = cat(inv_bind), cat(rest_q), cat(rest_t)
        ids = np.zeros(len(counts), dtype=np.int32)
        self._ck(self.lib.anim_create_skeletons(self.h, len(counts), _np_ptr(counts), _np_ptr(par), _np_ptr(ib),
                                                _np_ptr(rq), _np_ptr(rt), _np_ptr(ids)))
        self.type_sizes += [int(c) for c in counts]
        return [int(i) for i in ids]

    def upload_clips(self, type_id: int, keys, rate_hz: float):
        k = np.ascontiguousarray(keys, dtype=np.float32)
        nc, nk, n, eight = k.shape
        assert eight == 8
        self._ck(self.lib.anim_upload_clips(self.h, int(type_id), nc, nk, float(rate_hz), _np_ptr(k)))

    def upload_additive(self, type_id: int, keys, rate_hz: float):
        k = np.ascontiguousarray(keys, dtype=np.float32)
        nk, n, eight = k.shape
        assert eight == 8
        self._ck(self.lib.anim_upload_additive(self.h, int(type_id), nk, float(rate_hz), _np_ptr(k)))

    def evaluate_frame_layers(self, plan, time, weights, add_w=None, out=None, stream=None):
        """Frame with layered blending: clip weights [n_chars, 4], additive weights [n_chars] or None."""
        out = self._out(plan, 12, out)
        self._ck(self.lib.anim_evaluate_frame_layers(self.h, plan.h, _dptr(time), _dptr(weights), _dptr(add_w),
                                                     _dptr(out), _stream(stream)))
        return out

    def upload_faces(self, type_id: int, faces):
        f = np.ascontiguousarray(faces, dtype=np.int32)
        self._ck(self.lib.anim_upload_faces(self.h, int(type_id), len(f), _np_ptr(f)))

    def raster(self, plan, verts, width, height, cols, spacing, ox, oy, scale, ids=True, rgba=False, vis=None,
               stream=None):
        """Headless rasterization of the skinned characters: (ids [h, w] int32
        view of uint32 or None, rgba [h, w] int32 view or None); ids / rgba
        may be given as tensors to write into, or True / False."""
        import torch
        dev = f"cuda:{self.device}"
        vis = vis if vis is not None else torch.empty((height, width), dtype=torch.int64, device=dev)
        pick = lambda x: x if isinstance(x, torch.Tensor) else (
            torch.empty((height, width), dtype=torch.int32, device=dev) if x else None)
        out_ids, out_rgba = pick(ids), pick(rgba)
        p = _RasterParams(int(width), int(height), int(cols), float(spacing), float(ox), float(oy), float(scale))
        self._ck(self.lib.anim_raster(self.h, plan.h, _dptr(verts), ctypes.byref(p), _dptr(vis), _dptr(out_ids),
                                      _dptr(out_rgba), _stream(stream)))
        return out_ids, out_rgba

    def upload_mesh(self, type_id: int, mesh: dict):
        """mesh: pos [nv,3], nrm [nv,3], bones [nv,4] int, weights [nv,4]."""
        pos = np.ascontiguousarray(mesh["pos"], dtype=np.float32)
        nrm = np.ascontiguousarray(mesh["nrm"], dtype=np.float32)
        bones = np.ascontiguousarray(mesh["bones"], dtype=np.int32)
        wts = np.ascontiguousarray(mesh["weights"], dtype=np.float32)
        self._ck(self.lib.anim_upload_mesh(self.h, int(type_id), len(pos), _np_ptr(pos), _np_ptr(nrm),
                                           _np_ptr(bones), _np_ptr(wts)))

    def vertex_offsets(self, plan):
        out = np.zeros(plan.n_chars + 1, dtype=np.int64)
        self._ck(self.lib.anim_plan_vertex_offsets(self.h, plan.h, _np_ptr(out)))
        return out

    def evaluate_frame_skinned(self, plan, time, blend_w, verts=None, skin=None, stream=None):
        """Frame + fused linear blend skinning: vertices [total vertices, 6];
        pass a skin tensor [total, 12] to also receive the skin matrices."""
        import torch
        if verts is None:
            nv = int(self.vertex_offsets(plan)[-1])
            verts = torch.empty((max(nv, 1), 6), dtype=torch.float32, device=f"cuda:{self.device}")
        self._ck(self.lib.anim_evaluate_frame_skinned(self.h, plan.h, _dptr(time), _dptr(blend_w), _dptr(skin),
                                                      _dptr(verts), _stream(stream)))
        return verts

    def plan(self, char_type):
        return Plan(self, char_type)

    def status(self, stream=None) -> int:
        v = c_int()
        self._ck(self.lib.anim_get_status(self.h, _stream(stream), ctypes.byref(v)))
        return v.value

    # ---------------------------------------------------------- evaluation
    def _out(self, plan, cols, out):
        import torch
        if out is None:
            out = torch.empty((plan.total, cols), dtype=torch.float32, device=f"cuda:{self.device}")
        return out

    def evaluate_frame(self, plan, time, blend_w, out=None, stream=None, levelsync=False):
        """Fused frame: skin matrices [total, 12] from per-character time and blend weight."""
        out = self._out(plan, 12, out)
        fn = self.lib.anim_evaluate_frame_levelsync if levelsync else self.lib.anim_evaluate_frame
        self._ck(fn(self.h, plan.h, _dptr(time), _dptr(blend_w), _dptr(out), _stream(stream)))
        return out

    def evaluate_frame_host(self, plan, time, blend_w, out=None, stream=None):
        """The frame from and to host memory: time, blend_w are CPU float32
        tensors [n_chars] (page-locked for asynchronous copies); returns the
        CPU tensor [total, 12] the skin matrices are copied into (page-locked
        when allocated here).  Complete once `stream` has synchronized."""
        import torch
        for x in (time, blend_w):
            if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous() or x.numel() != plan.n_chars:
                raise ValueError("time and blend_w must be contiguous CPU float32 tensors [n_chars]")
        if out is None:
            out = torch.empty((plan.total, 12), dtype=torch.float32, pin_memory=True)
        if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != plan.total * 12:
            raise ValueError("out must be a contiguous CPU float32 tensor [total, 12]")
        self._ck(self.lib.anim_evaluate_frame_host(self.h, plan.h, c_void_p(time.data_ptr()),
                                                   c_void_p(blend_w.data_ptr()), c_void_p(out.data_ptr()),
                                                   _stream(stream)))
        return out

    def frame_build_queue(self, plan, time, stream=None):
        self._ck(self.lib.anim_frame_build_queue(self.h, plan.h, _dptr(time), _stream(stream)))

    def frame_run_queue(self, plan, time, blend_w, out, stream=None):
        self._ck(self.lib.anim_frame_run_queue(self.h, plan.h, _dptr(time), _dptr(blend_w), _dptr(out),
                                               _stream(stream)))
        return out

    def forward_local(self, plan, q, t, skin=True, model=False, stream=None, levelsync=False):
        """(skin or None, model or None) from local poses q [total,4], t [total,3]."""
        s = self._out(plan, 12, None) if skin else None
        m = self._out(plan, 12, None) if model else None
        if levelsync:
            assert skin and not model
            self._ck(self.lib.anim_forward_local_levelsync(self.h, plan.h, _dptr(q), _dptr(t), _dptr(s),
                                                           _stream(stream)))
        else:
            self._ck(self.lib.anim_forward_local(self.h, plan.h, _dptr(q), _dptr(t), _dptr(s), _dptr(m),
                                                 _stream(stream)))
        return s, m

    def forward_local_paper(self, plan, algorithm, q, t, out=None, stream=None):
        """Skin matrices from local poses with the paper's Algorithm 1-4
        (one CTA per character, one thread per joint): a comparator."""
        s = self._out(plan, 12, out)
        self._ck(self.lib.anim_forward_local_paper(self.h, plan.h, int(algorithm), _dptr(q), _dptr(t), _dptr(s),
                                                   _stream(stream)))
        return s

    def backward(self, plan, q, t, grad_pos, grad_q=None, grad_t=None, stream=None):
        grad_q = self._out(plan, 4, grad_q)
        grad_t = self._out(plan, 3, grad_t)
        self._ck(self.lib.anim_backward(self.h, plan.h, _dptr(q), _dptr(t), _dptr(grad_pos), _dptr(grad_q),
                                        _dptr(grad_t), _stream(stream)))
        return grad_q, grad_t

    def loss_backward(self, plan, q, t, target, grad_q=None, grad_t=None, loss=None, stream=None):
        import torch
        grad_q = self._out(plan, 4, grad_q)
        grad_t = self._out(plan, 3, grad_t)
        if loss is None:
            loss = torch.empty(plan.n_chars, dtype=torch.float32, device=f"cuda:{self.device}")
        self._ck(self.lib.anim_loss_backward(self.h, plan.h, _dptr(q), _dptr(t), _dptr(target), _dptr(grad_q),
                                             _dptr(grad_t), _dptr(loss), _stream(stream)))
        return grad_q, grad_t, loss

    def ik(self, plan, effectors):
        return IK(self, plan, effectors)

    def tune(self, plan, which: int = 0):
        self._ck(self.lib.anim_tune(self.h, plan.h, int(which)))

    def tune_ik(self, plan, effectors):
        """Autotune the schedule for the IK step (effectors: [n_types][n_eff])."""
        e = np.ascontiguousarray(effectors, dtype=np.int32)
        self._ck(self.lib.anim_tune_ik(self.h, plan.h, int(e.shape[1]), _np_ptr(e)))

    def get_schedule(self, plan):
        """[seg_len, ctas_per_sm, joints_per_item, walk, adj_ctas]"""
        out = np.zeros(5, dtype=np.int32)
        self._ck(self.lib.anim_get_schedule(self.h, plan.h, _np_ptr(out)))
        return [int(x) for x in out]

    def set_schedule(self, plan, sched):
        """Five values as get_schedule returns; four keep the current adjoint kernel."""
        sched = list(sched)
        if len(sched) == 4:
            sched.append(self.get_schedule(plan)[4])
        if len(sched) != 5:
            raise ValueError("a schedule has 5 values")
        a = np.ascontiguousarray(sched, dtype=np.int32)
        self._ck(self.lib.anim_set_schedule(self.h, plan.h, _np_ptr(a)))


class _RasterParams(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("cols", c_int32), ("spacing", c_float), ("ox", c_float),
                ("oy", c_float), ("scale", c_float)]


class Plan:
    def __init__(self, ctx: Context, char_type):
        self.ctx = ctx
        ct = np.ascontiguousarray(char_type, dtype=np.int32)
        self.n_chars = len(ct)
        h = c_void_p()
        ctx._ck(ctx.lib.anim_plan_create(ctx.h, len(ct), _np_ptr(ct), ctypes.byref(h)))
        self.h = h
        tot = c_int64()
        ctx._ck(ctx.lib.anim_plan_total_joints(h, ctypes.byref(tot)))
        self.total = tot.value
        self.row_off = np.zeros(len(ct) + 1, dtype=np.int64)
        ctx._ck(ctx.lib.anim_plan_row_offsets(h, _np_ptr(self.row_off)))

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            self.ctx.lib.anim_plan_destroy(self.ctx.h, self.h)
        self.h = None


class IK:
    def __init__(self, ctx: Context, plan: Plan, effectors):
        self.ctx, self.plan = ctx, plan
        eff = np.ascontiguousarray(effectors, dtype=np.int32)
        self.n_eff = eff.shape[1]
        h = c_void_p()
        ctx._ck(ctx.lib.anim_ik_create(ctx.h, plan.h, self.n_eff, _np_ptr(eff), ctypes.byref(h)))
        self.h = h

    def reset(self, stream=None):
        self.ctx._ck(self.ctx.lib.anim_ik_reset(self.ctx.h, self.h, _stream(stream)))

    def step(self, q, m, v, t, targets, lr=1e-2, betas=(0.9, 0.999), eps=1e-8, loss=None, stream=None):
        """One fused IK step; m = v = None keeps Adam's moments in the IK
        object's own state (active joints only; zeroed by reset())."""
        self.ctx._ck(self.ctx.lib.anim_ik_step(self.ctx.h, self.h, _dptr(q), _dptr(m), _dptr(v), _dptr(t),
                                               _dptr(targets), float(lr), float(betas[0]), float(betas[1]),
                                               float(eps), _dptr(loss), _stream(stream)))


def hierarchy_fn():
    """torch.autograd.Function: model-space joint positions p [total, 3] of
    local poses (q, t); its backward is the library's adjoint kernel."""
    import torch

    class HierarchyFn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, q, t, actx, plan):
            q = q.contiguous()
            t = t.contiguous()
            _, model = actx.forward_local(plan, q, t, skin=False, model=True)
            fctx.save_for_backward(q, t)
            fctx.actx, fctx.plan = actx, plan
            return model.view(-1, 3, 4)[:, :, 3]

        @staticmethod
        def backward(fctx, grad_pos):
            q, t = fctx.saved_tensors
            gq, gt = fctx.actx.backward(fctx.plan, q, t, grad_pos.contiguous())
            return gq, gt, None, None

    return HierarchyFn
