"""Helpers for the GPU tests: set a workload up in the CUDA library through
its Python binding (which calls the C ABI) and compare with the oracle."""
import numpy as np


def tol_for_depth(depth: int) -> float:
    """Max-abs tolerance on skeletons of unit extent: 1e-4, and 5e-4 for
    depth >= 1024 (FP32 against the FP64 oracle)."""
    return 5e-4 if depth >= 1024 else 1e-4


def setup(w: dict, device: int = 0, with_clips: bool = True):
    """Context + plan for a workload dict from synth; inverse binds are
    derived on the GPU from the rest pose (the oracle derives its own)."""
    import paper_2505_06703_gb300 as pk
    ctx = pk.Context(device)
    types = w["types"]
    ids = ctx.create_skeletons([t["parents"] for t in types], rest_q=[t["rest_q"] for t in types],
                               rest_t=[t["rest_t"] for t in types])
    if with_clips:
        for i, t in zip(ids, types):
            if "keys" in t:
                ctx.upload_clips(i, t["keys"], t["rate_hz"])
    for i, t in zip(ids, types):
        if "mesh" in t:
            ctx.upload_mesh(i, t["mesh"])
            if "faces" in t["mesh"] and len(t["mesh"]["faces"]):
                ctx.upload_faces(i, t["mesh"]["faces"])
        if with_clips and "add_keys" in t:
            ctx.upload_additive(i, t["add_keys"], t["rate_hz"])
    plan = ctx.plan(np.asarray(ids, np.int32)[w["char_type"]])
    return ctx, plan


def cuda(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def per_type_maxabs(got, ref, w):
    """Max |got - ref| per type over all characters of that type."""
    types = w["types"]
    off = np.zeros(len(w["char_type"]) + 1, np.int64)
    np.cumsum([len(types[t]["parents"]) for t in w["char_type"]], out=off[1:])
    err = np.abs(got.reshape(-1, 12) - ref.reshape(-1, 12)).max(axis=1)
    out = {}
    for ty in range(len(types)):
        rows = np.concatenate([np.arange(off[c], off[c + 1]) for c in np.nonzero(w["char_type"] == ty)[0]] or
                              [np.zeros(0, np.int64)])
        if len(rows):
            out[ty] = float(err[rows].max())
    return out


def assert_skin_close(got, ref, w):
    errs = per_type_maxabs(got, ref, w)
    for ty, e in errs.items():
        tol = tol_for_depth(w["types"][ty]["depth"])
        assert e <= tol, f"type {ty} (depth {w['types'][ty]['depth']}): max-abs {e:.3e} > {tol:.0e}"
    return errs
