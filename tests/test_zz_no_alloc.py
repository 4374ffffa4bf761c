"""anim_forward_local_noalloc: the forward scan + bind for callers that may
not allocate device memory (code under a fixed device-memory budget or a
custom allocator that owns every byte, plug-ins handed only pre-allocated
buffers, processes that must not grow after start-up).  It uses a static
device array for its scratch instead of cudaMalloc, so this test checks it
against the regular entry point anim_forward_local on two calls in a row,
with two different skeletons so the second call must replace the first
call's tables in the shared array.  The file name makes pytest collect it
last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _rigid(rng, n):
    from scipy.spatial.transform import Rotation
    B = np.zeros((n, 3, 4), np.float32)
    B[:, :, :3] = Rotation.from_quat(synth.random_unit_quats(rng, n, 180.0)).as_matrix()
    B[:, :, 3] = rng.uniform(-1, 1, (n, 3))
    return B


def test_noalloc_matches_forward_local_twice():
    import torch
    import paper_2505_06703_gb300 as pk
    lib = pk.load()
    rng = np.random.default_rng(2024)
    cases = [synth.relabel_dfs(synth.random_tree(256, 96, rng, spine=96), rng)[0],
             synth.relabel_random_topological(synth.random_tree(64, 12, rng, spine=12), rng)[0]]
    for parents, n_chars in zip(cases, (96, 257)):
        n = len(parents)
        B = _rigid(rng, n)
        q, t = synth.local_poses(rng, n_chars * n, t_half=0.01)
        ctx = pk.Context(0)
        ids = ctx.create_skeletons([parents], inv_bind=[B])
        plan = ctx.plan(np.full(n_chars, ids[0], np.int32))
        dq, dt = torch.as_tensor(q).cuda(), torch.as_tensor(t).cuda()
        ref, _ = ctx.forward_local(plan, dq, dt, skin=True, model=False)
        dB = torch.as_tensor(B.reshape(n, 12)).cuda()
        out = torch.full((n_chars * n, 12), float("nan"), device="cuda")
        par = np.ascontiguousarray(parents, dtype=np.int32)
        rc = lib.anim_forward_local_noalloc(n, ctypes.c_void_p(par.ctypes.data), n_chars,
                                            ctypes.c_void_p(dq.data_ptr()), ctypes.c_void_p(dt.data_ptr()),
                                            ctypes.c_void_p(dB.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= 1e-4, err
    # sizes beyond the static array's limits are rejected, not run
    one = np.array([-1], np.int32)
    big = torch.zeros(16, device="cuda")
    assert lib.anim_forward_local_noalloc(4096, ctypes.c_void_p(one.ctypes.data), 1, ctypes.c_void_p(big.data_ptr()),
                                          ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                          ctypes.c_void_p(big.data_ptr()), None) == -7
