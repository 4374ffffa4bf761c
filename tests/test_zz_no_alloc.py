"""anim_forward_local_noalloc: the forward scan + bind for callers that may
not allocate device memory (code under a fixed device-memory budget or a
custom allocator that owns every byte, plug-ins handed only pre-allocated
buffers, processes that must not grow after start-up).  Its scratch is a
static device array instead of cudaMalloc, shared by every call.

The output is compared element by element with the FP64 oracle (the
sequential parent-before-child product of Eq. 1, then the bind product) and
with the regular entry point anim_forward_local, on two calls in a row with
two different skeletons, so the second call must replace the first call's
tables in the shared array.  Then the documented refusals: sizes beyond the
limits, bad arguments, an empty batch, and a stream under graph capture.
The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4  # skeletons of unit extent, depth < 1024


def _rigid(rng, n):
    from scipy.spatial.transform import Rotation
    B = np.zeros((n, 3, 4), np.float32)
    B[:, :, :3] = Rotation.from_quat(synth.random_unit_quats(rng, n, 180.0)).as_matrix()
    B[:, :, 3] = rng.uniform(-1, 1, (n, 3))
    return B


def _call(lib, n, parents, n_chars, dq, dt, dB, out, stream=None):
    import torch
    par = np.ascontiguousarray(parents, dtype=np.int32)
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    return lib.anim_forward_local_noalloc(n, ctypes.c_void_p(par.ctypes.data), n_chars,
                                          ctypes.c_void_p(dq.data_ptr()), ctypes.c_void_p(dt.data_ptr()),
                                          ctypes.c_void_p(dB.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(st))


def _oracle_skin(parents, q, t, B, n_chars):
    n = len(parents)
    types = [{"parents": np.asarray(parents, np.int32)}]
    _, model = oracle.forward_qt(types, np.zeros(n_chars, np.int32), q, t, with_skin=False)
    Bt = np.tile(B.reshape(n, 12).astype(np.float64), (n_chars, 1))
    return oracle.bind(model, Bt).reshape(-1, 12)


def test_noalloc_matches_oracle_and_forward_local_twice():
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
        ref = _oracle_skin(parents, q, t, B, n_chars)
        ctx = pk.Context(0)
        ids = ctx.create_skeletons([parents], inv_bind=[B])
        plan = ctx.plan(np.full(n_chars, ids[0], np.int32))
        dq, dt = torch.as_tensor(q).cuda(), torch.as_tensor(t).cuda()
        regular, _ = ctx.forward_local(plan, dq, dt, skin=True, model=False)
        dB = torch.as_tensor(B.reshape(n, 12)).cuda()
        out = torch.full((n_chars * n, 12), float("nan"), device="cuda")
        assert _call(lib, n, parents, n_chars, dq, dt, dB, out) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err_oracle = np.abs(got - ref).max()
        assert err_oracle <= TOL, err_oracle
        err_regular = (out - regular).abs().max().item()
        assert err_regular <= TOL, err_regular


def test_noalloc_edge_cases_and_refusals():
    import torch
    import paper_2505_06703_gb300 as pk
    lib = pk.load()
    rng = np.random.default_rng(7)
    z = torch.zeros(64, device="cuda")
    one = np.array([-1], np.int32)
    # beyond the joint limit, and a 2,048-joint star whose one-character item
    # does not fit in shared memory
    assert _call(lib, 4096, one, 1, z, z, z, z) == -7
    star = np.zeros(2048, np.int32)
    star[0] = -1
    q, t = synth.local_poses(rng, 2048, t_half=0.01)
    dq, dt = torch.as_tensor(q).cuda(), torch.as_tensor(t).cuda()
    dB = torch.zeros((2048, 12), device="cuda")
    out = torch.zeros((2048, 12), device="cuda")
    assert _call(lib, 2048, star, 1, dq, dt, dB, out) == -7
    # bad parent, misaligned output
    bad = np.array([-1, 1], np.int32)
    assert _call(lib, 2, bad, 1, z, z, z, z) == -1
    assert lib.anim_forward_local_noalloc(1, ctypes.c_void_p(one.ctypes.data), 1, ctypes.c_void_p(z.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr() + 4), None) == -1
    # an empty batch succeeds and writes nothing
    sentinel = torch.full((4, 12), 7.0, device="cuda")
    assert _call(lib, 1, one, 0, z, z, z, sentinel) == 0
    torch.cuda.synchronize()
    assert bool((sentinel == 7.0).all())
    # a one-joint skeleton: S = L B
    n_chars = 33
    q1, t1 = synth.local_poses(rng, n_chars, t_half=0.01)
    B1 = _rigid(rng, 1)
    dq1, dt1 = torch.as_tensor(q1).cuda(), torch.as_tensor(t1).cuda()
    dB1 = torch.as_tensor(B1.reshape(1, 12)).cuda()
    out1 = torch.full((n_chars, 12), float("nan"), device="cuda")
    assert _call(lib, 1, one, n_chars, dq1, dt1, dB1, out1) == 0
    torch.cuda.synchronize()
    ref1 = _oracle_skin(one, q1, t1, B1, n_chars)
    assert np.abs(out1.cpu().numpy() - ref1).max() <= TOL
    # a stream under graph capture is refused and the capture stays usable
    s = torch.cuda.Stream()
    x = torch.zeros(8, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = _call(lib, 1, one, n_chars, dq1, dt1, dB1, out1, stream=s.cuda_stream)
        x.add_(1.0)
    assert rc == -7
    g.replay()
    torch.cuda.synchronize()
    assert bool((x == 1.0).all())
