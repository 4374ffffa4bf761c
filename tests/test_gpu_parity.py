"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle,
element by element, on the five workloads at full size and on edge cases.

Tolerances: max-abs 1e-4 on skeletons of unit extent, 5e-4 for depth >= 1024
(skin/model matrices); gradients 1e-4 * max(1, max |oracle gradient|) per
character (5e-4 for depth >= 1024)."""
import numpy as np
import pytest

import oracle
import synth
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def run_frame(w, levelsync=False):
    ctx, plan = _gpu.setup(w)
    tm, wt = _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])
    out = ctx.evaluate_frame(plan, tm, wt, levelsync=levelsync)
    skin = out.cpu().numpy()
    assert ctx.status() == 0
    return skin


def test_config1_forward_local(torch):
    w = synth.config1()
    ref, model_ref = oracle.forward_qt(w["types"], w["char_type"], w["q"], w["t"])
    ctx, plan = _gpu.setup(w, with_clips=False)
    q, t = _gpu.cuda(w["q"]), _gpu.cuda(w["t"])
    skin, model = ctx.forward_local(plan, q, t, skin=True, model=True)
    _gpu.assert_skin_close(skin.cpu().numpy(), ref, w)
    _gpu.assert_skin_close(model.cpu().numpy(), model_ref, w)
    s_only, _ = ctx.forward_local(plan, q, t, skin=True, model=False)
    _, m_only = ctx.forward_local(plan, q, t, skin=False, model=True)
    np.testing.assert_array_equal(s_only.cpu().numpy(), skin.cpu().numpy())
    np.testing.assert_array_equal(m_only.cpu().numpy(), model.cpu().numpy())
    lv, _ = ctx.forward_local(plan, q, t, levelsync=True)
    _gpu.assert_skin_close(lv.cpu().numpy(), ref, w)


def test_config2_frame_full(torch):
    w = synth.config2()
    ref = oracle.frame(w)
    errs = _gpu.assert_skin_close(run_frame(w), ref, w)
    print("config2 fused max-abs per type:", errs)


def test_config2_frame_levelsync(torch):
    w = synth.subset(synth.config2(), list(range(0, 4096, 7)) + [4096])
    _gpu.assert_skin_close(run_frame(w, levelsync=True), oracle.frame(w), w)


def test_config3_frame_full(torch):
    w = synth.config3()
    ref = oracle.frame(w)
    errs = _gpu.assert_skin_close(run_frame(w), ref, w)
    print("config3 fused max-abs per type:", errs)


def test_config3_frame_levelsync(torch):
    w = synth.subset(synth.config3(), list(range(0, 10000, 13)))
    _gpu.assert_skin_close(run_frame(w, levelsync=True), oracle.frame(w), w)


def test_frame_repeatable_and_graph_capturable(torch):
    """Two evaluations agree bit for bit (the work queue order changes
    nothing), and a captured CUDA graph replays the same frame."""
    w = synth.subset(synth.config3(), list(range(600)))
    ctx, plan = _gpu.setup(w)
    tm, wt = _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])
    a = ctx.evaluate_frame(plan, tm, wt).clone()
    b = ctx.evaluate_frame(plan, tm, wt).clone()
    assert torch.equal(a, b)
    out = torch.zeros_like(a)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.evaluate_frame(plan, tm, wt, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g):
        ctx.evaluate_frame(plan, tm, wt, out=out)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, a)


def test_frame_from_host_buffers(torch):
    """The host-buffer entry point (inputs copied in, skin matrices copied
    back inside the call) gives the device entry point's frame bit for bit,
    for page-locked and pageable buffers, and the oracle's within tolerance."""
    w = synth.subset(synth.config3(), list(range(0, 10000, 7)))
    ctx, plan = _gpu.setup(w)
    ref = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])).cpu()
    h_t = torch.as_tensor(w["time"]).pin_memory()
    h_w = torch.as_tensor(w["weight"]).pin_memory()
    out = ctx.evaluate_frame_host(plan, h_t, h_w)
    torch.cuda.synchronize()
    assert out.is_pinned() and torch.equal(out, ref)
    pageable = torch.zeros((plan.total, 12), dtype=torch.float32)
    ctx.evaluate_frame_host(plan, torch.as_tensor(w["time"]).clone(), torch.as_tensor(w["weight"]).clone(),
                            out=pageable)
    torch.cuda.synchronize()
    assert torch.equal(pageable, ref)
    _gpu.assert_skin_close(out.numpy(), oracle.frame(w), w)


@pytest.mark.parametrize("walk", [0, 1, 2])
def test_back_to_back_frames(torch, walk):
    """Frames enqueued back to back (each work-queue kernel and frame kernel
    launched with programmatic stream serialization after the previous one),
    with the times of each frame written by a torch kernel just before it,
    equal the same frames run one at a time -- on a stream and in a CUDA
    graph."""
    w = synth.subset(synth.config3(), list(range(0, 10000, 9)))
    ctx, plan = _gpu.setup(w)
    ctx.set_schedule(plan, [16, 3, 2048, walk])
    base, wt = _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])
    shifts = [0.0, 0.37, 0.71]
    refs = []
    for sh in shifts:
        tm = torch.remainder(base + sh, 1.0)
        refs.append(ctx.evaluate_frame(plan, tm, wt).clone())
        torch.cuda.synchronize()
    tms = [torch.empty_like(base) for _ in shifts]
    outs = [torch.zeros((plan.total, 12), device="cuda") for _ in shifts]

    def enqueue():
        for tm, sh, o in zip(tms, shifts, outs):
            torch.remainder(base + sh, 1.0, out=tm)  # the frame's input, written by the preceding kernel
            ctx.evaluate_frame(plan, tm, wt, out=o)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        enqueue()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        enqueue()
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


@pytest.mark.parametrize("walk", [1, 2])
def test_walk_frame_several_ranges(torch, walk):
    """8,192 characters of config 2's 512-joint type plus the dragon chain: the
    walk types' work queue cuts them into eight ranges of 1,024 characters,
    each with its own item region.  Sampled characters (the ends of ranges
    among them) equal the oracle's frame."""
    w = synth.config2(n_chars=8192)
    ctx, plan = _gpu.setup(w)
    ctx.set_schedule(plan, [16, 3, 4096, walk, 0])
    skin = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])).cpu().numpy()
    assert ctx.status() == 0
    sel = list(range(0, 8192, 37)) + [1023, 1024, 4095, 4096, 8191, 8192]
    ws = synth.subset(w, sel)
    off = oracle.offsets(w["char_type"], w["types"])
    _gpu.assert_skin_close(skin[_rows(off, sel)], oracle.frame(ws), ws)


@pytest.mark.parametrize("sched", [[16, 3, 2048, 0, 7], [16, 2, 2048, 0, 0]])
def test_back_to_back_adjoint(torch, sched):
    """Forward + adjoint launches enqueued back to back (the one-item kernel
    stages its items before waiting on the preceding grid), each on poses a
    torch kernel rescales just before it, equal the launches run one at a
    time -- on a stream and in a CUDA graph."""
    w = synth.subset(synth.config4(), list(range(0, 1024, 3)))
    ctx, plan = _gpu.setup(w, with_clips=False)
    ctx.set_schedule(plan, sched)
    q0, t, tg = _gpu.cuda(w["q"]), _gpu.cuda(w["t"]), _gpu.cuda(w["target"])
    scales = [1.0, 1.1, 0.9]
    refs = []
    for sc in scales:
        gq, gt, loss = ctx.loss_backward(plan, q0 * sc, t, tg)
        torch.cuda.synchronize()
        refs.append((gq.clone(), gt.clone(), loss.clone()))
    qs = [torch.empty_like(q0) for _ in scales]
    outs = [(torch.zeros_like(r[0]), torch.zeros_like(r[1]), torch.zeros_like(r[2])) for r in refs]

    def enqueue():
        for q, sc, (gq, gt, loss) in zip(qs, scales, outs):
            torch.mul(q0, sc, out=q)  # the launch's input, written by the preceding kernel
            ctx.loss_backward(plan, q, t, tg, grad_q=gq, grad_t=gt, loss=loss)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        enqueue()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for a, b in zip(o, r):
            assert torch.equal(a, b)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        enqueue()
    for o in outs:
        for a in o:
            a.zero_()
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for a, b in zip(o, r):
            assert torch.equal(a, b)


def test_autotuned_frame_parity(torch):
    """anim_tune picks a schedule by timing candidates; the tuned frame still
    matches the oracle and a second tune of the same mix hits the cache."""
    import time
    w = synth.subset(synth.config3(), list(range(0, 10000, 5)))
    ctx, plan = _gpu.setup(w)
    t0 = time.perf_counter()
    ctx.tune(plan, 0)
    t1 = time.perf_counter()
    ctx.tune(plan, 0)
    t2 = time.perf_counter()
    assert t2 - t1 < 0.5 * (t1 - t0)
    out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
    _gpu.assert_skin_close(out.cpu().numpy(), oracle.frame(w), w)
    ctx.tune(plan, 2)  # the adjoint's schedule search runs too


@pytest.mark.parametrize("sched", [[2, 1, 1024, 0, 0], [8, 2, 2048, 0, 6], [32, 3, 4096, 0, 4], [16, 2, 2048, 1, 8],
                                   [16, 3, 1024, 1, 0], [16, 2, 256, 1, 6], [16, 3, 2048, 2, 0]])
def test_every_schedule_variant_parity(torch, sched):
    """Each schedule the autotuner may pick (segment length, CTAs per SM --
    3 selects the other compiled kernel variant --, item size, chain-walk
    frame kernel, persistent or one-item adjoint kernel)
    gives oracle results for the frame, the forward and the adjoint, run one
    after another on the same plan (they share its work-queue counters)."""
    import paper_2505_06703_gb300 as pk
    w = synth.subset(synth.config3(), list(range(0, 10000, 25)) + [i for i in range(10000) if i % 997 == 3])
    ctx, plan = _gpu.setup(w)
    ctx.set_schedule(plan, sched)
    assert ctx.get_schedule(plan) == sched
    out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
    _gpu.assert_skin_close(out.cpu().numpy(), oracle.frame(w), w)
    rng = np.random.default_rng(sched[0] * 10 + sched[1])
    types, ct = w["types"], w["char_type"]
    off = oracle.offsets(ct, types)
    q, t = synth.local_poses(rng, int(off[-1]), t_half=0.0005)
    ref, mref = oracle.forward_qt(types, ct, q, t)
    s_, m_ = ctx.forward_local(plan, _gpu.cuda(q), _gpu.cuda(t), skin=True, model=True)
    _gpu.assert_skin_close(s_.cpu().numpy(), ref, w)
    _gpu.assert_skin_close(m_.cpu().numpy(), mref, w)
    g = rng.normal(size=(int(off[-1]), 3))
    dq_ref, dt_ref = oracle.grad(types, ct, q, t, g)
    args = (plan, _gpu.cuda(q), _gpu.cuda(t), _gpu.cuda(g.astype(np.float32)))
    if sched[0] == 2:
        # 1,024 segments of the 2,048-joint chain: the forward fits one CTA's
        # shared memory, the adjoint's two extra vectors per joint do not
        with pytest.raises(pk.AnimError, match="EUNSUPPORTED"):
            ctx.backward(*args)
        # a schedule the forward cannot take either is refused and the
        # previous one stays in force
        with pytest.raises(pk.AnimError, match="EUNSUPPORTED"):
            ctx.set_schedule(plan, [1, 2, 2048, 0])
        assert ctx.get_schedule(plan) == sched
        ctx.set_schedule(plan, [8] + sched[1:])
    gq, gt = ctx.backward(*args)
    tol = _grad_tol(dq_ref, dt_ref, w)
    assert (np.abs(gq.cpu().numpy() - dq_ref).max(axis=1) <= tol).all()
    assert (np.abs(gt.cpu().numpy() - dt_ref).max(axis=1) <= tol).all()


def _grad_tol(dq_ref, dt_ref, w):
    """Per-joint tolerance: 1e-4 * max(1, max |oracle grad| of the character)."""
    off = oracle.offsets(w["char_type"], w["types"])
    tol = np.empty(len(dq_ref))
    for c, ty in enumerate(w["char_type"]):
        sl = slice(off[c], off[c + 1])
        scale = max(1.0, np.abs(dq_ref[sl]).max(), np.abs(dt_ref[sl]).max())
        tol[sl] = _gpu.tol_for_depth(w["types"][ty]["depth"]) * scale
    return tol


def test_config4_loss_backward_full(torch):
    w = synth.config4()
    types, ct = w["types"], w["char_type"]
    _, M = oracle.forward_qt(types, ct, w["q"], w["t"], with_skin=False)
    g = 2 * (M[:, :, 3] - w["target"])
    dq_ref, dt_ref = oracle.grad(types, ct, w["q"], w["t"], g)
    off = oracle.offsets(ct, types)
    loss_ref = np.array([np.sum((M[off[c]:off[c + 1], :, 3] - w["target"][off[c]:off[c + 1]]) ** 2)
                         for c in range(len(ct))])
    ctx, plan = _gpu.setup(w, with_clips=False)
    q, t, tg = _gpu.cuda(w["q"]), _gpu.cuda(w["t"]), _gpu.cuda(w["target"])
    gq, gt, loss = ctx.loss_backward(plan, q, t, tg)
    gq, gt, loss = gq.cpu().numpy(), gt.cpu().numpy(), loss.cpu().numpy()
    tol = _grad_tol(dq_ref, dt_ref, w)
    assert (np.abs(gq - dq_ref).max(axis=1) <= tol).all(), np.abs(gq - dq_ref).max()
    assert (np.abs(gt - dt_ref).max(axis=1) <= tol).all(), np.abs(gt - dt_ref).max()
    np.testing.assert_allclose(loss, loss_ref, rtol=1e-4)
    # anim_backward with the same dLoss/dp given explicitly
    gq2, gt2 = ctx.backward(plan, q, t, _gpu.cuda(g.astype(np.float32)))
    assert (np.abs(gq2.cpu().numpy() - dq_ref).max(axis=1) <= tol).all()
    assert (np.abs(gt2.cpu().numpy() - dt_ref).max(axis=1) <= tol).all()


def test_autograd_function(torch):
    import paper_2505_06703_gb300 as pk
    w = synth.subset(synth.config4(), list(range(32)))
    types, ct = w["types"], w["char_type"]
    ctx, plan = _gpu.setup(w, with_clips=False)
    q = _gpu.cuda(w["q"]).requires_grad_(True)
    t = _gpu.cuda(w["t"]).requires_grad_(True)
    tg = _gpu.cuda(w["target"])
    p = pk.hierarchy_fn().apply(q, t, ctx, plan)
    loss = ((p - tg) ** 2).sum()
    loss.backward()
    _, M = oracle.forward_qt(types, ct, w["q"], w["t"], with_skin=False)
    np.testing.assert_allclose(p.detach().cpu().numpy(), M[:, :, 3], atol=1e-4)
    g = 2 * (M[:, :, 3] - w["target"])
    dq_ref, dt_ref = oracle.grad(types, ct, w["q"], w["t"], g)
    tol = _grad_tol(dq_ref, dt_ref, w)
    assert (np.abs(q.grad.cpu().numpy() - dq_ref).max(axis=1) <= tol).all()
    assert (np.abs(t.grad.cpu().numpy() - dt_ref).max(axis=1) <= tol).all()


def _ik_setup(torch, w):
    ctx, plan = _gpu.setup(w, with_clips=False)
    t = _gpu.cuda(w["t"])
    # the GPU derives its own targets: effector positions of the target pose
    _, mt = ctx.forward_local(plan, _gpu.cuda(w["q_target"]), t, skin=False, model=True)
    mt = mt.view(-1, 3, 4)[:, :, 3]
    off = torch.as_tensor(plan.row_off[:-1], device="cuda")
    ct = torch.as_tensor(w["char_type"], device="cuda").long()
    eff_t = torch.as_tensor(w["effectors"], device="cuda").long()[ct]
    targets = mt[off[:, None] + eff_t].contiguous()
    return ctx, plan, t, targets


@pytest.mark.parametrize("tuned", [False, True])
def test_config5_ik_first_step(torch, tuned):
    """The first fused IK step (forward, effector loss, adjoint, Adam) equals
    the oracle's first step wherever the gradient is above FP32 noise (Adam's
    first update is lr * g / (|g| + eps), a sign-like step) -- under the
    default schedule and under the one anim_tune_ik picks."""
    w = synth.subset(synth.config5(), list(range(32)))
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    targets_ref = oracle.ik_targets(w)
    q1_ref, hist = oracle.ik(types, ct, w["t"], w["q0"], eff, targets_ref, 1)
    ctx, plan, t, targets = _ik_setup(torch, w)
    if tuned:
        ctx.tune_ik(plan, eff)
        sched = ctx.get_schedule(plan)
        ctx.tune_ik(plan, eff)  # cached: applies the same schedule without timing
        assert ctx.get_schedule(plan) == sched
    assert np.abs(targets.cpu().numpy() - targets_ref).max() < 1e-5
    q = _gpu.cuda(w["q0"])
    m, v = torch.zeros_like(q), torch.zeros_like(q)
    loss = torch.zeros(len(ct), device="cuda")
    ik = ctx.ik(plan, eff)
    ik.reset()
    ik.step(q, m, v, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
    assert abs(loss.sum().item() - hist[0]) <= 1e-4 * max(1.0, hist[0])
    # the oracle's gradient at the start decides which components are above noise
    off = oracle.offsets(ct, types)
    _, M = oracle.forward_qt(types, ct, w["q0"], w["t"], with_skin=False)
    g = np.zeros((int(off[-1]), 3))
    for c, ty in enumerate(ct):
        for e, j in enumerate(eff[ty]):
            g[off[c] + j] = 2 * (M[off[c] + j, :, 3] - targets_ref[c, e])
    dq, _ = oracle.grad(types, ct, w["q0"], w["t"], g)
    clear = np.abs(dq) > 1e-4 * np.abs(dq).max()
    d = np.abs(q.cpu().numpy() - q1_ref)
    assert d[clear].max() < 1e-5, d[clear].max()


def test_config5_ik_subset(torch):
    """200 Adam steps of IK on 64 characters (32 of each type): final
    effector positions of the GPU run against the FP64 oracle run of the
    same schedule, and the loss must fall."""
    w = synth.subset(synth.config5(), list(range(64)))
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    steps = w["n_steps"]
    targets_ref = oracle.ik_targets(w)
    q_ref, hist = oracle.ik(types, ct, w["t"], w["q0"], eff, targets_ref, steps)
    ctx, plan, t, targets = _ik_setup(torch, w)
    q = _gpu.cuda(w["q0"])
    m, v = torch.zeros_like(q), torch.zeros_like(q)
    loss = torch.zeros(len(ct), device="cuda")
    ik = ctx.ik(plan, eff)
    ik.reset()
    first = None
    for s in range(steps):
        ik.step(q, m, v, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
        if s == 0:
            first = loss.sum().item()
    last = loss.sum().item()
    assert abs(first - hist[0]) <= 1e-4 * max(1, hist[0])
    assert last < 0.5 * first
    _, Mg = oracle.forward_qt(types, ct, q.cpu().numpy().astype(np.float64), w["t"], with_skin=False)
    _, Mr = oracle.forward_qt(types, ct, q_ref, w["t"], with_skin=False)
    offn = oracle.offsets(ct, types)
    pe_g = np.stack([Mg[offn[c] + eff[ty], :, 3] for c, ty in enumerate(ct)])
    pe_r = np.stack([Mr[offn[c] + eff[ty], :, 3] for c, ty in enumerate(ct)])
    err_g = np.linalg.norm(pe_g - targets_ref, axis=-1)
    err_r = np.linalg.norm(pe_r - targets_ref, axis=-1)
    print("IK final effector error: gpu mean %.3e oracle mean %.3e, max |p_gpu - p_oracle| %.3e" % (
        err_g.mean(), err_r.mean(), np.abs(pe_g - pe_r).max()))
    # Adam normalizes each step by the running RMS of the gradient, so FP32
    # rounding in near-zero gradient components can flip the sign of an
    # lr-sized update; the trajectories then separate by a fraction of lr
    # while converging to the same optimum.  The bar is on the outcome: every
    # effector ends within 1% of the (unit) skeleton extent of the FP64 run,
    # and the mean remaining error (a few 1e-4) agrees within 25%.
    assert np.abs(pe_g - pe_r).max() < 1e-2
    assert abs(err_g.mean() - err_r.mean()) <= 0.25 * err_r.mean()


def test_config5_ik_full_vs_oracle(torch):
    """The whole config-5 run: 200 Adam steps on all 8,192 characters in the
    bench's configuration (schedule from anim_tune_ik, Adam's moments in the
    IK object's own state), against the FP64 oracle running the same
    schedule from the same start (every host core, characters split into
    shares).  Each side derives its targets with its own forward.  Adam
    divides each coordinate's step by its running RMS, so FP32 rounding of
    near-zero gradient components changes individual trajectories; at this
    size some effectors of characters that have not converged after 200 steps
    end more than 1% of the unit extent apart (96 of 65,536 measured), so the
    bar compares the outcome: mean and largest remaining effector error within
    25% of the FP64 run's, and at least 99.5% of the effectors within 1% of
    the unit extent of their FP64 positions."""
    w = synth.config5()
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    steps = w["n_steps"]
    targets_ref = oracle.ik_targets(w)
    q_ref, hist, procs = oracle.ik_all_cores(types, ct, w["t"], w["q0"], eff, targets_ref, steps, lr=w["lr"],
                                             betas=w["betas"], eps=w["eps"])
    ctx, plan, t, targets = _ik_setup(torch, w)
    ctx.tune_ik(plan, eff)
    q = _gpu.cuda(w["q0"])
    loss = torch.zeros(len(ct), device="cuda")
    ik = ctx.ik(plan, eff)
    ik.reset()
    for s in range(steps):
        ik.step(q, None, None, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
        if s == 0:
            first = loss.sum().item()
    last = loss.sum().item()
    assert abs(first - hist[0]) <= 1e-4 * max(1, hist[0])
    assert last < 0.1 * first
    offn = oracle.offsets(ct, types)
    _, Mg = oracle.forward_qt(types, ct, q.cpu().numpy().astype(np.float64), w["t"], with_skin=False)
    _, Mr = oracle.forward_qt(types, ct, q_ref, w["t"], with_skin=False)
    rows = (offn[:-1, None] + eff[ct]).ravel()
    pe_g = Mg[rows, :, 3].reshape(len(ct), -1, 3)
    pe_r = Mr[rows, :, 3].reshape(len(ct), -1, 3)
    err_g = np.linalg.norm(pe_g - targets_ref, axis=-1)
    err_r = np.linalg.norm(pe_r - targets_ref, axis=-1)
    d = np.linalg.norm(pe_g - pe_r, axis=-1)
    conv = (err_g <= 1e-3) & (err_r <= 1e-3)
    print("IK full size (%d oracle processes): final effector error gpu mean %.3e max %.3e, oracle mean %.3e "
          "max %.3e; |p_gpu - p_oracle| max %.3e, 99.9th pct %.3e, > 1e-2: %d, > 5e-3: %d of %d; converged "
          "(both <= 1e-3): %d, their max %.3e; max over the others %.3e" % (
              procs, err_g.mean(), err_g.max(), err_r.mean(), err_r.max(), d.max(), np.percentile(d, 99.9),
              int((d > 1e-2).sum()), int((d > 5e-3).sum()), d.size, int(conv.sum()), d[conv].max(),
              d[~conv].max() if (~conv).any() else 0.0))
    assert abs(err_g.mean() - err_r.mean()) <= 0.25 * err_r.mean()
    assert abs(err_g.max() - err_r.max()) <= 0.25 * err_r.max()
    assert (d <= 1e-2).mean() >= 0.995


def _rows(off, chars):
    return np.concatenate([np.arange(off[c], off[c + 1]) for c in chars])


def test_forward_local_full_back_to_back(torch):
    """The forward from local poses on config 2's 2,098,176 joints under the
    schedule the bench times ([32, 3, 2048, 0]: 1,025 work items on 456
    persistent CTAs, so the producer warps prefetch their first items' rows
    ahead of the grid-dependency wait and each next item's rows during the
    current one).  Three launches back to back on one stream: two input sets,
    then the first set rewritten in place by a torch kernel and run again;
    sampled characters against the oracle."""
    w = synth.config2()
    types, ct = w["types"], w["char_type"]
    off = oracle.offsets(ct, types)
    n = int(off[-1])
    ctx, plan = _gpu.setup(w)
    ctx.set_schedule(plan, [32, 3, 2048, 0])
    rng = np.random.default_rng(77)
    q1, t1 = synth.local_poses(rng, n, unnormalized=True)
    q2, t2 = synth.local_poses(rng, n)
    dq1, dt1, dq2, dt2 = _gpu.cuda(q1), _gpu.cuda(t1), _gpu.cuda(q2), _gpu.cuda(t2)
    s1, _ = ctx.forward_local(plan, dq1, dt1, skin=True, model=False)
    s2, _ = ctx.forward_local(plan, dq2, dt2, skin=True, model=False)
    dq1.copy_(dq1[:, [3, 0, 1, 2]])
    dt1.mul_(2.0)
    s3, m3 = ctx.forward_local(plan, dq1, dt1, skin=True, model=True)
    sel = list(range(0, len(ct), 61)) + [len(ct) - 1]
    rows = _rows(off, sel)
    ws = synth.subset(w, sel)
    for got, q, t in ((s1, q1, t1), (s2, q2, t2), (s3, q1[:, [3, 0, 1, 2]], 2.0 * t1)):
        ref, mref = oracle.forward_qt(types, ct[sel], q[rows], t[rows])
        _gpu.assert_skin_close(got.cpu().numpy().reshape(n, 12)[rows], ref, ws)
    _gpu.assert_skin_close(m3.cpu().numpy().reshape(n, 12)[rows], mref, ws)


@pytest.mark.parametrize("sched", [[8, 2, 4096, 1, 0], [4, 3, 1024, 1, 0]])
def test_config5_ik_full_second_step(torch, sched):
    """Two IK steps on all 8,192 characters of config 5 under schedules the IK
    autotuner picks (persistent kernel, its 2- and 3-CTA/SM builds, several
    items per CTA, rows prefetched ahead of the grid-dependency wait).  The second launch
    reads the q, m and v the first one wrote; on sampled characters its
    result must equal one oracle Adam step (gradient of the effector loss by
    the oracle's reverse pass) taken from the GPU's own state after step 1."""
    w = synth.config5()
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    ctx, plan, t, targets = _ik_setup(torch, w)
    ctx.set_schedule(plan, sched)
    q = _gpu.cuda(w["q0"])
    m, v = torch.zeros_like(q), torch.zeros_like(q)
    loss = torch.zeros(len(ct), device="cuda")
    ik = ctx.ik(plan, eff)
    ik.reset()
    ik.step(q, m, v, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
    q1, m1, v1 = (x.cpu().numpy().astype(np.float64) for x in (q, m, v))
    ik.step(q, m, v, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
    q2, m2, v2 = (x.cpu().numpy() for x in (q, m, v))
    off = oracle.offsets(ct, types)
    sel = list(range(0, len(ct), 257)) + [len(ct) - 2, len(ct) - 1]
    rows = _rows(off, sel)
    offs = oracle.offsets(ct[sel], types)
    tg = targets.cpu().numpy().astype(np.float64)
    _, M = oracle.forward_qt(types, ct[sel], q1[rows], w["t"][rows], with_skin=False)
    g = np.zeros((len(rows), 3))
    for k, c in enumerate(sel):
        for e, j in enumerate(eff[ct[c]]):
            g[offs[k] + j] = 2 * (M[offs[k] + j, :, 3] - tg[c, e])
    dq, _ = oracle.grad(types, ct[sel], q1[rows], w["t"][rows], g)
    p_ref, m_ref, v_ref = q1[rows].copy(), m1[rows].copy(), v1[rows].copy()
    oracle.adam(p_ref, np.ascontiguousarray(dq), m_ref, v_ref, 2, w["lr"], *w["betas"], w["eps"])
    scale = max(1.0, np.abs(dq).max())
    # m and v are linear in the gradient, within the gradient tolerance
    # (1e-4 * max(1, max |gradient|)); a stale q, m or v read by the second
    # launch would be off by orders more
    assert np.abs(m2[rows] - m_ref).max() <= 1e-4 * scale
    assert np.abs(v2[rows] - v_ref).max() <= 1e-4 * scale * scale
    # q moves by lr * m_hat / (sqrt(v_hat) + eps), whose error grows as the
    # gradient shrinks: compare where it is well above FP32 noise in both
    # steps (1 % of the largest), to 1 % of a step of size lr
    big = np.abs(dq).max()
    clear = (np.abs(dq) > 1e-2 * big) & (np.abs(m1[rows]) > 1e-3 * big)
    assert clear.sum() > 100
    assert np.abs(q2[rows] - p_ref)[clear].max() < 1e-2 * w["lr"]


@pytest.mark.parametrize("sched", [[4, 3, 1024, 1, 0], [8, 2, 4096, 1, 0], [16, 2, 512, 1, 4]])
def test_ik_own_adam_state_matches_caller_state(torch, sched):
    """Five IK steps on all of config 5 with Adam's moments in the caller's
    [total][4] rows and, after a reset, in the IK object's own compact state
    (the same arithmetic on other rows): bit-identical poses and losses, also
    for a second run after another reset; persistent (2- and 3-CTA/SM builds)
    and one-item kernels."""
    w = synth.config5()
    ct, eff = w["char_type"], w["effectors"]
    ctx, plan, t, targets = _ik_setup(torch, w)
    ctx.set_schedule(plan, sched)
    ik = ctx.ik(plan, eff)
    q0 = _gpu.cuda(w["q0"])

    def run(own):
        q = q0.clone()
        m, v = (None, None) if own else (torch.zeros_like(q), torch.zeros_like(q))
        loss = torch.zeros(len(ct), device="cuda")
        ik.reset()
        for _ in range(5):
            ik.step(q, m, v, t, targets, lr=w["lr"], betas=w["betas"], eps=w["eps"], loss=loss)
        torch.cuda.synchronize()
        return q, loss

    q_c, l_c = run(False)
    q_o, l_o = run(True)
    q_o2, _ = run(True)
    assert torch.equal(q_c, q_o) and torch.equal(l_c, l_o)
    assert torch.equal(q_o, q_o2)
    assert not torch.equal(q_c, q0)
    import paper_2505_06703_gb300 as pk
    with pytest.raises(pk.AnimError, match="EINVAL"):  # one moment array alone
        ik.step(q0.clone(), torch.zeros_like(q0), None, t, targets)


# ------------------------------------------------------------------ edge cases
def _edge_types(rng):
    return [synth.make_type(np.array([-1], np.int32), rng, with_clips=True),               # one joint
            synth.make_type(synth.chain(3), rng, with_clips=True),                         # tiny chain
            synth.make_type(np.array([-1, 0, -1, 2, 2, -1], np.int32), rng, with_clips=True),  # forest
            synth.make_type(synth.relabel_random_topological(synth.random_tree(33, 9, rng, spine=9), rng)[0],
                            rng, with_clips=True),                                         # non depth-first
            synth.make_type(synth.random_tree(1000, 40, rng, spine=40), rng, with_clips=True),
            synth.make_type(np.array([-1] + [0] * 599, np.int32), rng, with_clips=True),     # star: 32 walk lanes
            synth.make_type(synth.chain(2048), rng, with_clips=True)]                      # maximum size


def test_edge_types_frame_and_local(torch):
    rng = np.random.default_rng(77)
    types = _edge_types(rng)
    ct = np.array(list(range(len(types))) * 3 + [0] * 70 + [1] * 5, np.int32)
    rng.shuffle(ct)
    w = {"types": types, "char_type": ct, "time": rng.uniform(-3, 5, len(ct)).astype(np.float32),
         "weight": rng.uniform(0, 1, len(ct)).astype(np.float32)}
    ref_frame = oracle.frame(w)
    _gpu.assert_skin_close(run_frame(w), ref_frame, w)
    _gpu.assert_skin_close(run_frame(w, levelsync=True), ref_frame, w)
    for walk in (1, 2):  # both chain-walk kernels (4-, 2- and 1-step chunks among these types)
        ctx, plan = _gpu.setup(w)
        ctx.set_schedule(plan, [16, 3, 2048, walk, 0])
        out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
        assert ctx.status() == 0
        _gpu.assert_skin_close(out.cpu().numpy(), ref_frame, w)
    off = oracle.offsets(ct, types)
    q, t = synth.local_poses(rng, int(off[-1]), t_half=0.0005)
    ref, mref = oracle.forward_qt(types, ct, q, t)
    ctx, plan = _gpu.setup(w)
    s, m = ctx.forward_local(plan, _gpu.cuda(q), _gpu.cuda(t), skin=True, model=True)
    _gpu.assert_skin_close(s.cpu().numpy(), ref, w)
    _gpu.assert_skin_close(m.cpu().numpy(), mref, w)
    g = rng.normal(size=(int(off[-1]), 3))
    dq_ref, dt_ref = oracle.grad(types, ct, q, t, g)
    gq, gt = ctx.backward(plan, _gpu.cuda(q), _gpu.cuda(t), _gpu.cuda(g.astype(np.float32)))
    tol = _grad_tol(dq_ref, dt_ref, {"types": types, "char_type": ct})
    assert (np.abs(gq.cpu().numpy() - dq_ref).max(axis=1) <= tol).all()
    assert (np.abs(gt.cpu().numpy() - dt_ref).max(axis=1) <= tol).all()


@pytest.mark.parametrize("walk", [0, 2])
def test_frame_key_counts(torch, walk):
    """Clips of 3 and of 40 keys: the work-queue kernel sorts characters by
    key index with one warp's scan for at most 32 keys and with block-wide
    scans beyond; both frames match the oracle, with times over several
    clip loops and ranges of several hundred characters per type."""
    rng = np.random.default_rng(91)
    types = []
    for parents, nk in ((synth.random_tree(48, 9, rng, spine=9), 3), (synth.random_tree(96, 20, rng, spine=20), 40),
                        (synth.chain(64), 40)):
        t = synth.make_type(parents, rng, with_clips=True)
        keys = t["keys"]
        reps = -(-nk // keys.shape[1])
        t["keys"] = np.ascontiguousarray(np.concatenate([keys] * reps, axis=1)[:, :nk])
        types.append(t)
    ct = np.array([0] * 300 + [1] * 300 + [2] * 40, np.int32)
    rng.shuffle(ct)
    w = {"types": types, "char_type": ct, "time": rng.uniform(0.0, 3.0, len(ct)).astype(np.float32),
         "weight": rng.uniform(0, 1, len(ct)).astype(np.float32)}
    ref = oracle.frame(w)
    ctx, plan = _gpu.setup(w)
    ctx.set_schedule(plan, [16, 3, 2048, walk, 0])
    out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
    assert ctx.status() == 0
    _gpu.assert_skin_close(out.cpu().numpy(), ref, w)


@pytest.mark.parametrize("algorithm", [1, 2, 3, 4, 5])
def test_paper_algorithms_parity(torch, algorithm):
    """The paper's Algorithms 1-4 and the leaf walk it describes (5) as GPU
    kernels give the oracle's skin
    matrices: the 64-joint trees of the plain forward workload, the biped
    (depth 70), the 256-joint depth-96 tree, a 1,000-joint tree numbered in
    random topological order (blocks of 64 indices span many subtrees) and a
    1,024-joint chain (depth 1,024)."""
    import paper_2505_06703_gb300 as pk
    rng = np.random.default_rng(50 + algorithm)
    w1, w2, w4 = synth.config1(), synth.config2(), synth.config4()
    types = [w1["types"][0], w2["types"][0], w2["types"][1], w4["types"][0],
             synth.make_type(synth.relabel_random_topological(synth.random_tree(1000, 40, rng, spine=40), rng)[0],
                             rng, with_clips=False)]
    ct = np.array([0] * 40 + [1] * 12 + [2] * 2 + [3] * 20 + [4] * 3, np.int32)
    rng.shuffle(ct)
    w = {"types": types, "char_type": ct}
    off = oracle.offsets(ct, types)
    q, t = synth.local_poses(rng, int(off[-1]), t_half=0.0005)
    ref, _ = oracle.forward_qt(types, ct, q, t)
    ctx, plan = _gpu.setup(w, with_clips=False)
    s = ctx.forward_local_paper(plan, algorithm, _gpu.cuda(q), _gpu.cuda(t))
    _gpu.assert_skin_close(s.cpu().numpy(), ref, w)
    # one thread per joint: types above 1,024 joints are refused
    big = {"types": [synth.make_type(synth.chain(2048), rng, with_clips=False)], "char_type": np.zeros(2, np.int32)}
    ctx2, plan2 = _gpu.setup(big, with_clips=False)
    with pytest.raises(pk.AnimError, match="EUNSUPPORTED"):
        ctx2.forward_local_paper(plan2, algorithm, _gpu.cuda(np.tile([0, 0, 0, 1.0], (4096, 1))),
                                 _gpu.cuda(np.zeros((4096, 3))))


@pytest.mark.parametrize("walk", [0, 1])
def test_skinned_frame(torch, walk):
    """Frame + fused linear blend skinning against the oracle's skinning of
    the oracle's skin matrices: bipeds and the 1,024-joint chain with
    1,500-vertex meshes, the five mixed types with 300-vertex meshes and one
    type left without a mesh; with and without the skin matrices written."""
    w2 = synth.with_meshes(synth.subset(synth.config2(), list(range(0, 4096, 64)) + [4096]), n_verts=1500, seed=21)
    w3 = synth.subset(synth.config3(), list(range(0, 10000, 50)))
    w3 = synth.with_meshes(w3, n_verts=300, seed=22)
    w3["types"][2] = {k: v for k, v in w3["types"][2].items() if k != "mesh"}
    for w in (w2, w3):
        types = w["types"]
        S_ref = oracle.frame(w)
        V_ref = oracle.skin_vertices(w, S_ref)
        ctx, plan = _gpu.setup(w)
        sched = ctx.get_schedule(plan)
        ctx.set_schedule(plan, sched[:3] + [walk, sched[4]])
        voff = ctx.vertex_offsets(plan)
        assert list(voff) == list(oracle.vertex_offsets(w["char_type"], types))
        tm, wt = _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])
        skin = torch.empty((plan.total, 12), device="cuda")
        v1 = ctx.evaluate_frame_skinned(plan, tm, wt, skin=skin).cpu().numpy()[:int(voff[-1])]
        v2 = ctx.evaluate_frame_skinned(plan, tm, wt).cpu().numpy()[:int(voff[-1])]
        _gpu.assert_skin_close(skin.cpu().numpy(), S_ref, w)
        for v in (v1, v2):
            for c, ty in enumerate(w["char_type"]):
                sl = slice(voff[c], voff[c + 1])
                tol = 2 * _gpu.tol_for_depth(types[ty]["depth"])
                assert np.abs(v[sl] - V_ref[sl]).max(initial=0.0) <= tol, (c, ty)
        # the plain frame still works on the same plan afterwards
        _gpu.assert_skin_close(run_frame_on(ctx, plan, w), S_ref, w)


def test_tuned_skinned_and_layered_frames(torch):
    """anim_tune's searches for the frame with skinning (which = 3) and the
    frame with layered blending (which = 4) time those frames themselves;
    under the schedules they pick, both still match the oracle."""
    w = synth.with_meshes(synth.subset(synth.config2(), list(range(0, 4096, 64)) + [4096]), n_verts=600, seed=23)
    S_ref = oracle.frame(w)
    V_ref = oracle.skin_vertices(w, S_ref)
    ctx, plan = _gpu.setup(w)
    ctx.tune(plan, 3)
    voff = ctx.vertex_offsets(plan)
    v = ctx.evaluate_frame_skinned(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])).cpu().numpy()
    for c, ty in enumerate(w["char_type"]):
        sl = slice(voff[c], voff[c + 1])
        assert np.abs(v[sl] - V_ref[sl]).max(initial=0.0) <= 2 * _gpu.tol_for_depth(w["types"][ty]["depth"])
    w = synth.with_layers(synth.subset(synth.config3(), list(range(0, 10000, 50))), n_clips=4, seed=43)
    ctx, plan = _gpu.setup(w)
    ctx.tune(plan, 4)
    got = ctx.evaluate_frame_layers(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weights"]), _gpu.cuda(w["add_w"]))
    _gpu.assert_skin_close(got.cpu().numpy(), oracle.frame_layers(w), w)


def run_frame_on(ctx, plan, w):
    return ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"])).cpu().numpy()


@pytest.mark.parametrize("walk", [0, 1])
def test_layered_frame(torch, walk):
    """Frame with up to 4 clips blended by incremental slerp and an additive
    layer, against the oracle: the config-2 and config-3 types with 4 and 3
    clips, one type without the additive layer; the two-clip case equals the
    plain frame."""
    w2 = synth.with_layers(synth.subset(synth.config2(), list(range(0, 4096, 64)) + [4096]), n_clips=4, seed=41)
    w3 = synth.with_layers(synth.subset(synth.config3(), list(range(0, 10000, 50))), n_clips=3, seed=42)
    w3["types"][1] = {k: v for k, v in w3["types"][1].items() if k != "add_keys"}
    for w in (w2, w3):
        ref = oracle.frame_layers(w)
        ctx, plan = _gpu.setup(w)
        sched = ctx.get_schedule(plan)
        ctx.set_schedule(plan, sched[:3] + [walk, sched[4]])
        got = ctx.evaluate_frame_layers(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weights"]), _gpu.cuda(w["add_w"]))
        _gpu.assert_skin_close(got.cpu().numpy(), ref, w)
        # the plain two-clip frame on the same plan afterwards
        _gpu.assert_skin_close(run_frame_on(ctx, plan, w), oracle.frame(w), w)
    # weights (1 - w, w, 0, 0) without additive weight: the two-clip frame
    w = synth.subset(synth.config2(), list(range(0, 4096, 128)) + [4096])
    m = len(w["char_type"])
    wl = np.stack([1 - w["weight"], w["weight"], np.zeros(m), np.zeros(m)], 1).astype(np.float32)
    ctx, plan = _gpu.setup(w)
    got = ctx.evaluate_frame_layers(plan, _gpu.cuda(w["time"]), _gpu.cuda(wl))
    _gpu.assert_skin_close(got.cpu().numpy(), oracle.frame(w), w)


def _raster_tri(V, voff, faces, ct, ident, cols, spacing, ox, oy, scale):
    """Screen-space vertices (pixels, FP64) and depths of triangle `ident`."""
    c, f = int(ident) >> 12, int(ident) & 4095
    tri = faces[int(ct[c])][f]
    wx, wy = (c % cols) * spacing, -(c // cols) * spacing
    v = V[voff[c] + tri]
    xy = np.stack([ox + scale * (v[:, 0] + wx), oy - scale * (v[:, 1] + wy)], 1)
    return xy, (2.0 - v[:, 2]) / 4.0


def _edge_distance(xy, p):
    """Distance in pixels from point p to the closest edge of triangle xy."""
    best = np.inf
    for k in range(3):
        a, b = xy[k], xy[(k + 1) % 3]
        d = b - a
        t = np.clip(np.dot(p - a, d) / max(np.dot(d, d), 1e-30), 0.0, 1.0)
        best = min(best, np.linalg.norm(a + t * d - p))
    return best


def _depth_at(xy, dz, p):
    m = np.array([[xy[0, 0], xy[1, 0], xy[2, 0]], [xy[0, 1], xy[1, 1], xy[2, 1]], [1.0, 1.0, 1.0]])
    lam = np.linalg.solve(m, [p[0], p[1], 1.0])
    return float(lam @ dz)


def test_crowd_raster(torch):
    """The headless raster of the skinned crowd (65 characters, 1,500-vertex
    meshes) against the oracle's rasterizer run on the oracle's skinned
    vertices: the id images agree except where both answers are valid -- a
    pixel centre within 1/32 pixel of an edge of one of the two triangles
    (FP32 and FP64 vertices snap apart there), or two triangles whose depths
    at the centre agree to 1e-4."""
    EMPTY = 0xFFFFFFFF
    w = synth.with_meshes(synth.subset(synth.config2(), list(range(0, 4096, 64)) + [4096]), n_verts=1500, seed=51)
    types, ct = w["types"], w["char_type"]
    V_ref = oracle.skin_vertices(w, oracle.frame(w))
    voff = oracle.vertex_offsets(ct, types)
    ctx, plan = _gpu.setup(w)
    verts = ctx.evaluate_frame_skinned(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
    W, H, cols, spacing, ox, oy, scale = 640, 520, 9, 2.5, 60.0, 60.0, 24.0
    ids_gpu, rgba = ctx.raster(plan, verts, W, H, cols, spacing, ox, oy, scale, rgba=True)
    g = ids_gpu.cpu().numpy().view(np.uint32)
    faces = [t["mesh"]["faces"] for t in types]
    ref = oracle.raster([faces[int(t)] for t in ct], V_ref, voff, cols, spacing, ox, oy, scale, W, H)
    covered = (g != EMPTY) | (ref != EMPTY)
    assert covered.sum() > 0.1 * W * H
    bad = np.argwhere((g != ref) & covered)
    assert len(bad) <= 0.002 * covered.sum(), (len(bad), int(covered.sum()))
    for py, px in bad:
        p = np.array([px + 0.5, py + 0.5])
        tris = [_raster_tri(V_ref, voff, faces, ct, i, cols, spacing, ox, oy, scale)
                for i in (g[py, px], ref[py, px]) if i != EMPTY]
        near_edge = any(_edge_distance(xy, p) < 1 / 32 for xy, _ in tris)
        same_depth = len(tris) == 2 and abs(_depth_at(*tris[0], p) - _depth_at(*tris[1], p)) < 1e-4
        assert near_edge or same_depth, (py, px, g[py, px], ref[py, px])
    # every covered pixel is shaded, the background is not
    img = rgba.cpu().numpy().view(np.uint32)
    assert ((img != 0xFF201810) == (g != EMPTY)).all()


def test_empty_plan_and_errors(torch):
    import paper_2505_06703_gb300 as pk
    rng = np.random.default_rng(5)
    w = {"types": [synth.make_type(synth.chain(4), rng, with_clips=True)], "char_type": np.zeros(0, np.int32),
         "time": np.zeros(0, np.float32), "weight": np.zeros(0, np.float32)}
    ctx, plan = _gpu.setup(w)
    assert plan.total == 0
    dummy = torch.zeros(4, device="cuda")
    ctx.evaluate_frame(plan, dummy, dummy, out=torch.zeros((0, 12), device="cuda"))
    with pytest.raises(pk.AnimError) as e:
        ctx.create_skeletons([np.array([-1, 1], np.int32)], inv_bind=[np.zeros((2, 12), np.float32)])
    assert e.value.code == -1
    with pytest.raises(pk.AnimError):
        ctx.create_skeletons([np.array([-1, 0], np.int32)])  # neither inverse binds nor rest pose
    with pytest.raises(pk.AnimError):
        ctx.plan(np.array([0, 7], np.int32))  # unknown type id
    # a type without clips cannot be evaluated as a frame
    ids = ctx.create_skeletons([np.array([-1, 0], np.int32)], inv_bind=[np.tile(np.eye(3, 4), (2, 1, 1))])
    p2 = ctx.plan(np.array(ids, np.int32))
    with pytest.raises(pk.AnimError) as e:
        ctx.evaluate_frame(p2, torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda"))
    assert e.value.code == -6
    # misaligned output pointer
    buf = torch.zeros(2 * 12 + 1, device="cuda")
    with pytest.raises(pk.AnimError):
        ctx._ck(ctx.lib.anim_forward_local(ctx.h, p2.h, torch.zeros((2, 4), device="cuda").data_ptr(),
                                           torch.zeros((2, 3), device="cuda").data_ptr(), buf.data_ptr() + 4,
                                           None, None))


def test_nonfinite_time_sets_status(torch):
    rng = np.random.default_rng(6)
    w = {"types": [synth.make_type(synth.chain(5), rng, with_clips=True)], "char_type": np.zeros(3, np.int32),
         "time": np.array([0.2, np.nan, np.inf], np.float32), "weight": np.full(3, 0.5, np.float32)}
    ctx, plan = _gpu.setup(w)
    out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
    assert ctx.status() & 1
    assert ctx.status() == 0  # read-and-clear
    w2 = dict(w, time=np.array([0.2, 0.0, 0.0], np.float32))  # non-finite times sample key 0
    ref = oracle.frame(w2)
    _gpu.assert_skin_close(out.cpu().numpy(), ref, w2)


@pytest.mark.parametrize("bind", ["rest", "rigid_matrices", "scaled_matrices"])
def test_walk_kernel_bind_sources(torch, bind):
    """The chain-walk frame kernel folds rigid inverse binds into its key
    records (skin-space walk).  Inverse binds derived from the rest pose,
    given as rigid 3x4 matrices, or given with a scale (not rigid: such a
    type runs on the segmented kernel instead) all give the oracle's skin
    matrices S = M B with the oracle's model poses M, under the walk kernel
    on and off."""
    rng = np.random.default_rng(31)
    w = synth.subset(synth.config2(), list(range(0, 4096, 9)) + [4096])
    types = w["types"]
    Bs = [oracle.inverse_bind(t["parents"], t["rest_q"], t["rest_t"]).astype(np.float32) for t in types]
    if bind == "scaled_matrices":
        for B in Bs:
            B[:, :, :3] *= 1.5
    _, M = oracle.frame(w, want_model=True)
    off = oracle.offsets(w["char_type"], types)
    Bj = np.concatenate([Bs[t] for t in w["char_type"]]).astype(np.float64)
    ref = oracle.bind(M, Bj)
    assert Bj.shape[0] == off[-1]
    import paper_2505_06703_gb300 as pk
    for walk in (2, 1, 0):
        ctx = pk.Context(0)
        if bind == "rest":
            ids = ctx.create_skeletons([t["parents"] for t in types], rest_q=[t["rest_q"] for t in types],
                                       rest_t=[t["rest_t"] for t in types])
        else:
            ids = ctx.create_skeletons([t["parents"] for t in types], inv_bind=Bs)
        for i, t in zip(ids, types):
            ctx.upload_clips(i, t["keys"], t["rate_hz"])
        plan = ctx.plan(np.asarray(ids, np.int32)[w["char_type"]])
        sched = ctx.get_schedule(plan)
        ctx.set_schedule(plan, sched[:3] + [walk, sched[4]])
        out = ctx.evaluate_frame(plan, _gpu.cuda(w["time"]), _gpu.cuda(w["weight"]))
        scale = 1.5 if bind == "scaled_matrices" else 1.0
        errs = _gpu.per_type_maxabs(out.cpu().numpy(), ref, w)
        for ty, e in errs.items():
            assert e <= scale * _gpu.tol_for_depth(types[ty]["depth"]), (walk, ty, e)
        assert ctx.status() == 0
