"""Pins for the oracle's gradient, Adam and IK.

  * central finite differences (h = 1e-6, fp64) on 16 characters of the
    256-joint differentiation workload;
  * the single-joint closed form dL/dtheta = sum_k (z x (p_k - p_root)) . g_k
    for a rotation of the root about z;
  * agreement of the two independent derivations (generic 4x4 reverse pass
    and subtree force/moment sums);
  * Adam against torch.optim.Adam in fp64 (a library routine);
  * IK against torch autograd + torch.optim.Adam in fp64.
"""
import numpy as np
import pytest

import oracle
import synth


def loss_per_char(types, ct, q, t, target):
    _, M = oracle.forward_qt(types, ct, q, t, with_skin=False)
    d = M[:, :, 3] - target
    off = oracle.offsets(ct, types)
    return np.array([np.sum(d[off[c]:off[c + 1]] ** 2) for c in range(len(ct))]), M


def test_grad_vs_central_fd():
    w = synth.config4()
    types = w["types"]
    n = len(types[0]["parents"])
    C = 16
    ct = np.zeros(C, np.int32)
    q = w["q"][: C * n].astype(np.float64)
    t = w["t"][: C * n].astype(np.float64)
    tg = w["target"][: C * n].astype(np.float64)
    _, M = loss_per_char(types, ct, q, t, tg)
    g = 2 * (M[:, :, 3] - tg)
    dq, dt = oracle.grad(types, ct, q, t, g)
    h = 1e-6
    fd_q = np.zeros_like(q)
    fd_t = np.zeros_like(t)
    for arr, fd, width in ((q, fd_q, 4), (t, fd_t, 3)):
        for j in range(n):
            for k in range(width):
                rows = np.arange(C) * n + j
                save = arr[rows, k].copy()
                arr[rows, k] = save + h
                lp, _ = loss_per_char(types, ct, q, t, tg)
                arr[rows, k] = save - h
                lm, _ = loss_per_char(types, ct, q, t, tg)
                arr[rows, k] = save
                fd[rows, k] = (lp - lm) / (2 * h)
    scale = max(1.0, np.abs(dq).max(), np.abs(dt).max())
    assert np.abs(dq - fd_q).max() <= 1e-6 * scale
    assert np.abs(dt - fd_t).max() <= 1e-6 * scale


def test_grad_single_joint_closed_form():
    rng = np.random.default_rng(9)
    parents = synth.random_tree(40, 10, rng, spine=10)
    n = len(parents)
    q = synth.random_unit_quats(rng, n, 40.0)
    th = 0.7
    q[0] = [0, 0, np.sin(th / 2), np.cos(th / 2)]
    t = rng.uniform(-0.2, 0.2, (n, 3))
    g = rng.normal(size=(n, 3))
    types = [{"parents": parents}]
    dq, _ = oracle.grad(types, np.zeros(1, np.int32), q, t, g)
    dtheta = dq[0] @ np.array([0, 0, np.cos(th / 2) / 2, -np.sin(th / 2) / 2])
    _, M = oracle.forward_qt(types, np.zeros(1, np.int32), q, t, with_skin=False)
    p = M[:, :, 3]
    ref = sum(np.cross([0, 0, 1.0], p[k] - p[0]) @ g[k] for k in range(n))
    assert abs(dtheta - ref) < 1e-12 * max(1, abs(ref))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_two_derivations_agree(seed):
    rng = np.random.default_rng(seed)
    types = [{"parents": synth.random_tree(120, 40, rng, spine=40)},
             {"parents": synth.relabel_random_topological(synth.random_tree(60, 12, rng, spine=12), rng)[0]},
             {"parents": synth.chain(50)}]
    ct = np.array([0, 1, 2, 0, 2], np.int32)
    off = oracle.offsets(ct, types)
    N = int(off[-1])
    q = synth.random_unit_quats(rng, N, 120.0) * rng.uniform(0.5, 2.0, (N, 1))
    t = rng.uniform(-0.3, 0.3, (N, 3))
    g = rng.normal(size=(N, 3))
    a = oracle.grad(types, ct, q, t, g)
    b = oracle.grad_force_moment(types, ct, q, t, g)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, atol=1e-11 * max(1, np.abs(y).max()))


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    p = rng.normal(size=64)
    m, v = np.zeros(64), np.zeros(64)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for s in range(1, 40):
        g = rng.normal(size=64) * (0.1 if s % 3 else 10.0)
        oracle.adam(p, g, m, v, s, 1e-2)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-14)


def _torch_rot(q):
    import torch
    u = q / q.norm(dim=-1, keepdim=True)
    x, y, z, w = u.unbind(-1)
    return torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w),
        2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
        2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1).reshape(q.shape[:-1] + (3, 3))


def test_ik_matches_torch_autograd():
    """200 Adam steps of IK on 4 characters of the IK workload: the oracle's
    trajectory (analytic gradient + its Adam) equals torch autograd + torch
    Adam in fp64.  The torch side composes transforms with its own ops and
    differentiates them by autograd."""
    torch = pytest.importorskip("torch")
    w = synth.subset(synth.config5(), [0, 1, 2, 3])
    types, ct, eff = w["types"], w["char_type"], w["effectors"]
    targets = oracle.ik_targets(w)
    steps = 60
    q_or, hist = oracle.ik(types, ct, w["t"], w["q0"], eff, targets, steps)
    off = oracle.offsets(ct, types)
    q = torch.tensor(w["q0"], dtype=torch.float64, requires_grad=True)
    t = torch.tensor(w["t"], dtype=torch.float64)
    opt = torch.optim.Adam([q], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for s in range(steps):
        opt.zero_grad()
        R = _torch_rot(q)
        loss = 0
        for c, ty in enumerate(ct):
            par = types[ty]["parents"]
            o = int(off[c])
            Rw, pw = [None] * len(par), [None] * len(par)
            for i, pp in enumerate(par):
                if pp < 0:
                    Rw[i], pw[i] = R[o + i], t[o + i]
                else:
                    Rw[i] = Rw[pp] @ R[o + i]
                    pw[i] = Rw[pp] @ t[o + i] + pw[pp]
            for e in range(eff.shape[1]):
                d = pw[eff[ty, e]] - torch.tensor(targets[c, e])
                loss = loss + (d * d).sum()
        assert abs(loss.item() - hist[s]) <= 1e-10 * max(1, hist[s])
        loss.backward()
        opt.step()
    np.testing.assert_allclose(q_or, q.detach().numpy(), atol=1e-9)
    assert hist[-1] < 0.5 * hist[0]
