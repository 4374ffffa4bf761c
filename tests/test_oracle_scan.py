"""Pins for the oracle's Hierarchy-Scan (Eq. 1) and Bind MeshPose.

The oracle computes M_i = M_parent(i) L_i by one pass in index order.  These
tests check it against things that are not the oracle:
  * a brute-force product over the explicit root-to-joint path, for every
    parent array of up to 7 joints (and every forest of up to 5);
  * the paper's own parallel schedules (Algorithms 1-4), emulated with their
    barriers as phases, which must give the same product (it is associative);
  * the paper's per-thread operation counts for those schedules;
  * closed forms: same-axis rotation chains, pure translations;
  * special cases: local pose = rest pose gives identity skin matrices;
  * rigidity invariants.
"""
import itertools

import os

import numpy as np
import pytest

import oracle
import synth
from tests import _paper_schedules as ps


def rand_affine(rng, n):
    """General (non-rigid) 3x4 matrices: the scan is defined for any affine."""
    return rng.normal(size=(n, 3, 4))


def rand_rigid(rng, n, t_half=0.3):
    q = synth.random_unit_quats(rng, n, 180.0)
    R = rot_from_quat_scipy(q)
    L = np.zeros((n, 3, 4))
    L[:, :, :3] = R
    L[:, :, 3] = rng.uniform(-t_half, t_half, size=(n, 3))
    return L


def rot_from_quat_scipy(q):
    from scipy.spatial.transform import Rotation
    return Rotation.from_quat(np.asarray(q, float)).as_matrix()


def h(A):
    H = np.zeros(A.shape[:-2] + (4, 4))
    H[..., :3, :] = A
    H[..., 3, 3] = 1
    return H


def brute(parents, L):
    """Root-to-joint product by explicit path collection, per joint."""
    out = np.empty((len(parents), 3, 4))
    for j in range(len(parents)):
        path = []
        a = j
        while a >= 0:
            path.append(a)
            a = parents[a]
        m = np.eye(4)
        for a in reversed(path):
            m = m @ h(L[a])
        out[j] = m[:3]
    return out


def all_parent_arrays(n, forests=False):
    choices = [range(-1 if forests else 0, i) for i in range(1, n)]
    for tail in itertools.product(*choices):
        yield np.array((-1,) + tail, dtype=np.int32)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_bruteforce_every_tree(n):
    rng = np.random.default_rng(100 + n)
    count = 0
    for parents in all_parent_arrays(n):
        L = rand_affine(rng, n)
        np.testing.assert_allclose(oracle.forward(parents, L), brute(parents, L), rtol=1e-12, atol=1e-12)
        count += 1
    assert count == int(np.prod(range(1, n))) if n > 1 else count == 1


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_bruteforce_every_forest(n):
    rng = np.random.default_rng(200 + n)
    for parents in all_parent_arrays(n, forests=True):
        L = rand_affine(rng, n)
        np.testing.assert_allclose(oracle.forward(parents, L), brute(parents, L), rtol=1e-12, atol=1e-12)


def _schedule_trees():
    rng = np.random.default_rng(7)
    trees = [synth.random_tree(300, 15, rng, spine=15), synth.random_tree(300, 120, rng, spine=120),
             synth.chain(200), synth.relabel_dfs(synth.random_tree(300, 40, rng, spine=40), rng)[0],
             synth.relabel_random_topological(synth.random_tree(150, 30, rng, spine=30), rng)[0]]
    return trees


def _paper_counts():
    """The paper's stated per-thread product and barrier counts
    (tests/golden/paper_schedule_counts.txt, with their passages)."""
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_schedule_counts.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, base, per64, barriers = line.split()[:4]
                out[name] = (base, int(per64), barriers)
    return out


@pytest.mark.parametrize("k", range(5))
def test_paper_schedules_equal_oracle(k):
    parents = _schedule_trees()[k]
    rng = np.random.default_rng(11 + k)
    L = rand_rigid(rng, len(parents))
    ref = oracle.forward(parents, L)
    D = ps.depths(parents).max()
    n = len(parents)

    m1, p1 = ps.alg1_gateau(parents, L)
    np.testing.assert_allclose(m1, ref, atol=1e-10)
    assert (p1 == ps.depths(parents) - 1).all()  # O(depth) per thread (Sec. 2)

    counts = _paper_counts()
    m2, p2, rounds = ps.alg2_jump(parents, L)
    np.testing.assert_allclose(m2, ref, atol=1e-10)
    assert counts["alg2"] == ("log2", 0, "log2")
    assert rounds == int(np.ceil(np.log2(D)))  # log2 rounds and barriers (Sec. 3.1)
    assert p2.max() <= rounds

    m3, p3, b3 = ps.alg3_blocks(parents, L)
    np.testing.assert_allclose(m3, ref, atol=1e-10)
    base, per64, bars = counts["alg3"]  # 6 + n/64, 6 rounds (Sec. 3.2.1)
    assert b3 == int(bars) and p3.max() <= int(base) + per64 * int(np.ceil(n / 64))

    m4, p4, b4 = ps.alg4_compress(parents, L)
    np.testing.assert_allclose(m4, ref, atol=1e-10)
    base, per64, bars = counts["alg4"]  # 14 + n/64, 2 barriers (Sec. 3.2.2)
    assert b4 == int(bars) and p4.max() <= int(base) + per64 * int(np.ceil(n / 64))


def test_same_axis_chain_closed_form():
    """z-rotations theta_k and translations (l_k, 0, 0) along a chain:
    R_j = Rz(sum_{k<=j} theta_k), p_j = sum_{k<=j} Rz(sum_{m<k} theta_m)(l_k,0,0)."""
    rng = np.random.default_rng(3)
    n = 500
    th = rng.uniform(-0.3, 0.3, n)
    ell = rng.uniform(0.01, 0.1, n)
    q = np.zeros((n, 4))
    q[:, 2] = np.sin(th / 2)
    q[:, 3] = np.cos(th / 2)
    t = np.zeros((n, 3))
    t[:, 0] = ell
    _, M = oracle.forward_qt([{"parents": synth.chain(n)}], np.zeros(1, np.int32), q, t, with_skin=False)
    cum = np.cumsum(th)
    prev = np.concatenate([[0.0], cum[:-1]])
    px = np.cumsum(np.cos(prev) * ell)
    py = np.cumsum(np.sin(prev) * ell)
    np.testing.assert_allclose(M[:, 0, 0], np.cos(cum), atol=1e-12)
    np.testing.assert_allclose(M[:, 1, 0], np.sin(cum), atol=1e-12)
    np.testing.assert_allclose(M[:, 0, 3], px, atol=1e-12)
    np.testing.assert_allclose(M[:, 1, 3], py, atol=1e-12)
    np.testing.assert_allclose(M[:, 2, 3], 0, atol=1e-15)


def test_identity_rotations_sum_translations():
    rng = np.random.default_rng(4)
    parents = synth.random_tree(200, 30, rng, spine=30)
    n = len(parents)
    q = np.tile([0.0, 0, 0, 1], (n, 1))
    t = rng.uniform(-1, 1, (n, 3))
    _, M = oracle.forward_qt([{"parents": parents}], np.zeros(1, np.int32), q, t, with_skin=False)
    p = np.zeros((n, 3))
    for i in range(n):
        a = i
        while a >= 0:
            p[i] += t[a]
            a = parents[a]
    np.testing.assert_allclose(M[:, :, :3], np.broadcast_to(np.eye(3), (n, 3, 3)), atol=1e-15)
    np.testing.assert_allclose(M[:, :, 3], p, atol=1e-12)


@pytest.mark.parametrize("cfg", [synth.config1, synth.config4])
def test_rest_pose_gives_identity_skin(cfg):
    w = cfg()
    ty = w["types"][0]
    skin, _ = oracle.forward_qt([ty], np.zeros(1, np.int32), ty["rest_q"].astype(np.float64),
                                ty["rest_t"].astype(np.float64))
    n = len(ty["parents"])
    ident = np.zeros((n, 3, 4))
    ident[:, :, :3] = np.eye(3)
    np.testing.assert_allclose(skin, ident, atol=1e-12)


def test_rigidity_invariants():
    w = synth.config4()
    ty = w["types"][0]
    n = len(ty["parents"])
    q, t = w["q"][: 8 * n], w["t"][: 8 * n]
    _, M = oracle.forward_qt([ty], np.zeros(8, np.int32), q, t, with_skin=False)
    R = M[:, :, :3]
    np.testing.assert_allclose(np.einsum("nji,njk->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    par = ty["parents"]
    p = M[:, :, 3].reshape(8, n, 3)
    tt = t.reshape(8, n, 3).astype(np.float64)
    for c in range(8):
        for i in range(1, n):
            assert abs(np.linalg.norm(p[c, i] - p[c, par[i]]) - np.linalg.norm(tt[c, i])) < 1e-12


def test_inverse_bind_is_inverse():
    w = synth.config1()
    ty = w["types"][0]
    B = oracle.inverse_bind(ty["parents"], ty["rest_q"], ty["rest_t"])
    _, M = oracle.forward_qt([ty], np.zeros(1, np.int32), ty["rest_q"].astype(np.float64),
                             ty["rest_t"].astype(np.float64), with_skin=False)
    prod = np.einsum("nij,njk->nik", h(M), h(B))
    np.testing.assert_allclose(prod, np.broadcast_to(np.eye(4), prod.shape), atol=1e-12)
    np.testing.assert_allclose(h(B), np.linalg.inv(h(M)), atol=1e-12)
