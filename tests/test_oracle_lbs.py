"""Pins of the oracle's linear blend skinning (the skinning step after Bind
MeshPose, Sec. 1 of the paper; textbook form since the paper gives none).

Each case has a result fixed by something other than the oracle's formula:
  * identity skin matrices leave every vertex and normal where it is;
  * one influence of weight 1 is the rigid transform of that bone, checked
    against scipy's rotation applied to the points;
  * bones that share one skin matrix act as that matrix whatever the split
    of the weights;
  * pure translations move a vertex by the weighted mean of the bones'
    translations and leave its normal;
  * a rotation by angle a about z on one bone and by -a on another with
    equal weights gives the cosine-scaled (x, y) of the rest point, whose
    closed form follows from cos(a) R_z(0) = (R_z(a) + R_z(-a)) / 2.
A mistake in the index of the bone, the order of the product, a dropped
translation or a missing weight fails one of them.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth


def _mesh(rng, n_joints, n_verts, k=4):
    # bones drawn over a random tree of n_joints (any valid ids will do)
    return synth.make_mesh(synth.random_tree(n_joints, max(2, n_joints // 2), rng), n_verts, rng, max_influences=k)


def _rigid(rng, n):
    R = Rotation.random(n, random_state=int(rng.integers(1 << 31))).as_matrix()
    t = rng.uniform(-1, 1, size=(n, 3))
    return np.concatenate([R, t[:, :, None]], axis=2)  # [n][3][4]


def test_identity_skin_keeps_rest_mesh():
    rng = np.random.default_rng(1)
    mesh = _mesh(rng, 12, 200)
    S = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1), (12, 1, 1))
    out = oracle.lbs(mesh, S)
    np.testing.assert_allclose(out[:, :3], mesh["pos"], atol=1e-6)
    np.testing.assert_allclose(out[:, 3:], mesh["nrm"], atol=1e-6)


def test_single_influence_is_the_bone_transform():
    rng = np.random.default_rng(2)
    n, nv = 9, 300
    mesh = _mesh(rng, n, nv)
    mesh["weights"][:] = 0
    mesh["weights"][:, 0] = 1
    S = _rigid(rng, n)
    out = oracle.lbs(mesh, S)
    b = mesh["bones"][:, 0]
    p = mesh["pos"].astype(np.float64)
    rot = Rotation.from_matrix(S[b, :, :3])
    np.testing.assert_allclose(out[:, :3], rot.apply(p) + S[b, :, 3], atol=1e-12)
    nr = rot.apply(mesh["nrm"].astype(np.float64))
    np.testing.assert_allclose(out[:, 3:], nr / np.linalg.norm(nr, axis=1, keepdims=True), atol=1e-12)


def test_shared_skin_matrix_ignores_the_weight_split():
    rng = np.random.default_rng(3)
    n, nv = 6, 250
    mesh = _mesh(rng, n, nv)
    S1 = _rigid(rng, 1)[0]
    S = np.tile(S1, (n, 1, 1))
    out = oracle.lbs(mesh, S)
    p = mesh["pos"].astype(np.float64)
    rot = Rotation.from_matrix(S1[:, :3])
    # the float32 weights sum to 1 within 1e-7
    np.testing.assert_allclose(out[:, :3], rot.apply(p) + S1[:, 3], atol=1e-6)
    nr = rot.apply(mesh["nrm"].astype(np.float64))
    np.testing.assert_allclose(out[:, 3:], nr / np.linalg.norm(nr, axis=1, keepdims=True), atol=1e-6)


def test_translations_move_by_the_weighted_mean():
    rng = np.random.default_rng(4)
    n, nv = 10, 300
    mesh = _mesh(rng, n, nv)
    t = rng.uniform(-2, 2, size=(n, 3))
    S = np.concatenate([np.tile(np.eye(3), (n, 1, 1)), t[:, :, None]], axis=2)
    out = oracle.lbs(mesh, S)
    w = mesh["weights"].astype(np.float64)
    expect = mesh["pos"] + np.einsum("vk,vkr->vr", w, t[mesh["bones"]])
    np.testing.assert_allclose(out[:, :3], expect, atol=1e-6)
    np.testing.assert_allclose(out[:, 3:], mesh["nrm"], atol=1e-6)


@pytest.mark.parametrize("angle", [0.3, 1.1, 2.5])
def test_opposite_rotations_blend_to_cosine_scaling(angle):
    rng = np.random.default_rng(5)
    nv = 100
    mesh = _mesh(rng, 2, nv)
    mesh["bones"][:, :2] = [0, 1]
    mesh["weights"][:] = 0
    mesh["weights"][:, :2] = 0.5
    c = np.cos(angle)
    Rz = lambda a: np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    S = np.stack([np.concatenate([Rz(angle), np.zeros((3, 1))], 1), np.concatenate([Rz(-angle), np.zeros((3, 1))], 1)])
    out = oracle.lbs(mesh, S)
    p = mesh["pos"].astype(np.float64)
    np.testing.assert_allclose(out[:, 0], c * p[:, 0], atol=1e-12)
    np.testing.assert_allclose(out[:, 1], c * p[:, 1], atol=1e-12)
    np.testing.assert_allclose(out[:, 2], p[:, 2], atol=1e-12)
    n = mesh["nrm"].astype(np.float64) * [c, c, 1.0]
    np.testing.assert_allclose(out[:, 3:], n / np.linalg.norm(n, axis=1, keepdims=True), atol=1e-12)


def test_workload_vertex_offsets():
    w = synth.with_meshes(synth.subset(synth.config1(), list(range(5))), n_verts=7)
    off = oracle.vertex_offsets(w["char_type"], w["types"])
    assert list(off) == [0, 7, 14, 21, 28, 35]
