"""Pins for the oracle's Simulation stage (Sec. 1 step 1; Sec. 2 keeps
keyframe interpolation and blending): slerp, key sampling and the two-clip
blend.  Checked against scipy's Slerp (a library routine; for general keys
and weights the whole sample-and-blend composed from it), closed forms for
same-axis rotations, the constant-angular-velocity property, and exact
special cases (key times, wrap-around, blend weights 0 and 1)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation, Slerp

import oracle
import synth


def axis_angle_q(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([axis * np.sin(ang / 2), [np.cos(ang / 2)]])


def same_rot(a, b, tol=1e-12):
    return min(np.abs(a - b).max(), np.abs(a + b).max()) < tol


def test_slerp_endpoints():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = synth.random_unit_quats(rng, 2, 170.0)
        assert same_rot(oracle.slerp(a, b, 0.0), a)
        assert same_rot(oracle.slerp(a, b, 1.0), b)


def test_slerp_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(300):
        a, b = synth.random_unit_quats(rng, 2, 179.0)
        if rng.random() < 0.5:
            b = -b  # the shorter arc must be taken either way
        al = rng.uniform(0, 1)
        ref = Slerp([0, 1], Rotation.from_quat([a, b]))([al]).as_matrix()[0]
        got = Rotation.from_quat(oracle.slerp(a, b, al)).as_matrix()
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_slerp_same_axis_closed_form():
    rng = np.random.default_rng(2)
    for _ in range(200):
        axis = rng.normal(size=3)
        p0, p1 = rng.uniform(-1.5, 1.5, 2)
        al = rng.uniform(0, 1)
        got = oracle.slerp(axis_angle_q(axis, p0), axis_angle_q(axis, p1), al)
        assert same_rot(got, axis_angle_q(axis, (1 - al) * p0 + al * p1), 1e-12)


def test_slerp_constant_angular_velocity():
    rng = np.random.default_rng(3)
    a, b = synth.random_unit_quats(rng, 2, 120.0)
    total = np.arccos(min(1.0, abs(a @ b)))
    for al1, al2 in rng.uniform(0, 1, size=(50, 2)):
        q1, q2 = oracle.slerp(a, b, al1), oracle.slerp(a, b, al2)
        ang = np.arccos(min(1.0, abs(q1 @ q2)))
        assert abs(ang - abs(al1 - al2) * total) < 1e-7


def test_slerp_near_parallel_and_antipodal():
    a = axis_angle_q([0, 0, 1], 0.3)
    for eps in (0.0, 1e-15, 1e-13, 1e-9):
        b = axis_angle_q([0, 0, 1], 0.3 + eps)
        r = oracle.slerp(a, b, 0.37)
        assert np.isfinite(r).all() and abs(np.linalg.norm(r) - 1) < 1e-15
        assert same_rot(r, axis_angle_q([0, 0, 1], 0.3 + 0.37 * eps), 1e-12)
    # q and -q are the same rotation: interpolating towards -b is interpolating towards b
    b = axis_angle_q([1, 2, 3], 1.1)
    assert same_rot(oracle.slerp(a, -b, 0.4), oracle.slerp(a, b, 0.4))


def _keys(rng, n=7, nk=30):
    keys = np.zeros((2, nk, n, 8), np.float32)
    for c in range(2):
        for k in range(nk):
            keys[c, k, :, :4] = synth.random_unit_quats(rng, n, 60.0)
            keys[c, k, :, 4:7] = rng.uniform(-1, 1, (n, 3))
    return keys


def test_sample_exact_key_times_and_weights():
    rng = np.random.default_rng(4)
    keys = _keys(rng)
    for k in (0, 1, 7, 29):
        tm = np.float32(k) / np.float32(30.0)
        # float32 time * 30 may land just below k; take the time whose float32 product is exactly k
        while np.float32(tm) * np.float32(30.0) < k:
            tm = np.nextafter(np.float32(tm), np.float32(2))
        for wgt, clip in ((0.0, 0), (1.0, 1)):
            q, t = oracle.sample_local(keys, 30.0, float(tm), wgt)
            ref = keys[clip, k, :, :4].astype(np.float64)
            ref /= np.linalg.norm(ref, axis=1, keepdims=True)
            for j in range(keys.shape[2]):
                assert same_rot(q[j], ref[j], 1e-12)
            np.testing.assert_allclose(t, keys[clip, k, :, 4:7], atol=1e-12)


def test_sample_wraps_and_is_continuous():
    rng = np.random.default_rng(5)
    keys = _keys(rng)
    # the last segment runs from key 29 to key 0: just before t = 1 s the pose approaches key 0
    q_end, t_end = oracle.sample_local(keys, 30.0, float(np.nextafter(np.float32(1.0), np.float32(0))), 0.0)
    q0, t0 = oracle.sample_local(keys, 30.0, 0.0, 0.0)
    np.testing.assert_allclose(t_end, t0, atol=1e-5)
    for j in range(keys.shape[2]):
        assert same_rot(q_end[j], q0[j], 1e-5)
    # periodicity: t and t + 1 s sample the same pose (when float32 maps them to the same fraction)
    for tm in (0.125, 0.25, 0.5, 0.75):
        qa, ta = oracle.sample_local(keys, 30.0, tm, 0.3)
        qb, tb = oracle.sample_local(keys, 30.0, tm + 2.0, 0.3)
        qc, tc = oracle.sample_local(keys, 30.0, tm - 1.0, 0.3)
        np.testing.assert_allclose(qa, qb, atol=1e-15)
        np.testing.assert_allclose(qa, qc, atol=1e-15)
        np.testing.assert_allclose(ta, tc, atol=1e-15)


def test_sample_same_axis_closed_form():
    """Keys rotating about one axis: the sampled and blended angle is the
    bilinear interpolation of the four key angles; translations likewise."""
    rng = np.random.default_rng(6)
    n, nk = 3, 30
    axis = np.array([0.3, -0.5, 0.8])
    ang = rng.uniform(-0.6, 0.6, size=(2, nk, n))
    keys = np.zeros((2, nk, n, 8), np.float32)
    for c in range(2):
        for k in range(nk):
            for j in range(n):
                keys[c, k, j, :4] = axis_angle_q(axis, ang[c, k, j])
    keys[..., 4:7] = rng.uniform(-1, 1, (2, nk, n, 3))
    for tm, wgt in ((0.4321, 0.2), (0.9876, 0.75), (0.05, 0.5)):
        wgt = float(np.float32(wgt))  # the weight crosses the interface as float32
        u = np.float32(tm) * np.float32(30.0)
        k0 = int(np.floor(u)) % nk
        k1 = (k0 + 1) % nk
        al = float(u - np.floor(u))
        q, t = oracle.sample_local(keys, 30.0, tm, wgt)
        for j in range(n):
            a0 = (1 - al) * ang[0, k0, j] + al * ang[0, k1, j]
            a1 = (1 - al) * ang[1, k0, j] + al * ang[1, k1, j]
            # use the float32-rounded keys' angles: compare with tolerance of float32 rounding
            assert same_rot(q[j], axis_angle_q(axis, (1 - wgt) * a0 + wgt * a1), 2e-7)
            kt = keys[..., 4:7].astype(np.float64)
            tref = (1 - wgt) * ((1 - al) * kt[0, k0, j] + al * kt[0, k1, j]) + \
                wgt * ((1 - al) * kt[1, k0, j] + al * kt[1, k1, j])
            np.testing.assert_allclose(t[j], tref, atol=1e-12)


def test_sample_general_matches_scipy_composition():
    """General keys (random axes, random quaternion signs), times and
    weights: the sampled pose is scipy's Slerp of each clip's bracketing keys
    at the key fraction, then scipy's Slerp of the two clip poses at the
    blend weight; translations lerp likewise."""
    rng = np.random.default_rng(8)
    keys = _keys(rng, n=9)
    flip = rng.random(keys.shape[:3]) < 0.5
    keys[..., :4][flip] *= -1.0  # q and -q: the shorter arc must be taken either way
    nk = keys.shape[1]
    for tm, wgt in zip(rng.uniform(-1.5, 2.5, 40), rng.uniform(0, 1, 40)):
        tm, wgt = float(np.float32(tm)), float(np.float32(wgt))
        u = np.float32(tm) * np.float32(30.0)
        k0 = int(np.floor(u)) % nk
        k1 = (k0 + 1) % nk
        al = float(u - np.floor(u))
        q, t = oracle.sample_local(keys, 30.0, tm, wgt)
        kq = keys[..., :4].astype(np.float64)
        kt = keys[..., 4:7].astype(np.float64)
        for j in range(keys.shape[2]):
            qa = Slerp([0, 1], Rotation.from_quat([kq[0, k0, j], kq[0, k1, j]]))([al])
            qb = Slerp([0, 1], Rotation.from_quat([kq[1, k0, j], kq[1, k1, j]]))([al])
            ref = Slerp([0, 1], Rotation.concatenate([qa, qb]))([wgt]).as_matrix()[0]
            # the oracle interpolates the float32 keys as stored, whose norms
            # differ from 1 by float32 rounding, while scipy normalizes them
            # first: the two paths differ by up to about 2e-8 (a wrong term,
            # sign, key or weight shows at 1e-3 and above)
            np.testing.assert_allclose(Rotation.from_quat(q[j]).as_matrix(), ref, atol=1e-7)
            ta = (1 - al) * kt[0, k0, j] + al * kt[0, k1, j]
            tb = (1 - al) * kt[1, k0, j] + al * kt[1, k1, j]
            np.testing.assert_allclose(t[j], (1 - wgt) * ta + wgt * tb, atol=1e-12)


def test_frame_chain_matches_stagewise():
    """frame() = sample_local -> forward -> bind, on a small config-2 subset."""
    w = synth.subset(synth.config2(), [0, 5, 4096])
    skin = oracle.frame(w)
    off = oracle.offsets(w["char_type"], w["types"])
    for c, ty in enumerate(w["char_type"]):
        T = w["types"][ty]
        q, t = oracle.sample_local(T["keys"], T["rate_hz"], float(w["time"][c]), float(w["weight"][c]))
        s2, _ = oracle.forward_qt([T], np.zeros(1, np.int32), q, t)
        np.testing.assert_allclose(skin[off[c]:off[c + 1]], s2, atol=1e-13)
