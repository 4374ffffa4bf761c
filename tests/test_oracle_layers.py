"""Pins of the oracle's layered blend (up to 4 clips blended by incremental
slerp, translations by weighted mean, an additive layer on top; the paper
asks to keep clip blending, Sec. 2, without a method, so this is a reading).

  * two clips with weights (1 - w, w) and no additive layer give the
    two-clip blend, itself pinned in test_oracle_simulation;
  * one-hot weights give that clip alone;
  * clips whose keys all rotate about one axis blend to the weighted mean of
    their angles (closed form), translations to the weighted mean;
  * scaling every weight changes nothing;
  * an additive layer of weight 0, or of identity keys, leaves the pose; on
    an identity base, an additive rotation about one axis by b gives the
    angle a * b;
  * for general keys, weights and an additive layer, the whole layered
    sample equals the same steps composed from scipy's Slerp (a library
    routine).
"""
import numpy as np
import pytest

import oracle
import synth


def _keys_axis(rng, n_clips, n_keys, n, angles):
    """Keys whose rotation is angles[c, j] about z for every key of clip c."""
    k = np.zeros((n_clips, n_keys, n, 8), np.float32)
    for c in range(n_clips):
        h = angles[c] / 2
        k[c, :, :, 2] = np.sin(h)
        k[c, :, :, 3] = np.cos(h)
        k[c, :, :, 4:7] = rng.uniform(-0.1, 0.1, (n, 3))
    return k


def test_two_clips_reduce_to_the_two_clip_blend():
    w = synth.subset(synth.config2(), list(range(0, 4096, 256)) + [4096])
    m = len(w["char_type"])
    wl = dict(w, weights=np.stack([1 - w["weight"], w["weight"], np.zeros(m), np.zeros(m)], 1).astype(np.float32),
              add_w=np.zeros(m, np.float32))
    np.testing.assert_allclose(oracle.frame_layers(wl), oracle.frame(w), atol=1e-7)


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_one_hot_weights_pick_one_clip(i):
    rng = np.random.default_rng(i)
    n, nk = 7, 30
    keys = np.zeros((4, nk, n, 8), np.float32)
    for c in range(4):
        for k in range(nk):
            keys[c, k, :, :4] = synth.random_unit_quats(rng, n, 40.0)
            keys[c, k, :, 4:7] = rng.uniform(-1, 1, (n, 3))
    wts = np.zeros(4, np.float32)
    wts[i] = 0.7
    q, t = oracle.sample_layers(keys, 30.0, 0.4567, wts)
    q1, t1 = oracle.sample_layers(keys[i:i + 1], 30.0, 0.4567, [1.0])
    np.testing.assert_allclose(q, q1, atol=1e-12)
    np.testing.assert_allclose(t, t1, atol=1e-6)


def test_same_axis_clips_blend_to_the_weighted_mean_angle():
    rng = np.random.default_rng(5)
    n, nk = 9, 30
    angles = rng.uniform(-0.8, 0.8, size=(4, n))
    keys = _keys_axis(rng, 4, nk, n, angles)
    wts = np.array([0.1, 0.4, 0.0, 0.5], np.float32)
    q, t = oracle.sample_layers(keys, 30.0, 0.1234, wts)
    ang = (wts.astype(np.float64)[:, None] * angles).sum(0) / wts.sum()
    np.testing.assert_allclose(q[:, 2], np.sin(ang / 2), atol=1e-7)
    np.testing.assert_allclose(q[:, 3], np.cos(ang / 2), atol=1e-7)
    tt = (wts.astype(np.float64)[:, None, None] * keys[:, 0, :, 4:7]).sum(0) / wts.sum()
    np.testing.assert_allclose(t, tt, atol=1e-6)


def test_weight_scale_does_not_matter():
    w = synth.with_layers(synth.subset(synth.config2(), list(range(6))))
    k = w["types"][0]["keys"]
    q1, t1 = oracle.sample_layers(k, 30.0, 0.77, [0.2, 0.3, 0.1, 0.4])
    q2, t2 = oracle.sample_layers(k, 30.0, 0.77, [2.0, 3.0, 1.0, 4.0])
    # exact in real arithmetic; the weights reach the oracle as float32, whose
    # rounding of 0.2 and 2.0 differ by ~1e-8 relative
    np.testing.assert_allclose(q1, q2, atol=1e-7)
    np.testing.assert_allclose(t1, t2, atol=1e-6)


def test_additive_layer_special_cases():
    rng = np.random.default_rng(9)
    n, nk = 6, 30
    keys = np.zeros((2, nk, n, 8), np.float32)
    for c in range(2):
        for k in range(nk):
            keys[c, k, :, :4] = synth.random_unit_quats(rng, n, 40.0)
            keys[c, k, :, 4:7] = rng.uniform(-1, 1, (n, 3))
    add = np.zeros((nk, n, 8), np.float32)
    for k in range(nk):
        add[k, :, :4] = synth.random_unit_quats(rng, n, 20.0)
        add[k, :, 4:7] = rng.uniform(-0.1, 0.1, (n, 3))
    base_q, base_t = oracle.sample_layers(keys, 30.0, 0.31, [0.6, 0.4])
    q, t = oracle.sample_layers(keys, 30.0, 0.31, [0.6, 0.4], add_keys=add, add_w=0.0)
    np.testing.assert_allclose(q, base_q, atol=1e-12)
    np.testing.assert_allclose(t, base_t, atol=1e-12)
    ident = np.zeros_like(add)
    ident[:, :, 3] = 1.0
    q, t = oracle.sample_layers(keys, 30.0, 0.31, [0.6, 0.4], add_keys=ident, add_w=0.8)
    np.testing.assert_allclose(q, base_q, atol=1e-12)
    np.testing.assert_allclose(t, base_t, atol=1e-12)
    # identity base, additive rotation about z by b: angle a * b
    base = np.zeros((1, nk, n, 8), np.float32)
    base[..., 3] = 1.0
    b = rng.uniform(-1.0, 1.0, n)
    za = np.zeros((nk, n, 8), np.float32)
    za[:, :, 2] = np.sin(b / 2)
    za[:, :, 3] = np.cos(b / 2)
    q, _ = oracle.sample_layers(base, 30.0, 0.5, [1.0], add_keys=za, add_w=0.3)
    np.testing.assert_allclose(q[:, 2], np.sin(0.3 * b / 2), atol=1e-7)
    np.testing.assert_allclose(q[:, 3], np.cos(0.3 * b / 2), atol=1e-7)


def test_general_layers_match_scipy_composition():
    """General keys (random axes and quaternion signs), weights and an
    additive layer: each clip is scipy's Slerp of its bracketing keys at the
    key fraction, the clips blend by incremental scipy Slerp (weight w_i / W
    after W += w_i), translations by weighted mean, and the additive layer
    multiplies on the right by scipy's Slerp from identity to its sampled
    rotation at weight a (translation + a * t_a)."""
    from scipy.spatial.transform import Rotation, Slerp
    rng = np.random.default_rng(17)
    n, nk, nc = 6, 30, 4
    keys = np.zeros((nc, nk, n, 8), np.float32)
    add = np.zeros((nk, n, 8), np.float32)
    for k in range(nk):
        for c in range(nc):
            keys[c, k, :, :4] = synth.random_unit_quats(rng, n, 70.0)
            keys[c, k, :, 4:7] = rng.uniform(-1, 1, (n, 3))
        add[k, :, :4] = synth.random_unit_quats(rng, n, 50.0)
        add[k, :, 4:7] = rng.uniform(-0.2, 0.2, (n, 3))
    keys[..., :4][rng.random(keys.shape[:3]) < 0.5] *= -1.0
    add[..., :4][rng.random(add.shape[:2]) < 0.5] *= -1.0

    def sample(kk, k0, k1, al, j):
        r = Slerp([0, 1], Rotation.from_quat([kk[k0, j, :4].astype(np.float64), kk[k1, j, :4].astype(np.float64)]))
        t = (1 - al) * kk[k0, j, 4:7].astype(np.float64) + al * kk[k1, j, 4:7].astype(np.float64)
        return r([al]), t

    for trial in range(12):
        tm = float(np.float32(rng.uniform(-1, 2)))
        wts = rng.uniform(0, 1, nc).astype(np.float32)
        if trial % 3 == 0:
            wts[rng.integers(0, nc)] = 0.0  # a zero weight inside the sequence
        aw = float(np.float32(rng.uniform(0, 1)))
        u = np.float32(tm) * np.float32(30.0)
        k0 = int(np.floor(u)) % nk
        k1 = (k0 + 1) % nk
        al = float(u - np.floor(u))
        q, t = oracle.sample_layers(keys, 30.0, tm, wts, add_keys=add, add_w=aw)
        wd = wts.astype(np.float64)
        for j in range(n):
            rot, W, tsum = None, 0.0, np.zeros(3)
            t0 = None
            for c in range(nc):
                rc, tc = sample(keys[c], k0, k1, al, j)
                if c == 0:
                    rot, t0 = rc, tc
                elif W + wd[c] > 0:
                    rot = Slerp([0, 1], Rotation.concatenate([rot, rc]))([wd[c] / (W + wd[c])])
                W += wd[c]
                tsum += wd[c] * tc
            tref = tsum / W if W > 0 else t0
            ra, ta = sample(add, k0, k1, al, j)
            rref = rot * Slerp([0, 1], Rotation.concatenate([Rotation.identity(), ra]))([aw])
            tref = tref + aw * ta
            # float32 keys as stored (norms off 1 by rounding) against scipy's
            # normalized inputs: agreement to about 1e-7
            np.testing.assert_allclose(Rotation.from_quat(q[j]).as_matrix(), rref.as_matrix()[0], atol=1e-7)
            np.testing.assert_allclose(t[j], tref, atol=1e-12)
