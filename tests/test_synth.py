"""The seeded input recipes: each workload generator yields the shapes,
sizes, depths and value ranges its configuration states (the benchmark's five
workloads; the paper's experiment shape for config 3's mix), deterministically
per seed.  The generators hold no method arithmetic; these checks use numpy
only."""
import numpy as np
import pytest

import synth


def depths(parents):
    d = np.zeros(len(parents), np.int64)
    for i, p in enumerate(parents):
        d[i] = 1 if p < 0 else d[p] + 1
    return d


def max_path_length(parents, t):
    """Largest root-to-joint sum of translation lengths."""
    s = np.zeros(len(parents))
    for i, p in enumerate(parents):
        s[i] = np.linalg.norm(t[i]) + (s[p] if p >= 0 else 0.0)
    return s.max()


def check_type(ty, n, depth):
    par = ty["parents"]
    assert len(par) == n and par[0] == -1
    assert all(par[i] < i for i in range(1, n))  # topological order, parent first
    assert int(depths(par).max()) == depth == ty["depth"]
    if "keys" in ty:
        assert ty["keys"].shape == (2, 30, n, 8) and ty["keys"].dtype == np.float32
        assert ty["rate_hz"] == 30.0
        np.testing.assert_allclose(np.linalg.norm(ty["keys"][..., :4], axis=-1), 1.0, atol=1e-6)


@pytest.mark.parametrize("name", ["config2", "config3", "config4", "config5"])
def test_unit_extent(name):
    """Unit-extent types: no root-to-joint path of the rest pose or of any key
    is longer than 1."""
    for ty in getattr(synth, name)()["types"]:
        assert max_path_length(ty["parents"], ty["rest_t"]) <= 1.0 + 1e-6
        if "keys" in ty:
            for c in range(2):
                for k in range(0, 30, 7):
                    assert max_path_length(ty["parents"], ty["keys"][c, k, :, 4:7]) <= 1.0 + 1e-6


def test_config1():
    w = synth.config1()
    assert len(w["char_type"]) == 64
    check_type(w["types"][0], 64, 12)
    assert w["q"].shape == (64 * 64, 4) and w["t"].shape == (64 * 64, 3)
    ang = 2 * np.degrees(np.arccos(np.clip(np.abs(w["q"][:, 3]), 0, 1)))
    assert ang.max() <= 30.0 + 1e-3 and np.abs(w["t"]).max() <= 0.1


def test_config2():
    w = synth.config2()
    ct = w["char_type"]
    assert len(ct) == 4097 and (ct[:4096] == 0).all() and ct[4096] == 1
    check_type(w["types"][0], 512, 70)
    check_type(w["types"][1], 1024, 1024)  # the dragon: a pure chain
    assert sum(len(w["types"][t]["parents"]) for t in ct) == 2_098_176
    assert (w["time"] >= 0).all() and (w["time"] < 1).all()
    assert (w["weight"] >= 0).all() and (w["weight"] <= 1).all()


def test_config3():
    w = synth.config3()
    ct = w["char_type"]
    assert len(ct) == 10_000
    for i, (n, d) in enumerate(synth.CONFIG3_MIX):
        check_type(w["types"][i], n, d)
    assert np.bincount(ct).tolist() == [4000, 3000, 1500, 1000, 500]
    assert sum(len(w["types"][t]["parents"]) for t in ct) == 3_328_000
    assert not (np.diff(ct) >= 0).all()  # shuffled


def test_config4():
    w = synth.config4()
    assert len(w["char_type"]) == 1024
    check_type(w["types"][0], 256, 96)
    nq = np.linalg.norm(w["q"], axis=1)
    assert nq.min() >= 0.8 - 1e-6 and nq.max() <= 1.2 + 1e-6  # unnormalized local rotations
    assert w["target"].shape == (1024 * 256, 3) and np.abs(w["target"]).max() <= 0.5


def test_config5():
    w = synth.config5()
    ct = w["char_type"]
    assert len(ct) == 8192 and (ct[0::2] == 0).all() and (ct[1::2] == 1).all()  # alternating
    check_type(w["types"][0], 128, 16)
    check_type(w["types"][1], 1024, 256)
    eff = w["effectors"]
    assert eff.shape == (2, 8)
    for ty, e in zip(w["types"], eff):
        assert len(set(e.tolist())) == 8 and (e > 0).all() and (e < len(ty["parents"])).all()
    q0 = w["q0"]
    assert (q0[:, :3] == 0).all() and (q0[:, 3] == 1).all()  # IK starts from identity rotations
    assert w["n_steps"] == 200 and w["lr"] == 1e-2


def test_deterministic_per_seed():
    a, b = synth.config2(), synth.config2()
    np.testing.assert_array_equal(a["time"], b["time"])
    np.testing.assert_array_equal(a["types"][0]["keys"], b["types"][0]["keys"])
    c = synth.config2(seed=9)
    assert not np.array_equal(a["time"], c["time"])
