"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/anim.h declares, the Python binding's
signature table matches the header, and the host-only skeleton analysis
(segments and pointer-jumping rounds of the scan) is right."""
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "anim.h")).read()
    return sorted(set(re.findall(r"ANIM_API\s+(?:const\s+)?\w+\s*\*?\s*(anim_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_06703_gb300 import anim
    return anim.load()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ("anim_create_skeletons", "anim_upload_clips", "anim_evaluate_frame", "anim_backward",
                 "anim_forward_local", "anim_loss_backward", "anim_ik_step", "anim_tune", "anim_get_status",
                 "anim_evaluate_frame_levelsync"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    for name in header_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_signatures_match_header():
    from paper_2505_06703_gb300 import anim
    assert sorted(anim.SIGNATURES) == header_functions()


def test_library_exports_nothing_else(lib):
    import subprocess
    from paper_2505_06703_gb300 import anim
    out = subprocess.run(["nm", "-D", "--defined-only", anim.lib_path()], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == set(header_functions())


def test_version_and_no_device_error(lib):
    import ctypes
    assert lib.anim_version() >= 10000
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = lib.anim_create(ctypes.byref(h), 0)
    assert rc in (-5, -3)  # EDEVICE (or ECUDA) without a usable device, never a crash
    assert lib.anim_last_error(None)


def _seg_depth(parents, starts):
    n = len(parents)
    seg_of = np.zeros(n, int)
    for g in range(len(starts) - 1):
        seg_of[starts[g]:starts[g + 1]] = g
    d = []
    for g in range(len(starts) - 1):
        p = parents[starts[g]]
        d.append(1 if p < 0 else d[seg_of[p]] + 1)
    return max(d)


@pytest.mark.parametrize("seg_len", [1, 4, 8, 16])
def test_analyze_segments(seg_len):
    from paper_2505_06703_gb300 import analyze_skeleton
    rng = np.random.default_rng(seg_len)
    trees = [synth.chain(2048), synth.random_tree(300, 40, rng, spine=40),
             synth.relabel_dfs(synth.biped_with_chains(rng), rng)[0],
             synth.relabel_random_topological(synth.random_tree(100, 12, rng, spine=12), rng)[0],
             np.array([-1] + [0] * 63, np.int32), np.array([-1, -1, 1, -1], np.int32), np.array([-1], np.int32)]
    for par in trees:
        starts, rounds, depth = analyze_skeleton(par, seg_len)
        assert starts[0] == 0 and starts[-1] == len(par) and (np.diff(starts) > 0).all()
        assert np.diff(starts).max() <= seg_len
        for g in range(len(starts) - 1):  # a segment is a run of parent = previous joint
            for j in range(starts[g] + 1, starts[g + 1]):
                assert par[j] == j - 1
        D = _seg_depth(par, starts)
        assert rounds == (math.ceil(math.log2(D)) if D > 1 else 0)
        assert depth == synth.depths_of(par).max()


def test_analyze_rejects_bad_parents():
    from paper_2505_06703_gb300 import AnimError, analyze_skeleton
    for bad in ([0], [-1, 1], [-1, 0, 5], [-2]):
        with pytest.raises(AnimError):
            analyze_skeleton(np.array(bad, np.int32))


def test_chain_2048_segments():
    from paper_2505_06703_gb300 import analyze_skeleton
    starts, rounds, depth = analyze_skeleton(synth.chain(2048), 16)
    assert len(starts) - 1 == 128 and rounds == 7 and depth == 2048
