"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol
include/cgh.h declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cgh_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2211_09938_gb300 import build_lib, cgh
    if not os.path.exists(cgh.LIB_PATH):
        build_lib.build()
    return cgh.lib()


def test_header_declares_the_path():
    names = declared_functions()
    for n in ("cgh_plan_create", "cgh_haar_decompose", "cgh_select_blocks",
              "cgh_progressive_hologram", "cgh_reconstruct", "cgh_plain_direct"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    from paper_2211_09938_gb300 import cgh
    for n in declared_functions():
        assert hasattr(L, n), n
        assert n in cgh.SIGNATURES, n  # the binding marshals every entry point


def test_host_argument_checks_without_gpu(L):
    h = ctypes.c_void_p()
    z = (ctypes.c_double * 1)(0.1)
    # levels other than 3 are rejected before any CUDA call
    assert L.cgh_plan_create(ctypes.byref(h), 64, 64, 256, 256, 8e-6, 532e-9, 1, z, 2, 0, None) == 3
    assert h.value is None
    # hologram not an integer multiple of the object
    assert L.cgh_plan_create(ctypes.byref(h), 64, 64, 250, 256, 8e-6, 532e-9, 1, z, 3, 0, None) == 1
    assert b"integer" in L.cgh_last_error()
    # object not a multiple of 8
    assert L.cgh_plan_create(ctypes.byref(h), 60, 60, 240, 240, 8e-6, 532e-9, 1, z, 3, 0, None) == 1
    # bad layer count / distances
    assert L.cgh_plan_create(ctypes.byref(h), 64, 64, 256, 256, 8e-6, 532e-9, 0, z, 3, 0, None) == 1
    # unknown plan flags
    assert L.cgh_plan_create(ctypes.byref(h), 64, 64, 256, 256, 8e-6, 532e-9, 1, z, 3, 4, None) == 1
    zneg = (ctypes.c_double * 1)(-0.1)
    assert L.cgh_plan_create(ctypes.byref(h), 64, 64, 256, 256, 8e-6, 532e-9, 1, zneg, 3, 0, None) == 1
    # NULL plan
    assert L.cgh_haar_decompose(None, None, None, None, None) == 1
    assert L.cgh_select_blocks(None, None, None, -1, 1, None, None, 0, None) == 1
    assert L.cgh_progressive_hologram(None, None, None, None, None, 0, 0, None) == 1
    assert L.cgh_progressive_step(None, None, None, None, None, None, None, None, None, None, 0, 1, None) == 1
    assert b"cgh_progressive_step" in L.cgh_last_error()
    tiles = ctypes.c_int(-1)
    assert L.cgh_plan_stage2_tiles_used(None, ctypes.byref(tiles)) == 1
    assert tiles.value == -1  # nothing written on error
    assert L.cgh_plan_set_stage2_tiles(None, 0) == 1
    assert L.cgh_plan_destroy(None) == 0
    assert L.cgh_version() >= 10000


def test_operator_count_of_device_counts_matches_oracle():
    """Plan.operator_count (host arithmetic on the counts the selection writes) agrees with
    the pinned oracle's operator_count on the same lists, stage by stage."""
    import numpy as np
    import torch
    from oracle import cgh_oracle as O
    from paper_2211_09938_gb300 import Plan
    from synth import scenes
    sc = scenes.random_scene(55, 64, 128, 3, graded=True)
    lists = O.progressive_lists(sc["saliency"], sc["layer"], 3, scenes.THRESHOLDS_U8)
    counts = torch.tensor([[len(x), len(x)] for x in lists], dtype=torch.int32)
    e = np.zeros(0, np.int32)
    for stage, keep in enumerate(Plan._STAGE_LISTS):
        st = [lists[k] if k in keep else e for k in range(4)]
        assert Plan.operator_count(Plan.level_counts(counts, stage)) == O.operator_count(st)
