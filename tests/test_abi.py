"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, exports every function include/perch.h declares, the binding's
structures match the header's layouts, and calls fail cleanly without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1510_05613_gb300 import perch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "perch.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(perch.LIB_PATH):
        from paper_1510_05613_gb300 import build
        build.build()
    return perch.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(perch_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(perch.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layouts():
    assert ctypes.sizeof(perch.perch_obj) == 8 == perch.OBJ.itemsize
    assert perch.COST.itemsize == 28
    assert ctypes.sizeof(perch.perch_mesh) == 40
    assert ctypes.sizeof(perch.perch_search_params) == 48
    # objs, n_objs + pad, cost, expansions, successors, seconds, proven_optimal + pad, found_seconds,
    # found_expansions
    assert ctypes.sizeof(perch.perch_result) == 16 * 8 + 4 + 4 + 8 * 4 + 4 + 4 + 8 + 8
    assert perch.perch_result.found_seconds.offset == 176
    # kind, n, p[4], zlo, zhi, normals
    assert ctypes.sizeof(perch.perch_volume) == 4 + 4 + 16 + 8 + 8
    assert perch.perch_volume.normals.offset == 32
    # c, s, tx, ty (double), n_model, n_corr, iters, status
    assert perch.ICP.itemsize == 48 and perch.ICP.fields["status"][1] == 44


def test_null_context_and_null_args_are_rejected(lib):
    assert lib.perch_destroy(None) == perch.PERCH_OK
    assert lib.perch_load_meshes(None, None, 0) == perch.PERCH_E_ARG
    assert lib.perch_eval_successors(None, None, 0, None, 0, None, None, 0, 1, None) == perch.PERCH_E_ARG
    assert lib.perch_search(None, None, None) == perch.PERCH_E_ARG
    assert lib.perch_create(None, 0, None) == perch.PERCH_E_ARG
    assert lib.perch_set_volumes(None, None, 0) == perch.PERCH_E_ARG
    assert lib.perch_set_wait_limit(None, 0) == perch.PERCH_E_ARG
    assert lib.perch_set_share_renders(None, 1) == perch.PERCH_E_ARG
    assert lib.perch_set_render_cache(None, 1) == perch.PERCH_E_ARG
    assert lib.perch_launch_config(None, None, None, None) == perch.PERCH_E_ARG
    assert lib.perch_set_inline_pixels(None, -1, 16) == perch.PERCH_E_ARG
    assert lib.perch_set_bin_depth(None, -1, 64) == perch.PERCH_E_ARG
    assert lib.perch_launch_bin_depths(None, None) == perch.PERCH_E_ARG
    assert lib.perch_set_cost_stages(None, -1, 2) == perch.PERCH_E_ARG
    assert lib.perch_launch_cost_stages(None, None) == perch.PERCH_E_ARG
    assert lib.perch_icp_refine(None, None, 0, None, 0, None, None, 0, 0.02, 20, None) == perch.PERCH_E_ARG
    assert lib.perch_icp_refine_dev(None, None, 0, None, 0, None, None, 0, 0.02, 20, None) == perch.PERCH_E_ARG


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.perch_create(ctypes.byref(h), 0, None) == perch.PERCH_E_CUDA
    assert not h.value
