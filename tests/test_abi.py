"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

No call here touches a GPU: only argument validation that the library
performs before any CUDA call is exercised.
"""

import ctypes

import pytest

from paper_2110_01172_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_expected_entry_points():
    names = binding.declared_functions()
    for n in ("gbdct_plan_create", "gbdct_plan_create_batched", "gbdct_exec_forward",
              "gbdct_exec_inverse", "gbdct_plan_destroy", "gbdct_plan_workspace_bytes",
              "gbdct_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in binding.declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.gbdct_status_string(0) == b"GBDCT_OK"
    assert lib.gbdct_status_string(2) == b"GBDCT_ERR_UNSUPPORTED"
    assert lib.gbdct_status_string(99) == b"GBDCT_ERR_UNKNOWN"
    assert b"sm_103a" in lib.gbdct_version()


def _create(lib, dims, ndim=None, kind=0, dtype=0, batch=1):
    arr = (ctypes.c_int64 * max(1, len(dims)))(*dims)
    h = ctypes.c_void_p()
    st = lib.gbdct_plan_create_batched(ctypes.byref(h), len(dims) if ndim is None else ndim,
                                       arr, batch, kind, dtype)
    return st, h


@pytest.mark.parametrize("dims,ndim,kind,dtype,batch,expect", [
    ((0, 8), None, 0, 0, 1, binding.ERR_INVALID_ARG),       # dim <= 0
    ((8, -4), None, 0, 0, 1, binding.ERR_INVALID_ARG),
    ((8, 8), 4, 0, 0, 1, binding.ERR_INVALID_ARG),           # rank out of range
    ((8, 8), 0, 0, 0, 1, binding.ERR_INVALID_ARG),
    ((8, 8), None, 9, 0, 1, binding.ERR_INVALID_ARG),        # unknown kind
    ((8, 8), None, 0, 0, 0, binding.ERR_INVALID_ARG),        # batch < 1
    ((8, 8), None, 0, 3, 1, binding.ERR_UNSUPPORTED),        # dtype
    ((12, 8), None, 0, 0, 1, binding.ERR_UNSUPPORTED),       # not a power of two
    ((1, 8), None, 0, 0, 1, binding.ERR_UNSUPPORTED),        # below the smallest size
    ((8, 32768), None, 0, 0, 1, binding.ERR_UNSUPPORTED),    # above the largest size
    ((8,), None, 0, 0, 1, binding.ERR_UNSUPPORTED),          # 1D
    ((8, 8, 8), None, 1, 0, 1, binding.ERR_UNSUPPORTED),     # 3D: DCT-II only
    ((12, 8, 8), None, 0, 0, 1, binding.ERR_UNSUPPORTED),    # 3D: not a power of two
    ((8192, 8, 8), None, 0, 0, 1, binding.ERR_UNSUPPORTED),  # 3D: axis 0 above 4096
    ((4096, 8, 8), None, 0, 0, 16, binding.ERR_UNSUPPORTED), # 3D: batch * N0 > 65535
    ((8, 0, 8), None, 0, 0, 1, binding.ERR_INVALID_ARG),     # 3D: dim <= 0
])
def test_plan_create_rejects_before_touching_the_gpu(lib, dims, ndim, kind, dtype, batch, expect):
    st, h = _create(lib, dims, ndim, kind, dtype, batch)
    assert st == expect
    assert not h.value


def test_null_handles(lib):
    assert lib.gbdct_exec_forward(None, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.gbdct_exec_inverse(None, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.gbdct_plan_destroy(None) == binding.OK
    assert lib.gbdct_plan_workspace_bytes(None) == 0
    assert lib.gbdct_plan_launches_per_exec(None) == 0
    h = ctypes.c_void_p()
    assert lib.gbdct_plan_create(ctypes.byref(h), 2, None, 0, 0) == binding.ERR_INVALID_ARG
    assert lib.gbdct_plan_create(None, 2, (ctypes.c_int64 * 2)(8, 8), 0, 0) == binding.ERR_INVALID_ARG


def test_multi_and_family_rejections_before_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    shapes = (ctypes.c_int64 * 4)(64, 64, 128, 64)
    assert lib.gbdct_multi_create(ctypes.byref(h), 0, shapes, 0, 0) == binding.ERR_INVALID_ARG      # count
    assert lib.gbdct_multi_create(ctypes.byref(h), 2, None, 0, 0) == binding.ERR_INVALID_ARG        # shapes
    assert lib.gbdct_multi_create(None, 2, shapes, 0, 0) == binding.ERR_INVALID_ARG                 # out
    assert lib.gbdct_multi_create(ctypes.byref(h), 2, shapes, 7, 0) == binding.ERR_INVALID_ARG      # kind
    assert lib.gbdct_multi_create(ctypes.byref(h), 2, shapes, 0, 8) == binding.ERR_INVALID_ARG      # flags
    bad = (ctypes.c_int64 * 4)(64, 64, 96, 64)
    assert lib.gbdct_multi_create(ctypes.byref(h), 2, bad, 0, 0) == binding.ERR_UNSUPPORTED        # not pow2
    neg = (ctypes.c_int64 * 2)(64, 0)
    assert lib.gbdct_multi_create(ctypes.byref(h), 1, neg, 0, 0) == binding.ERR_INVALID_ARG
    assert not h.value
    assert lib.gbdct_multi_offset(None, 0) == -1
    assert lib.gbdct_multi_total_elems(None) == 0
    assert lib.gbdct_multi_group_count(None) == 0
    assert lib.gbdct_multi_group_family(None, 0) == b""
    assert lib.gbdct_multi_exec(None, 0, None, None, None) == binding.ERR_INVALID_ARG
    assert lib.gbdct_multi_destroy(None) == binding.OK
    dims = (ctypes.c_int64 * 2)(256, 256)
    assert lib.gbdct_plan_create_family(ctypes.byref(h), 2, dims, 1, 0, 0, b"fft") == binding.ERR_INVALID_ARG
    assert lib.gbdct_plan_create_family(ctypes.byref(h), 2, dims, 1, 0, 0, None) == binding.ERR_INVALID_ARG
    assert lib.gbdct_plan_create_tuned(ctypes.byref(h), 2, dims, 0, 0, 0, None, 0) == binding.ERR_INVALID_ARG
    assert not h.value


def test_multi_layout_is_a_dense_grouped_packing():
    """The packed layout of an uneven batch, computed on the host: every
    transform gets its own 16-byte-aligned range, the ranges tile the buffer
    exactly, equal shapes are contiguous in index order, larger shapes first."""
    from paper_2110_01172_gb300 import inputs
    shapes = inputs.batched_shapes(512, seed=0, lo=64, hi=1024)
    offs, total, groups = binding.multi_layout(shapes)
    sizes = [a * b for a, b in shapes]
    assert total == sum(sizes)
    assert groups == len(set(shapes))
    spans = sorted((o, o + s) for o, s in zip(offs, sizes))
    assert spans[0][0] == 0 and spans[-1][1] == total
    assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))       # no gap, no overlap
    assert all(o % 4 == 0 for o in offs)                               # 16-byte aligned
    by_shape = {}
    for i, sh in enumerate(shapes):
        by_shape.setdefault(sh, []).append(i)
    starts = []
    for sh, idx in by_shape.items():
        o = [offs[i] for i in idx]
        assert o == sorted(o)                                          # index order within a group
        assert all(b - a == sh[0] * sh[1] for a, b in zip(o, o[1:]))  # contiguous batch
        starts.append((o[0], sh[0] * sh[1]))
    starts.sort()
    assert [s for _, s in starts] == sorted((s for _, s in starts), reverse=True)   # largest first
    with pytest.raises(ValueError):
        binding.multi_layout([(64, 64), (96, 64)])


def test_precision_and_layout_null_paths(lib):
    assert lib.gbdct_plan_set_precision(None, 1) == binding.ERR_INVALID_ARG
    assert lib.gbdct_plan_set_precision(None, 0) == binding.ERR_INVALID_ARG
    shapes = (ctypes.c_int64 * 2)(64, 64)
    assert lib.gbdct_multi_layout(0, shapes, None, None) == -1
    assert lib.gbdct_multi_layout(1, None, None, None) == -1
    assert lib.gbdct_multi_layout(1, shapes, None, None) == 64 * 64
    bad = (ctypes.c_int64 * 2)(64, 65)
    assert lib.gbdct_multi_layout(1, bad, None, None) == -1
