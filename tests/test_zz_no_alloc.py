"""The forward 2D DCT entry point that allocates no device memory.

Some callers cannot allocate device memory on the call path (a host framework
that owns all device memory through its own pool, or a loop where cudaMalloc
would synchronise the device); gbdct_dct2d_forward_noalloc serves them from a
static device array.  These tests call it through the C ABI and compare it
with the plan-based gbdct_exec_forward on two calls in a row, so a second call
that wrongly depended on what the first left in the shared array would fail.
This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from paper_2110_01172_gb300 import binding, inputs

torch = pytest.importorskip("torch")

REL_L2 = 1e-5
MAX_ABS = 1e-4


def _compare(got, ref):
    got = got.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= REL_L2 and mx <= MAX_ABS, (err, mx)


def _noalloc_call(lib, x, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.gbdct_dct2d_forward_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           x.shape[0], x.shape[1], ctypes.c_void_p(stream))


@pytest.mark.gpu
def test_noalloc_matches_plan_forward_on_two_calls_in_a_row():
    from paper_2110_01172_gb300 import Plan
    lib = binding.load()
    for shape, seed in (((1024, 1024), 1), ((256, 2048), 2)):
        x = torch.from_numpy(inputs.uniform(shape, seed=seed)).cuda()
        out = torch.empty_like(x)
        assert _noalloc_call(lib, x, out) == binding.OK
        ref = Plan(shape, "dct2").forward(x)
        torch.cuda.synchronize()
        _compare(out, ref)


@pytest.mark.gpu
def test_noalloc_one_sequence_kernels_and_in_place():
    """Shapes with a side below 16 or equal to 16384 take the one-sequence
    passes (a different grid and shared-memory size); in == out is allowed."""
    from paper_2110_01172_gb300 import Plan
    lib = binding.load()
    for shape, seed in (((16384, 64), 3), ((8, 4096), 4), ((2, 2), 5), ((64, 16384), 6)):
        x = torch.from_numpy(inputs.uniform(shape, seed=seed)).cuda()
        out = torch.empty_like(x)
        assert _noalloc_call(lib, x, out) == binding.OK
        ref = Plan(shape, "dct2").forward(x)
        torch.cuda.synchronize()
        _compare(out, ref)
    x = torch.from_numpy(inputs.uniform((512, 512), seed=7)).cuda()
    ref = Plan((512, 512), "dct2").forward(x)
    assert _noalloc_call(lib, x, x) == binding.OK    # in place
    torch.cuda.synchronize()
    _compare(x, ref)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = binding.load()
    x = torch.zeros((2048, 1024), device="cuda")
    assert _noalloc_call(lib, x, x) == binding.ERR_UNSUPPORTED
    y = torch.zeros((24, 64), device="cuda")
    assert _noalloc_call(lib, y, y) == binding.ERR_UNSUPPORTED
