"""Host buffers passed straight to the transforms (needs a GB300).

Page-locked host memory is mapped into the device's address space; the first
kernel of a transform reads such an input and the last kernel writes such an
output over the host link, so no staging copy is needed.  The results must be
bit-identical to the same transform on device buffers.
"""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,family", [((4096, 4096), "fs2"), ((256, 1024), "pair"), ((64, 64), None)])
def test_pinned_host_input_and_output_match_device_buffers(shape, family):
    from paper_2110_01172_gb300 import Plan
    plan = Plan(shape, family=family)
    xh = torch.from_numpy(inputs.uniform(shape, seed=70)).pin_memory()
    xd = xh.cuda()
    ref_fwd = plan.forward(xd)
    ref_inv = plan.inverse(ref_fwd)
    got_fwd = plan.forward(xh, torch.empty_like(xd))   # host in -> device out
    assert got_fwd.is_cuda
    assert not plan.forward(xh).is_cuda                # host in, no out: page-locked host out
    yh = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    plan.inverse(ref_fwd, yh)                      # device in -> host out
    hh = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    plan.forward(xh, hh)                           # host in -> host out
    torch.cuda.synchronize()
    assert torch.equal(got_fwd, ref_fwd)
    assert torch.equal(yh, ref_inv.cpu())
    assert torch.equal(hh, ref_fwd.cpu())
    if shape[0] * shape[1] <= 256 * 1024:
        X = hh.numpy().astype(np.float64)
        ref = oracle.dct2_2d(xh.numpy())
        assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e-5


def test_pinned_host_in_place_and_kinds():
    from paper_2110_01172_gb300 import Plan
    shape = (512, 512)
    x = inputs.uniform(shape, seed=71)
    buf = torch.from_numpy(x.copy()).pin_memory()
    plan = Plan(shape, "dst2")
    plan.forward(buf, buf)
    torch.cuda.synchronize()
    ref = oracle.dst2_2d(x)
    got = buf.numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    plan.inverse(buf, buf)
    torch.cuda.synchronize()
    assert np.abs(buf.numpy() - x).max() <= 1e-4 * np.abs(x).max()


def test_pageable_host_memory_is_used_only_where_the_device_can_access_it():
    """A pageable pointer gives INVALID_ARG, or (on devices with pageable
    memory access) the correct transform; never a fault."""
    from paper_2110_01172_gb300 import Plan, binding
    shape = (256, 256)
    x = np.ascontiguousarray(inputs.uniform(shape, seed=72))
    out = np.zeros(shape, dtype=np.float32)
    plan = Plan(shape)
    assert x.ctypes.data % 16 == 0 and out.ctypes.data % 16 == 0
    st = plan.forward_ptr(x.ctypes.data, out.ctypes.data, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if st == binding.OK:
        ref = oracle.dct2_2d(x)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-5
    else:
        assert st == binding.ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(4096, 4096), (1024, 2048)])
def test_two_pass_plan_on_host_buffers_runs_the_four_step_kernels(shape):
    """A two-pass plan runs full transforms on host-mapped buffers with the
    four-step kernels (whole-row host accesses): bit-identical to a four-step
    plan on device buffers, and within FP32 rounding of the two-pass result."""
    from paper_2110_01172_gb300 import Plan
    tp, fs2 = Plan(shape, family="tp"), Plan(shape, family="fs2")
    xh = torch.from_numpy(inputs.uniform(shape, seed=73)).pin_memory()
    xd = xh.cuda()
    ref_fs2 = fs2.forward(xd)
    ref_tp = tp.forward(xd)
    hf = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    tp.forward(xh, hf)
    hi = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    tp.inverse(ref_fs2, hi)
    inv_fs2 = fs2.inverse(ref_fs2)
    torch.cuda.synchronize()
    assert torch.equal(hf, ref_fs2.cpu())
    assert torch.equal(hi, inv_fs2.cpu())
    d = (hf - ref_tp.cpu()).norm() / ref_tp.norm().cpu()
    assert d <= 2e-6


@pytest.mark.parametrize("shape", [(4096, 4096), (1024, 2048)])
def test_two_pass_single_steps_on_host_buffers_match_bulk_copy_path(shape):
    """Single steps of a two-pass plan keep its launch sequence: the column
    pass moves device buffers with bulk tensor copies and host-mapped buffers
    with per-thread loads and stores, with bit-identical results."""
    from paper_2110_01172_gb300 import Plan
    plan = Plan(shape, family="tp")
    xh = torch.from_numpy(inputs.uniform(shape, seed=74)).pin_memory()
    xd = xh.cuda()
    fwd_dev, fwd_host = torch.empty_like(xd), torch.empty_like(xd)
    for k in range(plan.launches_per_exec):
        plan.step(False, k, xd, fwd_dev)
    for k in range(plan.launches_per_exec):
        plan.step(False, k, xh, fwd_host)          # column pass reads the host input
    inv_dev = torch.empty_like(xd)
    inv_host = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    for k in range(plan.launches_per_exec):
        plan.step(True, k, fwd_dev, inv_dev)
    for k in range(plan.launches_per_exec):
        plan.step(True, k, fwd_dev, inv_host)      # column pass writes the host output
    torch.cuda.synchronize()
    assert torch.equal(fwd_host, fwd_dev)
    assert torch.equal(inv_host, inv_dev.cpu())
    assert torch.equal(fwd_dev, plan.forward(xd))
