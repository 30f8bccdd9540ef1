"""Split-BF16 DFT-GEMM precision mode (hand-written tcgen05 tensor-core
kernels) against the FP64 oracle (needs a GB300).

The mode's error is that of the bf16 hi+lo split (each operand to ~2^-17
relative, the lo*lo products dropped), about 5e-6 relative in L2 — stated per
result here, with a bound of 5e-5 asserted (the FP32 FFT path is held to
1e-5).  The timeout path of the kernels' bounded waits is exercised by forcing
a one-poll bound: the error word reports it, the context stays usable, and
the next call with the default bound is correct again."""

import numpy as np
import pytest

import oracle
from paper_2110_01172_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = 5e-5


def rel(got, ref):
    got = np.asarray(got, np.float64)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("shape", [(128, 128), (256, 512), (1024, 1024), (2048, 256), (128, 2048), (2048, 2048)])
def test_split_bf16_forward_and_inverse_error(shape):
    from paper_2110_01172_gb300 import Plan
    x = inputs.uniform(shape, seed=90)
    p = Plan(shape).set_precision("split_bf16")
    X = p.forward(torch.from_numpy(x).cuda())
    y = p.inverse(X)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    ef = rel(Xh, oracle.dct2_2d(x))
    ei = rel(y.cpu().numpy(), oracle.idct2_2d(Xh))
    print(f"split-bf16 {shape}: forward rel-L2 {ef:.2e}, inverse rel-L2 {ei:.2e}")
    assert ef <= BOUND and ei <= BOUND


def test_split_bf16_batched_in_place_and_switch_back():
    from paper_2110_01172_gb300 import Plan, GbdctError
    shape, b = (128, 256), 3
    xs = np.stack([inputs.uniform(shape, seed=91 + i) for i in range(b)])
    p = Plan(shape, batch=b).set_precision("split_bf16")
    xd = torch.from_numpy(xs).cuda()
    X = p.forward(xd)
    buf = xd.clone()
    p.forward(buf, out=buf)
    torch.cuda.synchronize()
    assert torch.equal(buf, X)
    for i in range(b):
        assert rel(X[i].cpu().numpy(), oracle.dct2_2d(xs[i])) <= BOUND
    with pytest.raises(GbdctError):
        p.step(False, 0, xd, buf)
    p.set_precision("fp32")
    fp32 = Plan(shape, batch=b).forward(xd)
    again = p.forward(xd)
    torch.cuda.synchronize()
    assert torch.equal(again, fp32)


def test_split_bf16_unsupported_plans():
    from paper_2110_01172_gb300 import Plan, GbdctError
    for args in (((4096, 256), "dct2"), ((256, 256), "dst2"), ((16, 16, 16), "dct2"), ((64, 256), "dct2"),
                 ((256, 64), "dct2")):
        with pytest.raises(GbdctError):
            Plan(args[0], args[1]).set_precision("split_bf16")


def test_split_bf16_wait_timeout_is_reported_and_recovers():
    from paper_2110_01172_gb300 import Plan, binding
    shape = (256, 256)
    x = inputs.uniform(shape, seed=95)
    p = Plan(shape).set_precision("split_bf16")
    xd = torch.from_numpy(x).cuda()
    assert p.check_device_error() == binding.OK
    p.set_wait_limit(1)               # every wait gives up after one poll
    p.forward(xd)
    torch.cuda.synchronize()
    assert p.check_device_error() == binding.ERR_TIMEOUT
    assert p.check_device_error() == binding.OK   # reported once, then cleared
    p.set_wait_limit(0)               # default bound again
    X = p.forward(xd)
    torch.cuda.synchronize()
    assert p.check_device_error() == binding.OK
    assert rel(X.cpu().numpy(), oracle.dct2_2d(x)) <= BOUND
