"""The rate probes the benchmark uses for its L2 and L1 ceilings
(dash_probe_rate): each must do exactly the operations it reports, or the
rates it yields mean nothing.  Reductions add 1.0 per float they touch, so
the buffer's total is fixed by the reported count; gathers from a buffer of
ones sum to the per-thread count in every thread's sink."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,floats_per_op", [(1, 2), (2, 4), (3, 2)])
def test_reduction_probes_do_the_reported_work(dashlib, kind, floats_per_op):
    buf = torch.zeros(1_000_003 * 4, dtype=torch.float32, device="cuda")   # an odd number of 16-byte groups
    ops = dashlib.dash_probe_rate(kind, buf, 7)
    torch.cuda.synchronize()
    assert ops == dashlib.dash_probe_threads(kind) * 7
    assert float(buf.double().sum()) == floats_per_op * ops
    assert float(buf.max()) < 2 ** 24   # every per-float count exact in FP32


@pytest.mark.parametrize("kind", [4, 5])
def test_gather_probes_do_the_reported_work(dashlib, kind):
    buf = torch.ones(333_331 * 4, dtype=torch.float32, device="cuda")
    sink = torch.zeros(dashlib.dash_probe_threads(kind), dtype=torch.float32, device="cuda")
    ops = dashlib.dash_probe_rate(kind, buf, 9, sink)
    torch.cuda.synchronize()
    assert ops == sink.numel() * 9
    assert bool(torch.all(sink == 9.0))


def test_probe_arguments_are_checked(dashlib):
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(dashlib.DashError):
        dashlib.dash_probe_rate(9, buf, 1)          # unknown kind
    with pytest.raises(dashlib.DashError):
        dashlib.dash_probe_rate(1, buf, 0)          # iters out of range
    with pytest.raises(dashlib.DashError):
        dashlib.dash_probe_rate(1, buf[1:], 1)      # not 16-byte aligned
