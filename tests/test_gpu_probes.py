"""The measurement probes run and report sane figures: empty launches,
random reads from an L2-resident table (the gather's ceiling), and the host
cost of a skeleton call against a bare launch of its kernel."""
import pytest

from helpers import skel

pytestmark = pytest.mark.gpu


def test_probe_empty_launches_count():
    import torch
    sk = skel()
    l0 = sk.lib.skel_launch_count()
    sk.skel_probe_empty_launches(50)
    torch.cuda.synchronize()
    assert sk.lib.skel_launch_count() - l0 == 50
    sk.skel_check_device()


def test_probe_l2_random_reads_and_rejects_bad_tables():
    import torch
    sk = skel()
    table = torch.rand(1 << 20, device="cuda")
    sink = torch.zeros(1, device="cuda")
    made = sk.skel_probe_l2_random(table, 1 << 24, sink)
    torch.cuda.synchronize()
    assert made >= 1 << 24 and made % 8 == 0
    assert float(sink.item()) == 0.0            # never written
    with pytest.raises(sk.SkelError):
        sk.skel_probe_l2_random(torch.rand(1000, device="cuda"), 1 << 20, sink)   # not a power of two


def test_probe_call_overhead_positive():
    sk = skel()
    us_call, us_launch = sk.skel_probe_call_overhead(100, 1024)
    assert 0 < us_launch < 1000 and 0 < us_call < 1000
