"""The library's peak probes (pttk_peak_probe): every kind runs to completion and reports a
rate inside the part's physical range, the streaming MMA probes order by width as the tensor
pipe's cost per MMA implies (flat up to N = 128), and an unknown kind is rejected."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_06344_gb300 import pttk
    pttk.load()
    return pttk


# (kind, loop trips, an upper bound in TFLOP/s well above the part's nominal rate)
KINDS = [("dfma", 2000, 5.0), ("ffma", 20000, 300.0), ("dmma", 2000, 5.0), ("tf32", 20000, 3000.0),
         ("f16", 20000, 6000.0), ("f16s64", 20000, 6000.0), ("f16s128", 20000, 6000.0), ("f16s256", 20000, 6000.0)]


@pytest.mark.parametrize("kind,iters,hi", KINDS)
def test_probe_reports_a_physical_rate(P, kind, iters, hi):
    tf, ms = P.peak_probe(kind, iters)
    assert math.isfinite(tf) and 0.0 < tf < hi
    assert ms > 0.0


def test_streaming_probe_rates_grow_with_width(P):
    r = {n: max(P.peak_probe(f"f16s{n}", 50000)[0] for _ in range(2)) for n in (64, 128, 256)}
    assert r[128] > 1.3 * r[64]
    assert r[256] > r[128]


def test_unknown_probe_kind_is_rejected(P):
    for kind in (-1, 8):
        with pytest.raises(P.PttkError) as e:
            P.peak_probe(kind, 10)
        assert e.value.status == P.EINVAL
