"""Host-side logic of bench.py that needs no GPU: the sweep's setting filter and
the roofline traffic lookup keyed by the extension kernels' source."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_filter(bench):
    w = bench.sweep_wanted
    assert w("", "c3", 20, 0) and w("", "splicing")
    assert w("c5", "c5") and w("c5", "c5", 25, 128) and not w("c5", "c3") and not w("c5", "splicing")
    assert w("c5:20", "c5", 20, 1024) and not w("c5:20", "c5", 25, 1024)
    assert w("c5:20:inf", "c5", 20, 0) and not w("c5:20:inf", "c5", 20, 1024)
    assert w("c5:20:inf", "c5")  # the workload itself is wanted when any of its settings is
    assert w("c3:25,c5:20:128", "c3", 25, 0) and w("c3:25,c5:20:128", "c5", 20, 128)
    assert not w("c3:25,c5:20:128", "c5", 20, 0) and not w("c3:25,c5:20:128", "splicing")


def test_traffic_follows_the_kernel_source(bench):
    """The committed DRAM capture counts only while the extension source it was
    taken on is unchanged; then its bytes scale with the cells of a launch."""
    import json
    cap = json.load(open(os.path.join(ROOT, "profiles", "k_extend_dram_traffic_c2.json")))
    t = bench.traffic_per_launch(1e9)
    if cap["kernel_sha256_16"] != bench.kernel_hash():
        assert t is None
        return
    assert t == pytest.approx(cap["dram_bytes_per_cell"] * 1e9)
    assert bench.traffic_per_launch(2e9) == pytest.approx(2 * t)
