"""bench.py's per-kernel table (host logic, no GPU)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kernel_table_rates_and_shares():
    b = _bench()
    # name: [launches, total ms, keys]
    kt = {"sample_scatter": [2, 1.0, 2 * 268435456], "transfer": [5, 0.01, 0],
          "counting_fill": [1, 0.2, 268435456]}
    t = b.kernel_table(kt, 6674.8)
    assert list(t) == ["sample_scatter", "counting_fill", "transfer"]   # by time
    # 2 x 2^28 keys x 8 bytes in 1 ms; 2^28 keys x 4 bytes in 0.2 ms.
    assert abs(t["sample_scatter"]["gbs"] - 2 * 268435456 * 8 / 1e-3 / 1e9) < 0.1
    assert abs(t["counting_fill"]["gbs"] - 268435456 * 4 / 0.2e-3 / 1e9) < 0.1
    assert abs(t["counting_fill"]["frac"] - t["counting_fill"]["gbs"] / 6674.8) < 1e-4
    assert "gbs" not in t["transfer"]                   # no algorithmic bytes
    assert abs(sum(e["share"] for e in t.values()) - 1.0) < 1e-3
