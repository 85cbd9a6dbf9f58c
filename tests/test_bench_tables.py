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


def test_traffic_is_used_only_for_the_source_it_was_taken_on(tmp_path):
    """profiles/traffic.json's DRAM bytes are scaled to a launch only while the
    kernel's source still hashes to the value recorded with the capture."""
    import json
    b = _bench()
    csrc = tmp_path / "paper_2506_20677_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "samplesort.cu").write_text("// partition pass, first version\n")
    b.ROOT = str(tmp_path)
    h = b.kernel_source_hash("sample_scatter")
    assert h is not None and b.kernel_source_hash("no_such_kernel") is None
    with open(tmp_path / "profiles" / "traffic.json", "w") as fh:
        json.dump({"sample_scatter": {"dram_bytes_per_item": 7.5, "source_hash": h}}, fh)
    assert b.ncu_traffic("sample_scatter", 1000) == 7500.0
    assert b.ncu_traffic("msd_scatter", 1000) is None          # same source, no entry
    (csrc / "samplesort.cu").write_text("// partition pass, changed\n")
    assert b.ncu_traffic("sample_scatter", 1000) is None        # source changed since
