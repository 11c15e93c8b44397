"""The traffic table behind the bench line's `roofline.traffic`: the ncu CSV
reader and entry writer (paper_1505_02037_gb300/traffic_table.py), and the
bench's rule that an entry counts only when it was captured on the sources
it is read with. No GPU."""
import importlib.util
import json
import os

import pytest

from paper_1505_02037_gb300 import traffic_table as TT

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ncu_csv(path, rows):
    """A file in the layout `ncu --csv --log-file` writes: a header row and
    one row per (launch, metric), values with thousands separators."""
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",' \
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",' \
           '"Metric Value"'
    with open(path, "w") as f:
        f.write("==PROF== a line ncu prints before the table\n")
        f.write(head + "\n")
        for (lid, kernel, name, unit, value) in rows:
            f.write(f'"{lid}","1","python","127.0.0.1","{kernel}","1","7","(128, 1, 1)",'
                    f'"(16384, 1, 1)","0","10.3","Command line profiler metrics","{name}",'
                    f'"{unit}","{value}"\n')


def test_reader_scales_units_and_keeps_launches_apart(tmp_path):
    p = tmp_path / "cap.csv"
    ncu_csv(p, [
        (0, "void k_aux<19, float>(...)", "dram__bytes_read.sum", "Mbyte", "1.5"),
        (1, "void k_collide_w<19, float>(...)", "dram__bytes_read.sum", "Gbyte", "2.5"),
        (1, "void k_collide_w<19, float>(...)", "dram__bytes_write.sum", "Kbyte", "1,024"),
        (1, "void k_collide_w<19, float>(...)", "gpu__time_duration.sum", "usecond", "756.5"),
        (2, "void k_collide_w<19, float>(...)", "gpu__time_duration.sum", "nsecond", "1,000,000"),
    ])
    rows = TT.read_ncu_csv(str(p), "k_collide")
    assert len(rows) == 2
    assert rows[0]["dram__bytes_read.sum"] == pytest.approx(2.5e9)
    assert rows[0]["dram__bytes_write.sum"] == pytest.approx(1.024e6)
    assert rows[0]["gpu__time_duration.sum"] == pytest.approx(0.7565)   # milliseconds
    assert rows[1]["gpu__time_duration.sum"] == pytest.approx(1.0)
    assert TT.read_ncu_csv(str(p), "k_aux")[0]["dram__bytes_read.sum"] == pytest.approx(1.5e6)


def test_entry_is_per_cell_and_stamped_with_the_current_sources(tmp_path):
    p = tmp_path / "cap.csv"
    cells = 2 ** 21
    ncu_csv(p, [
        (5, "void k_collide_w<19>(...)", "dram__bytes_read.sum", "byte", str(1300 * cells)),
        (5, "void k_collide_w<19>(...)", "dram__bytes_write.sum", "byte", str(1200 * cells)),
        (5, "void k_collide_w<19>(...)", "gpu__time_duration.sum", "msecond", "0.75"),
        (5, "void k_collide_w<19>(...)", "smsp__sass_thread_inst_executed_op_dadd_pred_on.sum",
         "inst", str(10 * cells)),
        (5, "void k_collide_w<19>(...)", "smsp__sass_thread_inst_executed_op_dmul_pred_on.sum",
         "inst", str(20 * cells)),
        (5, "void k_collide_w<19>(...)", "smsp__sass_thread_inst_executed_op_dfma_pred_on.sum",
         "inst", str(30 * cells)),
    ])
    out = tmp_path / "table.json"
    assert TT.main([str(p), "--key", "k:w:f", "--cells", str(cells), "--out", str(out),
                    "--captured-on", "test", "--command", "ncu ..."]) == 0
    e = json.loads(out.read_text())["k:w:f"]
    assert e["dram_read_bytes_per_cell"] == 1300.0 and e["dram_write_bytes_per_cell"] == 1200.0
    assert e["dram_bytes_per_cell"] == 2500.0 and e["launch_ms_under_ncu"] == 0.75
    assert e["fp64_instructions_per_cell"] == 60.0
    assert e["fp64_flops_per_cell"] == 10 + 20 + 2 * 30   # a fused multiply-add is two flops
    assert e["source_hash"] == TT.source_hash(TT.COLLIDE_SOURCES)
    # a second capture adds to the same file without touching the first
    assert TT.main([str(p), "--key", "k:w:g", "--cells", str(2 * cells), "--out", str(out),
                    "--captured-on", "test", "--command", "ncu ..."]) == 0
    table = json.loads(out.read_text())
    assert set(table) == {"k:w:f", "k:w:g"}
    assert table["k:w:g"]["dram_bytes_per_cell"] == 1250.0


def test_source_hash_follows_every_byte_of_the_kernel_sources(tmp_path, monkeypatch):
    src = tmp_path / "csrc"
    src.mkdir()
    for n in TT.BATCH_SOURCES:
        (src / n).write_text(f"// {n}\n")
    monkeypatch.setattr(TT, "HERE", str(tmp_path))
    h0 = TT.source_hash(TT.BATCH_SOURCES)
    (src / TT.BATCH_SOURCES[0]).write_text(f"// {TT.BATCH_SOURCES[0]} \n")  # one byte more
    assert TT.source_hash(TT.BATCH_SOURCES) != h0


@pytest.fixture
def bench(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(mod, "ROOT", str(tmp_path))
    return mod


def test_bench_takes_only_entries_captured_on_its_sources(bench, tmp_path):
    current = TT.source_hash(TT.COLLIDE_SOURCES)
    table = {
        "fresh": {"source_hash": current, "dram_bytes_per_cell": 2456.0},
        "stale": {"source_hash": "0" * 16, "dram_bytes_per_cell": 2456.0},
        "restamped": {"source_hash": current, "dram_bytes_per_cell": 2456.0,
                      "sources_note": "counters taken before an edit"},
    }
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    assert bench.traffic_for("fresh", 1000) == pytest.approx(2456.0 * 1000)
    assert bench.traffic_for("stale", 1000) is None
    assert bench.traffic_for("restamped", 1000) is None
    assert bench.traffic_for("absent", 1000) is None
    # the 37-field and batched kernels are checked against their own sources
    assert bench.traffic_for("fresh", 1000, TT.AD_SOURCES) is None


def test_fp64_flop_count_falls_back_to_the_recorded_figure(bench):
    assert bench.profile_entry("absent", "fp64_flops_per_cell") is None
    assert bench.FP64_FLOPS_PER_CELL == 2948.0
