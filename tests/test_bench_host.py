"""Host-side logic of bench.py (no GPU): the instruction-count table it reads
its roofline numerators from, and the summary that writes that table from an
ncu capture."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_count_table_is_current():
    """The committed count table was taken on the kernels as they are now: a
    code change to any elementwise kernel source fails this test until the
    table is captured again (the command is in the table's file)."""
    counts, stamp = bench.load_counts()
    assert stamp is not None, f"{bench.COUNTS_FILE} has no kernel source hash"
    assert stamp == bench.kernel_source_hash(), (
        f"the elementwise kernels changed since {os.path.basename(bench.COUNTS_FILE)} was captured: capture it again")
    for f in bench.FUNCS:
        assert f in counts, f"no counts for {f}"
        c = counts[f]
        assert c["alu"] > 0 and c["fp64"] > 0 and c["inst"] >= c["alu"] + c["fp64"]
        # at the capture's n = 2^24 part of the output is still in L2 when a launch ends
        assert 0.85 * bench.BYTES_PER_ELEM[f] <= c["traffic_per_elem"] <= 1.2 * bench.BYTES_PER_ELEM[f]


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    src = tmp_path / "paper_1502_05216_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (src / name).write_text("int a = 1; // one\n/* block */ int b;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (src / "tf_core.cuh").write_text("int a = 1; // another comment\n/* other */   int b;\n")
    assert bench.kernel_source_hash() == h0
    (src / "tf_core.cuh").write_text("int a = 2;\nint b;\n")
    assert bench.kernel_source_hash() != h0


def test_ncu_summary_parses_a_capture(tmp_path, monkeypatch):
    """The summary of a (synthetic) ncu --csv capture: the first launch of each
    kernel, per-element counts = warp instructions x 32 / n, DRAM bytes per
    element, and a table load_counts reads back."""
    hdr = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')
    n = 1 << 20
    vals = {"gpu__time_duration.sum": ("msecond", "0.05"), "dram__bytes_read.sum": ("Mbyte", "16.78"),
            "dram__bytes_write.sum": ("Mbyte", "16.78"), "sm__inst_executed_pipe_alu.sum": ("inst", str(10 * n)),
            "sm__inst_executed_pipe_fp64.sum": ("inst", str(n // 4)), "sm__inst_executed_pipe_fma.sum": ("inst", "0"),
            "smsp__inst_executed.sum": ("inst", str(20 * n)),
            "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active": ("%", "71.5"),
            "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active": ("%", "60.2")}
    lines = [hdr]
    for i, kern in enumerate(["(anonymous namespace)::unary_v2<(anonymous namespace)::OpExp>(const double *, ...)",
                              "(anonymous namespace)::unary_v2<(anonymous namespace)::OpExp>(const double *, ...)",
                              "(anonymous namespace)::binary_v2<(anonymous namespace)::OpMul>(const double *, ...)"]):
        for k, (u, v) in vals.items():
            v2 = str(float(v) * (2 if i == 1 else 1))  # the second texp launch must be ignored
            lines.append(f'"{i}","1","python","h","{kern}","1","7","(256, 1, 1)","(64, 1, 1)","0","10.3","",'
                         f'"{k}","{u}","{v2}"')
    csvp = tmp_path / "c.csv"
    csvp.write_text("==PROF== noise\n" + "\n".join(lines) + "\n")
    old = bench.N_FOR_SUMMARY[0]
    bench.N_FOR_SUMMARY[0] = n
    try:
        table = bench.ncu_summary(str(csvp))
    finally:
        bench.N_FOR_SUMMARY[0] = old
    md = tmp_path / "t.md"
    md.write_text(table + "\n")
    counts, stamp = bench.load_counts(str(md))
    assert stamp == bench.kernel_source_hash()
    assert set(counts) == {"texp", "tmul"}
    assert counts["texp"]["alu"] == pytest.approx(320.0)
    assert counts["texp"]["fp64"] == pytest.approx(8.0)
    assert counts["texp"]["inst"] == pytest.approx(640.0)
    assert counts["texp"]["traffic_per_elem"] == pytest.approx(2 * 16.78e6 / n, rel=1e-3)
