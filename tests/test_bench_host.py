"""Host logic of the benchmark (no GPU): the summary of a one-pass ncu capture
that gives the traversal pass's DRAM bytes per ray, and the check that ties a
stored summary to the kernel sources it was taken on."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEAD = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
       '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'


def _row(i, kernel, metric, unit, value):
    return f'"{i}","1","python","h","{kernel}","1","7","(256, 1, 1)","(1216, 1, 1)","0","10.3",' \
           f'"Command line profiler metrics","{metric}","{unit}","{value}"\n'


TIMED = "void <unnamed>::k_wf_trace<0, 0, 0, 0>(DevScene, WfParams, const unsigned int *)"
COUNTING = "void <unnamed>::k_wf_trace<0, 1, 0, 0>(DevScene, WfParams, const unsigned int *)"


def test_profile_summary_sums_the_timed_launches_only(tmp_path):
    csv = tmp_path / "trace_dram.csv"
    rows = ["==PROF== Connected to process 1\n", HEAD]
    for i, (k, rd, wr, us) in enumerate([(TIMED, "1,000.00", "250.00", "800.50"),
                                         (TIMED, "2.00", "0.50", "1,200.00"),
                                         (COUNTING, "9,999.00", "9,999.00", "99,999.00")]):
        rd_unit = "Gbyte" if i == 1 else "Mbyte"
        rows += [_row(i, k, "dram__bytes_read.sum", rd_unit, rd),
                 _row(i, k, "dram__bytes_write.sum", rd_unit, wr),
                 _row(i, k, "gpu__time_duration.sum", "usecond", us)]
    rows.append(_row(3, "void k_wf_shade<0>(DevScene)", "dram__bytes_read.sum", "Mbyte", "5.00"))
    csv.write_text("".join(rows))
    log = tmp_path / "trace.log"
    log.write_text("building\n" + json.dumps({"profile_case": "trace", "rays": 1000000, "paths": 10}) + "\n")
    out = tmp_path / "prof.json"
    # a stored summary's ncu --set full issue figures are carried over
    out.write_text(json.dumps({"issue": {"threads_per_executed_instruction": 8.86}}))
    bench.profile_summary(str(csv), str(log), str(out))
    d = json.load(open(out))
    assert d["launches"] == 2
    assert d["rays"] == 1000000
    assert abs(d["dram_bytes_read"] - (1000e6 + 2e9)) < 1
    assert abs(d["dram_bytes_write"] - (250e6 + 0.5e9)) < 1
    assert abs(d["gpu_time_ms_serialised"] - 2.0005) < 1e-9
    assert abs(d["dram_bytes_per_ray"] - (3750e6 / 1e6)) < 1e-9
    assert d["issue"] == {"threads_per_executed_instruction": 8.86}
    assert d["kernel_hash"] == bench._kernel_hash()


def test_stored_profile_is_used_only_at_its_kernel_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.json").write_text(json.dumps({"kernel_hash": "abc", "dram_bytes_per_ray": 87.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profile("abc", "x")["dram_bytes_per_ray"] == 87.0
    assert bench._profile("def", "x") is None
    assert bench._profile("abc", "missing") is None
