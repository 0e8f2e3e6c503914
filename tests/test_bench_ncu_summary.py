"""The launch-list summary bench.py prints from an ncu CSV (`--summarize-ncu`), which
the committed profile summaries quote: kernel names stripped of their argument lists
and anonymous namespaces, launches counted, device time summed across units, shares
of the total, and every other metric and every log line ignored (no GPU needed)."""
import bench

CSV = '''==PROF== Connected to process 1 (/usr/bin/python3)
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python3","127.0.0.1","void <unnamed>::k_patch_warp<3, float, __nv_bfloat16, 2, 0, 2>(<unnamed>::PatchArgs)","1","7","(512, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ms","3.000"
"1","1","python3","127.0.0.1","void (anonymous namespace)::k_patch_sum<float>(int, int, int, int, int, const float *, long long, const double *, float *)","1","7","(256, 1, 1)","(9, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","500"
"2","1","python3","127.0.0.1","void <unnamed>::k_patch_warp<3, float, __nv_bfloat16, 2, 0, 2>(<unnamed>::PatchArgs)","1","7","(512, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","1,500,000"
"2","1","python3","127.0.0.1","void <unnamed>::k_patch_warp<3, float, __nv_bfloat16, 2, 0, 2>(<unnamed>::PatchArgs)","1","7","(512, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","1154188032"
==PROF== Disconnected from process 1
'''


def test_summary_of_a_launch_list(tmp_path):
    path = tmp_path / "launches.csv"
    path.write_text(CSV)
    lines = bench.summarize_ncu_launches(str(path)).splitlines()
    rows = {ln[:70].strip(): ln[70:].split() for ln in lines[1:]}
    assert rows["k_patch_warp<3, float, __nv_bfloat16, 2, 0, 2>"] == ["2", "4.500", "90.00%"]
    assert rows["k_patch_sum<float>"] == ["1", "0.500", "10.00%"]
    assert rows["all"] == ["3", "5.000"]
    assert len(rows) == 3          # the DRAM metric row is not a launch


def test_summary_rejects_a_file_without_the_csv_header(tmp_path):
    import pytest
    path = tmp_path / "log.txt"
    path.write_text("==PROF== nothing here\n")
    with pytest.raises(ValueError):
        bench.summarize_ncu_launches(str(path))
