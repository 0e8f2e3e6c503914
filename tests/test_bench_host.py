"""Host logic of bench.py (no GPU needed).

- The launch-list summary printed from an ncu CSV (`--summarize-ncu`), which the
  committed profile summaries quote: kernel names stripped of their argument lists and
  anonymous namespaces, launches counted, device time summed across units, shares of
  the total, every other metric and every log line ignored.
- The clock record of the timed region, parsed from nvidia-smi's sampling."""
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


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_throttle_reasons(tmp_path):
    """The clock record of the timed region: median SM clock of the benchmarked device,
    its maximum, and the throttle reasons seen Active (other devices and malformed lines
    are skipped), from nvidia-smi's csv,noheader,nounits sampling."""
    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "1, 1200, 2070, 300.0, 0x0000000000000004, Not Active, Active, Not Active, Not Active\n"
        "0, 1965, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    c = bench.Clocks()
    c.proc, c.path = _DoneProcess(), str(path)
    rec = c.stop(dev_index=0)
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
