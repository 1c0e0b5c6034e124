"""The ncu launch-list summary used for the committed profiles (host code, no GPU)."""
import csv

from paper_1903_04395_gb300 import ncu_summary


def _write(path, rows):
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(["ID", "Process ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"])
        for r in rows:
            w.writerow(r)


def test_launch_table_groups_by_kernel_and_converts_units(tmp_path):
    p = tmp_path / "launches.csv"
    name_a = "void (anonymous namespace)::k_spmm_u<float, 8, 9>(const int *, int)"
    name_b = "void (anonymous namespace)::k_hist<float, 8>(const int *)"
    _write(p, [
        ["0", "1", name_a, "gpu__time_duration.sum", "msecond", "7.5"],
        ["0", "1", name_a, "dram__bytes_read.sum", "Gbyte", "10.5"],
        ["0", "1", name_a, "dram__bytes_write.sum", "Mbyte", "1,850"],
        ["1", "1", name_b, "gpu__time_duration.sum", "usecond", "550"],
        ["2", "1", name_a, "gpu__time_duration.sum", "nsecond", "7,400,000"],
        ["2", "1", name_a, "dram__bytes_read.sum", "byte", "10000000000"],
    ])
    t = ncu_summary.launch_table(str(p))
    a, b = t["k_spmm_u<float, 8, 9>"], t["k_hist<float, 8>"]
    assert a["launches"] == 2 and abs(a["ms"] - 14.9) < 1e-9
    assert abs(a["read"] - 20.5e9) < 1 and abs(a["write"] - 1.85e9) < 1
    assert b["launches"] == 1 and abs(b["ms"] - 0.55) < 1e-12 and b["read"] == 0.0


def test_launches_prints_shares(tmp_path, capsys):
    p = tmp_path / "launches.csv"
    _write(p, [
        ["0", "1", "void k_color(int)", "gpu__time_duration.sum", "msecond", "1"],
        ["1", "1", "void k_final_sum(int)", "gpu__time_duration.sum", "msecond", "3"],
    ])
    ncu_summary.launches(str(p))
    out = capsys.readouterr().out.splitlines()
    assert out[1].startswith("k_final_sum") and "75.0%" in out[1]
    assert out[2].startswith("k_color") and "25.0%" in out[2]
    assert out[-1].split()[1] == "2"
