"""Host logic of bench.py that needs no GPU: the DRAM-traffic record behind
roofline.traffic (per-launch averages from an ncu launch list, keyed by the
kernel sources' digest and the workload)."""
import csv
import json

import pytest

import bench


def _write_launch_list(path, rows):
    """An ncu --csv launch list: a preamble line, the header, one row per
    (launch, metric)."""
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.writer(f)
        w.writerow(["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
                    "Section Name", "Metric Name", "Metric Unit", "Metric Value"])
        for launch, kernel, metric, unit, value in rows:
            w.writerow([str(launch), "1", "python", "box", kernel, "1", "7", "Command line profiler metrics",
                        metric, unit, value])


@pytest.fixture()
def traffic_file(tmp_path, monkeypatch):
    path = tmp_path / "kernel_traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    return path


def test_record_traffic_averages_per_launch(tmp_path, traffic_file):
    g = "void idg::gridder_kernel<96, 8, 0, 0>(idg::GridArgs)"
    d = "void idg::degridder_kernel<96, 0>(idg::DegridArgs)"
    rows = [
        (0, g, "dram__bytes_read.sum", "Mbyte", "400"), (0, g, "dram__bytes_write.sum", "Gbyte", "1.0"),
        (0, g, "gpu__time_duration.sum", "msecond", "21.2"),
        (1, "void idg::fft_adder_kernel<96, 0>(idg::FftArgs)", "dram__bytes_read.sum", "Gbyte", "1.0"),
        (2, g, "dram__bytes_read.sum", "Mbyte", "200"), (2, g, "dram__bytes_write.sum", "Mbyte", "1,000"),
        (3, d, "dram__bytes_read.sum", "Gbyte", "1.05"), (3, d, "dram__bytes_write.sum", "byte", "35000000"),
        (4, "void idg::gridder_noalloc_kernel<96>(idg::GridArgs)", "dram__bytes_read.sum", "Gbyte", "9"),
    ]
    csv_path = tmp_path / "launches.csv"
    _write_launch_list(csv_path, rows)
    bench.record_traffic(str(csv_path), "workload A", "the command")
    rec = json.loads(traffic_file.read_text())
    assert set(rec) == {"gridder", "degridder"}
    assert rec["gridder"]["launches"] == 2
    assert rec["gridder"]["dram_bytes_per_launch"] == pytest.approx((1.4e9 + 1.2e9) / 2)
    assert rec["degridder"]["launches"] == 1
    assert rec["degridder"]["dram_bytes_per_launch"] == pytest.approx(1.085e9)
    for k in ("gridder", "degridder"):
        assert rec[k]["source_sha256"] == bench.source_digest(k)
        assert rec[k]["workload"] == "workload A" and rec[k]["command"] == "the command"


def test_recorded_traffic_needs_same_sources_and_workload(tmp_path, traffic_file, monkeypatch):
    d = "void idg::degridder_kernel<96, 0>(idg::DegridArgs)"
    csv_path = tmp_path / "launches.csv"
    _write_launch_list(csv_path, [(0, d, "dram__bytes_read.sum", "Gbyte", "1.0"),
                                  (0, d, "dram__bytes_write.sum", "Mbyte", "100")])
    bench.record_traffic(str(csv_path), "workload A", "cmd")
    assert bench.recorded_traffic("degridder", "workload A") == pytest.approx(1.1e9)
    assert bench.recorded_traffic("degridder", "workload B") is None
    assert bench.recorded_traffic("gridder", "workload A") is None       # no gridder launch recorded
    monkeypatch.setattr(bench, "source_digest", lambda kern: "0" * 64)  # the sources changed since
    assert bench.recorded_traffic("degridder", "workload A") is None


def test_recorded_traffic_without_a_record(traffic_file):
    assert not traffic_file.exists()
    assert bench.recorded_traffic("degridder", "workload A") is None
