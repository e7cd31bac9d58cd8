"""Host logic of bench.py that needs no GPU: the DRAM-traffic record behind
roofline.traffic (per-launch averages of single-kernel ncu captures on the
90-station case, scaled to a full-size launch by algorithmic bytes, keyed
by the kernel sources' digest and the workload)."""
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


def _captures(tmp_path, gridder_rows, degridder_rows):
    _write_launch_list(tmp_path / "traffic_gridder.csv", gridder_rows)
    _write_launch_list(tmp_path / "traffic_degridder.csv", degridder_rows)
    return str(tmp_path)


@pytest.fixture(scope="module")
def full_obs(idg_mod):
    from paper_2502_17789_gb300 import synth
    return synth.config(2, seed=0)


def test_record_traffic_scales_per_launch_captures(tmp_path, traffic_file, full_obs):
    """Each kernel's capture (its first launches on the 90-station case) is
    averaged per launch and scaled to a full-size launch by the ratio of
    algorithmic bytes per launch (host-only plans of both workloads)."""
    from paper_2502_17789_gb300 import synth
    g = "void idg::gridder_kernel<96, 8, false, false>(idg::GridArgs)"
    d = "void idg::degridder_kernel<96, 1, false>(idg::DegridArgs)"
    folder = _captures(tmp_path, [
        (0, g, "dram__bytes_read.sum", "Mbyte", "400"), (0, g, "dram__bytes_write.sum", "Gbyte", "1.0"),
        (2, g, "dram__bytes_read.sum", "Mbyte", "200"), (2, g, "dram__bytes_write.sum", "Mbyte", "1,000"),
    ], [
        (3, d, "dram__bytes_read.sum", "Gbyte", "1.05"), (3, d, "dram__bytes_write.sum", "byte", "35000000"),
    ])
    bench.record_traffic(folder, full_obs, "workload A")
    rec = json.loads(traffic_file.read_text())
    assert set(rec) == {"gridder", "degridder"}
    small = synth.config(2, seed=0, n_stations=bench.TRAFFIC_STATIONS)
    for kern, measured, n in (("gridder", (1.4e9 + 1.2e9) / 2, 2), ("degridder", 1.085e9, 1)):
        r = rec[kern]
        assert r["captured_launches"] == n
        assert r["captured_bytes_per_launch"] == pytest.approx(measured)
        alg_small = bench.algorithmic_bytes_per_launch(kern, small, small.subgrid_size)
        alg_full = bench.algorithmic_bytes_per_launch(kern, full_obs, full_obs.subgrid_size)
        assert r["algorithmic_bytes_per_launch"] == pytest.approx(alg_full)
        assert r["dram_bytes_per_launch"] == pytest.approx(measured * alg_full / alg_small)
        assert r["source_sha256"] == bench.source_digest(kern) and r["workload"] == "workload A"
        assert f"-k regex:\"idg::{kern}_kernel<\" -c 2" in r["command"] and "--stations 90" in r["command"]
    # the full-size degridder launch of the MWA-like workload: 3270 subgrids of 96^2 pixels read
    # (32 B each) and their 2.73 M visibilities written (32 B each), on average over 4 batches
    assert rec["degridder"]["algorithmic_bytes_per_launch"] == pytest.approx(
        (13082 * 96 * 96 * 32 + 32 * full_obs.n_vis) / 4)


def test_recorded_traffic_needs_same_sources_and_workload(tmp_path, traffic_file, monkeypatch, full_obs):
    d = "void idg::degridder_kernel<96, 1, false>(idg::DegridArgs)"
    folder = _captures(tmp_path, [], [(0, d, "dram__bytes_read.sum", "Gbyte", "1.0"),
                                      (0, d, "dram__bytes_write.sum", "Mbyte", "100")])
    bench.record_traffic(folder, full_obs, "workload A")
    got = bench.recorded_traffic("degridder", "workload A")
    assert got is not None and got > 1e9
    assert bench.recorded_traffic("degridder", "workload B") is None
    assert bench.recorded_traffic("gridder", "workload A") is None       # no gridder launch recorded
    monkeypatch.setattr(bench, "source_digest", lambda kern: "0" * 64)  # the sources changed since
    assert bench.recorded_traffic("degridder", "workload A") is None


def test_recorded_traffic_without_a_record(traffic_file):
    assert not traffic_file.exists()
    assert bench.recorded_traffic("degridder", "workload A") is None


def test_tensor_core_kernels_recorded_under_their_own_names(tmp_path, traffic_file, full_obs):
    """The tensor-core kernels have their own traffic entries; the gridder's
    capture ignores degridder rows whose name contains its own."""
    assert bench.kernel_of("gridder", 1) == "gridder" and bench.kernel_of("gridder", 3) == "gridder"
    assert bench.kernel_of("gridder", 2) == "gridder_tc"
    assert bench.kernel_of("degridder", 1) == "degridder"
    assert bench.kernel_of("degridder", 2) == bench.kernel_of("degridder", 3) == "degridder_tc"
    gt = "void idg::gridder_tc_kernel<96, false>(idg::GridArgs)"
    dt = "void idg::degridder_tc_kernel<96, false>(idg::DegridArgs)"
    _write_launch_list(tmp_path / "traffic_gridder_tc.csv", [
        (0, gt, "dram__bytes_read.sum", "Mbyte", "300"), (0, gt, "dram__bytes_write.sum", "Gbyte", "1.0"),
        (1, dt, "dram__bytes_read.sum", "Gbyte", "9.0"), (1, dt, "dram__bytes_write.sum", "Gbyte", "9.0")])
    _write_launch_list(tmp_path / "traffic_degridder_tc.csv", [
        (0, dt, "dram__bytes_read.sum", "Gbyte", "1.0"), (0, dt, "dram__bytes_write.sum", "Mbyte", "90")])
    bench.record_traffic(str(tmp_path), full_obs, "workload A")
    rec = json.loads(traffic_file.read_text())
    assert set(rec) == {"gridder_tc", "degridder_tc"}
    assert rec["gridder_tc"]["captured_launches"] == 1
    assert rec["gridder_tc"]["captured_bytes_per_launch"] == pytest.approx(1.3e9)
    assert rec["degridder_tc"]["captured_bytes_per_launch"] == pytest.approx(1.09e9)
    assert bench.recorded_traffic("degridder_tc", "workload A") is not None


def test_traffic_recipe_runs_the_kernel_it_captures():
    """Each kernel's capture command runs the bench with the MAC unit whose
    plan launches that kernel, and names the kernel exactly."""
    for mac in (1, 2, 3):
        for kind in ("gridder", "degridder"):
            kern = bench.kernel_of(kind, mac)
            cmd = bench.ncu_traffic_command(kern)
            assert f'regex:"idg::{kern}_kernel<"' in cmd
            chosen = int(cmd.split("--mac-unit ")[1].split()[0]) if "--mac-unit" in cmd else 2  # the default plan
            assert bench.kernel_of(kind, chosen) == kern
            assert "--clock-control none" in cmd and "-c 2" in cmd
