"""Host-side pieces of bench.py, no GPU: whether a clock record is accepted, the peak lookup and the
reference arm's JSON line (the oracle on a small workload)."""
import json
import types

import pytest


def _sampler(tmp_path, rows):
    import bench
    path = tmp_path / "clocks.csv"
    path.write_text("".join(", ".join(r) + "\n" for r in rows))
    s = bench.ClockSampler(0, str(path))
    s.proc = object()  # as if nvidia-smi had run
    return s


def _row(mhz, power="900.0", hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return ["0", str(mhz), "2070", power, "0x0000000000000000", hw, hw_th, sw_th, cap]


def test_clock_summary_median_and_power_cap(tmp_path):
    s = _sampler(tmp_path, [_row(2070), _row(1950, cap="Active"), _row(2040), ["garbage line"]])
    d = s.summary()
    assert d["sm_mhz"] == 2040.0 and d["sm_max_mhz"] == 2070.0
    assert d["reasons"] == ["sw_power_cap"]
    assert d["samples"] == 3 and d["power_w_max"] == 900.0


@pytest.mark.parametrize("field,name", [("hw", "hw_slowdown"), ("hw_th", "hw_thermal_slowdown"),
                                        ("sw_th", "sw_thermal_slowdown")])
def test_clock_summary_names_each_slowdown(tmp_path, field, name):
    s = _sampler(tmp_path, [_row(2070), _row(1500, **{field: "Active"})])
    assert s.summary()["reasons"] == [name]


def test_clock_summary_without_samples(tmp_path):
    import bench
    assert bench.ClockSampler(0, str(tmp_path / "x.csv")).summary()["reasons"] == ["nvidia-smi unavailable"]
    assert _sampler(tmp_path, []).summary()["reasons"] == ["no samples"]


def test_measured_peaks_reads_the_file_else_falls_back(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks("hbm_gbs") == (6800.0, "fallback")
    assert bench.measured_peaks("bf16_tflops") == (1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6758.5}))
    assert bench.measured_peaks("hbm_gbs") == (6758.5, "measured")
    assert bench.measured_peaks("bf16_tflops") == (1900.0, "fallback")


def test_reference_arm_line(capsys, monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    args = types.SimpleNamespace(workload="syc12_3x4_d8", cpu_sample_gates=42, warmup=1, steps=2)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # 8 gates of 2^12 amplitudes per step
    assert line["value"] == pytest.approx(2 * 8 * 4096 / (line["ms_per_step"] * 2 / 1e3))


def test_reference_arm_other_ranks_print_nothing(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(types.SimpleNamespace(workload="syc12_3x4_d8", cpu_sample_gates=42, warmup=1, steps=1))
    assert capsys.readouterr().out == ""


def test_large_cases_plan_on_the_host(monkeypatch):
    """Each --large-case configuration parses, and its workload, sliced sets and phases plan on
    the host (the GPU run itself is not part of this test)."""
    import sys

    import bench
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si
    for name, cfg in bench.LARGE_CASES.items():
        monkeypatch.setattr(sys, "argv", ["bench.py", "--large-case", name])
        assert bench.parse().large_case == name
        circ = si.workload_circuit(name, seed=0)
        n, s = circ.n_qubits, cfg["slice_bits"]
        gates = pkg.gates_array(circ)
        if cfg["sets"] == "chosen":
            set_a, set_b, _, _ = pkg.sim_phases_choose_sets(n, gates, s, kmax=cfg["kmax"])
        else:
            set_a, set_b = list(range(s)), list(range(n - s, n))
        assert len(set_a) == len(set_b) == s and not set(set_a) & set(set_b)
        assert 0 <= cfg["device_regions"] < (1 << s)
        ph = pkg.sim_phases_create(n, gates, s, set_a, set_b, kmax=cfg["kmax"], precision=pkg.SIM_FP16X3_TMEM)
        n_phases, n_blocks = pkg.sim_phases_info(ph)
        pkg.sim_phases_destroy(ph)
        assert n_phases == 4 and n_blocks > 0
