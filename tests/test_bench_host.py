"""Host-side bookkeeping of bench.py, on CPU: the algorithmic bytes it credits each force-evaluation
kernel with against the DRAM bytes ncu measured for the same launches (the committed 1024^3 /
2048^3 summary), the per-evaluation floor against those kernels, the clock sampler's
throttle-reason window, and the bench commands the profile summaries give."""
import glob
import json
import os
import re
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_P, NG = 1024, 2048

# kernel of the launch list -> the name bench.py accounts it under
BENCH_NAME = {
    "k_keys_x4": "keys",
    "k_scatter_x4": "scatter",
    "k_deposit_fftx": f"deposit_fftx_{NG}",
    "k_fft_y_fwd_wide": f"fft_cols_{NG}",
    "k_fft_z_green_wide": f"fft_z_green_{NG}",
    "k_fft_y_inv3_wide": f"fft_y_inv3_{NG}",
    "k_fft_x_c2r3": f"fft_x_c2r3_{NG}",
    "k_gather_binned4": "gather_binned4",
    "k_kick_drift4": "kick_drift4",
}


def dram_table():
    """Rows of the DRAM table: kernel -> (read GB, write GB, algorithmic GB)."""
    text = open(os.path.join(ROOT, "profiles", "launches_cola_1024p_2048g.md")).read()
    body = text.split("## DRAM bytes per launch", 1)[1]
    rows = {}
    for m in re.finditer(r"^\| `([^`]+)` \| [\d.]+ \| ([\d.]+) \| ([\d.]+) \| \d+ \| [\d.]+ \| ([\d.]+) \|", body, re.M):
        rows[m.group(1).split("<")[0]] = tuple(float(m.group(i)) for i in (2, 3, 4))
    return rows


def test_every_force_evaluation_kernel_has_a_dram_row():
    assert set(dram_table()) == set(BENCH_NAME)


def test_algorithmic_bytes_agree_with_the_profile_and_stay_below_dram():
    for kernel, (rd, wr, alg_gb) in dram_table().items():
        alg = bench.algorithmic_bytes(BENCH_NAME[kernel], N_P, NG)
        assert alg is not None, kernel
        assert abs(alg / 1e9 - alg_gb) <= 0.006, (kernel, alg / 1e9, alg_gb)
        # the credited bytes are a floor: no launch moved less through DRAM (within ncu's rounding)
        assert (rd + wr) * 1e9 >= 0.99 * alg, (kernel, rd + wr, alg / 1e9)


def test_half_spectrum_passes_count_whole_half_spectra():
    # one half spectrum of a 2048^3 mesh: 2048^2 x 1025 complex64 modes
    h = 2048 * 2048 * 1025 * 8
    assert bench.algorithmic_bytes(f"fft_cols_{NG}", N_P, NG) == 2 * h
    assert bench.algorithmic_bytes(f"fft_z_green_{NG}", N_P, NG) == 3 * h
    assert bench.algorithmic_bytes(f"fft_y_inv3_{NG}", N_P, NG) == 5 * h
    assert bench.algorithmic_bytes(f"fft_x_c2r3_{NG}", N_P, NG) == 3 * (h + 4 * NG**3)


def test_evaluation_floor_is_below_what_the_kernels_must_move():
    floor = bench.eval_floor_bytes(N_P, NG)
    assert floor == 56 * NG**3 + 84 * N_P**3
    moved = sum(bench.algorithmic_bytes(name, N_P, NG) for name in BENCH_NAME.values())
    assert floor < moved


def test_dominant_kernel_traffic_matches_the_dram_table():
    # the traffic bench.py reports for the dominant kernel is the DRAM table's read + write
    data = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))["cola_1024p_2048g_L1000"]
    kernel_of = {name: kernel for kernel, name in BENCH_NAME.items()}
    table = dram_table()
    assert data
    for name, rec in data.items():
        rd, wr, _ = table[kernel_of[name]]
        assert abs(rec["dram_bytes_per_launch"] / 1e9 - (rd + wr)) <= 0.011, name


class _FakeSmi:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_sampler_reads_reasons_inside_the_timed_window_only():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.proc = _FakeSmi()
    na, a = "Not Active", "Active"
    cs.samples = [
        (9.0, ["1200", "2070", "300", a, na, na, na]),      # before the window
        (10.0, ["2070", "2070", "900", na, na, na, na]),
        (10.5, ["1980", "2070", "1400", na, na, na, a]),    # power cap: kept and reported
        (11.0, ["2070", "2070", "1100", na, na, na, na]),
        (14.0, ["600", "2070", "120", na, a, na, na]),      # after the window
    ]
    cs.mark(10.0, 11.0)
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_profile_commands_run_committed_files_with_valid_bench_flags(monkeypatch):
    # every bench command a profile summary was made with still parses, on a known workload
    from paper_1301_0322_gb300 import inputs
    n = 0
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        assert "_work" not in text, path
        for m in re.finditer(r"python bench\.py([^\\`\n#]*)", text):
            monkeypatch.setattr(sys, "argv", ["bench.py"] + m.group(1).split())
            args = bench.parse_args()  # argparse exits on a flag bench.py does not take
            assert args.workload in inputs.WORKLOADS, (path, args.workload)
            n += 1
    assert n > 0
