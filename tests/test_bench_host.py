"""Host-side arithmetic of bench.py that decides its JSON line: the clock
summary taken during the timed region, the algorithmic bytes of the step
kernel, and the DRAM-traffic record that holds only for the sources it was
measured on.  CPU only."""
import pytest

import bench


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    s.proc = object()  # summary() reads the file of a sampler that ran
    return s


def test_clock_summary_takes_the_median_under_load(tmp_path):
    na, a = "Not Active", "Active"
    lines = [
        "0, 1980, 2070, 120.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),   # idle: left out
        "0, 2070, 2070, 900.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),
        "0, 2055, 2070, 1200.0, 0x4, %s, %s, %s, %s" % (na, na, na, a),
        "0, 2040, 2070, 1100.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),
        "garbage line",
        "0, [N/A], 2070, 1100.0, 0x0, %s, %s, %s, %s" % (na, na, na, na),
    ]
    out = _sampler(tmp_path, lines).summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["samples"] == 4
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_throttling(tmp_path):
    na, a = "Not Active", "Active"
    lines = ["0, 1500, 2070, 1300.0, 0x8, %s, %s, %s, %s" % (a, na, a, na)]
    out = _sampler(tmp_path, lines).summary()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _sampler(tmp_path, ["nothing"]).summary()["reasons"] == ["no samples"]


def test_step_kernel_bytes():
    # five 4-vectors (position in and out, velocity in and out, build
    # position), bond slots and list count per particle; 4 B per list entry
    assert bench.step_kernel_bytes(1000, 12900, 1) == 1000 * (5 * 16 + 12) + 4 * 12900
    assert bench.step_kernel_bytes(1000, 12900, 2) == 1000 * (5 * 32 + 12) + 4 * 12900
    # the KG melt at about 12.9 entries per bead: 143.5 B per particle-step
    assert bench.step_kernel_bytes(10 ** 6, 12_881_152, 1) / 1e6 == pytest.approx(143.52, abs=0.01)


def test_traffic_record_holds_only_for_its_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "step_kernel_traffic.txt").write_text(
        "# a capture\nk_step_sha: 0123abcd\ndram_bytes_per_particle_step: 150.25\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "step_kernel_digest", lambda: "0123abcd")
    assert bench.read_traffic_record() == 150.25
    monkeypatch.setattr(bench, "step_kernel_digest", lambda: "ffff0000")
    assert bench.read_traffic_record() is None
    (prof / "step_kernel_traffic.txt").unlink()
    assert bench.read_traffic_record() is None


def test_structure_correction_is_an_ibi_step_that_keeps_the_core():
    np = pytest.importorskip("numpy")
    n = 175
    g_t = np.ones(n)
    g = np.ones(n)
    g[60:80] = 1.2           # too many pairs there: the correction must rise
    g[100:120] = 0.8         # too few: it must fall
    counts = np.full(n, 1e4)
    counts[:20] = 0          # an unsampled core
    C = bench._correction_update(np.zeros(n), g, g_t, counts, first_t=10)
    assert np.all(C[:20] == C[20])                     # held below the first reliable bin
    assert C[70] == pytest.approx(0.3 * np.log(1.2), rel=1e-12)
    assert C[110] == pytest.approx(0.3 * np.log(0.8), rel=1e-12)
    assert np.all(np.abs(C[30:50]) < 1e-15)            # no error, no correction
    # corrections accumulate over iterations
    C2 = bench._correction_update(C, g, g_t, counts, first_t=10)
    assert C2[70] == pytest.approx(2 * C[70], rel=1e-12)
