"""Host logic of bench.py on CPU: the algorithmic work behind every roofline figure, the
clock-record parsing that decides whether a run is kept, and the whole-job throughput.

The per-launch work is checked against the sizes written out independently here (a_lm
count, ring pairs, pixels), so that a wrong factor in the bench's table (a dropped parity,
a complex counted as one float, launches per step) fails.
"""
import pytest

import bench

L, R, NPHI, P, CHUNK = 2000, 2001, 4096, 16, 32
N_MAX, N_PAIR = 816, 136
PEAKS = {"hbm_gbs": 6683.8, "bf16_tflops_sustained": 1710.9}


def _prof(ms=10.0):
    stages = ["legendre", "legendre_adjoint", "ring_c2r", "ring_r2c", "adjoint_pixel", "cubic", "linear_term",
              "pair_means", "legendre_prep", "legendre_adjoint_prep"]
    return {s: (ms, 1) for s in stages}


def _by_stage(rows):
    return {r["stage"]: r for r in rows}


def test_algorithmic_work_per_launch_at_the_bench_workload():
    rows = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, _prof(), 1, PEAKS))
    n_alm = 2001 * 2002 // 2                       # m >= 0 entries, l <= 2000
    pairs_of_rings = 1001                          # 1000 north/south pairs and the equator
    npix = 2001 * 4096
    # each (l, m, ring pair) is one multiply-add (2 flop) into re/im of P outputs of one parity
    legendre = 2 * 2 * P * n_alm * pairs_of_rings * CHUNK
    assert float(rows["legendre"]["per_launch"].split()[0]) == pytest.approx(legendre, rel=1e-3)
    assert float(rows["legendre_adjoint"]["per_launch"].split()[0]) == pytest.approx(legendre, rel=1e-3)
    # ring FFT: E and O complex64 rows in (16 B per (m, ring pair)), float maps out
    c2r = (CHUNK * P * pairs_of_rings * (L + 1) * 16 + CHUNK * P * npix * 4) / 1e9
    assert float(rows["ring_c2r"]["per_launch"].split()[0]) == pytest.approx(c2r, rel=1e-3)
    assert float(rows["ring_r2c"]["per_launch"].split()[0]) == pytest.approx(c2r, rel=1e-3)
    assert c2r == pytest.approx(33.19, abs=0.01)
    # cubic: one multiply-add per mode and pixel; adjoint: per pair, basis function, pixel
    assert float(rows["cubic"]["per_launch"].split()[0]) == pytest.approx(2 * N_MAX * npix * CHUNK, rel=1e-3)
    # linear term of a split plan: the pair-mean table (complex64 per pair and a_lm) and the a_lm
    lin = (N_PAIR + CHUNK) * n_alm * 8 / 1e9
    assert rows["linear_term"]["bound"] == "hbm"
    assert float(rows["linear_term"]["per_launch"].split()[0]) == pytest.approx(lin, rel=1e-3)
    # the FP32 plan's pixel-space product: one multiply-add per pair, basis function and pixel
    f32 = _by_stage(bench.stage_rooflines("fp32", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, _prof(), 1, PEAKS))
    assert float(f32["linear_term"]["per_launch"].split()[0]) == pytest.approx(2 * N_PAIR * P * npix * CHUNK,
                                                                              rel=1e-3)
    assert float(rows["adjoint_pixel"]["per_launch"].split()[0]) == pytest.approx(2 * P * N_PAIR * npix * CHUNK,
                                                                                 rel=1e-3)
    # pair sums: the maps once, the FP64 sums read and written
    pm = (CHUNK * P * npix * 4 + 2 * N_PAIR * npix * 8) / 1e9
    assert float(rows["pair_means"]["per_launch"].split()[0]) == pytest.approx(pm, rel=1e-3)
    # operand preparation: a_lm in (complex64), hi and lo FP16 copies of 2P real columns out
    prep = (CHUNK * n_alm * 8 + CHUNK * 2 * P * n_alm * 2 * 2) / 1e9
    assert float(rows["legendre_prep"]["per_launch"].split()[0]) == pytest.approx(prep, rel=1e-3)


def test_launches_per_step_and_achieved_rates():
    prof = _prof(ms=30.0)
    three = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, prof, 1, PEAKS))
    two = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, prof, 1, PEAKS,
                                          nsynth=2))
    for s in ("legendre", "ring_c2r", "legendre_prep"):
        assert three[s]["launches_per_step"] == 3 and two[s]["launches_per_step"] == 2
    for s in ("cubic", "ring_r2c", "adjoint_pixel", "legendre_adjoint"):
        assert three[s]["launches_per_step"] == two[s]["launches_per_step"] == 1
    # 64 maps in chunks of 32: every stage runs twice as often
    six = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, 64, prof, 1, PEAKS))
    assert six["legendre"]["launches_per_step"] == 6 and six["cubic"]["launches_per_step"] == 2
    # achieved = work per step / stage time; fraction against the stated peak
    c2r = three["ring_c2r"]
    gb = float(c2r["per_launch"].split()[0])
    assert c2r["achieved"] == pytest.approx(3 * gb / 0.030, rel=1e-3)
    assert c2r["peak"] == pytest.approx(6683.8) and c2r["frac"] == pytest.approx(c2r["achieved"] / 6683.8, rel=1e-3)
    # split FP16 runs three products per useful multiply-add; 3xTF32 at half the bf16 rate, three products
    assert three["legendre"]["peak"] == pytest.approx(1710.9 / 3, rel=1e-3)
    assert three["adjoint_pixel"]["peak"] == pytest.approx(1710.9 / 6, rel=1e-3)
    assert three["cubic"]["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12, rel=1e-3)
    # rows come largest time first, and stages that did not run are left out
    prof2 = dict(prof)
    prof2["cubic"] = (90.0, 1)
    del prof2["ring_r2c"]
    rows = bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, prof2, 1, PEAKS)
    assert rows[0]["stage"] == "cubic" and "ring_r2c" not in _by_stage(rows)


def test_traffic_only_for_the_captured_workload():
    rows = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, _prof(), 1, PEAKS))
    assert rows["ring_c2r"]["traffic"] == pytest.approx(16.52 + 16.74, abs=0.01)
    assert rows["linear_term"]["traffic"] == pytest.approx(2.815, abs=0.01)
    small = _by_stage(bench.stage_rooflines("fp16x3", 1000, 1001, 2048, P, N_MAX, N_PAIR, 8, 8, _prof(), 1, PEAKS))
    assert all(r["traffic"] is None for r in small.values())


def test_clock_record_flags_slowdowns():
    c = bench.ClockSampler(0)
    # clocks.sm, clocks.max.sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    c.lines = [
        "2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1995, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 950.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # unreadable sample
        "garbage",
    ]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == pytest.approx(2070.0)
    assert s["sm_max_mhz"] == pytest.approx(2070.0)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_job_throughput_is_whole_job_maps_per_second():
    assert bench.job_throughput(32, 4, 1, 160.0) == pytest.approx(32 * 4 / 0.160)
    assert bench.job_throughput(32, 4, 8, 160.0) == pytest.approx(8 * 32 * 4 / 0.160)


def test_probed_peaks_replace_the_derived_ones():
    """With the library's throughput probes of this run, the FP32-SIMT stages use the probed
    FP32 rate and the 3xTF32 stages a third of the probed tf32 tensor rate; the split-FP16
    stages keep the sustained bf16 figure of the measured-peaks file."""
    probe = {"fp32_simt": 70.0, "tf32_tensor": 900.0}
    rows = _by_stage(bench.stage_rooflines("fp16x3", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, _prof(), 1, PEAKS,
                                           probe=probe))
    assert rows["cubic"]["peak"] == pytest.approx(70.0)
    assert rows["adjoint_pixel"]["peak"] == pytest.approx(300.0)
    assert rows["legendre"]["peak"] == pytest.approx(1710.9 / 3, rel=1e-3)
    assert "measured in this run" in rows["cubic"]["peak_source"]
    tf = _by_stage(bench.stage_rooflines("3xtf32", L, R, NPHI, P, N_MAX, N_PAIR, CHUNK, CHUNK, _prof(), 1, PEAKS,
                                         probe=probe))
    assert tf["legendre"]["peak"] == pytest.approx(300.0)


def test_no_function_reads_an_undefined_global():
    """Every global name a function of bench.py or of the Python package reads is defined at
    module level or built in (a stray name fails only when its workload runs on a GPU)."""
    import builtins
    import os
    import symtable
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for rel in ("bench.py", "__graft_entry__.py", "paper_1105_2791_gb300/modal.py",
                "paper_1105_2791_gb300/binding.py", "paper_1105_2791_gb300/tuning.py"):
        top = symtable.symtable(open(os.path.join(root, rel)).read(), rel, "exec")
        defined = set(top.get_identifiers())
        bad = []

        def walk(t):
            for sym in t.get_symbols():
                name = sym.get_name()
                if sym.is_global() and sym.is_referenced() and name not in defined and not hasattr(builtins, name):
                    bad.append((t.get_name(), name))
            for child in t.get_children():
                walk(child)

        walk(top)
        assert not bad, (rel, bad)
