"""Host-side logic of bench.py and of the learned-correction driver (no GPU):
the pencil count and FFT flop model behind the reported roofline, the clock-record
parsing that decides whether a run is kept, the peak lookup, the residual
statistics of the learned entry, and the seeded mock sizes."""
import json
import math
import types

import numpy as np
import pytest

import bench


def _plan(n, box_len, k_min, dk, n_bins):
    cfg = types.SimpleNamespace(box_len=box_len, n_mesh=n, k_min=k_min, dk=dk, n_bins=n_bins)
    return types.SimpleNamespace(cfg=cfg)


def _pencils_brute(n, box_len, k_min, dk, n_bins):
    """(k_y, k_z >= 0) pairs with a kept shell reachable along k_x, by enumeration."""
    kf = 2 * math.pi / box_len
    n2s = [m for m in range(1, (n // 2) ** 2)
           if kf * math.sqrt(m) < kf * n / 2 and 0 <= math.floor((kf * math.sqrt(m) - k_min) / dk) < n_bins]
    n2_hi = max(n2s) + 1
    pairs = [(ky, kz) for kz in range(n) for ky in range(-n, n + 1) if ky * ky + kz * kz < n2_hi]
    return len(pairs), max(kz for _, kz in pairs) + 1


@pytest.mark.parametrize("n,box,k_min,dk,nb", [(32, 500.0, 0.0, 0.01, 21), (64, 1000.0, 0.0, 0.007, 25),
                                               (96, 700.0, 0.02, 0.01, 30), (128, 3500.0, 0.0, 0.01, 11)])
def test_plan_pencils_matches_enumeration(n, box, k_min, dk, nb):
    got = bench.plan_pencils(_plan(n, box, k_min, dk, nb), with_nzc=True)
    assert got == _pencils_brute(n, box, k_min, dk, nb)


def test_survey_pencils_and_flops():
    # the 512^3 survey workload: box 3500 Mpc/h, shells of 0.01 to 0.4 h/Mpc
    n_p, nzc = bench.plan_pencils(_plan(512, 3500.0, 0.0, 0.01, 40), with_nzc=True)
    assert (n_p, nzc) == (78217, 223)
    line = 5 * 512 * 9
    assert bench.fft_flops("yz_stage", 512, 2, n_p, nzc) == line * (2 * 512 * 512 * 8 + 2 * 512 * nzc * 16)
    assert bench.fft_flops("x_combine", 512, 2, n_p, nzc) == line * 2 * 9 * n_p
    assert bench.fft_flops("tile_deposit", 512, 2, n_p, nzc) == 0.0
    b = bench.alg_bytes(10_000_000, 50_000_000, 512, 2, 9, n_p)
    assert b == 14_641_049_600
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.54784)


def _sampler(tmp_path, lines):
    f = tmp_path / "clocks.csv"
    f.write_text("\n".join(lines) + "\n")
    s = bench.ClockSampler(0)
    s.proc = object()
    s.file = open(f, "a+")
    return s


def test_clock_summary_median_and_reasons(tmp_path):
    s = _sampler(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal(tmp_path):
    s = _sampler(tmp_path, ["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"])
    assert s.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_peaks_prefers_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6778.0, "bf16_tflops": 1900.0}))
    assert bench._peaks() == (6778.0, "measured")


def test_residual_stats_of_learned_entry():
    torch = pytest.importorskip("torch")
    from paper_1505_05341_gb300 import learned
    nb = learned.N_BINS
    stride = 5 * nb + 5
    rows = np.zeros((2, stride))
    rows[:, nb:2 * nb] = 10                       # modes in every shell
    rows[:, 2 * nb:3 * nb] = 300.0                # P0
    rows[:, 5 * nb + 2] = 100.0                   # S/I, so D = 400
    fine = rows.copy()
    fine[:, 2 * nb:3 * nb] += 4.0                 # P0 off by 1 % of D everywhere
    fine[1, 4 * nb + 3] = 40.0                    # one P4 shell off by 10 % of D
    st = learned.residual_stats(torch.from_numpy(rows), torch.from_numpy(fine))
    assert st["rms0"] == pytest.approx(0.01) and st["max0"] == pytest.approx(0.01)
    assert st["rms2"] == 0.0
    assert st["max4"] == pytest.approx(0.1)
    assert st["rms4"] == pytest.approx(math.sqrt(0.01 / (2 * nb)))
    same = learned.residual_stats(torch.from_numpy(rows), torch.from_numpy(rows))
    assert all(v == 0.0 for v in same.values())


def test_mock_sizes_are_seeded_and_in_range():
    import synth.gpu as sg
    a = [sg.mock_sizes(s) for s in range(10_000, 10_050)]
    assert a == [sg.mock_sizes(s) for s in range(10_000, 10_050)]
    assert all(200_000 <= g <= 2_000_000 and r == 5 * g for g, r in a)
    assert len({g for g, _ in a}) > 45


@pytest.mark.parametrize("k_max,box,n", [(0.2, 500.0, 32), (0.05, 1000.0, 64), (10.0, 300.0, 16)])
def test_half_mode_count_matches_binning(k_max, box, n):
    """The mode count behind the galaxy-sum extrapolation equals the oracle's
    half-grid mode weights (Hermitian weight 2 counted as two modes, halved)."""
    from oracle.binning import BinSpec, mode_bins
    kn = math.pi * n / box
    top = min(k_max, kn)
    bins = BinSpec(0.0, top / 7, 7)
    bidx, w, _ = mode_bins(n, box, bins)
    want = float(np.sum(w[bidx >= 0])) / 2
    assert bench.half_modes_below(k_max, box, n) == pytest.approx(want)


@pytest.mark.parametrize("n,m,groups,launches", [(512, 2, 9, 1), (256, 1, 4, 2), (128, 2, 1, 3)])
def test_kernel_bytes_add_up_to_the_step(n, m, groups, launches):
    """The per-kernel algorithmic bytes behind the roofline add up to the step's: the
    deposit writes each mesh, the y,z stage reads it and writes the grouped pencils
    (split over its launches), the x stage reads them, and the particles are read once."""
    ng, nr, npen = 1_000_000, 5_000_000, 12_345
    per_step = (bench.kernel_bytes("tile_deposit", ng, nr, n, m, groups, npen, 1, None)
                + launches * bench.kernel_bytes("yz_stage", ng, nr, n, m, groups, npen, launches, None)
                + bench.kernel_bytes("x_combine", ng, nr, n, m, groups, npen, 1, None)
                + 16 * (ng + nr))
    assert per_step == pytest.approx(bench.alg_bytes(ng, nr, n, m, groups, npen), rel=1e-12)
    # the counting launches (one per catalogue) read x, y, z, w and the randoms' nbar
    assert 2 * bench.kernel_bytes("particle_count", ng, nr, n, m, groups, npen, 1, None) == 16 * (ng + nr) + 4 * nr
    assert bench.kernel_bytes("finalize", ng, nr, n, m, groups, npen, 1, None) == 0.0


def test_seeds_record_matches_the_workload_seeds():
    assert bench.seeds_record(0) == {"galaxies": 4, "randoms": 5, "rank": 0,
                                     "other_ranks": "both seeds + 100 per rank"}
    r = bench.seeds_record(3, "cone256_tsc_il")
    assert (r["galaxies"], r["randoms"]) == bench.rank_seeds(3, "cone256_tsc_il") == (302, 303)
