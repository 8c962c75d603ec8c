"""Host logic of the benchmark (no GPU): the per-launch unit counts and
algorithmic bytes behind the roofline, the peaks file and its fallback, and
the parsing of the clock samples that decides whether a run is kept."""
import json

import bench


def test_units_per_launch():
    n = (128, 96, 64)
    nx, ny, nz = n
    assert bench.kernel_units("c2p", n) == nx * ny * nz == bench.kernel_units("update", n)
    # faces: every face along d, over the cells and 3 ghost layers across
    assert bench.kernel_units("faces_x", n) == (nx + 1) * (ny + 6) * (nz + 6)
    assert bench.kernel_units("faces_z", n) == (nx + 6) * (ny + 6) * (nz + 1)
    # edges along e: one per owned edge, faces + 1 across
    assert bench.kernel_units("emf_y", n) == (nx + 1) * ny * (nz + 1)
    # the 128^3 capture the traffic per face is taken from
    assert bench.kernel_units("faces_x", (128, 128, 128)) == 2316324


def test_bytes_per_unit():
    # FP64: every value 8 B; FP32: 4 B except the Newton unknown Z (FP64)
    assert bench.kernel_bytes_per_unit("c2p", 64) == 18 * 8
    assert bench.kernel_bytes_per_unit("c2p", 32) == 16 * 4 + 2 * 8
    assert bench.kernel_bytes_per_unit("faces_y", 32) == 19 * 4
    assert bench.kernel_bytes_per_unit("update", 64) == 42 * 8


def test_peaks_file_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.load_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0}))
    peaks, src = bench.load_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 7000.0


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(gpu, sm, mx, w, *reasons):
    flags = ["Active" if r else "Not Active" for r in reasons]
    return f"{gpu}, {sm} MHz, {mx} MHz, {w} W, 0x0, " + ", ".join(flags)


def test_clock_samples_parsed():
    s = bench.ClockSampler(gpu_index=1)
    s.proc = _Proc()
    s.lines = [_row(0, 900, 2070, 100.0, 1, 1, 0, 0),
               _row(1, 2070, 2070, 300.0, 0, 0, 0, 0),
               _row(1, 2055, 2070, 320.5, 0, 0, 0, 1),
               _row(1, 2070, 2070, 310.0, 0, 0, 0, 0),
               "garbage"]
    out = s.stop()
    # only the selected GPU's rows; the other GPU's slowdown is not ours
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["power_w_max"] == 320.5


def test_clock_sampler_without_nvidia_smi():
    out = bench.ClockSampler().stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_flops_from_the_oracle_counts(tmp_path):
    """The roofline numerator: per unit, the counts the oracle's counting
    build wrote; c2p's per-cell part plus its per-iteration part times the
    iterations the inversion took."""
    counts = {"flops_per_unit": {"faces": 480.0, "emf": 250.0}, "update_per_cell": 87.0,
              "c2p_per_cell_fixed": 49.0, "c2p_per_newton_iteration": 55.0}
    assert bench.algorithmic_flops(counts, "faces_y", 3.0) == 480.0
    assert bench.algorithmic_flops(counts, "emf_z", 3.0) == 250.0
    assert bench.algorithmic_flops(counts, "update", 3.0) == 87.0
    assert bench.algorithmic_flops(counts, "c2p", 3.0) == 49.0 + 3 * 55.0
    # the committed file has every figure the numerator needs
    got = bench.load_op_counts()
    for key in ("faces", "emf", "c2p", "assemble", "ct", "rk"):
        assert got["flops_per_unit"][key] > 0.0, key
    assert got["c2p_per_newton_iteration"] > 0.0 and got["update_per_cell"] > 0.0


def test_reference_arm_labels_what_it_times():
    """The reference arm (the oracle on the host cores) names the workload of
    the GPU arm and, in the same label, the sample it actually times."""
    import argparse
    args = argparse.Namespace(size=12, precision=64, steps=1, warmup=1, gpus=1)
    line = bench.run_reference(args, 1, 0)
    assert line["impl"] == "reference" and line["value"] > 0.0
    assert "12^3" in line["config"]["workload"] and "sample" in line["config"]["workload"]
    assert line["config"]["sample_grid"] == [12, 12, 12]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_torus_frame_l1_measure():
    """The torus FP32 line's frame-based L1: zero for equal states; a change
    in one momentum component moves only that component's figure (and not D
    or tau); invariant under a common scale of both states; an S_theta
    change of d in one cell reads d sqrt(gamma^thth) / sum |S| there."""
    import numpy as np
    import bench
    from paper_1810_04597_gb300 import inputs
    prob = inputs.fm_torus((12, 6, 4))
    N = prob.ncells
    rng = np.random.default_rng(3)
    a = rng.normal(size=8 * N + 50)
    assert all(v == 0.0 for v in bench.torus_frame_l1(prob, a, a).values())
    b = a.copy()
    cell = 1 * prob.n[0] * prob.n[1] + 3 * prob.n[0] + 7        # (k, j, i) = (1, 3, 7)
    b[2 * N + cell] += 1e-3                                     # S_theta of that cell
    m = bench.torus_frame_l1(prob, a, b)
    assert m["D"] == 0.0 and m["tau"] == 0.0 and m["S_r"] == 0.0 and m["S_phi"] == 0.0
    x1 = prob.x0[0] + 7.5 * prob.dx[0]
    th = prob.x0[1] + 3.5 * prob.dx[1]
    _, _, g11, g13, g22, g33 = inputs.ks_metric_arrays(np.array([[x1]]), np.array([[th]]), prob.spin)
    X1, TH = np.meshgrid(prob.x0[0] + (np.arange(prob.n[0]) + 0.5) * prob.dx[0],
                         prob.x0[1] + (np.arange(prob.n[1]) + 0.5) * prob.dx[1])
    _, _, G11, G13, G22, G33 = inputs.ks_metric_arrays(X1, TH, prob.spin)
    det = G11 * G33 - G13 ** 2
    S = [a[(1 + q) * N:(2 + q) * N].reshape(prob.n[2], prob.n[1], prob.n[0]) for q in range(3)]
    Smag = np.sqrt(G33 / det * S[0] ** 2 + S[1] ** 2 / G22 + G11 / det * S[2] ** 2 - 2 * G13 / det * S[0] * S[2])
    want = 1e-3 / np.sqrt(g22[0, 0]) / np.sum(Smag)
    assert abs(m["S_theta"] - want) <= 1e-12 * want
    s = bench.torus_frame_l1(prob, 3.0 * a, 3.0 * b)
    assert all(abs(s[k] - m[k]) <= 1e-14 + 1e-12 * m[k] for k in m)


def test_fp64_mix_cap():
    """At the nominal FP64 peak, an FMA-only kernel (2 flop per FP64
    instruction) can reach the whole peak and a DADD-only kernel half of it;
    the listed kernels' caps lie between."""
    import bench
    assert abs(bench.fp64_mix_cap(2.0, 1.0, bench.FP64_PEAK_TFLOPS) - 1.0) < 1e-12
    assert abs(bench.fp64_mix_cap(1.0, 1.0, bench.FP64_PEAK_TFLOPS) - 0.5) < 1e-12
    for prec, fl in bench.FLOPS64.items():
        for k, f in fl.items():
            cap = bench.fp64_mix_cap(f, bench.FP64_INSTR[prec][k], bench.FP64_PEAK_TFLOPS)
            assert 0.5 <= cap <= 1.0, (prec, k, cap)
