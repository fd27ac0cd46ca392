"""The benchmark's reference arm keeps the JSON-line contract on a machine without a GPU: one line with
impl = reference, the metric, unit and config of the GPU arm, a CPU baseline that states its cores and
sample, an end-to-end figure with no host-device copies, and an extrapolated per-step time that says so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-seconds", "2"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    res = json.loads(lines[0])
    assert res["impl"] == "reference" and res["unit"] == "field·screen steps/s" and res["value"] > 0
    assert res["metric"].startswith("field·screen steps/s at N=1024")
    assert res["config"]["workload"].startswith("ar-evolution N=1024")
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == res["value"]
    assert res["e2e"] == {"value": res["value"], "unit": res["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "extrapolated" in res["ms_per_step_note"] and res["samples_timed"] == 1


def test_monte_carlo_theory_column_follows_the_oracle_amplitudes():
    # the bench reports SI and W_LT per Cn^2 beside theory computed in numpy from the phase PSD; the
    # same sums over the oracle's FP64 amplitudes (psd_amplitude, sh_amplitude) must agree
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    from paper_2604_07248_gb300 import workloads as W

    K = 2 * np.pi / W.LAMBDA
    for cn2 in (W.config2_cn2()[0], W.config2_cn2()[5]):
        wl = W.config2(cn2)
        got = bench.mc_theory(cn2, wl, 3)
        dz = wl.L / wl.S
        md = O.medium(W.LAMBDA, wl.N, wl.dx, l0=W.L0_INNER, L0=W.L0_OUTER)
        s2 = O.psd_amplitude(md, cn2, dz) ** 2
        f = np.fft.fftfreq(wl.N, 1 / wl.N) * 2 * np.pi / (wl.N * wl.dx)
        k2 = f[None, :] ** 2 + f[:, None] ** 2
        d = [wl.L - s * dz for s in range(1, wl.S + 1)]
        rytov = sum(4 * np.sum(s2 * np.sin(k2 * ds / (2 * K)) ** 2) for ds in d)
        grad2 = np.sum(k2 * s2)
        b = O.sh_amplitude(md, cn2, dz)
        dk = 2 * np.pi / (wl.N * wl.dx)
        for p in range(1, 4):
            for q in range(9):
                grad2 += (((q % 3 - 1) ** 2 + (q // 3 - 1) ** 2) * (dk / 3 ** p) ** 2) * b[p - 1, q] ** 2
        Wv = 0.02 * np.sqrt(1 + (wl.L / (np.pi * 0.02 ** 2 / W.LAMBDA)) ** 2)
        w_mom = np.sqrt(Wv ** 2 + 2 * sum((ds / K) ** 2 for ds in d) * grad2)
        assert abs(got["SI_rytov_discrete"] / rytov - 1) < 1e-3
        assert abs(got["W_LT_moment_m"] / w_mom - 1) < 1e-4
        assert abs(got["sigma_R2"] / (1.23 * cn2 * K ** (7 / 6) * wl.L ** (11 / 6)) - 1) < 1e-3
