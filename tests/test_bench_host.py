"""Host side of the benchmark: the JSON line of the reference arm (the FP64
oracle on the CPU), the algorithmic byte model behind the roofline, the
fixed-tuning argument, the DRAM traffic lookup and the digest built from
ncu captures.  No GPU."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N, M = 512 ** 3, 1024 ** 3
K = 1024 * 1024 * 520          # modes per field on the blocked 1024^3 spectrum


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["dtype"] == "f64"
    assert line["config"]["workload"] == "pm512_mesh1024"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_algorithmic_bytes_per_launch():
    ab = lambda kind: bench.algorithmic_bytes(kind, N, M, K)  # noqa: E731
    assert ab("paint_density") == 12 * N + 4 * M            # s in; one field out
    assert ab("paint_adj") == 24 * N + 16 * M               # s, mu in; four fields out
    assert ab("fft_z_fwd_4") == 4 * (4 * M + 8 * K)         # reals in, half spectra out
    assert ab("fft_z_inv_3") == 3 * 8 * K + 16 * M          # spectra in, 4-slot mesh out
    assert ab("fft_z_inv_1") == 8 * K + 4 * M
    assert ab("fft_y_fwd_4") == 4 * 16 * K                  # pencil pass: read + write
    assert ab("spectral_force") == 32 * K and ab("spectral_adj") == 64 * K
    assert ab("fft_x_round_1") == 32 * K and ab("fft_x_round_4") == 64 * K
    assert ab("no_such_kernel") is None
    # the fused x round trip saves two spectrum round trips per evaluation
    assert ab("fft_x_fwd_1") + ab("spectral_force") + ab("fft_x_inv_3") - ab("fft_x_round_1") == 64 * K
    assert ab("fft_x_fwd_4") + ab("spectral_adj") + ab("fft_x_inv_4") - ab("fft_x_round_4") == 128 * K
    # the potential pipeline: one field each way per force x pass, two per
    # adjoint x pass, the adjoint source stencil, the planar 2-field z inverse
    assert ab("fft_x_pot_1") == 16 * K and ab("fft_x_pot_2") == 32 * K and ab("fft_x_pot_4") == 48 * K
    assert ab("vjp_source") == 24 * M and ab("grad_stencil_1") == 20 * M
    assert ab("fft_z_inv_2") == 2 * 8 * K + 8 * M and ab("fft_z_fwd_2") == 2 * (4 * M + 8 * K)
    # reads from the potential mesh count one float per cell (two for the adjoint's phi, psi)
    pr = lambda kind: bench.algorithmic_bytes(kind, N, M, K, pot_read=True)  # noqa: E731
    assert pr("read_kick_drift") == 48 * N + 4 * M and ab("read_kick_drift") == 48 * N + 12 * M
    assert pr("read_adj") == 96 * N + 8 * M and ab("read_adj") == 96 * N + 16 * M


def test_tuning_argument():
    assert bench._tuning_arg("paint=512,read=128,x_round=3") == {"paint": 512, "read": 128, "x_round": 3}


def test_traffic_lookup_needs_the_current_sources(monkeypatch):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    with open(path) as fh:
        digest = json.load(fh)["source_digest"]
    monkeypatch.setattr(bench, "_source_digest", lambda: digest)
    direct = bench._ncu_traffic("paint_adj", "pm512_mesh1024")
    assert direct is not None and direct > bench.algorithmic_bytes("paint_adj", N, M, K)
    assert bench._ncu_traffic("no_such_kernel", "pm512_mesh1024") is None
    monkeypatch.setattr(bench, "_source_digest", lambda: "changed")
    assert bench._ncu_traffic("paint_adj", "pm512_mesh1024") is None


def test_workloads_of_the_bench():
    from paper_2211_09958_gb300.configs import WORKLOADS
    w = WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert (w.n_p, w.n_m, w.box, w.n_steps, w.n_batch) == (512, 1024, 1000.0, 100, 1)
    assert w.n_m ** 3 * 4 > 129e6                      # every mesh field exceeds the 129 MB L2
    small = WORKLOADS["pm32_mesh64"]
    assert (small.n_p, small.n_m, small.n_steps) == (32, 64, 10)
    batch = WORKLOADS["batch32_pm64_mesh128"]
    assert (batch.n_batch, batch.n_p, batch.n_m, batch.n_steps) == (32, 64, 128, 20)
    learned = WORKLOADS[bench.LEARNED_WORKLOAD]
    assert (learned.n_p, learned.n_m, learned.n_steps) == (128, 128, 40)


def test_kernel_kinds_from_ncu_names():
    # the names ncu prints (template arguments plain or with C-style casts)
    kind = bench._kernel_kind
    assert kind("void pmgb::<unnamed>::k_read<(int)3, (bool)0, (int)128, (int)2, (bool)1>(pmgb::ReadArgs)",
                "(1, 1, 1)", 256) == "read_adj"
    assert kind("void pmgb::<unnamed>::k_read<1, false, 128, 2, true>(pmgb::ReadArgs)", "(1, 1, 1)", 256) == \
        "read_kick_drift"
    assert kind("void pmgb::<unnamed>::k_paint<(int)2, (int)512, (int)2>(pmgb::PaintArgs)", "(1, 1, 1)", 256) == \
        "paint_adj"
    assert kind("void pmgb::<unnamed>::k_deposit<(int)1, (int)256>(pmgb::DepositArgs)", "(1, 1, 1)", 256) == \
        "deposit_density"
    assert kind("void pmgb::<unnamed>::k_deposit_halo<(int)4>(pmgb::DepositArgs)", "(1, 1, 1)", 256) == \
        "deposit_halo_4"
    assert kind("pmgb::<unnamed>::k_bin_count(pmgb::DepositArgs)", "(1, 1, 1)", 256) == "bin_count"
    assert kind("void pmgb::<unnamed>::k_fft_xpot<(int)256, (int)1>(float2 *, ...)", "(1, 1, 1)", 256) == \
        "fft_x_pot_1"
    assert kind("void pmgb::<unnamed>::k_fft_z_inv<(int)256, (int)2, (int)2, (int)256, (bool)1>(...)",
                "(1, 1, 1)", 256) == "fft_z_inv_2"
    # y pass: one block per (field, run, kz block of 8) and x; 256^3 has 136 / 8 kz blocks
    assert kind("void pmgb::<unnamed>::k_fft_pencil<(int)256, (bool)1, (int)8>(...)", f"({2 * 17 * 256}, 1, 1)",
                256) == "fft_y_inv_2"
    assert kind("void regular_fft<512, EPT<8>>(kernel_arguments_t)", "(1, 1, 1)", 256) is None


def test_traffic_digest_from_a_capture(tmp_path, monkeypatch):
    # a two-launch capture of one kernel: mean DRAM bytes per launch, its ratio to
    # the algorithmic bytes and the factor to the headline workload
    csv_text = "\n".join([
        '"ID","Kernel Name","Grid Size","Metric Name","Metric Unit","Metric Value"',
        '"0","void pmgb::<unnamed>::k_vjp_source<32>(const float4 *, float2 *, int, float)","(512, 1, 1)",'
        '"dram__bytes_read.sum","byte","300,000,000"',
        '"0","void pmgb::<unnamed>::k_vjp_source<32>(const float4 *, float2 *, int, float)","(512, 1, 1)",'
        '"dram__bytes_write.sum","byte","100,000,000"',
        '"1","void pmgb::<unnamed>::k_vjp_source<32>(const float4 *, float2 *, int, float)","(512, 1, 1)",'
        '"dram__bytes_read.sum","byte","320,000,000"',
        '"1","void pmgb::<unnamed>::k_vjp_source<32>(const float4 *, float2 *, int, float)","(512, 1, 1)",'
        '"dram__bytes_write.sum","byte","80,000,000"'])
    path = tmp_path / "k.csv"
    path.write_text("==PROF== noise\n" + csv_text + "\n")
    out = bench.traffic_digest([str(path)], out_path=str(tmp_path / "traffic.json"))
    ent = out["kernels"]["vjp_source"]
    assert ent["launches"] == 2 and ent["dram_bytes_per_launch"] == 4e8
    ab = bench.algorithmic_bytes("vjp_source", 128 ** 3, 256 ** 3, 256 ** 2 * 129)
    assert ent["ratio"] == round(4e8 / ab, 3)
    assert ent["scale_to"]["pm512_mesh1024"] == pytest.approx(1024 ** 3 / 256 ** 3)
    assert json.load(open(tmp_path / "traffic.json"))["source_digest"] == bench._source_digest()
