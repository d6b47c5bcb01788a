"""Host-side logic of the benchmark: flop counts, tile_cfg decoding, the traffic guard."""
import bench


def test_flops_per_snp_counts_the_triangle_and_the_linear_rows():
    n, q, t = 10, 3, 2
    # n(n+1) flops for W x (lower triangle incl. diagonal), 2n per row of [X_L|Y]
    assert bench.flops_per_snp(n, q, t) == n * (n + 1) + 2 * n * (q + 1 + t)
    assert bench.bf16_flops_per_snp(n, q, t, 3) == 3 * (n * (n + 1) + 2 * n * (q + t))


def test_tile_cfg_fields_match_the_bit_layout():
    assert bench.tile_cfg_fields(None) == bench.tile_cfg_fields(-1)
    d = bench.tile_cfg_fields(8832)           # pair forced, group 40 MB, stages auto
    assert d == {"stages": 0, "group_mb": 40, "single_cta": False, "pair": True,
                 "fuse": False, "ztail": False}
    d = bench.tile_cfg_fields(4 | (160 << 4) | (1 << 12) | (1 << 17))
    assert d["stages"] == 4 and d["group_mb"] == 160 and d["single_cta"] and d["fuse"]
    assert not bench.tile_cfg_fields((1 << 17) | (1 << 14))["fuse"]   # bit 14 wins
    assert bench.tile_cfg_fields(0)["group_mb"] == 40   # group 0 = the default
    assert bench.tile_cfg_fields((1 << 21) | (1 << 13))["ztail"]
    assert not bench.tile_cfg_fields((1 << 21) | (1 << 17))["ztail"]   # fused wins


def test_traffic_guard_rejects_other_shapes_and_groupings():
    rec = bench.TRAFFIC["k_block_mixed<3>"][0]
    n, mb = rec["n"], rec["m_blk"]
    assert bench.traffic_for("k_block_mixed<3>", n + 1, mb) is None
    assert bench.traffic_for("k_block_mixed<3>", n, mb // 2) is None
    assert bench.traffic_for("k_block_mixed<3>", n, mb, 120 << 4) is None   # not captured
    assert bench.traffic_for("k_block_mixed<3>", n, mb, 1 << 12) is None
    assert bench.traffic_for("k_block_mixed<9>", n, mb) is None
    for g in (40, 80, 160):
        got = bench.traffic_for("k_block_mixed<3>", n, mb, (1 << 13) | (g << 4) | (rec["fuse"] << 17))
        # None once the kernel source changes
        assert got is None or got == rec["bytes_by_group_mb"][g]
    fused = rec["fuse"] << 17
    assert bench.traffic_for("k_block_mixed<3>", n, mb, 8832 | fused) == \
        bench.traffic_for("k_block_mixed<3>", n, mb, (1 << 13) | fused)


def test_pack_2bit_layout():
    import numpy as np
    import synth
    rng = np.random.default_rng(3)
    for n in (1, 4, 5, 11):
        X = rng.integers(-1, 4, size=(n, 6)).astype(np.int8)
        for call_of, miss in (((0, 1, 2), 3), ((3, 2, 0), 1)):
            P = synth.pack_2bit(X, call_of=call_of, missing_call=miss)
            assert P.shape == (-(-n // 4), 6) and P.flags.f_contiguous
            for j in range(6):
                for k in range(n):
                    d = int(X[k, j])
                    want = call_of[d] if d in (0, 1, 2) else miss
                    assert (int(P[k // 4, j]) >> (2 * (k % 4))) & 3 == want
                for k in range(n, 4 * P.shape[0]):      # padding calls are zero
                    assert (int(P[k // 4, j]) >> (2 * (k % 4))) & 3 == 0


def test_device_arguments_are_checked_before_the_call():
    """Tensors with the wrong element type or layout are refused by the binding without
    reaching the library (CPU tensors stand in for device ones)."""
    import pytest
    import torch
    from paper_1304_2272_gb300 import gwas
    X = torch.zeros((4, 8), dtype=torch.int8)
    b = torch.zeros((4, 1, 4), dtype=torch.float64)
    with pytest.raises(TypeError):
        gwas._require_dev(torch.zeros(3, dtype=torch.float32), gwas.np.float64, "b")
    with pytest.raises(ValueError):
        gwas._require_dev(torch.zeros((4, 8), dtype=torch.int8).t(), gwas.np.int8, "X")
    with pytest.raises(ValueError):
        gwas._require_dev(X, gwas.np.int8, "X")        # host tensor
    assert gwas._require_dev(None, gwas.np.int8, "X") is None
    assert gwas._require_dev(1234, gwas.np.int8, "X") == 1234
    del b


def test_autotune_cache_roundtrip_on_the_host(tmp_path, monkeypatch):
    """The tuning cache: one entry per (device, shape, precision, limbs, m_blk) key, written
    atomically and read back; a read-only or corrupt cache never raises."""
    from paper_1304_2272_gb300 import autotune
    monkeypatch.setenv("GWAS_AUTOTUNE_CACHE", str(tmp_path / "c" / "tune.json"))
    k1 = autotune.key_for(10000, 4, 1, 1, 3, 16384)
    k2 = autotune.key_for(10000, 4, 1, 1, 5, 16384)
    assert k1 != k2 and "n=10000" in k1 and "limbs=3" in k1
    autotune._store({k1: {"tile_cfg": 8832, "m_blk": 16384}})
    assert autotune._load()[k1]["tile_cfg"] == 8832
    (tmp_path / "c" / "tune.json").write_text("{not json")
    assert autotune._load() == {}


def test_code_sha_ignores_comments_only():
    src = "// a kernel\n__global__ void k(int* x) {  /* body */\n    x[0] = 1;  // one\n}\n"
    same = "// another comment\n__global__ void k(int* x) {\n  x[0] = 1;\n}\n"
    other = "__global__ void k(int* x) { x[0] = 2; }"
    assert bench.code_sha(src) == bench.code_sha(same)
    assert bench.code_sha(src) != bench.code_sha(other)


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` (the CPU oracle arm) prints one JSON line with the
    contract's keys, on a small n."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "300",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=str(bench.ROOT))
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "impl", "cpu_baseline", "e2e", "config"):
        assert k in d
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_host_arrays_are_refused_for_device_arguments():
    import numpy as np
    import pytest
    from paper_1304_2272_gb300 import gwas
    with pytest.raises(TypeError):
        gwas._require_dev(np.zeros(8, dtype=np.float64), np.float64, "b")


def test_cpu_baseline_flavours_on_a_small_cohort():
    """The CPU legs on a small cohort: the multithreaded Algorithm 1 route and the three
    single-threaded flavours (same route, textbook substitution, one process per core
    over disjoint SNPs), each with its rate and thread count."""
    import synth
    c = synth.make_cohort(5, 600, n_markers=300)
    X = c.snps(64)
    rec, L = bench.cpu_baseline(c, X, 0.2)
    assert rec["kind"] == "oracle" and rec["value"] > 0 and rec["cores"] >= 1
    assert L.shape == (600, 600)
    names = [f["flavour"] for f in rec["flavours"]]
    assert names[:3] == ["algorithm1_blas_all_threads", "algorithm1_blas_1_thread",
                         "plain_row_loop_substitution_1_thread"], rec["flavours"]
    assert names[3].startswith("processes_over_snps_")
    for f in rec["flavours"]:
        assert f["value"] > 0 and f["threads"] >= 1 and f["snps"] > 0
    assert rec["flavours"][1]["threads"] in (1, None) or rec["flavours"][1]["threads"] == 1


def test_oracle_errors_report_a_planted_error():
    """oracle_errors finds an error planted into otherwise exact outputs, in b and in the
    Wald statistic, and flags a status that differs."""
    import numpy as np
    import synth
    from oracle import gls as G
    c = synth.make_cohort(6, 300, n_markers=300)
    X = c.snps(40)
    L = G.factor(c.phi, c.h, c.sigma2)
    b, w, st = G.gls_hoisted(L, c.XL, c.Y, X)
    sample = {"X": X, "b": b.copy(), "wald": w.copy(), "status": st.copy(), "snps": 40}
    e = bench.oracle_errors(L, c, sample)
    assert e["err_b"] == 0.0 and e["err_wald"] == 0.0 and e["status_match"]
    scale = np.max(np.abs(b[7, 0]))
    sample["b"][7, 0, 3] += 1e-7 * scale
    sample["wald"][3, 0] += 1e-6 * max(w[3, 0], 1.0)
    sample["status"][5] = 1
    e = bench.oracle_errors(L, c, sample)
    assert abs(e["err_b"] - 1e-7) < 1e-9 and abs(e["err_wald"] - 1e-6) < 1e-8
    assert not e["status_match"]


def test_factor_record_excludes_the_upload():
    """The factor's rate is taken over its device time without the host uploads, at
    2n^3/3 flops, and compared with the probed FP64 fma rate when there is one."""
    import types
    st = {"factor_ms": 600.0, "factor_upload_ms": 80.0, "factor_launches": 500}
    args = types.SimpleNamespace(fp64_probe={"tflops": 1.25})
    r = bench.factor_record(st, 10000, args)
    assert r["compute_ms"] == 520.0 and r["upload_ms"] == 80.0 and r["launches"] == 500
    assert abs(r["fp64_tflops"] - 2e12 / 3 / 0.52 / 1e12) < 1e-12
    assert abs(r["frac_of_fma_rate"] - r["fp64_tflops"] / 1.25) < 1e-12
    r = bench.factor_record(st, 10000, types.SimpleNamespace(fp64_probe=None))
    assert "frac_of_fma_rate" not in r
