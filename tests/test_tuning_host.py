"""Host logic of the autotuner (no GPU): the candidate launch shapes it
times for one lattice, and its on-disk cache."""
from paper_1405_6162_gb300 import tuning


def test_candidates_cover_each_family_and_respect_its_limits():
    dims = (256, 256, 256)
    c32 = tuning.candidates("fp32_shifted", dims, ("two_pass", "bulk", "fused"))
    fams = {c[0] for c in c32}
    assert fams == {"two_pass", "bulk", "fused"}
    # two-pass: threads per CTA x phi sites per thread (the paper's TPB and VVL)
    assert {(c[1], c[2]) for c in c32 if c[0] == "two_pass"} == {(t, v) for t in (128, 256) for v in (1, 2, 4)}
    # bulk: the lean form (2 slots) only in FP32; cluster sizes divide ny;
    # planes per CTA include 20 and 24 (fuller last waves at 256^3)
    assert {c[1] for c in c32 if c[0] == "bulk"} == {2, 3, 4}
    assert {c[3] for c in c32 if c[0] == "bulk"} == {16, 20, 24, 32, 64}
    c64 = tuning.candidates("fp64", dims, ("bulk",))
    assert {c[1] for c in c64} == {3, 4}
    odd = tuning.candidates("fp32_shifted", (256, 6, 8), ("bulk",))
    assert {c[2] for c in odd} == {1, 2}
    # rows that are not whole 16-byte units, or longer than 256: no bulk shapes
    assert tuning.candidates("fp32_shifted", (13, 8, 8), ("bulk",)) == []
    assert tuning.candidates("fp32_shifted", (260, 8, 8), ("bulk",)) == []
    # double-float: no fused kernel
    assert tuning.candidates("fp64_df", dims, ("fused",)) == []


def test_reduced_form_shapes_only_at_tau_g_one():
    dims = (64, 64, 64)
    assert tuning.candidates("fp32_shifted", dims, ("taug1",), tau_g=0.9) == []
    t1 = tuning.candidates("fp32_shifted", dims, ("taug1",), tau_g=1.0)
    assert {c[1] for c in t1} == {1, 2, 4} and {c[2] for c in t1} == {4, 8} and {c[3] for c in t1} == {0, 32, 64}
    # four rows per warp spill in double-float: not offered there
    df = tuning.candidates("fp64_df", dims, ("taug1",), tau_g=1.0)
    assert {c[1] for c in df} == {1, 2}


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "CACHE", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(tuning, "_gpu_name", lambda: "probe-gpu")
    dims = (32, 16, 8)
    assert tuning.bench_config(dims, "fp32_shifted") == tuning.DEFAULT
    assert tuning.cached_table(dims, "fp32_shifted") is None
    tuning._save(tuning._key(dims, "fp32_shifted"),
                 {"config": ["bulk", 3, 2, 16], "seconds_per_step": 1e-3, "table": [[["bulk", 3, 2, 16], 1e-3]]})
    assert tuning.bench_config(dims, "fp32_shifted") == ("bulk", 3, 2, 16)
    # another family set or precision is another entry
    assert tuning.bench_config(dims, "fp32_shifted", ("taug1",)) == tuning.DEFAULT
    assert tuning.bench_config(dims, "fp64") == tuning.DEFAULT
