"""Host logic of bench.py (no GPU): the roofline's traffic is read from a
committed ncu summary only while that summary was taken on the current
kernel sources, and every committed step summary is current."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _summary(tmp_path, monkeypatch, body):
    """profiles/probe.md under a scratch root that holds a copy of the
    kernel sources (which the hash is taken of)."""
    import shutil
    csrc = tmp_path / "paper_1405_6162_gb300" / "csrc"
    if not csrc.exists():
        shutil.copytree(os.path.join(ROOT, "paper_1405_6162_gb300", "csrc"), csrc)
    prof = tmp_path / "profiles"
    prof.mkdir(exist_ok=True)
    (prof / "probe.md").write_text(body)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))


def test_value_read_only_when_sources_match(tmp_path, monkeypatch):
    sha = bench._kernel_sha(bench.STEP_SOURCES)
    _summary(tmp_path, monkeypatch, f"dram_bytes_per_step: 123.5\n\nkernel_sources_sha256_16: {sha}\n")
    assert bench._profile_value("probe", "dram_bytes_per_step") == 123.5


def test_stale_summary_gives_none(tmp_path, monkeypatch):
    _summary(tmp_path, monkeypatch, "dram_bytes_per_step: 123.5\n\nkernel_sources_sha256_16: 0000000000000000\n")
    assert bench._profile_value("probe", "dram_bytes_per_step") is None
    # a figure that does not depend on the kernel sources can still be read
    assert bench._profile_value("probe", "dram_bytes_per_step", need_current=False) == 123.5


def test_listed_sources_are_the_ones_hashed(tmp_path, monkeypatch):
    src = ("d3q19.cuh", "df64.cuh")
    sha = bench._kernel_sha(src)
    body = f"x: 7\n(sources: {', '.join(src)})\n\nkernel_sources_sha256_16: {sha}\n"
    _summary(tmp_path, monkeypatch, body)
    assert bench._profile_value("probe", "x") == 7.0
    # the same hash under the default list does not match
    (tmp_path / "profiles" / "probe.md").write_text(body.replace(f"(sources: {', '.join(src)})\n", ""))
    assert bench._profile_value("probe", "x") is None


def test_missing_summary_or_key():
    assert bench._profile_value("no_such_summary", "x") is None
    assert bench._profile_value("step_fp32_shifted_256cubed", "no_such_key") is None


def test_committed_step_summaries_are_current():
    # the figures bench.py reports beside its timings come from these
    for name, key in (("step_fp32_shifted_256cubed", "dram_bytes_per_step"),
                      ("step_bulk_fp32_shifted_256cubed", "dram_bytes_per_step"),
                      ("step_fp64_256cubed", "dram_bytes_per_step"),
                      ("step_fp64_256cubed", "fp64_instr_per_site"),
                      ("step_fp64_df_256cubed", "dram_bytes_per_step"),
                      ("step_taug1_256cubed", "dram_bytes_per_step_fp32_shifted"),
                      ("step_mrt_256cubed", "fp64_flops_per_site"),
                      ("step_isotropic_stencils_256cubed", "fp64_flops_per_site_27"),
                      ("adjoint_reverse_step_64cubed", "fp64_flops_per_site"),
                      ("reduce_128cubed", "fp64_adds_per_site_fp32_shifted"),
                      ("reduce_128cubed", "dram_bytes_per_site_fp64")):
        assert bench._profile_value(name, key) is not None, (name, key)
