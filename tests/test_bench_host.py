"""Host logic of bench.py (no GPU): the numbers it takes from the committed
ncu summaries, and when it refuses them."""
import pytest

import bench


@pytest.fixture
def profile(tmp_path, monkeypatch):
    path = tmp_path / "heat.md"
    monkeypatch.setitem(bench.PROFILES, "heat", str(path))
    return path


def test_summary_values_are_used_only_for_the_current_kernel_sources(profile):
    h = bench.kernel_source_hash()
    profile.write_text("dram_bytes_per_full_launch[v1]: 70000000\n"
                       "instructions_per_site[v1]: 229.5\n"
                       f"kernel_source_sha256_16: {h}\n")
    assert bench.ncu_traffic("heat", "v1") == 70000000.0
    assert bench.ncu_instructions("heat", "v1") == 229.5
    assert bench.ncu_traffic("heat", "v2") is None          # another launch shape
    profile.write_text("dram_bytes_per_full_launch[v1]: 70000000\n"
                       "kernel_source_sha256_16: 0000000000000000\n")
    assert bench.ncu_traffic("heat", "v1") is None          # taken on other code
    profile.unlink()
    assert bench.ncu_instructions("heat", "v1") is None     # no summary


def test_heat_flops_take_the_timed_variants_count_else_the_counted_variants(profile):
    h = bench.kernel_source_hash()
    v = bench.HEAT_COUNTED_VARIANT
    profile.write_text(f"flops_per_site[{v}]: 261.6\n"
                       "flops_per_site[other]: 250.0\n"
                       f"kernel_source_sha256_16: {h}\n")
    assert bench.heat_flops("other") == (250.0, "other")
    assert bench.heat_flops("uncounted") == (261.6, v)
    profile.write_text(f"flops_per_site[{v}]: 261.6\n"
                       "kernel_source_sha256_16: 0000000000000000\n")
    assert bench.heat_flops(v) == (None, None)              # taken on other code


def test_source_hash_ignores_comments_and_white_space(tmp_path, monkeypatch):
    a, b, c = tmp_path / "a.cuh", tmp_path / "b.cuh", tmp_path / "c.cuh"
    a.write_text("int f(int x) { return x + 1; }  // one\n")
    b.write_text("/* two */\nint f(int x)\n{\n    return x + 1;\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_1911_10747_gb300" / "csrc").mkdir(parents=True)
    for src in (a, b, c):
        (tmp_path / "paper_1911_10747_gb300" / "csrc" / src.name).write_text(src.read_text())
    ha = bench.kernel_source_hash(("a.cuh",))
    assert ha == bench.kernel_source_hash(("b.cuh",))
    assert ha != bench.kernel_source_hash(("c.cuh",))


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "max_sm_mhz", lambda: 2000.0)
    r = bench.issue_roofline(320.0, 1_000_000, 1.0)  # 10 M warp instructions in 1 ms
    assert r["peak"] == pytest.approx(152 * 4 * 2.0e9 / 1e12)
    assert r["achieved"] == pytest.approx(0.01)
    assert r["frac"] == pytest.approx(0.01 / r["peak"])
    assert bench.issue_roofline(None, 1, 1.0) is None


def test_fp64_counts_are_used_only_for_the_current_fp64_sources(tmp_path, monkeypatch):
    path = tmp_path / "fp64.md"
    monkeypatch.setitem(bench.PROFILES, "fp64", str(path))
    h = bench.kernel_source_hash(bench.FP64_SOURCES)
    path.write_text("fp64_instructions_per_site[flow]: 370.4\n"
                    "fp64_flops_per_site[flow]: 464.1\n"
                    f"fp64_source_sha256_16: {h}\n")
    assert bench.ncu_fp64_instructions("flow") == 370.4
    assert bench.ncu_fp64_flops("flow") == 464.1
    assert bench.ncu_fp64_instructions("heat") is None      # not counted
    path.write_text("fp64_instructions_per_site[flow]: 370.4\n"
                    "fp64_source_sha256_16: 0000000000000000\n")
    assert bench.ncu_fp64_instructions("flow") is None      # taken on other code
