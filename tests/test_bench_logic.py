"""Host logic of bench.py that decides what the bench line reports.

* The clock summary parses nvidia-smi's CSV samples (median SM clock, the
  throttle reasons seen active), and a run is rejected on a hardware or
  thermal slowdown or on clocks stuck low with no reason; a power-cap
  reason alone is kept.
* The roofline's DRAM traffic comes from a committed profile summary only
  while the hash of the profiled sources matches: any edit to those sources
  makes it null.
"""
import os

import pytest

import bench

Q = "0, {sm}, 2070, 900.5, 0x0, {hw}, {hwt}, {swt}, {pc}"


def sampler(lines):
    cs = bench.ClockSampler(0)
    cs.lines = lines
    return cs


def line(sm, hw="Not Active", hwt="Not Active", swt="Not Active", pc="Not Active"):
    return Q.format(sm=sm, hw=hw, hwt=hwt, swt=swt, pc=pc)


def test_clock_summary_and_acceptance():
    clk = sampler([line(2070), line(2070), line(2055), "garbage"]).summary()
    assert clk == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    assert not bench.rejected(clk)
    assert sampler([]).summary() is None
    assert not bench.rejected(None)


@pytest.mark.parametrize("field,reason", [("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                                          ("swt", "sw_thermal_slowdown")])
def test_slowdowns_are_rejected(field, reason):
    clk = sampler([line(2070), line(1500, **{field: "Active"})]).summary()
    assert reason in clk["reasons"]
    assert bench.rejected(clk)


def test_power_cap_is_kept_and_a_stuck_clock_rejected():
    capped = sampler([line(1900, pc="Active"), line(1950, pc="Active")]).summary()
    assert capped["reasons"] == ["sw_power_cap"]
    assert not bench.rejected(capped)
    stuck = sampler([line(1000), line(1005)]).summary()
    assert stuck["reasons"] == [] and bench.rejected(stuck)


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1302_1125_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("kernel a\n")
    (csrc / "b.cuh").write_text("header b\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.csrc_hash(["b.cuh", "a.cu"])
    assert h == bench.csrc_hash(["a.cu", "b.cuh"])          # order does not matter
    (tmp_path / "profiles" / "k.md").write_text(
        f"# k\n\ncsrc_sha256: {h}   (note)\ncsrc_files: a.cu b.cuh\ntraffic_bytes_per_cell: 350.5\n")
    assert bench.profiled_traffic("k.md", 1000) == pytest.approx(350500.0)
    (csrc / "b.cuh").write_text("header b, edited\n")
    assert bench.profiled_traffic("k.md", 1000) is None      # stale capture: no traffic
    assert bench.profiled_traffic("missing.md", 1000) is None


def test_committed_profiles_name_existing_sources():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in os.listdir(os.path.join(root, "profiles")):
        text = open(os.path.join(root, "profiles", name)).read()
        for ln in text.splitlines():
            if ln.startswith("csrc_files:"):
                for f in ln.split(":", 1)[1].split():
                    assert os.path.exists(os.path.join(root, "paper_1302_1125_gb300", "csrc", f)), (name, f)


def _oracle_import_sites(path):
    """(enclosing top-level function or None, line) of every import of oracle"""
    import ast
    tree = ast.parse(open(path).read())
    sites = []
    for top in tree.body:
        name = top.name if isinstance(top, (ast.FunctionDef, ast.AsyncFunctionDef)) else None
        for node in ast.walk(top):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            if any(m == "oracle" or m.startswith("oracle.") for m in mods):
                sites.append((name, node.lineno))
    return sites


def test_oracle_is_used_only_by_the_baseline_legs_and_the_entry_checks():
    """the product path never reaches the oracle: bench.py imports it only in
    its CPU-baseline functions, __graft_entry__ only in build (which compiles
    it) and smoke (which checks against it), the package not at all"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sites = _oracle_import_sites(os.path.join(root, "bench.py"))
    assert sites and all(f is not None and f.startswith("cpu_baseline") for f, _ in sites), sites
    sites = _oracle_import_sites(os.path.join(root, "__graft_entry__.py"))
    assert {f for f, _ in sites} <= {"build", "smoke"}, sites
    pkg = os.path.join(root, "paper_1302_1125_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith(".py"):
                assert not _oracle_import_sites(os.path.join(dirpath, fn)), fn
            if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "rlb_oracle" not in text and "orc_" not in text, fn


def test_reference_arm_line_has_the_contract_keys(capsys, monkeypatch):
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the benchmark's keys, the reference marker, its CPU
    baseline and an end-to-end entry without host copies"""
    import json
    monkeypatch.delenv("RANK", raising=False)
    args = type("A", (), {"steps": 2, "warmup": 1, "gpus": 1})()
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_peak_bandwidth_is_the_measured_one_else_the_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6778.0, "bf16_tflops": 1873.2}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6778.0, "measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench.peaks() == (6800.0, "fallback")


def _quoted_commands():
    """(module, argv) of every bench.py or profile_step command the committed
    profile summaries quote"""
    import re
    import shlex
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    found = []
    for name in sorted(os.listdir(os.path.join(root, "profiles"))):
        for ln in open(os.path.join(root, "profiles", name)):
            m = re.search(r"python (-m paper_1302_1125_gb300\.profile_step|bench\.py)((?: --?[\w-]+(?: [\w.,]+)?)*)", ln)
            if m:
                found.append((name, "profile_step" if "profile_step" in m.group(1) else "bench",
                              shlex.split(m.group(2))))
    return found


def test_profile_commands_parse_with_the_committed_clis():
    """every command quoted in profiles/ uses only options that the committed
    bench.py and profile_step accept"""
    from paper_1302_1125_gb300 import profile_step
    cmds = _quoted_commands()
    assert {m for _, m, _ in cmds} == {"bench", "profile_step"}
    for name, module, argv in cmds:
        parser = bench.arg_parser() if module == "bench" else profile_step.arg_parser()
        parser.exit = lambda status=0, message=None: (_ for _ in ()).throw(AssertionError((name, argv, message)))
        parser.error = lambda message: (_ for _ in ()).throw(AssertionError((name, argv, message)))
        parser.parse_args(argv)
