"""Host-side checks of bench.py (no GPU): every workload's constants and helpers exist, every name the
functions read is defined, and the sampled-oracle estimate and pixel weights are consistent."""
import ast
import builtins
import pathlib

import numpy as np

import aprsynth as S
import bench

SRC = pathlib.Path(bench.__file__).read_text()


def test_workload_constants_and_choices():
    assert bench.WORKLOAD in S.CONFIGS and bench.MC_WORKLOAD in S.CONFIGS and bench.RL_WORKLOAD in S.CONFIGS
    assert bench.RL_ITERS == 20 and bench.K == 5 and bench.MC_C == 16
    for w in ("blob1024", "blob256_mc", "blob512_rl", "surrogate"):
        assert f'"{w}"' in SRC


def test_functions_read_only_defined_names():
    tree = ast.parse(SRC)
    defined = set(dir(builtins))
    for node in tree.body:
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            defined.add(node.name)
        elif isinstance(node, ast.Assign):
            defined.update(t.id for t in node.targets if isinstance(t, ast.Name))
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            defined.update((a.asname or a.name).split(".")[0] for a in node.names)
    missing = set()
    for fn in (n for n in tree.body if isinstance(n, ast.FunctionDef)):
        local = {a.arg for a in fn.args.args} | {a.arg for a in fn.args.kwonlyargs}
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Store):
                local.add(n.id)
            elif isinstance(n, ast.FunctionDef):
                local.add(n.name)
                local.update(a.arg for a in n.args.args)
            elif isinstance(n, ast.Lambda):
                local.update(a.arg for a in n.args.args)
            elif isinstance(n, (ast.Import, ast.ImportFrom)):
                local.update((a.asname or a.name).split(".")[0] for a in n.names)
            elif isinstance(n, ast.ExceptHandler) and n.name:
                local.add(n.name)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in local | defined:
                missing.add((fn.name, n.id))
    assert not missing, sorted(missing)


def test_pixels_per_particle_partition_the_image():
    apr = S.random_balanced_apr((9, 14, 21), 1, seed=4, p_fine=0.05)
    assert bench.pixels_per_particle(apr).sum() == 9 * 14 * 21


def test_oracle_sampled_step_estimate():
    import time
    calls = []

    def run(smp):   # a fixed cost plus a cost per sampled particle
        calls.append(smp.size)
        time.sleep(0.01 + 1e-5 * smp.size)

    est, t_fixed, t_s = bench.oracle_sampled_step(100000, 0.5, run, 2000, np.random.default_rng(0))
    assert calls == [16, 2000]
    assert 0.5 + 0.01 <= est and abs(est - (0.5 + 0.01 + 1.0)) < 0.5


def test_recorded_traffic_follows_the_kernel_sources():
    """roofline.traffic comes from the committed ncu record only while the kernel sources hash to the
    recorded value: the committed record matches the tree, and a changed source hash gives None."""
    import json
    rec = json.loads((pathlib.Path(bench.ROOT) / "profiles" / "traffic.json").read_text())
    assert rec["sha1_prefix"] == bench.kernel_source_hash()
    assert rec["mc"]["sha1_prefix"] == bench.kernel_source_hash(bench.MC_TRAFFIC_SOURCES)
    adj = bench.recorded_traffic("apr_convolve_adjoint")
    assert adj == rec["dram_bytes_per_call"]["apr_convolve_adjoint"] and adj > 0
    assert bench.recorded_traffic("data_adjoint", "mc") == rec["mc"]["dram_bytes_per_call"]["data_adjoint"]
    saved = bench.kernel_source_hash
    try:
        bench.kernel_source_hash = lambda sources=None: "000000000000"
        assert bench.recorded_traffic("apr_convolve_adjoint") is None
        assert bench.recorded_traffic("data_adjoint", "mc") is None
    finally:
        bench.kernel_source_hash = saved
