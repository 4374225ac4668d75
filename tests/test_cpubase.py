"""The multi-core FP32 CPU baseline (cpubase/, timed by bench.py) against the FP64 oracle (CPU only).

Tolerances as for the GPU path: tree and forward max relative error 1e-5 (positive data),
backward normwise 1e-5. Multi-threaded runs equal single-threaded ones (forward and data gradient
bit for bit: every output is computed by one thread in a fixed order)."""
import numpy as np
import pytest

import aprsynth as S
import cpubase
import oracle

CASES = {
    "blob64": lambda: S.make_config("blob64"),
    "rand_ragged": lambda: S.random_balanced_apr((21, 13, 150), 1, seed=7, p_fine=0.01),
    "rand_thin": lambda: S.random_balanced_apr((3, 40, 9), 0, seed=8, p_fine=0.05),
    "all_max": lambda: S.uniform_level_apr((9, 17, 70), 7, l_min=2),
    "tiny": lambda: S.random_balanced_apr((2, 3, 5), 0, seed=9, p_fine=0.3),
}


def _stencils(apr, k, kind, seed=0):
    if kind == "restricted":
        w = S.gaussian_stencil(k, 1.0 if k == 3 else 1.5)
        return oracle.restrict_stencil(w, apr.l_max, apr.l_min).reshape(apr.n_levels, -1).astype(np.float32)
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, size=(apr.n_levels, k ** 3)).astype(np.float32)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("k", [3, 5])
@pytest.mark.parametrize("bc", [0, 1])
def test_cpu_baseline_matches_oracle(case, k, bc):
    apr = CASES[case]()
    c = cpubase.CpuApr(apr, threads=3)
    o = oracle.Oracle(apr)
    t = c.tree_restrict(apr.values)
    rt = o.tree()[:, 0]
    assert t.shape == rt.shape
    if rt.size:
        assert np.max(np.abs(t - rt) / np.abs(rt)) <= 1e-6
    for kind in ("restricted", "random"):
        st = _stencils(apr, k, kind)
        out = c.convolve(apr.values, t, st, k, bc)
        ref = o.conv(st.astype(np.float64), k, bc)[:, 0]
        if kind == "restricted":
            assert np.max(np.abs(out - ref) / np.abs(ref)) <= 1e-5
        else:
            assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) <= 1e-5
    g = np.random.default_rng(1).normal(size=apr.n_particles).astype(np.float32)
    for kind in ("restricted", "random"):
        st = _stencils(apr, k, kind, seed=2)
        gp, gw = c.backward(apr.values, t, st, k, g, bc)
        rp, rw = o.conv_backward(st.astype(np.float64), k, g.astype(np.float64), bc)
        assert np.max(np.abs(gp - rp[:, 0])) / np.max(np.abs(rp)) <= 1e-5
        assert np.max(np.abs(gw - rw.reshape(gw.shape))) / np.max(np.abs(rw)) <= 1e-5


def test_cpu_baseline_thread_count_does_not_change_results():
    apr = CASES["blob64"]()
    st = _stencils(apr, 5, "random")
    g = np.random.default_rng(3).normal(size=apr.n_particles).astype(np.float32)
    res = []
    for th in (1, 4):
        c = cpubase.CpuApr(apr, threads=th)
        t = c.tree_restrict(apr.values)
        res.append((t, c.convolve(apr.values, t, st, 5), *c.backward(apr.values, t, st, 5, g)))
    for a, b in zip(res[0][:3], res[1][:3]):  # tree, forward, data gradient
        np.testing.assert_array_equal(a, b)
    # stencil gradient: FP64 per-thread partials summed in thread order
    np.testing.assert_allclose(res[0][3], res[1][3], rtol=1e-6, atol=1e-6 * np.abs(res[0][3]).max())
