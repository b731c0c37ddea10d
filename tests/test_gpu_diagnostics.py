"""The per-cell entropy check (Section 4) runs inside the kernels that the timed runs use.

With diagnostics on, every entropic relaxation evaluates F(omega - 1) = B(omega - 1) - B(-1) in
FP64 (the change of the cell's microscopic entropy) and counts the cells above the rounding level
of the arithmetic that chose omega.  The check reads what the relaxation computed and writes
nothing back: the distributions are bit for bit those of the same kernel without it.  Cases cover
the temporally blocked 1D and 2D kernels, the per-stage kernels (the staged 2D stage kernel for rows
on 16-byte boundaries) and the batched cooperative kernel, in FP32, FP64 and FP32 with the entropy
difference in FP64.
"""
import numpy as np
import pytest

from paper_2403_13406_gb300 import eslbm, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

EPS = {"fp32": 1.1920929e-7, "fp64": 2.220446e-16, "fp32_mixed": 2.220446e-16}

CASES = {
    # 1D: one temporally blocked launch per composite step
    "sw1d": (1, "sw", 1000, 1, dict(V=4.0, g=9.81), lambda: inputs.sw_random_1d(1000, seed=3, h_amp=0.2, u_amp=0.3)),
    "burgers1d": (1, "burgers", 1000, 1, dict(V=1.5), lambda: inputs.random_scalar_1d(1000, seed=2)),
    # 2D rows on 16-byte boundaries: the bulk-copy staged stage kernel, or the blocked 2D kernel
    "sw2d_rows": (2, "sw", 1032, 3, dict(V=8.0, g=9.81),
                  lambda: inputs.sw_random_2d(1032, 3, seed=9, h_amp=0.1, u_amp=0.2)),
    "burgers2d_rows": (2, "burgers", 1032, 6, dict(V=3.0, c=(1.0, 0.6)),
                       lambda: inputs.burgers_2d(1032, 6, seed=8, noise=1e-2)),
}


def run(name, precision, diag, steps=6, blocking=True):
    dim, system, nx, ny, kw, init = CASES[name]
    cfg = eslbm.make_config(dim, system, nx, ny, precision=precision, omega_mode="entropic", diagnostics=diag,
                            blocking=blocking, **kw)
    sim = eslbm.Simulation(cfg)
    sim.init_equilibrium(init())
    sim.step(steps)
    f = sim.distributions(host=True)
    d = sim.diagnostics()
    sim.close()
    return f, d


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_mixed"])
@pytest.mark.parametrize("blocking", [True, False, 6])
def test_diagnostics_leave_results_unchanged(name, precision, blocking):
    """Default: the 1D temporally blocked kernel, the 2D per-stage kernel (rows on 16-byte boundaries:
    the bulk-copy staged one); off: the per-stage kernels; 6: the temporally blocked 2D kernel."""
    f0, d0 = run(name, precision, False, blocking=blocking)
    f1, d1 = run(name, precision, True, blocking=blocking)
    assert np.array_equal(f0, f1)
    assert d0["fallbacks"] == d1["fallbacks"]
    assert d1["entropy_increases"] == 0
    assert d1["entropy_excess_max"] <= 64 * EPS[precision]
    assert 1.0 <= d1["omega_min"] <= d1["omega_max"] <= 4.0


@pytest.mark.parametrize("precision", ["fp32", "fp32_mixed"])
def test_batched_kernel_checks_every_cell(precision):
    """The cooperative batched kernel with diagnostics: same results, no per-cell increase."""
    sizes = [(96, 64), (64, 80), (128, 40)]
    outs, diags = [], []
    for diag in (False, True):
        cfg = eslbm.make_config(2, "sw", 1, 1, V=8.0, g=9.81, precision=precision, omega_mode="entropic",
                                diagnostics=diag)
        b = eslbm.Batch(cfg, sizes)
        b.init_equilibrium(b.pack([inputs.sw_random_2d(nx, ny, seed=20 + i, h_amp=0.1, u_amp=0.2)
                                   for i, (nx, ny) in enumerate(sizes)]))
        b.step(4)
        outs.append(b.moments_flat().cpu().numpy())
        diags.append(b.diagnostics())
        b.close()
    assert np.array_equal(outs[0], outs[1])
    assert diags[1]["entropy_increases"] == 0
    assert diags[1]["entropy_excess_max"] <= 64 * EPS[precision]
    assert 1.0 <= diags[1]["omega_min"] <= diags[1]["omega_max"] <= 4.0


def test_mixed_mode_is_never_above_the_root():
    """FP32 storage with the entropy difference in FP64: on rough data far from equilibrium every
    relaxation satisfies F(omega - 1) <= 0 to FP64 rounding (the chord correction), while the
    result stays within the FP32 bar of the all-FP32 run."""
    init = lambda: inputs.sw_random_1d(4096, seed=31, h_amp=0.3, u_amp=0.5, modes=12)
    res = {}
    for precision in ("fp32", "fp32_mixed"):
        cfg = eslbm.make_config(1, "sw", 4096, V=5.0, g=9.81, precision=precision, omega_mode="entropic",
                                diagnostics=True)
        sim = eslbm.Simulation(cfg)
        sim.init_equilibrium(init())
        sim.step(10)
        res[precision] = (sim.moments(host=True), sim.diagnostics())
        sim.close()
    d = res["fp32_mixed"][1]
    assert d["entropy_increases"] == 0 and d["entropy_excess_max"] <= 64 * 2.220446e-16
    a, b = res["fp32"][0], res["fp32_mixed"][0]
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
