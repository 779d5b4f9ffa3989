"""The random-cloud sweeps (Evaluation – Parameter Sensitivity and Scalability Analysis shapes): the sweep grid, the
table formatting, and one small point end to end on the GPU."""
import pytest

from paper_2511_18207_gb300 import sweeps


def test_sweep_grid_matches_the_studies():
    assert [p["D"] for p in sweeps.SWEEPS["dim"]] == [2, 4, 8, 16, 32, 64, 128, 256]
    assert [p["n_b"] / p["n_a"] for p in sweeps.SWEEPS["ratio"]] == [0.125, 0.25, 0.5, 1.0]
    assert [p["n_a"] + p["n_b"] for p in sweeps.SWEEPS["size"]] == [200_000, 500_000, 1_000_000, 2_000_000]
    assert all(p["alpha"] == 0.01 for k in ("dim", "ratio", "size") for p in sweeps.SWEEPS[k])
    assert all(p["alpha_max"] >= p["alpha"] for p in sweeps.SWEEPS["adaptive"])


def test_markdown_table():
    r = dict(n_a=100, n_b=50, D=4, alpha=0.01, m=2, seeds=3, rel_err_mean_abs=0.031, rel_err_mean_signed=-0.01,
             overestimates=2, refined_rel_err_mean=0.004, refined_rel_err_max=0.01, ms=1.5, refined_ms=2.5,
             exact_ms=10.0, subset_frac=0.05)
    md = sweeps.markdown({"ratio": [r]})
    assert "### ratio" in md and "| 100 | 50 | 4 | 0.01 | 5.00% | 3.10% | 2/3 | 0.40% / 1.00% |" in md


@pytest.mark.gpu
def test_one_small_point_on_the_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    r = sweeps.run_point(dict(n_a=3000, n_b=1500, D=4, alpha=0.02), seeds=2, torch=torch)
    # the refinement never exceeds the exact HD
    assert r["refined_rel_err_max"] < 1.0 and r["refined_rel_err_mean"] >= -1e-6
    assert 0 < r["subset_frac"] < 1 and r["exact_ms"] > 0
    a = sweeps.run_adaptive_point(dict(n_a=3000, n_b=1500, D=4, alpha=0.005, alpha_max=0.16, rel_tol=1e-3), seeds=2,
                                  torch=torch)
    assert a["rel_err_mean"] >= -1e-6 and a["steps_mean"] >= 1
    assert "adaptive" in sweeps.markdown({"adaptive": [a]})
