"""The bench's stated-error statistics on synthetic ensembles with a known
answer (host logic, no GPU): the unpaired per-cell z of two independent seed
ensembles and the paired bias of two ensembles that share their seeds."""
import numpy as np

import bench


def _ens(rng, m, cells, loc=0.0, scale=1.0):
    return [{"U": loc + scale * rng.standard_normal(cells), "k": 1.0 + 0.1 * rng.standard_normal(cells)}
            for _ in range(m)]


def test_unpaired_z_follows_students_t_without_a_bias():
    rng = np.random.default_rng(1)
    a, b = _ens(rng, 8, 4000), _ens(rng, 8, 4000)
    r = bench.z_cells(a, b)
    assert r["tests"] == 8000
    # Welch's t with about 14 degrees of freedom: P(|t| > 3) is close to 1 %
    assert 0.003 < r["frac_above_3"] < 0.03, r["frac_above_3"]


def test_unpaired_z_finds_a_shift_of_several_standard_errors():
    rng = np.random.default_rng(2)
    a, b = _ens(rng, 8, 500, loc=2.0), _ens(rng, 8, 500)
    r = bench.z_cells(a, b)
    # a shift of 2 against a standard error of sqrt(2 / 8) = 0.5: z near 4
    assert r["max_abs_z_per_stat"]["U"] > 3.0
    assert r["frac_above_3"] > 0.3


def test_paired_bias_is_zero_for_the_same_runs_and_states_a_planted_bias():
    rng = np.random.default_rng(3)
    b = _ens(rng, 8, 300)
    same = bench.paired_bias([dict(x) for x in b], b)
    assert same["max_bias_in_se"] == 0.0 and same["max_abs_paired_t"] == 0.0
    # the pair shares its noise: a bias of 0.35 (one standard error of the
    # 8-run mean, 1 / sqrt(8)) under a small independent jitter
    a = [{"U": x["U"] + 1.0 / np.sqrt(8.0) + 1e-3 * rng.standard_normal(300), "k": x["k"].copy()} for x in b]
    r = bench.paired_bias(a, b)
    se_b = np.array([x["U"] for x in b]).std(0, ddof=1) / np.sqrt(8.0)
    # stated in units of B's standard error of the mean: 0.354 / se_b per cell
    assert np.isclose(r["max_bias_in_se_per_stat"]["U"], np.max((1.0 / np.sqrt(8.0)) / se_b), rtol=0.05)
    assert r["max_abs_paired_t_per_stat"]["U"] > 100.0  # the jitter is tiny against the bias
    assert r["max_bias_in_se_per_stat"]["k"] == 0.0
