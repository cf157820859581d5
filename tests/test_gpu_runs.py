"""Whole MetaDE runs (Alg. 3): FP32 GPU runs and FP64 oracle runs diverge
trajectory by trajectory, so they are compared as distributions over 31
seeds with the paper's test, a Wilcoxon rank-sum test at 0.05 (Sec. IV-A).
Errors below 1e-8 count as 0, as the paper reports them."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SEEDS = range(31)


def _truncate(y):
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < 1e-8, 0.0, y)


def _gpu_runs(power_up=False, seeds=SEEDS, path=0, evolver=0):
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    p = wl.problems[0]
    ys = []
    for s in seeds:
        b = M.Batch([(p.dim, p.obj, p.shift, p.rot)], wl.inst_np, wl.inst_prob, wl.inst_group, seed=s,
                    one_shot=1, n_out=wl.n_out, path=path, evolver=evolver)
        _, ofit = b.run_metade(wl.outer_gens, wl.inner_gens, power_up=power_up,
                               use_graph=path == M.METADE_PATH_BATCHED)
        ys.append(float(ofit.min()))
        b.close()
    return np.array(ys)


def _oracle_runs(power_up=False, seeds=SEEDS, evolver=0):
    wl = synth.tiny()
    p = wl.problems[0]
    return np.array([oracle.metade_run(wl.n_out, 16, p.obj, p.shift, p.rot, wl.inner_gens, wl.outer_gens,
                                       seed=s, power_up=power_up, evolver=evolver)[0] for s in seeds])


def test_final_meta_fitness_distribution_matches_oracle():
    from scipy.stats import ranksums
    g = _truncate(_gpu_runs())
    o = _truncate(_oracle_runs())
    stat, pval = ranksums(g, o)
    print("median gpu %.4g oracle %.4g, rank-sum p = %.3f" % (np.median(g), np.median(o), pval))
    assert pval > 0.05


def test_power_up_never_hurts():
    """Sec. III-D: with one-shot evaluation an executor's best after 5 G'
    generations is at most its best after G', so the last evolver
    generation's trials only gain and the final best cannot rise."""
    seeds = range(6)
    base, pu = _gpu_runs(False, seeds), _gpu_runs(True, seeds)
    assert np.all(pu <= base)
    ob, op = _oracle_runs(False, seeds), _oracle_runs(True, seeds)
    assert np.all(op <= ob)


def test_one_shot_runs_are_reproducible():
    a = _gpu_runs(False, range(2))
    b = _gpu_runs(False, range(2))
    np.testing.assert_array_equal(a, b)


def test_batched_and_plain_runs_agree_in_distribution():
    """The metric compares the batched path with the plain FP32 path at an
    equal FE budget: whole MetaDE runs on both (the plain path launches one
    executor per generation, no graph, no tuning) must give final
    meta-fitness distributions that the paper's rank-sum test at 0.05 does not
    separate, over 31 seeds."""
    import paper_2502_10470_gb300 as M
    from scipy.stats import ranksums
    batched = _truncate(_gpu_runs(path=M.METADE_PATH_BATCHED))
    plain = _truncate(_gpu_runs(path=M.METADE_PATH_PLAIN))
    stat, pval = ranksums(batched, plain)
    print("median batched %.4g plain %.4g, rank-sum p = %.3f" % (np.median(batched), np.median(plain), pval))
    assert pval > 0.05


def test_pso_evolver_runs_match_oracle_in_distribution():
    """Whole MetaDE runs with the PSO evolver: GPU against the FP64 oracle's
    PSO, 31 seeds, rank-sum test at 0.05."""
    import paper_2502_10470_gb300 as M
    from scipy.stats import ranksums
    g = _truncate(_gpu_runs(evolver=M.EVOLVER_PSO))
    o = _truncate(_oracle_runs(evolver=1))
    stat, pval = ranksums(g, o)
    print("PSO evolver: median gpu %.4g oracle %.4g, rank-sum p = %.3f" % (np.median(g), np.median(o), pval))
    assert pval > 0.05


@pytest.mark.parametrize("evolver", [2, 3], ids=["cso", "nes"])
def test_cso_nes_evolver_runs_match_oracle_in_distribution(evolver):
    """Whole MetaDE runs with the CSO and NES (xNES) evolvers: GPU against the
    FP64 oracle's, 31 seeds, rank-sum test at 0.05."""
    from scipy.stats import ranksums
    g = _truncate(_gpu_runs(evolver=evolver))
    o = _truncate(_oracle_runs(evolver=evolver))
    stat, pval = ranksums(g, o)
    print("evolver %d: median gpu %.4g oracle %.4g, rank-sum p = %.3f" % (evolver, np.median(g), np.median(o), pval))
    assert pval > 0.05
