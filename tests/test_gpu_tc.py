"""Large-D executors on the tensor cores (tcgen05 rotation GEMM with the
objective fused into the epilogue), BF16 and bf16x3, against the FP64 oracle.

The trial vectors are built by the same FP32 code as the other paths, so they
must agree with the oracle to TRIAL_ATOL; the fitness carries the rotation's
reduced precision.  Against FP64 at the GPU's own trial it must be within
RTOL relative, or within the first-order effect of the precision's rounding
budget on z: each product's operands carry a relative error of 2^-8 for BF16
(two roundings to 8-bit mantissas) and about 2^-16 for bf16x3 (the dropped
lo*lo term and the lo parts' own rounding)."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TRIAL_ATOL, check_fitness, feasible_theta, make_batch, random_state, rel_err

pytestmark = pytest.mark.gpu

TOL = {1: 4e-3, 3: 1e-5}     # relative: 2^-8 (BF16), 1e-5 (bf16x3, as FP32)
UNIT = {1: 2.0 ** -8, 3: 2.0 ** -16}


def _wl(seed=41):
    rng = np.random.default_rng(seed)
    dims, nps, objs = [300, 260, 520, 256], [130, 64, 200, 17], [2, 0, 1, 4]
    probs = [synth.make_problem(rng, d, o) for d, o in zip(dims, objs)]
    n = len(probs)
    th = synth.random_theta(rng, n)
    th[:, 5] = [1, 2, 3, 1]
    wl = synth.Workload(name="tc-ragged", problems=probs, inst_np=np.array(nps, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=3, one_shot=0, theta=th)
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    return wl


@pytest.mark.parametrize("prec", [1, 3], ids=["bf16", "bf16x3"])
def test_tc_one_step_against_oracle(prec):
    import paper_2502_10470_gb300 as M
    wl = _wl()
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["tensor_core"]["executors"] == wl.n_inst
    pops, fits = random_state(wl, seed=5, fit_inf=True)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 1, 2, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    worst = 0.0
    for k in range(wl.n_inst):
        p = wl.problems[k]
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=1, gen=2)
        assert np.abs(npops[k] - out["trial"]).max() < TRIAL_ATOL
        f64 = oracle.eval_pop(p.obj, npops[k], p.shift, p.rot)
        worst = max(worst, float(rel_err(nfits[k], f64, 1e-30).max()))
        frac = check_fitness(nfits[k], npops[k], p, TOL[prec], UNIT[prec])
        print("executor", k, "D", p.dim, "obj", p.obj, "beyond rtol:", frac)
    print("worst relative fitness error", worst)
    b.close()


@pytest.mark.parametrize("prec", [1, 3], ids=["bf16", "bf16x3"])
def test_tc_selection_and_generations(prec):
    """Several generations with real stored fitness: the best never rises,
    and a generation's selection matches FP64 wherever the fitness gap
    exceeds the precision's tolerance."""
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=43)
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    pops, fits = random_state(wl, seed=7)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    last = [f.min() for f in fits]
    for g in range(3):
        pops, fits = b.get_population()
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, g, 1, b.best_f, b.best_i)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        npops, nfits = b.get_population()
        for k in range(wl.n_inst):
            p = wl.problems[k]
            out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                                  epoch=0, gen=g)
            decided = rel_err(out["ftrial"], fits[k]) > 0.1 if prec == 1 else rel_err(out["ftrial"], fits[k]) > 1e-3
            acc = np.any(npops[k] != pops[k], axis=1) | (nfits[k] != fits[k])
            np.testing.assert_array_equal(acc[decided], out["accept"].astype(bool)[decided])
            assert nfits[k].min() <= last[k]
            last[k] = nfits[k].min()
    b.close()
