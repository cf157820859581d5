"""Full-size workloads in the benchmark's launch configuration, checked on
sampled outputs that the FP64 oracle computes one by one, and by properties
that hold at any size.

- moderate: 600 executors x NP 100 x D 20, one-shot, the tuned batched plan
  (the headline benchmark's workload);
- precision: 64 executors x NP 512 x D 1000 on the tensor cores (BF16, FP8);
- full: 8 runs x 128 executors, NP 50..200, D 20..200, BF16 on the tensor
  cores for D >= the autotuned width (the headline benchmark's workload).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FIT_RTOL, TRIAL_ATOL, check_fitness, rel_err

pytestmark = pytest.mark.gpu

SAMPLE = [0, 57, 123, 199, 250, 333, 401, 478, 512, 599]   # spread over the six runs


def _moderate():
    import paper_2502_10470_gb300 as M
    wl = synth.moderate()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=1, n_out=wl.n_out)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 20)
    b.sync()
    return wl, b


def _compare_step(wl, k, pops, fits, theta, npops, nfits, gap_min, tol, unit, epoch=0, gen=0):
    """One generation of executor k against the oracle from the same state:
    selection bits wherever the fitness gap is decisive, trial rows of rows
    accepted on both sides, fitness against FP64 at the GPU's own rows, and
    rows the GPU kept unchanged."""
    p = wl.problems[int(wl.inst_prob[k])]
    out = oracle.pde_step(pops[k], fits[k], theta[k], p.obj, p.shift, p.rot, seed=wl.seed,
                          stream=oracle.stream_of(wl, k), epoch=epoch, gen=gen, lo=wl.lo, hi=wl.hi)
    decided = rel_err(out["ftrial"], fits[k].astype(np.float64)) > gap_min
    acc_or = out["accept"].astype(bool)
    acc_gpu = (nfits[k] != fits[k]) | np.any(npops[k] != pops[k], axis=1)
    np.testing.assert_array_equal(acc_gpu[decided], acc_or[decided], err_msg="selection, executor %d" % k)
    both = acc_gpu & acc_or
    if both.any():
        assert np.abs(npops[k][both] - out["trial"][both]).max() < TRIAL_ATOL
        check_fitness(nfits[k][both], npops[k][both], p, tol, unit)
    kept = ~acc_gpu
    np.testing.assert_array_equal(npops[k][kept], pops[k][kept])
    np.testing.assert_array_equal(nfits[k][kept], fits[k][kept])
    return int(decided.sum())


def test_moderate_full_size_generation_sampled():
    """The headline workload, tuned plan, one generation: ten executors
    spread over the six runs against the oracle's generation."""
    import paper_2502_10470_gb300 as M
    wl, b = _moderate()
    pops, fits = b.get_population()
    theta = b.theta.cpu().numpy()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    n = sum(_compare_step(wl, k, pops, fits, theta, npops, nfits, 2 * FIT_RTOL, FIT_RTOL, 0.0) for k in SAMPLE)
    assert n > 500
    b.close()


def test_moderate_full_size_500_generations_properties():
    """The benchmark's launch: 500 fused generations of all 600 executors in
    one call.  Every executor: rows inside the box, best_f / best_i the
    minimum of its stored fitness, and a best that never rose.  Sampled
    executors: each stored fitness agrees with the FP64 objective of its
    stored row (1e-4 relative: a stored value may carry the rounding of one
    accepted near tie, f(x) + difference, per generation)."""
    import paper_2502_10470_gb300 as M
    wl, b = _moderate()
    pops0, fits0 = b.get_population()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 500, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    best_f, best_i = b.best_f.cpu().numpy(), b.best_i.cpu().numpy()
    for k in range(wl.n_inst):
        assert np.all(npops[k] >= wl.lo) and np.all(npops[k] <= wl.hi)
        assert best_f[k] == nfits[k].min() and nfits[k][best_i[k]] == best_f[k]
        assert best_i[k] == int(np.argmin(nfits[k]))
        assert best_f[k] <= fits0[k].min()
    for k in SAMPLE:
        check_fitness(nfits[k], npops[k], wl.problems[int(wl.inst_prob[k])], 1e-4, 0.0, floor=1e-30)
    b.close()


@pytest.mark.parametrize("prec,tol,unit,gap", [(1, 4e-3, 2.0 ** -8, 0.1), (2, 3e-2, 2.0 ** -3, 0.3)],
                         ids=["bf16", "fp8e4m3"])
def test_precision_full_size_generation_sampled(prec, tol, unit, gap):
    """64 executors x NP 512 x D 1000 on the tensor cores, one generation:
    three executors (every row) against the oracle's generation, with the
    precision's fitness budget."""
    import paper_2502_10470_gb300 as M
    wl = synth.precision()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0, prec=prec)
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    b.sync()
    pops, fits = b.get_population()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    theta = wl.theta.astype(np.float32)
    for k in (0, 33, 63):
        _compare_step(wl, k, pops, fits, theta, npops, nfits, gap, tol, unit)
    b.close()


def _full():
    """The headline workload (8 runs x 128 executors, NP 50..200, D 20..200),
    BF16 context, autotuned plan, after the evolver's first trials."""
    import paper_2502_10470_gb300 as M
    wl = synth.full()
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=1, n_out=wl.n_out,
                prec=M.METADE_BF16)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 3)
    # the tuned width decides each executor's evaluation precision: initialise again under it
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    b.sync()
    return wl, b


def _full_budget(p, tc_min_dim):
    """(fitness rtol, operand unit, decisive gap) of an executor of the full
    workload: BF16 on the tensor cores, FP32 elsewhere."""
    return (4e-3, 2.0 ** -8, 0.1) if p.dim >= tc_min_dim else (FIT_RTOL, 0.0, 2 * FIT_RTOL)


def test_full_workload_generation_sampled():
    """The headline workload in the benchmark's launch configuration, one
    generation: two executors of every run (all rows) against the oracle's
    generation from the same state, with the budget of the precision each
    executor runs in."""
    import json
    import paper_2502_10470_gb300 as M
    wl, b = _full()
    tcmin = json.loads(M.metade_plan_info(b.ctx))["tc_min_dim"]
    pops, fits = b.get_population()
    theta = b.theta.cpu().numpy()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    n = 0
    for g in range(wl.n_groups):
        for k in (g * wl.n_out + 5, g * wl.n_out + 97):
            p = wl.problems[int(wl.inst_prob[k])]
            tol, unit, gap = _full_budget(p, tcmin)
            n += _compare_step(wl, k, pops, fits, theta, npops, nfits, gap, tol, unit)
    assert n > 500
    b.close()


def test_full_workload_200_generations_properties():
    """The benchmark's launch: 200 generations of all 1024 executors in one
    call.  Every executor: rows inside the box, best_f / best_i the minimum of
    its stored fitness, a best that never rose.  Sampled executors of every
    run: stored fitness against the FP64 objective of the stored row within
    the precision's budget (BF16 rows carry the GEMM's rounding; an accepted
    near tie stores f(x) + difference)."""
    import json
    import paper_2502_10470_gb300 as M
    wl, b = _full()
    tcmin = json.loads(M.metade_plan_info(b.ctx))["tc_min_dim"]
    pops0, fits0 = b.get_population()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 200, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    best_f, best_i = b.best_f.cpu().numpy(), b.best_i.cpu().numpy()
    for k in range(wl.n_inst):
        assert np.all(npops[k] >= wl.lo) and np.all(npops[k] <= wl.hi)
        assert best_f[k] == nfits[k].min() and best_i[k] == int(np.argmin(nfits[k]))
        assert best_f[k] <= fits0[k].min()
    for g in range(wl.n_groups):
        k = g * wl.n_out + 11
        p = wl.problems[int(wl.inst_prob[k])]
        tol, unit, _ = _full_budget(p, tcmin)
        check_fitness(nfits[k], npops[k], p, max(tol, 1e-4), unit, floor=1e-30)
    b.close()


def test_batching_full_size_generation_sampled():
    """512 ragged executors (NP 20..400, D 10..100: the small-D kernel and,
    by the autotuned FP32 width, the tile kernels or the CUDA-core GEMM
    pipeline), tuned plan, one generation: executors of every size class and
    objective against the oracle's generation."""
    import paper_2502_10470_gb300 as M
    from gpu_util import feasible_theta
    wl = synth.batching()
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    b = M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=0)
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 5)
    b.sync()
    pops, fits = b.get_population()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    theta = wl.theta.astype(np.float32)
    picked = []
    for d in (10, 20, 50, 100):          # two executors per dimension, different objectives
        ks = [k for k in range(wl.n_inst) if wl.problems[k].dim == d]
        objs_seen = set()
        for k in ks:
            if wl.problems[k].obj not in objs_seen:
                objs_seen.add(wl.problems[k].obj)
                picked.append(k)
            if len(objs_seen) == 2:
                break
    picked.append(int(np.argmax(wl.inst_np)))  # the largest population
    for k in picked:
        _compare_step(wl, k, pops, fits, theta, npops, nfits, 2 * FIT_RTOL, FIT_RTOL, 0.0)
    b.close()


def test_largest_executors_each_kernel():
    """Maximum sizes: the largest population the small-D kernel holds at
    D = 32 (population, trials and R in shared memory: NP 700), the largest
    accepted population (NP 1024) at D = 100 and 200 (tile kernels), and
    D = 300 (the per-generation pipeline in FP32); one generation against the
    oracle."""
    import json
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(99)
    dims, nps = [32, 100, 200, 300], [700, 1024, 1024, 600]   # NP 1024 is the largest accepted
    probs = [synth.make_problem(rng, d, k % 6) for k, d in enumerate(dims)]
    n = len(probs)
    th = synth.random_theta(rng, n)
    wl = synth.Workload(name="largest", problems=probs, inst_np=np.array(nps, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=4, one_shot=0, theta=th)
    b = M.Batch([(p.dim, p.obj, p.shift, p.rot) for p in probs], wl.inst_np, wl.inst_prob, wl.inst_group,
                seed=wl.seed, one_shot=0)
    kernels = {bk["kernel"] for bk in json.loads(M.metade_plan_info(b.ctx))["buckets"]}
    assert "fused_small" in kernels
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    b.sync()
    pops, fits = b.get_population()
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    theta = wl.theta.astype(np.float32)
    for k in range(n):
        _compare_step(wl, k, pops, fits, theta, npops, nfits, 2 * FIT_RTOL, FIT_RTOL, 0.0)
    b.close()
