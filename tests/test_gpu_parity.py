"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Bars: bit-exact for the initial population (one rounding of the same exact
value), for every index/mask/integer draw and for the decoded categorical
genes; FP32 trial coordinates within TRIAL_ATOL; FP32 fitness within 1e-5
relative of the FP64 value at the same point; selection bits equal wherever
the fitness gap exceeds the FP32 tolerance.
"""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_util import (FIT_RTOL, TRIAL_ATOL, check_fitness_fp32, feasible_theta, make_batch, random_state,
                      rel_err)

pytestmark = pytest.mark.gpu

PATHS = [0, 1]  # batched, plain
PATH_IDS = ["batched", "plain"]


def _wl_small():
    wl = synth.small_ragged()
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    return wl


def _wl_with_theta(wl, seed=3):
    rng = np.random.default_rng(seed)
    wl.theta = feasible_theta(synth.random_theta(rng, wl.n_inst), wl.inst_np)
    return wl


def _ragged_many():
    """Every strategy family across ragged sizes: 48 executors, NP 4..130,
    D 1..70 (tiles of 4/32 plus ragged tails)."""
    rng = np.random.default_rng(21)
    n = 48
    dims = rng.choice([1, 2, 3, 5, 10, 13, 20, 31, 33, 47, 64, 70], size=n)
    nps = rng.integers(4, 131, size=n)
    probs = [synth.make_problem(rng, int(d), int(k % 6)) for k, d in enumerate(dims)]
    th = synth.random_theta(rng, n)
    # make sure each (bl, br) pair and crossover appears
    for k in range(n):
        th[k, 2] = 1 + (k % 4)
        th[k, 3] = 1 + ((k // 4) % 4)
        th[k, 5] = 1 + (k % 3)
    wl = synth.Workload(name="ragged-many", problems=probs, inst_np=nps.astype(np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=2, outer_gens=1, seed=5, one_shot=0, theta=th)
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    return wl


# ------------------------------------------------------------------- init
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_init_bit_exact(path):
    for wl in (synth.tiny(), _wl_small()):
        b = make_batch(wl, path)
        import paper_2502_10470_gb300 as M
        M.metade_init(b.ctx, b.pop, b.fit, 0)
        b.sync()
        pops, fits = b.get_population()
        for k in range(wl.n_inst):
            p = wl.problems[int(wl.inst_prob[k])]
            want = oracle.init_pop(int(wl.inst_np[k]), p.dim, wl.seed, oracle.stream_of(wl, k), 0, wl.lo, wl.hi)
            np.testing.assert_array_equal(pops[k], want.astype(np.float32))
            check_fitness_fp32(fits[k], pops[k], p)
        b.close()


# ------------------------------------------------------------------- eval
@pytest.mark.parametrize("near", [False, True], ids=["box", "near-optimum"])
def test_eval_fp32_and_fp64(near):
    import torch
    import paper_2502_10470_gb300 as M
    wl = _ragged_many()
    b = make_batch(wl, 0)
    rng = np.random.default_rng(4)
    pops = []
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        if near:
            x = (p.shift[None, :] + rng.normal(0, 1e-2, (int(wl.inst_np[k]), p.dim))).astype(np.float32)
        else:
            x = synth.random_population(rng, int(wl.inst_np[k]), p.dim)
        pops.append(x)
    b.set_population(pops)
    f32 = torch.zeros(b.n_indiv, dtype=torch.float32, device="cuda")
    f64 = torch.zeros(b.n_indiv, dtype=torch.float64, device="cuda")
    M.metade_eval_pop(b.ctx, b.pop, M.METADE_FP32, f32)
    M.metade_eval_pop(b.ctx, b.pop, M.METADE_FP64, f64)
    b.sync()
    f32, f64 = f32.cpu().numpy(), f64.cpu().numpy()
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        want = oracle.eval_pop(p.obj, pops[k], p.shift, p.rot)
        sl = slice(b.fit_off[k], b.fit_off[k] + int(wl.inst_np[k]))
        check_fitness_fp32(f32[sl], pops[k], p, floor=1e-3 if near else 0.0)
        assert rel_err(f64[sl], want, 1e-12).max() < 1e-9, (k, p.obj, p.dim)
    b.close()


def test_eval_caller_points_fp64_and_fp32():
    """metade_eval on caller-given points (the final error f(x_best) - f* of
    Sec. IV-A is one such call): 300 points of random executors in one
    [n][ldx] buffer.  FP64 against the oracle's FP64 objective within 1e-12
    relative; FP32 bit-equal to the whole-population evaluation of the same
    rows (same kernel arithmetic); an executor id out of range latches EINVAL
    and yields NaN without touching the other points."""
    import torch
    import paper_2502_10470_gb300 as M
    wl = _ragged_many()
    b = make_batch(wl, 0)
    rng = np.random.default_rng(12)
    n = 300
    inst = rng.integers(0, wl.n_inst, n).astype(np.int32)
    ldx = int(np.max(b.dpad)) + 4
    x = np.zeros((n, ldx), dtype=np.float32)
    for r in range(n):
        d = int(b.dims[inst[r]])
        x[r, :d] = synth.random_population(rng, 1, d)[0]
    xd = torch.from_numpy(x).cuda()
    idd = torch.from_numpy(inst).cuda()
    f64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    f32 = torch.zeros(n, dtype=torch.float32, device="cuda")
    M.metade_eval(b.ctx, xd, n, idd, ldx, M.METADE_FP64, f64)
    M.metade_eval(b.ctx, xd, n, idd, ldx, M.METADE_FP32, f32)
    b.sync()
    f64, f32 = f64.cpu().numpy(), f32.cpu().numpy()
    for r in range(n):
        p = wl.problems[int(wl.inst_prob[inst[r]])]
        want = oracle.eval_pop(p.obj, x[r:r + 1, :p.dim], p.shift, p.rot)[0]
        assert abs(f64[r] - want) <= 1e-12 * max(abs(want), 1e-12), (r, p.obj, p.dim, f64[r], want)
    # FP32: the same rows placed in the population and evaluated there
    pops = [synth.random_population(rng, int(wl.inst_np[k]), int(b.dims[k])) for k in range(wl.n_inst)]
    first = {}
    for r in range(n):
        k = int(inst[r])
        if k not in first:
            first[k] = r
            pops[k][0] = x[r, :int(b.dims[k])]
    b.set_population(pops)
    fp = torch.zeros(b.n_indiv, dtype=torch.float32, device="cuda")
    M.metade_eval_pop(b.ctx, b.pop, M.METADE_FP32, fp)
    b.sync()
    fp = fp.cpu().numpy()
    for k, r in first.items():
        assert fp[b.fit_off[k]] == f32[r]
    # a bad executor id: EINVAL on the device, NaN for that point only
    bad = idd.clone()
    bad[7] = wl.n_inst
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    M.metade_eval(b.ctx, xd, n, bad, ldx, M.METADE_FP64, out)
    assert M.metade_sync(b.ctx) == M.METADE_EINVAL
    got = out.cpu().numpy()
    assert np.isnan(got[7]) and np.array_equal(np.delete(got, 7), np.delete(f64, 7))
    # host-side checks: ldx not a multiple of 4, unsupported precision
    with pytest.raises(M.MetadeError):
        M.metade_eval(b.ctx, xd, n, idd, ldx - 1, M.METADE_FP64, out)
    with pytest.raises(M.MetadeError):
        M.metade_eval(b.ctx, xd, n, idd, ldx, M.METADE_BF16, out)
    M.metade_eval(b.ctx, xd, 0, idd, ldx, M.METADE_FP64, out)  # n = 0: nothing to do
    assert M.metade_sync(b.ctx) == M.METADE_OK
    b.close()


# ---------------------------------------------------------------- records
@pytest.mark.parametrize("gen", [0, 7, 123456])
def test_draw_record_bit_exact(gen):
    import torch
    import paper_2502_10470_gb300 as M
    wl = _ragged_many()
    b = make_batch(wl, 0)
    pops, fits = random_state(wl, seed=gen % 97)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    rec = torch.zeros((b.n_indiv, M.REC_FIELDS), dtype=torch.int32, device="cuda")
    M.metade_draw_record(b.ctx, b.fit, b.theta, 3, gen, rec)
    assert b.sync() is None
    rec = rec.cpu().numpy()
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed,
                              stream=oracle.stream_of(wl, k), epoch=3, gen=gen, lo=wl.lo, hi=wl.hi)
        sl = slice(b.fit_off[k], b.fit_off[k] + int(wl.inst_np[k]))
        np.testing.assert_array_equal(rec[sl], out["rec"], err_msg="executor %d" % k)
    b.close()


# ---------------------------------------------------------------- one step
def _step_and_compare(wl, path, fit_inf, gen=4, epoch=2):
    import paper_2502_10470_gb300 as M
    b = make_batch(wl, path)
    pops, fits = random_state(wl, seed=gen, fit_inf=fit_inf)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, epoch, gen, 1, b.best_f, b.best_i)
    b.sync()
    npops, nfits = b.get_population()
    best_f = b.best_f.cpu().numpy()
    n_checked = 0
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed,
                              stream=oracle.stream_of(wl, k), epoch=epoch, gen=gen, lo=wl.lo, hi=wl.hi)
        gap = rel_err(out["ftrial"], fits[k].astype(np.float64))
        decided = gap > 2 * FIT_RTOL
        acc_or = out["accept"].astype(bool)
        # rows the GPU replaced: fitness or row changed
        acc_gpu = (nfits[k] != fits[k]) | np.any(npops[k] != pops[k], axis=1)
        np.testing.assert_array_equal(acc_gpu[decided], acc_or[decided], err_msg="selection, executor %d" % k)
        both = acc_gpu & acc_or
        if both.any():
            err = np.abs(npops[k][both] - out["trial"][both]).max()
            assert err < TRIAL_ATOL, ("trial", k, err)
            # FP32 fitness vs FP64 at the GPU's own float32 trial
            check_fitness_fp32(nfits[k][both], npops[k][both], p)
        kept = ~acc_gpu
        np.testing.assert_array_equal(npops[k][kept], pops[k][kept])
        np.testing.assert_array_equal(nfits[k][kept], fits[k][kept])
        assert best_f[k] == nfits[k].min()
        n_checked += int(both.sum())
    b.close()
    return n_checked


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_one_step_all_accepted_trials(path):
    """Stored fitness +inf: every trial is accepted, so the new population is
    the trial matrix itself, compared coordinate by coordinate."""
    wl = _ragged_many()
    n = _step_and_compare(wl, path, fit_inf=True)
    assert n == wl.individuals()


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("gen", [0, 9])
def test_one_step_with_selection(path, gen):
    wl = _ragged_many()
    _step_and_compare(wl, path, fit_inf=False, gen=gen)


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_tiny_and_small_ragged_step(path):
    _step_and_compare(_wl_with_theta(synth.tiny()), path, fit_inf=False)
    _step_and_compare(_wl_small(), path, fit_inf=True)


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_multi_generation_resynced(path):
    """Ten fused generations compared one generation at a time: the oracle
    restarts every generation from the GPU's state (trajectories of FP32 and
    FP64 runs legitimately drift apart, so whole runs are compared as
    distributions elsewhere)."""
    import paper_2502_10470_gb300 as M
    wl = _wl_with_theta(synth.tiny(), seed=8)
    b = make_batch(wl, path)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    b.set_theta(wl.theta)
    b.sync()
    for g in range(10):
        pops, fits = b.get_population()
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, g, 1, b.best_f, b.best_i)
        b.sync()
        npops, nfits = b.get_population()
        for k in range(wl.n_inst):
            p = wl.problems[0]
            out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed,
                                  stream=oracle.stream_of(wl, k), epoch=0, gen=g)
            decided = rel_err(out["ftrial"], fits[k]) > 2 * FIT_RTOL
            acc_gpu = nfits[k] != fits[k]
            np.testing.assert_array_equal(acc_gpu[decided], out["accept"].astype(bool)[decided])
            assert nfits[k].min() <= fits[k].min()
    b.close()


def test_fused_generations_equal_single_steps():
    """n_gens = 5 in one fused launch equals five launches of one generation
    (same kernels, same draws; the only state is the population)."""
    import paper_2502_10470_gb300 as M
    wl = _ragged_many()
    outs = []
    for split in (False, True):
        b = make_batch(wl, 0)
        pops, fits = random_state(wl, seed=1)
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        if split:
            for g in range(5):
                M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 10 + g, 1, None, None)
        else:
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 10, 5, None, None)
        b.sync()
        outs.append(b.get_population())
        b.close()
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(outs[0][0][k], outs[1][0][k])
        np.testing.assert_array_equal(outs[0][1][k], outs[1][1][k])


# ------------------------------------------------------------------ evolver
def test_fused_pbest_pool_with_equal_fitness():
    """Inside one fused launch the small-D kernel re-ranks the pbest pool
    among the previous pool and the individuals whose fitness fell; a launch
    of one generation ranks every individual.  With pairs of identical rows
    (equal fitness, so the index decides the order) and a 30% pool, eight
    fused generations equal eight single-generation launches bit for bit."""
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(33)
    n = 24
    dims = rng.choice([2, 5, 10, 20, 31], size=n)
    nps = rng.choice([8, 17, 40, 100, 130], size=n)
    probs = [synth.make_problem(rng, int(d), int(k % 6)) for k, d in enumerate(dims)]
    th = synth.random_theta(rng, n)
    for k in range(n):
        th[k, 2] = 3 if k % 2 == 0 else 1 + (k // 2) % 4   # pbest base or pbest right vector
        th[k, 3] = 3 if k % 2 == 1 else 1 + (k // 2) % 4
        th[k, 5] = 1 + (k % 3)
    wl = synth.Workload(name="pbest-equal", problems=probs, inst_np=nps.astype(np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=8, outer_gens=1, seed=7, one_shot=0, theta=th,
                        p_best_pct=30)
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    pops, fits = random_state(wl, seed=4)
    for k in range(n):
        pops[k][1::2] = pops[k][0:pops[k].shape[0] - 1:2][: pops[k][1::2].shape[0]]
        fits[k][1::2] = fits[k][0:fits[k].shape[0] - 1:2][: fits[k][1::2].shape[0]]
    outs = []
    for split in (False, True):
        b = make_batch(wl, 0)
        info = json.loads(M.metade_plan_info(b.ctx))
        assert all(bk["kernel"] == "fused_small" for bk in info["buckets"])
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        if split:
            for g in range(8):
                M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 20 + g, 1, None, None)
        else:
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 20, 8, None, None)
        b.sync()
        outs.append(b.get_population())
        b.close()
    for k in range(n):
        np.testing.assert_array_equal(outs[0][0][k], outs[1][0][k])
        np.testing.assert_array_equal(outs[0][1][k], outs[1][1][k])


def test_outer_init_trial_decode_select():
    import torch
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    wl2 = synth.Workload(name="two-runs", problems=wl.problems * 2, inst_np=np.full(16, 16, dtype=np.int32),
                         inst_prob=np.repeat([0, 1], 8).astype(np.int32),
                         inst_group=np.repeat([0, 1], 8).astype(np.int32), n_groups=2, n_out=8, inner_gens=2,
                         outer_gens=2, seed=11, one_shot=1)
    b = make_batch(wl2, 0)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    b.sync()
    opop = b.opop.cpu().numpy().reshape(2, 8, 6)
    for g in range(2):
        want, wfit = oracle.outer_init(8, wl2.seed, g)
        np.testing.assert_array_equal(opop[g], want.astype(np.float32))
        assert np.all(np.isinf(b.ofit.cpu().numpy()))
    for og in (0, 3):
        M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, og, 0)
        b.sync()
        trial = b.trial.cpu().numpy().reshape(2, 8, 6)
        theta = b.theta.cpu().numpy().reshape(2, 8, 6)
        for g in range(2):
            want = oracle.outer_trial(opop[g], wl2.seed, g, og)
            assert np.abs(trial[g] - want).max() < 2e-6
            for i in range(8):
                # decoding is compared on the GPU's own float32 trial (same input, same floor)
                np.testing.assert_array_equal(theta[g, i], oracle.decode(trial[g, i]).astype(np.float32))
    meta = torch.tensor(np.random.default_rng(0).uniform(0, 10, 16).astype(np.float32), device="cuda")
    meta[3] = float("nan")
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, meta, 0, 1)
    b.sync()
    npop, nfit = b.opop.cpu().numpy(), b.ofit.cpu().numpy()
    m = meta.cpu().numpy()
    for e in range(16):
        if e == 3:  # NaN counts as +inf and still beats the initial +inf
            assert np.isinf(nfit[e])
        else:
            assert nfit[e] == m[e]
            np.testing.assert_array_equal(npop[e], b.trial.cpu().numpy()[e])
    b.close()


def test_pso_evolver_move_and_select():
    """PSO evolver: generation 0 evaluates the initial swarm exactly; a later
    move matches the FP64 oracle's update from the same float32 state (two
    runs, so gbest is per run), decoding is the DE evolver's, and selection
    copies positions into the personal bests."""
    import torch
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    wl2 = synth.Workload(name="two-runs", problems=wl.problems * 2, inst_np=np.full(16, 16, dtype=np.int32),
                         inst_prob=np.repeat([0, 1], 8).astype(np.int32),
                         inst_group=np.repeat([0, 1], 8).astype(np.int32), n_groups=2, n_out=8, inner_gens=2,
                         outer_gens=2, seed=13, one_shot=1)
    b = make_batch(wl2, 0, evolver=M.EVOLVER_PSO)
    assert tuple(b.trial.shape) == (16, 12)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    b.sync()
    tr = b.trial.cpu().numpy()
    np.testing.assert_array_equal(tr[:, :6], b.opop.cpu().numpy())
    assert not tr[:, 6:].any()
    # a mid-run state: personal bests, fitness with a tie for the run best, positions, velocities
    rng = np.random.default_rng(3)
    lb, ub = synth.OUTER_LB, synth.OUTER_UB
    pbest = (lb + (ub - lb) * rng.random((16, 6))).astype(np.float32)
    x = (lb + (ub - lb) * rng.random((16, 6))).astype(np.float32)
    v = (0.4 * (ub - lb) * (rng.random((16, 6)) - 0.5)).astype(np.float32)
    pfit = rng.uniform(1, 10, 16).astype(np.float32)
    pfit[[2, 5]] = 0.5           # run 0: tie, index 2 is gbest
    pfit[12] = 0.25              # run 1: gbest 12
    b.opop.copy_(torch.from_numpy(pbest))
    b.ofit.copy_(torch.from_numpy(pfit))
    b.trial.copy_(torch.from_numpy(np.concatenate([x, v], axis=1)))
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 4, 0)
    b.sync()
    tr = b.trial.cpu().numpy()
    theta = b.theta.cpu().numpy()
    for g in range(2):
        sl = slice(8 * g, 8 * g + 8)
        wx, wv = oracle.pso_move(pbest[sl], pfit[sl], x[sl], v[sl], seed=wl2.seed, group=g, gen=4)
        assert np.abs(tr[sl, :6] - wx).max() < 1e-5
        assert np.abs(tr[sl, 6:] - wv).max() < 1e-5
        for i in range(8):
            np.testing.assert_array_equal(theta[8 * g + i], oracle.decode(tr[8 * g + i, :6]).astype(np.float32))
    meta = torch.tensor(np.where(np.arange(16) % 2 == 0, 0.1, 100.0).astype(np.float32), device="cuda")
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, meta, 4, 1)
    b.sync()
    npb, nf = b.opop.cpu().numpy(), b.ofit.cpu().numpy()
    for e in range(16):
        if e % 2 == 0:
            np.testing.assert_array_equal(npb[e], tr[e, :6])
            assert nf[e] == np.float32(0.1)
        else:
            np.testing.assert_array_equal(npb[e], pbest[e])
            assert nf[e] == pfit[e]
    b.close()


def _two_runs(n_out=8, seed=13):
    wl = synth.tiny()
    n = 2 * n_out
    return synth.Workload(name="two-runs", problems=wl.problems * 2, inst_np=np.full(n, 16, dtype=np.int32),
                          inst_prob=np.repeat([0, 1], n_out).astype(np.int32),
                          inst_group=np.repeat([0, 1], n_out).astype(np.int32), n_groups=2, n_out=n_out,
                          inner_gens=2, outer_gens=2, seed=seed, one_shot=1)


@pytest.mark.parametrize("n_out", [8, 9, 4095, 4096])  # 4096: the largest swarm the pairing holds
def test_cso_evolver_move_and_select(n_out):
    """CSO evolver: generation 0 evaluates the initial swarm, all flagged; a
    later move pairs each run exactly as the oracle (flags bit-exact: the
    permutation and the pair decisions are integer work on the same stored
    fitness), moves the losers within FP32 rounding of the FP64 update, keeps
    the winners; selection replaces the flagged particles unconditionally."""
    import torch
    import paper_2502_10470_gb300 as M
    wl2 = _two_runs(n_out)
    n = 2 * n_out
    b = make_batch(wl2, 0, evolver=M.EVOLVER_CSO)
    assert tuple(b.trial.shape) == (n, 13)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 0, 0)
    b.sync()
    tr = b.trial.cpu().numpy()
    np.testing.assert_array_equal(tr[:, :6], b.opop.cpu().numpy())
    assert not tr[:, 6:12].any() and (tr[:, 12] == 1).all()
    rng = np.random.default_rng(5)
    lb, ub = synth.OUTER_LB, synth.OUTER_UB
    x = (lb + (ub - lb) * rng.random((n, 6))).astype(np.float32)
    v = (0.3 * (ub - lb) * (rng.random((n, 6)) - 0.5)).astype(np.float32)
    fit = rng.uniform(1, 10, n).astype(np.float32)
    fit[[1, 3]] = 0.5                                           # an equal-fitness pair decides by index
    b.opop.copy_(torch.from_numpy(x))
    b.ofit.copy_(torch.from_numpy(fit))
    b.trial.copy_(torch.from_numpy(np.concatenate([x, v, np.zeros((n, 1), np.float32)], axis=1)))
    for gen in (1, 6):
        M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, gen, 0)
        b.sync()
        tr = b.trial.cpu().numpy()
        theta = b.theta.cpu().numpy()
        for g in range(2):
            sl = slice(n_out * g, n_out * (g + 1))
            wx, wv, wf = oracle.cso_move(x[sl], fit[sl], v[sl], seed=wl2.seed, group=g, gen=gen)
            np.testing.assert_array_equal(tr[sl, 12].astype(np.int32), wf)
            assert wf.sum() == n_out // 2
            assert np.abs(tr[sl, :6] - wx).max() < 1e-5
            assert np.abs(tr[sl, 6:12] - wv).max() < 1e-5
            np.testing.assert_array_equal(tr[sl, :6][wf == 0], x[sl][wf == 0])
            for i in range(n_out):
                np.testing.assert_array_equal(theta[n_out * g + i], oracle.decode(tr[n_out * g + i, :6]).astype(np.float32))
        b.trial.copy_(torch.from_numpy(np.concatenate([x, v, np.zeros((n, 1), np.float32)], axis=1)))
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, 6, 0)
    b.sync()
    tr = b.trial.cpu().numpy()
    meta = np.full(n, 50.0, dtype=np.float32)
    meta[0] = np.nan
    M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, torch.from_numpy(meta).cuda(), 6, 1)
    b.sync()
    npop, nf = b.opop.cpu().numpy(), b.ofit.cpu().numpy()
    for g in range(2):
        sl = slice(n_out * g, n_out * (g + 1))
        wp, wf = oracle.cso_select(x[sl], fit[sl], tr[sl, :6], tr[sl, 12].astype(np.int32), meta[sl])
        np.testing.assert_array_equal(npop[sl], wp.astype(np.float32))
        np.testing.assert_array_equal(nf[sl], wf.astype(np.float32))
    b.close()


def test_nes_evolver_sample_and_update():
    """NES (xNES) evolver: generation 0 sets the oracle's initial distribution;
    the samples (standard normals and clip(z)) and their decoding match the
    FP64 oracle from the same state; the update matches the oracle's
    natural-gradient step (the oracle's expm by Jacobi eigenvectors, the
    kernel's by Taylor scaling and squaring) and keeps det B = 1; population
    and fitness then hold the samples and their meta-fitness."""
    import torch
    import paper_2502_10470_gb300 as M
    n_out = 12
    wl2 = _two_runs(n_out, seed=17)
    b = make_batch(wl2, 0, evolver=M.EVOLVER_NES)
    assert tuple(b.trial.shape) == (2, 12 * n_out + 96)

    def state(g):
        blk = b.trial.cpu().numpy()[g]
        return blk[12 * n_out:12 * n_out + 86].copy().view(np.float64)

    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    rng = np.random.default_rng(2)
    st_prev = [oracle.nes_init(), oracle.nes_init()]
    for gen in range(4):
        M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, None, gen, 0)
        b.sync()
        blk = b.trial.cpu().numpy()
        theta = b.theta.cpu().numpy()
        for g in range(2):
            st = state(g)
            if gen == 0:
                np.testing.assert_allclose(st, st_prev[g], rtol=1e-14, atol=1e-15)
            ws, wz, wzc = oracle.nes_sample(st, n_out, seed=wl2.seed, group=g, gen=gen)
            smp = blk[g, :12 * n_out].reshape(n_out, 12)
            ds = np.abs(smp[:, 6:] - ws) / (1 + np.abs(ws))
            dz = np.abs(smp[:, :6] - wzc) / (1 + np.abs(wzc))
            assert ds.max() < 1e-6 and dz.max() < 1e-6, (gen, g, ds.max(), dz.max(), smp[:2], ws[:2], wzc[:2], st)
            for k in range(n_out):
                np.testing.assert_array_equal(theta[n_out * g + k], oracle.decode(smp[k, :6]).astype(np.float32))
        meta = rng.uniform(0, 5, 2 * n_out).astype(np.float32)
        meta[3] = meta[4]                                   # equal meta-fitness ranks by index
        meta[7] = np.nan
        before = [state(g) for g in range(2)]
        smps = [b.trial.cpu().numpy()[g, :12 * n_out].reshape(n_out, 12).copy() for g in range(2)]
        M.metade_outer_step(b.ctx, b.opop, b.ofit, b.trial, b.theta, torch.from_numpy(meta).cuda(), gen, 1)
        b.sync()
        opop, ofit = b.opop.cpu().numpy(), b.ofit.cpu().numpy()
        for g in range(2):
            sl = slice(n_out * g, n_out * (g + 1))
            want = oracle.nes_update(before[g], smps[g][:, 6:].astype(np.float64), meta[sl].astype(np.float64))
            got = state(g)
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
            assert abs(np.linalg.det(got[7:].reshape(6, 6)) - 1.0) < 1e-9
            np.testing.assert_array_equal(opop[sl], smps[g][:, :6])
            np.testing.assert_array_equal(ofit[sl], np.where(np.isnan(meta[sl]), np.inf, meta[sl]))
    b.close()


@pytest.mark.parametrize("evolver", [2, 3], ids=["cso", "nes"])
def test_cso_nes_outer_generation_graph_matches_direct(evolver):
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    res = []
    for use_graph in (False, True):
        b = make_batch(wl, 0, evolver=evolver)
        M.metade_outer_init(b.ctx, b.opop, b.ofit)
        for og in range(3):
            M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i,
                                      og, 10, use_graph)
        assert M.metade_sync(b.ctx) == 0
        res.append((b.opop.cpu().numpy(), b.ofit.cpu().numpy(), b.trial.cpu().numpy()))
        b.close()
    for a, c in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, c)
    assert np.isfinite(res[0][1]).all()


def test_cso_run_best_never_rises():
    """In CSO the swarm's best particle wins its pair and is kept, so each
    run's best stored meta-fitness never rises from one evolver generation
    to the next (generation 0 evaluates everyone)."""
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    b = make_batch(wl, 0, evolver=M.EVOLVER_CSO)
    M.metade_outer_init(b.ctx, b.opop, b.ofit)
    best = []
    for og in range(6):
        M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i,
                                  og, 10, True)
        b.sync()
        best.append(float(b.ofit.min().item()))
    assert M.metade_sync(b.ctx) == 0
    assert all(y1 <= y0 for y0, y1 in zip(best, best[1:])), best
    b.close()


def test_outer_generation_graph_matches_direct():
    import paper_2502_10470_gb300 as M
    wl = synth.tiny()
    res = []
    for use_graph in (False, True):
        b = make_batch(wl, 0)
        M.metade_outer_init(b.ctx, b.opop, b.ofit)
        for og in range(3):
            M.metade_outer_generation(b.ctx, b.opop, b.ofit, b.trial, b.theta, b.pop, b.fit, b.best_f, b.best_i,
                                      og, 20, use_graph)
        b.sync()
        res.append((b.opop.cpu().numpy(), b.ofit.cpu().numpy(), b.pop.cpu().numpy()))
        b.close()
    for a, c in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, c)


# -------------------------------------------------------------- edge cases
def test_invalid_theta_sets_sticky_status():
    import paper_2502_10470_gb300 as M
    wl = _wl_small()
    b = make_batch(wl, 0)
    th = wl.theta.copy()
    th[2, 4] = 9  # dn outside {1..4}
    b.set_theta(th)
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 2, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_EINVAL
    assert M.metade_sync(b.ctx) == M.METADE_OK  # cleared
    th = wl.theta.copy()
    th[0, 4] = 4  # NP = 4 cannot hold 2 dn + 1 distinct draws
    b.set_theta(th)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
    assert M.metade_sync(b.ctx) == M.METADE_EINVAL
    b.close()


def test_zero_generations_and_empty_batch():
    import paper_2502_10470_gb300 as M
    wl = _wl_small()
    b = make_batch(wl, 0)
    pops, fits = random_state(wl)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 0, b.best_f, b.best_i)
    b.sync()
    bf = b.best_f.cpu().numpy()
    bi = b.best_i.cpu().numpy()
    for k in range(wl.n_inst):
        assert bf[k] == fits[k].min() and bi[k] == int(np.argmin(fits[k]))
    b.close()
    e = M.Batch([(3, 0, np.zeros(3, np.float32), np.eye(3, dtype=np.float32))], [], [])
    M.metade_inner_step(e.ctx, e.pop, e.fit, e.theta, 0, 0, 3, None, None)
    assert M.metade_sync(e.ctx) == M.METADE_OK
    e.close()


def test_plain_path_one_launch_per_executor_generation():
    """The plain FP32 arm is one cooperative launch per executor per
    generation (its three phases separated by grid barriers inside the
    launch); the generation still matches the oracle (the parity tests above
    run the plain path too)."""
    import paper_2502_10470_gb300 as M
    wl = _wl_small()
    b = make_batch(wl, 1)
    pops, fits = random_state(wl, seed=6)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    l0 = M.metade_launch_count(b.ctx)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 3, None, None)
    assert M.metade_launch_count(b.ctx) - l0 == 3 * wl.n_inst
    assert M.metade_sync(b.ctx) == M.METADE_OK
    b.close()


def test_bad_configs_rejected_on_host():
    import paper_2502_10470_gb300 as M
    z = np.zeros(4, np.float32)
    eye = np.eye(2, dtype=np.float32)
    with pytest.raises(M.MetadeError):
        M.Batch([(2, 0, z[:2], eye)], [3], [0])           # NP < 4
    with pytest.raises(M.MetadeError):
        M.Batch([(2, 7, z[:2], eye)], [8], [0])           # unknown objective
    with pytest.raises(M.MetadeError):
        M.Batch([(2, 0, z[:2], eye)], [8], [1])           # problem index out of range
    with pytest.raises(M.MetadeError):
        M.Batch([(2, 0, z[:2], eye)], [8] * 6, [0] * 6, n_out=4)  # 6 executors, evolver of 4
    with pytest.raises(M.MetadeError):
        M.Batch([(2, 0, z[:2], eye)], [8], [0], lo=1.0, hi=-1.0)


# ------------------------------------------------------------ near ties
@pytest.mark.parametrize("tie_fp64", [0, 1], ids=["difference", "fp64"])
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_near_tie_decisions_match_fp64(tie_fp64, path):
    """Selection ties (|f(u) - f(x)| <= band(D) f(x), band(D) = max(1e-6,
    2^-21 sqrt(D))) are decided like FP64 does; the pairs checked lie within
    half the band, where the FP32 values alone already flag them as ties.
    Population on a grid of 8 and F = 2^-20 make the trial x_i + F (x_r0 - x_r1)
    exact in float32, so both implementations see the same u; the ground truth
    is the sign of the FP64 difference f(u) - f(x) of the oracle.  D spans the
    per-thread (<= 32), tile (<= 128) and group (<= 256) kernels; with FP64
    re-evaluation an accepted tie stores min(f32(f64 f(u)), f(x)) exactly."""
    import torch
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(31)
    n = 24
    dims = [2, 5, 10, 20, 33, 40, 100, 200] * 3
    probs = [synth.make_problem(rng, dims[k], k % 6) for k in range(n)]
    nps = np.full(n, 64, dtype=np.int32)
    wl = synth.Workload(name="near-ties", problems=probs, inst_np=nps, inst_prob=np.arange(n, dtype=np.int32),
                        inst_group=np.arange(n, dtype=np.int32), n_groups=n, n_out=0, inner_gens=1,
                        outer_gens=1, seed=9, one_shot=0)
    theta = np.tile(np.array([2.0 ** -20, 0.0, 4, 4, 1, 1], dtype=np.float32), (n, 1))
    pops = [(rng.integers(-12, 13, (64, probs[k].dim)) * 8.0).astype(np.float32) for k in range(n)]
    fits = [oracle.eval_pop(probs[k].obj, pops[k], probs[k].shift, probs[k].rot).astype(np.float32)
            for k in range(n)]
    b = make_batch(wl, path, tie_fp64=tie_fp64)
    b.set_population(pops, fits)
    b.set_theta(theta)
    rec = torch.zeros((b.n_indiv, M.REC_FIELDS), dtype=torch.int32, device="cuda")
    M.metade_draw_record(b.ctx, b.fit, b.theta, 0, 0, rec)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
    b.sync()
    rec = rec.cpu().numpy()
    npops, nfits = b.get_population()
    checked = 0
    for k in range(n):
        p = probs[k]
        r = rec[b.fit_off[k]:b.fit_off[k] + 64]
        out = oracle.pde_step(pops[k], fits[k], theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=0, gen=0)
        u = pops[k].astype(np.float64).copy()
        for i in range(64):
            j = r[i, 2]
            u[i, j] += 2.0 ** -20 * (float(pops[k][r[i, 9], j]) - float(pops[k][r[i, 10], j]))
        np.testing.assert_array_equal(u, out["trial"])           # the trial is exact on both sides
        assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
        fu = oracle.eval_pop(p.obj, u, p.shift, p.rot)
        fx = oracle.eval_pop(p.obj, pops[k], p.shift, p.rot)
        delta = fu - fx
        band = max(1e-6, 2.0 ** -21 * np.sqrt(p.dim))
        tie = (np.abs(delta) <= 0.5 * band * np.abs(fx)) & (np.abs(delta) > 1e-10 * np.abs(fx))
        took = np.any(npops[k] != pops[k], axis=1)
        np.testing.assert_array_equal(took[tie], (delta <= 0)[tie], err_msg="executor %d obj %d" % (k, p.obj))
        assert np.all(nfits[k] <= fits[k])                      # stored fitness never rises
        if tie_fp64:
            a = tie & took
            np.testing.assert_array_equal(nfits[k][a], np.minimum(fu[a].astype(np.float32), fits[k][a]))
        checked += int(tie.sum())
    b.close()
    assert checked > 200


def test_autotune_changes_speed_not_results():
    """The autotuner only picks block shapes; every individual's arithmetic
    and every reduction's tie-breaking are independent of them, so results
    are bit-identical before and after tuning."""
    import paper_2502_10470_gb300 as M
    wl = _ragged_many()
    outs = []
    for tune in (False, True):
        b = make_batch(wl, 0)
        pops, fits = random_state(wl, seed=2)
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        if tune:
            M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 2)
            info = json.loads(M.metade_plan_info(b.ctx))
            assert all("autotune_ms" in bk for bk in info["buckets"])
            # tuning used copies: the caller's state is untouched
            p2, f2 = b.get_population()
            for k in range(wl.n_inst):
                np.testing.assert_array_equal(p2[k], pops[k])
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 3, 4, b.best_f, b.best_i)
        b.sync()
        outs.append(b.get_population())
        b.close()
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(outs[0][0][k], outs[1][0][k])
        np.testing.assert_array_equal(outs[0][1][k], outs[1][1][k])


# ------------------------------------------------------------ bounded waits
def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The tensor-core pipeline's bounded mbarrier wait, on its own: on a
    barrier that nothing arrives at it gives up after its rounds with
    METADE_ETIMEOUT (no fault, no hang), on a completed phase it returns at
    once, and the device then runs a generation that matches the oracle."""
    import paper_2502_10470_gb300 as M
    st, done, sec = M.metade_wait_check(False, 1 << 16)
    assert st == M.METADE_ETIMEOUT and done == 0 and sec > 0.0
    st, done, sec1 = M.metade_wait_check(True, 1 << 16)
    assert st == M.METADE_OK and done == 1 and sec1 < sec
    assert M.metade_wait_check(2, 1)[0] == M.METADE_EINVAL
    _step_and_compare(_wl_with_theta(synth.tiny()), 0, fit_inf=False)
