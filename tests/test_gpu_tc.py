"""Large-D executors on the tensor cores (tcgen05 rotation GEMM with the
objective fused into the epilogue), BF16, bf16x3 and FP8-e4m3, against the
FP64 oracle; and the same pipeline in FP32 with the GEMM on the CUDA cores
(k_rot_simt, for D_pad > 256), whose operands are exact (unit 0).

The trial vectors are built by the same FP32 code as the other paths, so they
must agree with the oracle to TRIAL_ATOL; the fitness carries the rotation's
reduced precision.  Against FP64 at the GPU's own trial it must be within
RTOL relative, or within the first-order effect of the precision's rounding
budget on z: each product's operands carry a relative error of 2^-8 for BF16
(two roundings to 8-bit mantissas), about 2^-16 for bf16x3 (the dropped
lo*lo term and the lo parts' own rounding) and 2^-3 for e4m3 (two roundings
to 4-bit mantissas, both operands scaled so their largest entry is 448)."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TRIAL_ATOL, check_fitness, feasible_theta, make_batch, random_state, rel_err

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 4e-3, 2: 3e-2, 3: 1e-5}     # relative: FP32, 2^-8 (BF16), a few % (e4m3), 1e-5 (bf16x3)
UNIT = {0: 0.0, 1: 2.0 ** -8, 2: 2.0 ** -3, 3: 2.0 ** -16}
GAP = {0: 1e-4, 1: 0.1, 2: 0.3, 3: 1e-3}      # relative fitness gap beyond which selection must match FP64
PRECS = pytest.mark.parametrize("prec", [1, 2, 3], ids=["bf16", "fp8e4m3", "bf16x3"])
# FP32 runs the same pipeline with the GEMM on the CUDA cores (k_rot_simt) for D_pad > 256
PIPE = pytest.mark.parametrize("prec", [0, 1, 2, 3], ids=["fp32-simt", "bf16", "fp8e4m3", "bf16x3"])


def _on_pipeline(wl, prec):
    return sum(1 for p in wl.problems if (((p.dim + 3) // 4) * 4 > 256 if prec == 0 else p.dim >= 129))


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


@PIPE
def test_tc_one_step_against_oracle(prec):
    import paper_2502_10470_gb300 as M
    wl = _wl()
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["tensor_core"]["executors"] == _on_pipeline(wl, prec)
    assert plan["tensor_core"]["kernel"] == ("k_rot_simt" if prec == 0 else "k_rot_tc")
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


@PIPE
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
            decided = rel_err(out["ftrial"], fits[k]) > GAP[prec]
            acc = np.any(npops[k] != pops[k], axis=1) | (nfits[k] != fits[k])
            np.testing.assert_array_equal(acc[decided], out["accept"].astype(bool)[decided])
            assert nfits[k].min() <= last[k]
            last[k] = nfits[k].min()
    b.close()


def _bf16_bits(x32):
    """float32 -> bfloat16 bit patterns, round to nearest even (the
    conversion the operand packing uses)."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF


@pytest.mark.parametrize("D,tie_fp64", [(256, 0), (256, 1), (40, 0), (100, 0), (200, 0), (600, 0)],
                         ids=["D256-difference", "D256-fp64", "D40-difference", "D100-difference",
                              "D200-difference", "D600-difference"])
def test_tc_near_ties_decided_like_fp64(D, tie_fp64):
    """Near ties on the tensor-core path.  A first step with F = 0, CR = 1 and
    stored fitness +inf makes every trial a copy of another grid point and
    stores its BF16 fitness.  A second step moves one coordinate by
    2^-20 (x_r0 - x_r1), exact in float32; where that coordinate's BF16
    operand u_j - o_j rounds as before, the GEMM sees the same row, so f(u)
    equals the stored f(x) and the pair must be listed as a tie and decided
    like the sign of the FP64 difference of the oracle.  D = 40, 100 and
    200 take the four-kernel generation (tc_min_dim 33) whose batched tie
    kernel groups 8, 4 and 2 ties per row of z; D = 600 its row-split tie
    kernel; D = 256 both tie modes."""
    import torch
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(77 + D)
    n, NP = 6, 64
    probs = [synth.make_problem(rng, D, k) for k in range(n)]
    wl = synth.Workload(name="tc-ties", problems=probs, inst_np=np.full(n, NP, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=12, one_shot=0)
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=1, tie_fp64=tie_fp64, tc_min_dim=33)
    assert json.loads(M.metade_plan_info(b.ctx))["tensor_core"]["executors"] == n
    grid = [(rng.integers(-12, 13, (NP, D)) * 8.0).astype(np.float32) for _ in range(n)]
    b.set_population(grid, [np.full(NP, np.inf, dtype=np.float32)] * n)
    b.set_theta(np.tile(np.array([0.0, 1.0, 1, 1, 1, 1], dtype=np.float32), (n, 1)))
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    pops, fits = b.get_population()                       # grid copies, BF16 fitness
    theta = np.tile(np.array([2.0 ** -20, 0.0, 4, 4, 1, 1], dtype=np.float32), (n, 1))
    b.set_theta(theta)
    rec = torch.zeros((b.n_indiv, M.REC_FIELDS), dtype=torch.int32, device="cuda")
    M.metade_draw_record(b.ctx, b.fit, b.theta, 0, 1, rec)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 1, 1, None, None)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    rec = rec.cpu().numpy()
    npops, nfits = b.get_population()
    checked = 0
    for k in range(n):
        p = probs[k]
        r = rec[b.fit_off[k]:b.fit_off[k] + NP]
        u = pops[k].astype(np.float64).copy()
        j = r[:, 2]
        rows = np.arange(NP)
        u[rows, j] += 2.0 ** -20 * (pops[k][r[:, 9], j].astype(np.float64) - pops[k][r[:, 10], j])
        u32 = u.astype(np.float32)
        assert np.array_equal(u32.astype(np.float64), u)
        same_op = _bf16_bits(u32[rows, j] - p.shift[j]) == _bf16_bits(pops[k][rows, j] - p.shift[j])
        fu = oracle.eval_pop(p.obj, u, p.shift, p.rot)
        fx = oracle.eval_pop(p.obj, pops[k], p.shift, p.rot)
        delta = fu - fx
        sure = same_op & np.isfinite(fits[k]) & (fits[k] > 0) & (np.abs(delta) > 1e-10 * np.abs(fx))
        took = np.any(npops[k] != pops[k], axis=1)
        np.testing.assert_array_equal(took[sure], (delta <= 0)[sure], err_msg="executor %d obj %d" % (k, p.obj))
        assert np.all(nfits[k] <= fits[k])
        if tie_fp64:
            a = sure & took
            np.testing.assert_array_equal(nfits[k][a], np.minimum(fu[a].astype(np.float32), fits[k][a]))
        checked += int(sure.sum())
    b.close()
    assert checked > 200


@PRECS
def test_tc_init_evaluates_on_the_tensor_cores(prec):
    """metade_init: executors on the tensor cores get their initial fitness
    from the rotation GEMM in the context's precision (within its error
    budget against FP64 at the same points); executors on the CUDA-core path
    of the same context get exactly the FP32 values of an FP32 context."""
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(47)
    dims, nps, objs = [20, 300, 33, 256], [40, 130, 17, 64], [2, 1, 5, 3]
    probs = [synth.make_problem(rng, d, o) for d, o in zip(dims, objs)]
    n = len(probs)
    wl = synth.Workload(name="tc-init", problems=probs, inst_np=np.array(nps, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=5, one_shot=0)
    out = {}
    for pr in (M.METADE_FP32, prec):
        b = make_batch(wl, M.METADE_PATH_BATCHED, prec=pr)
        M.metade_init(b.ctx, b.pop, b.fit, 3)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        out[pr] = b.get_population()
        b.close()
    for k in range(n):
        np.testing.assert_array_equal(out[prec][0][k], out[M.METADE_FP32][0][k])   # same initial points
        if dims[k] < 256:
            np.testing.assert_array_equal(out[prec][1][k], out[M.METADE_FP32][1][k])
        else:
            assert not np.array_equal(out[prec][1][k], out[M.METADE_FP32][1][k])  # not the FP32 values
            check_fitness(out[prec][1][k], out[prec][0][k], probs[k], TOL[prec], UNIT[prec])


@pytest.mark.parametrize("prec", [1, 3], ids=["bf16", "bf16x3"])
def test_tc_epilogue_all_objectives_multi_chunk(prec):
    """The GEMM epilogue evaluates each 256-column chunk in two halves on
    separate warps and composes the halves' objective states in column order
    (sums; Griewank's product pair; Rosenbrock's pair across the boundary;
    Schwefel 1.2's prefix carry).  Every objective at D = 300 (second chunk
    ends in the first half), 511 and 777 (ragged last halves): the initial
    fitness from the GEMM agrees with the FP64 oracle within the precision's
    budget."""
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(91)
    dims = [300, 511, 777]
    probs = [synth.make_problem(rng, d, o) for d in dims for o in range(6)]
    n = len(probs)
    wl = synth.Workload(name="tc-objectives", problems=probs, inst_np=np.full(n, 40, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=6, one_shot=0)
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    assert json.loads(M.metade_plan_info(b.ctx))["tensor_core"]["executors"] == n
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    pops, fits = b.get_population()
    for k, p in enumerate(probs):
        frac = check_fitness(fits[k], pops[k], p, TOL[prec], UNIT[prec])
        print("D", p.dim, "obj", p.obj, "beyond rtol:", frac)
    b.close()


# ------------------------------------------------ 128 < D < 256 on the tensor cores
def _wl_mid(seed=53):
    """Widths between the tile kernels' reach and 256 (D = 129, 200, 255),
    three executors per problem with ragged populations (17 + 61 + 130 = 208
    rows), so that a 128-row GEMM tile spans several executors of one problem
    and the problem's last tile is partial."""
    rng = np.random.default_rng(seed)
    dims, objs = [129, 200, 255, 200], [2, 3, 5, 1]
    probs = [synth.make_problem(rng, d, o) for d, o in zip(dims, objs)]
    nps = [17, 61, 130]
    inst_prob = np.repeat(np.arange(len(probs)), len(nps)).astype(np.int32)
    inst_np = np.tile(np.array(nps, dtype=np.int32), len(probs))
    n = len(inst_np)
    th = synth.random_theta(rng, n)
    th[:, 5] = np.arange(n) % 3 + 1
    wl = synth.Workload(name="tc-mid", problems=probs, inst_np=inst_np, inst_prob=inst_prob,
                        inst_group=np.arange(n, dtype=np.int32), n_groups=n, n_out=0, inner_gens=1, outer_gens=1,
                        seed=4, one_shot=0, theta=th)
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    return wl


@PRECS
def test_tc_mid_width_one_step_against_oracle(prec):
    """D = 129, 200 and 255 run on the tensor cores by default (D_pad > 128):
    one step from a shared state, trials against the oracle at TRIAL_ATOL and
    fitness within the precision's budget against FP64 at the GPU's trials.
    The GEMM's tiles cross executor boundaries here, so a fitness written to
    the wrong executor or row fails the comparison."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid()
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["tc_min_dim"] == 129
    assert plan["tensor_core"]["executors"] == wl.n_inst
    assert plan["tensor_core"]["tiles"] == 2 * len(wl.problems)  # 208 rows per problem: tiles of 128 + 80
    pops, fits = random_state(wl, seed=8, fit_inf=True)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 2, 5, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=2, gen=5)
        assert np.abs(npops[k] - out["trial"]).max() < TRIAL_ATOL
        frac = check_fitness(nfits[k], npops[k], p, TOL[prec], UNIT[prec])
        print("executor", k, "D", p.dim, "obj", p.obj, "beyond rtol:", frac)
    bf = b.best_f.cpu().numpy()
    for k in range(wl.n_inst):
        assert bf[k] == nfits[k].min()
    b.close()


@pytest.mark.parametrize("prec", [1, 3], ids=["bf16", "bf16x3"])
def test_tc_mid_width_selection_over_generations(prec):
    """Three generations with stored fitness on the mid-width workload: the
    best never rises, and every selection whose fitness gap exceeds the
    precision's tolerance matches the oracle's FP64 decision."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid(seed=59)
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    pops, fits = random_state(wl, seed=9)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    last = [f.min() for f in fits]
    for g in range(3):
        pops, fits = b.get_population()
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, g, 1, b.best_f, b.best_i)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        npops, nfits = b.get_population()
        for k in range(wl.n_inst):
            p = wl.problems[int(wl.inst_prob[k])]
            out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                                  epoch=0, gen=g)
            decided = rel_err(out["ftrial"], fits[k]) > GAP[prec]
            acc = np.any(npops[k] != pops[k], axis=1) | (nfits[k] != fits[k])
            np.testing.assert_array_equal(acc[decided], out["accept"].astype(bool)[decided])
            assert nfits[k].min() <= last[k]
            last[k] = nfits[k].min()
    b.close()


def test_tc_min_dim_places_executors_and_autotune_picks_a_width():
    """tc_min_dim = 256 keeps D < 256 on the FP32 kernels: bit-identical to an
    FP32 context.  tc_min_dim = 0 lets metade_autotune time both widths (129
    and 256) and keep the faster; the plan reports both timings."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid(seed=61)
    pops, fits = random_state(wl, seed=3)
    outs = {}
    for name, kw in (("fp32", dict(prec=0)), ("bf16-256", dict(prec=1, tc_min_dim=256))):
        b = make_batch(wl, M.METADE_PATH_BATCHED, **kw)
        if name == "bf16-256":
            plan = json.loads(M.metade_plan_info(b.ctx))
            assert plan["tc_min_dim"] == 256 and "tensor_core" not in plan
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 3, None, None)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        outs[name] = b.get_population()
        b.close()
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(outs["fp32"][0][k], outs["bf16-256"][0][k])
        np.testing.assert_array_equal(outs["fp32"][1][k], outs["bf16-256"][1][k])
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=1, tc_min_dim=0)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_autotune(b.ctx, b.pop, b.fit, b.theta, 2)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["tc_min_dim_auto"] and plan["tc_min_dim"] in (33, 129, 256)
    assert set(plan["tc_autotune_ms"]) == {"33", "129", "256"}
    p2, f2 = b.get_population()  # tuning ran on copies
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(p2[k], pops[k])
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 2, None, None)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    b.close()


def test_tc_fused_generation_equals_the_pipeline():
    """The three-kernel generation (k_tc_rank, k_tc_trial2, k_tc_sel) against
    the five-kernel pipeline (tc_unfused = 1) on the same state: the same
    trial arithmetic, the same GEMM operands and epilogue, the same FP32 tie
    rotations and difference forms, so populations and fitness must be
    bit-identical -- over three generations of random states (D 129..255,
    tiles across executors), and over a near-tie step (grid copies, then
    trials 2^-20 away) where most selections go through the tie path."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid(seed=67)
    pops, fits = random_state(wl, seed=11)
    outs = []
    for unfused in (0, 1):
        b = make_batch(wl, M.METADE_PATH_BATCHED, prec=1, tc_unfused=unfused)
        assert json.loads(M.metade_plan_info(b.ctx))["tensor_core"]["kernel"] == ("k_rot_tc" if unfused else "k_tc_sel")
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 3, b.best_f, b.best_i)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        outs.append((b.get_population(), b.best_f.cpu().numpy(), b.best_i.cpu().numpy()))
        b.close()
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(outs[0][0][0][k], outs[1][0][0][k])
        np.testing.assert_array_equal(outs[0][0][1][k], outs[1][0][1][k])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])
    # near ties: D = 200 and 256 executors on a grid
    rng = np.random.default_rng(79)
    n, NP = 6, 64
    probs = [synth.make_problem(rng, 200 if k % 2 else 256, k) for k in range(n)]
    wt = synth.Workload(name="tc-ties-fused", problems=probs, inst_np=np.full(n, NP, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=13, one_shot=0)
    grid = [(rng.integers(-12, 13, (NP, p.dim)) * 8.0).astype(np.float32) for p in probs]
    res = []
    for unfused in (0, 1):
        b = make_batch(wt, M.METADE_PATH_BATCHED, prec=1, tc_unfused=unfused)
        b.set_population(grid, [np.full(NP, np.inf, dtype=np.float32)] * n)
        b.set_theta(np.tile(np.array([0.0, 1.0, 1, 1, 1, 1], dtype=np.float32), (n, 1)))
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
        b.set_theta(np.tile(np.array([2.0 ** -20, 0.0, 4, 4, 1, 1], dtype=np.float32), (n, 1)))
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 1, 2, None, None)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        res.append(b.get_population())
        b.close()
    for k in range(n):
        np.testing.assert_array_equal(res[0][0][k], res[1][0][k])
        np.testing.assert_array_equal(res[0][1][k], res[1][1][k])


def test_tc_wide_four_kernel_generation_equals_the_pipeline():
    """Operands wider than 256 elements: the four-kernel generation (k_tc_rank,
    k_tc_trial2, k_rot_tc selecting in its epilogue, k_tc_ties2 over row groups
    of 256) against the five-kernel pipeline (tc_unfused = 1), bit-identical
    over three generations of random states (D 256..520, K extents differing
    between tiles), and over a near-tie step on grids at D 129..1536, where the
    tie kernel stages the fewest ties per chunk and z spans six row groups."""
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=71)
    pops, fits = random_state(wl, seed=13)
    outs = []
    for unfused in (0, 1):
        b = make_batch(wl, M.METADE_PATH_BATCHED, prec=1, tc_unfused=unfused)
        tc = json.loads(M.metade_plan_info(b.ctx))["tensor_core"]
        assert tc["kernel"] == "k_rot_tc" and tc["kernels_per_generation"] == (5 if unfused else 4)
        b.set_population(pops, fits)
        b.set_theta(wl.theta)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 3, b.best_f, b.best_i)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        outs.append((b.get_population(), b.best_f.cpu().numpy(), b.best_i.cpu().numpy()))
        b.close()
    for k in range(wl.n_inst):
        np.testing.assert_array_equal(outs[0][0][0][k], outs[1][0][0][k])
        np.testing.assert_array_equal(outs[0][0][1][k], outs[1][0][1][k])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][2], outs[1][2])
    rng = np.random.default_rng(83)
    dims = [300, 1536, 129, 1000, 520, 256]
    n, NP = len(dims), 40
    probs = [synth.make_problem(rng, d, k) for k, d in enumerate(dims)]
    wt = synth.Workload(name="tc-ties-wide", problems=probs, inst_np=np.full(n, NP, dtype=np.int32),
                        inst_prob=np.arange(n, dtype=np.int32), inst_group=np.arange(n, dtype=np.int32),
                        n_groups=n, n_out=0, inner_gens=1, outer_gens=1, seed=17, one_shot=0)
    grid = [(rng.integers(-12, 13, (NP, p.dim)) * 8.0).astype(np.float32) for p in probs]
    res = []
    for unfused in (0, 1):
        b = make_batch(wt, M.METADE_PATH_BATCHED, prec=1, tc_unfused=unfused)
        b.set_population(grid, [np.full(NP, np.inf, dtype=np.float32)] * n)
        b.set_theta(np.tile(np.array([0.0, 1.0, 1, 1, 1, 1], dtype=np.float32), (n, 1)))
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 1, None, None)
        b.set_theta(np.tile(np.array([2.0 ** -20, 0.0, 4, 4, 1, 1], dtype=np.float32), (n, 1)))
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 1, 2, None, None)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        res.append(b.get_population())
        b.close()
    for k in range(n):
        np.testing.assert_array_equal(res[0][0][k], res[1][0][k])
        np.testing.assert_array_equal(res[0][1][k], res[1][1][k])


def test_fp32_width_runs_the_cuda_core_gemm_pipeline():
    """FP32 with tc_min_dim = 129: the D = 129 .. 255 executors leave the fused
    tile kernels for the per-generation pipeline with the FP32 GEMM on the
    CUDA cores (k_rot_simt, 64-row tiles of each executor).  One step against
    the oracle (trials at TRIAL_ATOL, FP32 fitness), then two generations with
    stored fitness whose clear selections match the oracle's; the default
    FP32 width (257) keeps them in the tile kernels."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid(seed=89)
    d0 = make_batch(wl, M.METADE_PATH_BATCHED, prec=0)
    plan = json.loads(M.metade_plan_info(d0.ctx))
    assert plan["tc_min_dim"] == 257 and "tensor_core" not in plan
    d0.close()
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=0, tc_min_dim=129)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["tensor_core"]["kernel"] == "k_rot_simt" and plan["tensor_core"]["executors"] == wl.n_inst
    pops, fits = random_state(wl, seed=12, fit_inf=True)
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 1, 3, 1, None, None)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=1, gen=3)
        assert np.abs(npops[k] - out["trial"]).max() < TRIAL_ATOL
        check_fitness(nfits[k], npops[k], p, TOL[0], UNIT[0])
    for g in range(4, 6):
        pops, fits = b.get_population()
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 1, g, 1, None, None)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        npops, nfits = b.get_population()
        for k in range(wl.n_inst):
            p = wl.problems[int(wl.inst_prob[k])]
            out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                                  epoch=1, gen=g)
            decided = rel_err(out["ftrial"], fits[k]) > GAP[0]
            acc = np.any(npops[k] != pops[k], axis=1) | (nfits[k] != fits[k])
            np.testing.assert_array_equal(acc[decided], out["accept"].astype(bool)[decided])
    b.close()


@pytest.mark.parametrize("prec", [1, 0], ids=["bf16-four-kernel", "fp32-cuda-core-gemm"])
def test_invalid_theta_rows_are_left_alone_by_the_draw_record_path(prec):
    """An executor with an invalid theta among valid ones, on the paths whose
    draws go through k_tc_rank's draw records (the BF16 four-kernel generation,
    and the FP32 pipeline's narrow rows at tc_min_dim = 129): the sticky status
    is METADE_EINVAL, the invalid executor's rows and fitness are unchanged,
    and every other executor ends exactly as in a run where that executor is
    valid (executors draw from their own Philox streams and share no rows).
    Then a run with every theta valid leaves the status OK."""
    import paper_2502_10470_gb300 as M
    wl = _wl_mid(seed=97)
    pops, fits = random_state(wl, seed=5)
    bad = 4  # the second executor of the D = 200 problem
    kw = dict(prec=prec) if prec else dict(prec=0, tc_min_dim=129)
    outs = []
    for invalid in (True, False):
        b = make_batch(wl, M.METADE_PATH_BATCHED, **kw)
        plan = json.loads(M.metade_plan_info(b.ctx))
        assert plan["tensor_core"]["kernel"] == ("k_tc_sel" if prec else "k_rot_simt")
        b.set_population(pops, fits)
        th = wl.theta.copy()
        if invalid:
            th[bad, 4] = 9  # dn outside {1..4}
        b.set_theta(th)
        M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 0, 3, None, None)
        assert M.metade_sync(b.ctx) == (M.METADE_EINVAL if invalid else M.METADE_OK)
        outs.append(b.get_population())
        b.close()
    (pa, fa), (pb, fb) = outs
    np.testing.assert_array_equal(pa[bad], pops[bad])
    np.testing.assert_array_equal(fa[bad], fits[bad])
    for k in range(wl.n_inst):
        if k != bad:
            np.testing.assert_array_equal(pa[k], pb[k])
            np.testing.assert_array_equal(fa[k], fb[k])
    assert any(not np.array_equal(pb[k], pops[k]) for k in range(wl.n_inst) if k != bad)  # the runs did work
