"""The MLP regression objective (id 6), a neuroevolution-like large-D
problem, on its own per-generation path: initial and FP64 evaluations, the
teacher optimum, one PDE step against the FP64 oracle, several generations
in one call against single calls, and its place in the plan (never the
rotation kernels).  h = 4 runs the forward pass four hidden units at a time,
h = 21 one at a time."""
import json

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TRIAL_ATOL, feasible_theta, make_batch, rel_err

pytestmark = pytest.mark.gpu


def _wl(seed=61, prec_dims=(4, 21)):
    rng = np.random.default_rng(seed)
    probs = [synth.make_mlp_problem(rng, h) for h in prec_dims] + [synth.make_problem(rng, 10, synth.OBJ_RASTRIGIN)]
    n = len(probs)
    nps = np.array([40, 64, 24, 32][:n], dtype=np.int32)
    th = synth.random_theta(rng, n)
    wl = synth.Workload(name="mlp-mixed", problems=probs, inst_np=nps, inst_prob=np.arange(n, dtype=np.int32),
                        inst_group=np.arange(n, dtype=np.int32), n_groups=n, n_out=0, inner_gens=1, outer_gens=1,
                        seed=8, one_shot=0, theta=th, lo=-2.0, hi=2.0)
    wl.theta = feasible_theta(wl.theta, wl.inst_np)
    return wl


def test_mlp_init_eval_and_teacher_optimum():
    import torch
    import paper_2502_10470_gb300 as M
    wl = _wl()
    b = make_batch(wl, M.METADE_PATH_BATCHED)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["mlp"]["executors"] == 2 and plan["mlp"]["rows"] == 104
    M.metade_init(b.ctx, b.pop, b.fit, 0)
    f64 = torch.empty(b.n_indiv, dtype=torch.float64, device="cuda")
    M.metade_eval_pop(b.ctx, b.pop, M.METADE_FP64, f64)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    pops, fits = b.get_population()
    f64 = f64.cpu().numpy()
    for k, p in enumerate(wl.problems):
        ref = oracle.eval_pop(p.obj, pops[k], p.shift, p.rot)
        assert rel_err(fits[k], ref, 1e-30).max() < 1e-5
        got64 = f64[b.fit_off[k]:b.fit_off[k] + wl.inst_np[k]]
        assert rel_err(got64, ref, 1e-30).max() < 1e-12
    # the teacher itself: f = 0 exactly in FP32 (the targets come from the same forward pass)
    for k in (0, 1):
        pops[k][3] = wl.problems[k].shift
    b.set_population(pops, fits)
    f32 = torch.empty(b.n_indiv, dtype=torch.float32, device="cuda")
    M.metade_eval_pop(b.ctx, b.pop, M.METADE_FP32, f32)
    b.sync()
    f32 = f32.cpu().numpy()
    for k in (0, 1):
        assert f32[b.fit_off[k] + 3] == 0.0
    b.close()


def test_mlp_one_step_against_oracle():
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=62)
    b = make_batch(wl, M.METADE_PATH_BATCHED)
    rng = np.random.default_rng(4)
    pops = [rng.uniform(-2, 2, (wl.inst_np[k], p.dim)).astype(np.float32) for k, p in enumerate(wl.problems)]
    fits = [oracle.eval_pop(p.obj, pops[k], p.shift, p.rot).astype(np.float32) for k, p in enumerate(wl.problems)]
    b.set_population(pops, fits)
    b.set_theta(wl.theta)
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 0, 5, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    for k, p in enumerate(wl.problems):
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=0, gen=5, lo=wl.lo, hi=wl.hi)
        took = np.any(npops[k] != pops[k], axis=1)
        assert np.abs(npops[k][took] - out["trial"][took]).max(initial=0.0) < TRIAL_ATOL
        fu = oracle.eval_pop(p.obj, npops[k][took], p.shift, p.rot)
        assert rel_err(nfits[k][took], fu, 1e-30).max(initial=0.0) < 1e-5
        decided = rel_err(out["ftrial"], fits[k], 1e-30) > 1e-4
        np.testing.assert_array_equal(took[decided], out["accept"].astype(bool)[decided])
        assert np.all(nfits[k] <= fits[k])
    b.close()


def test_mlp_generations_in_one_call_equal_single_calls():
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=63)
    res = []
    for split in (False, True):
        b = make_batch(wl, M.METADE_PATH_BATCHED)
        b.set_theta(wl.theta)
        M.metade_init(b.ctx, b.pop, b.fit, 1)
        if split:
            for g in range(4):
                M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 1, g, 1, b.best_f, b.best_i)
        else:
            M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 1, 0, 4, b.best_f, b.best_i)
        assert M.metade_sync(b.ctx) == M.METADE_OK
        res.append(b.get_population() + (b.best_f.cpu().numpy(),))
        b.close()
    for k in range(len(wl.problems)):
        np.testing.assert_array_equal(res[0][0][k], res[1][0][k])
        np.testing.assert_array_equal(res[0][1][k], res[1][1][k])
    np.testing.assert_array_equal(res[0][2], res[1][2])


def test_mlp_stays_off_the_rotation_paths():
    """A reduced-precision context sends D >= 256 rotation problems to the
    tensor cores, but an MLP problem of any size keeps its own path (its
    first layer on the tensor cores by k_mlp_tc in BF16, the CUDA-core kernel
    in FP32), never the rotation GEMM; the plain path rejects the objective."""
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=64, prec_dims=(14, 20))      # D = 268 and 382
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=M.METADE_BF16)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["mlp"]["executors"] == 2
    assert plan["mlp"]["kernels"][2] == "k_mlp_tc" and plan["mlp"]["precision"] == "bf16"
    assert "tensor_core" not in plan
    b.close()
    b = make_batch(wl, M.METADE_PATH_BATCHED)
    assert json.loads(M.metade_plan_info(b.ctx))["mlp"]["kernels"][2] == "k_mlp_eval"
    b.close()
    with pytest.raises(M.MetadeError):
        make_batch(wl, M.METADE_PATH_PLAIN)


def _mlp_budget(theta, teacher, unit, tanh_err=0.0):
    """FP64 objective of parameter rows and the first-order effect on it of
    rounding the first layer's operands (inputs and W1) with relative error
    `unit` each: |dz| <= 2 unit (|X| |W1|), propagated through tanh, the
    second layer and the mean squared error; plus a relative error
    `tanh_err` of each tanh value."""
    X = oracle.mlp_inputs().astype(np.float64)
    h = oracle.mlp_hidden(theta.shape[1])

    def parts(v):
        W1 = v[:16 * h].reshape(16, h)
        b1 = v[16 * h:17 * h]
        W2 = v[17 * h:19 * h].reshape(h, 2)
        b2 = v[19 * h:19 * h + 2]
        return W1, b1, W2, b2

    W1t, b1t, W2t, b2t = parts(np.asarray(teacher, dtype=np.float64))
    T = np.tanh(X @ W1t + b1t) @ W2t + b2t
    f, bound = [], []
    for v in np.asarray(theta, dtype=np.float64):
        W1, b1, W2, b2 = parts(v)
        t = np.tanh(X @ W1 + b1)
        e = t @ W2 + b2 - T
        dz = 2 * unit * (np.abs(X) @ np.abs(W1))
        dy = ((1 - t * t) * dz + tanh_err * np.abs(t)) @ np.abs(W2)
        f.append(float(np.mean(e * e)))
        bound.append(float(np.mean(2 * np.abs(e) * dy + dy * dy)))
    return np.array(f), np.array(bound)


@pytest.mark.parametrize("prec,unit,tanh_err", [(1, 2.0 ** -9, 2.0 ** -10), (3, 2.0 ** -16, 0.0)],
                         ids=["bf16", "bf16x3"])
def test_mlp_tensor_core_eval_and_step(prec, unit, tanh_err):
    """k_mlp_tc (the first layer on the tensor cores, BF16 or split BF16) at
    h = 4, 21 and 80 (N 16, 32, 80; D up to 1522): the initial evaluation
    against the FP64 oracle within the first-order effect of the operands'
    rounding (and, in BF16, of the hardware tanh's relative error, taken as
    2^-10 against its documented 2^-10.99), then one PDE step: trials at TRIAL_ATOL, accepted rows' fitness
    within the same budget, and the selections the budget cannot flip equal
    to the oracle's."""
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=66, prec_dims=(4, 21, 80))
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=prec)
    assert json.loads(M.metade_plan_info(b.ctx))["mlp"]["kernels"][2] == "k_mlp_tc"
    b.set_theta(wl.theta)
    M.metade_init(b.ctx, b.pop, b.fit, 2)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    pops, fits = b.get_population()
    for k, p in enumerate(wl.problems):
        if p.obj != synth.OBJ_MLP:
            continue
        fr, bd = _mlp_budget(pops[k], p.shift, unit, tanh_err)
        assert np.all(np.abs(fits[k] - fr) <= 2 * bd + 1e-5 * np.abs(fr) + 1e-7), "executor %d h %d" % (
            k, oracle.mlp_hidden(p.dim))
    M.metade_inner_step(b.ctx, b.pop, b.fit, b.theta, 2, 7, 1, b.best_f, b.best_i)
    assert M.metade_sync(b.ctx) == M.METADE_OK
    npops, nfits = b.get_population()
    for k, p in enumerate(wl.problems):
        if p.obj != synth.OBJ_MLP:
            continue
        out = oracle.pde_step(pops[k], fits[k], wl.theta[k], p.obj, p.shift, p.rot, seed=wl.seed, stream=k,
                              epoch=2, gen=7, lo=wl.lo, hi=wl.hi)
        took = np.any(npops[k] != pops[k], axis=1)
        assert np.abs(npops[k][took] - out["trial"][took]).max(initial=0.0) < TRIAL_ATOL
        fr, bd = _mlp_budget(npops[k][took], p.shift, unit, tanh_err)
        assert np.all(np.abs(nfits[k][took] - fr) <= 2 * bd + 1e-5 * np.abs(fr) + 1e-7)
        fu, bu = _mlp_budget(out["trial"], p.shift, unit, tanh_err)
        _, bx = _mlp_budget(pops[k], p.shift, unit, tanh_err)
        decided = np.abs(out["ftrial"] - fits[k]) > 4 * (bu + bx) + 1e-4 * np.abs(fits[k])
        np.testing.assert_array_equal(took[decided], out["accept"].astype(bool)[decided])
        assert np.all(nfits[k] <= fits[k])
    b.close()
