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
    nps = np.array([40, 64, 24], dtype=np.int32)
    n = len(probs)
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
    tensor cores, but an MLP problem of any size keeps its FP32 kernel; the
    plain path rejects the objective."""
    import paper_2502_10470_gb300 as M
    wl = _wl(seed=64, prec_dims=(14, 20))      # D = 268 and 382
    b = make_batch(wl, M.METADE_PATH_BATCHED, prec=M.METADE_BF16)
    plan = json.loads(M.metade_plan_info(b.ctx))
    assert plan["mlp"]["executors"] == 2
    assert "tensor_core" not in plan
    b.close()
    with pytest.raises(M.MetadeError):
        make_batch(wl, M.METADE_PATH_PLAIN)
