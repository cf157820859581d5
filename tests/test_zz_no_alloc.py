"""The allocation-free entry point, metade_plain_step_noalloc, against the
plain path of metade_inner_step on the same executor.

Callers whose device heap belongs to someone else (a host framework's caching
allocator, a plugin that must not grow the device footprint) cannot let this
library cudaMalloc; the entry point keeps its scratch in a fixed device array
inside the library instead.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth
from gpu_util import FIT_RTOL, TRIAL_ATOL, check_fitness_fp32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("np_,dim,obj", [(37, 13, 2), (100, 20, 1), (257, 130, 3), (16, 1, 5)])
def test_noalloc_matches_inner_step_on_two_calls(np_, dim, obj):
    import torch
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(np_ * 7 + dim)
    p = synth.make_problem(rng, dim, obj)
    theta = np.array([0.7, 0.6, 4, 2, 1, 1], dtype=np.float32)
    ref = M.Batch([(p.dim, p.obj, p.shift, p.rot)], [np_], [0], seed=5, path=M.METADE_PATH_PLAIN)
    pop0 = synth.random_population(rng, np_, dim)
    import oracle
    fit0 = oracle.eval_pop(obj, pop0, p.shift, p.rot).astype(np.float32)
    ref.set_population([pop0], [fit0])
    ref.set_theta(theta[None, :])
    dpad = int(ref.dpad[0])
    pop = ref.pop[:np_ * dpad].clone()
    fit = ref.fit[:np_].clone()
    th = torch.tensor(theta, device="cuda")
    shift = torch.tensor(p.shift, device="cuda")
    rot = torch.tensor(p.rot.reshape(-1), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for gen in (0, 1):
        start_pop = pop.view(np_, dpad)[:, :dim].cpu().numpy()
        start_fit = fit.cpu().numpy()
        M.metade_inner_step(ref.ctx, ref.pop, ref.fit, ref.theta, 0, gen, 1, None, None)
        st = M.metade_plain_step_noalloc(pop, fit, th, shift, rot, np_, dim, obj, -100.0, 100.0, 5, 0, 0, gen,
                                         10, stream)
        assert st == M.METADE_OK
        ref.sync()
        torch.cuda.synchronize()
        want_pop = ref.pop[:np_ * dpad].view(np_, dpad)[:, :dim].cpu().numpy()
        want_fit = ref.fit[:np_].cpu().numpy()
        got_pop = pop.view(np_, dpad)[:, :dim].cpu().numpy()
        got_fit = fit.cpu().numpy()
        assert np.abs(got_pop - want_pop).max() <= TRIAL_ATOL
        assert np.all(np.abs(got_fit - want_fit) <= FIT_RTOL * np.maximum(np.abs(want_fit), 1.0))
        check_fitness_fp32(got_fit, got_pop, p)
        assert not np.array_equal(got_pop, pop0)  # the generation did something
        assert M.metade_plain_step_noalloc_status() == 0
        # and against the FP64 oracle's generation from the same state: the
        # selection wherever the fitness gap is clear, the accepted trials
        out = oracle.pde_step(start_pop, start_fit, theta, obj, p.shift, p.rot, seed=5, stream=0, epoch=0, gen=gen)
        took = np.any(got_pop != start_pop, axis=1)
        gap = np.abs(out["ftrial"] - start_fit) / np.maximum(np.abs(start_fit), 1.0)
        decided = gap > 2e-5
        np.testing.assert_array_equal(took[decided], out["accept"].astype(bool)[decided])
        both = took & out["accept"].astype(bool)
        assert np.abs(got_pop[both] - out["trial"][both]).max(initial=0.0) < TRIAL_ATOL
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2502_10470_gb300 as M
    t = torch.zeros(8, device="cuda")
    # 1024 x 1536 trial rows exceed the fixed 2^20-float scratch
    st = M.metade_plain_step_noalloc(t, t, t, t, t, 1024, 1536, 0, -100.0, 100.0, 0, 0, 0, 0, 10, None)
    assert st == M.METADE_EINVAL
    st = M.metade_plain_step_noalloc(t, t, t, t, t, 3, 4, 0, -100.0, 100.0, 0, 0, 0, 0, 10, None)
    assert st == M.METADE_EINVAL
    # pop is read and written as float4 rows: a pointer off a 16-byte boundary is rejected on the host
    big = torch.zeros(16 * 8 + 1, device="cuda")
    st = M.metade_plain_step_noalloc(big[1:], t, t, t, t, 16, 8, 0, -100.0, 100.0, 0, 0, 0, 0, 10, None)
    assert st == M.METADE_EINVAL


def test_noalloc_reports_a_skipped_generation():
    """An invalid theta (np too small for dn = 4 difference pairs) leaves pop
    and fit unchanged, and the status word says the generation was skipped;
    a valid one afterwards says it ran."""
    import torch
    import paper_2502_10470_gb300 as M
    rng = np.random.default_rng(3)
    p = synth.make_problem(rng, 8, 0)
    np_, dpad = 6, 8
    pop = torch.tensor(synth.random_population(rng, np_, 8), device="cuda").reshape(-1).contiguous()
    import oracle
    fit = torch.tensor(oracle.eval_pop(0, pop.view(np_, dpad).cpu().numpy(), p.shift, p.rot).astype(np.float32),
                       device="cuda")
    shift = torch.tensor(p.shift, device="cuda")
    rot = torch.tensor(p.rot.reshape(-1), device="cuda")
    before = pop.clone()
    bad = torch.tensor([0.5, 0.5, 1, 1, 4, 1], dtype=torch.float32, device="cuda")  # 9 distinct draws, NP 6
    assert M.metade_plain_step_noalloc(pop, fit, bad, shift, rot, np_, 8, 0, -100.0, 100.0, 1, 0, 0, 0, 10,
                                       None) == M.METADE_OK
    assert M.metade_plain_step_noalloc_status() == 1
    assert torch.equal(pop, before)
    good = torch.tensor([0.5, 0.9, 1, 1, 1, 1], dtype=torch.float32, device="cuda")
    assert M.metade_plain_step_noalloc(pop, fit, good, shift, rot, np_, 8, 0, -100.0, 100.0, 1, 0, 0, 1, 10,
                                       None) == M.METADE_OK
    assert M.metade_plain_step_noalloc_status() == 0
