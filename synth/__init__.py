"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no step of the MetaDE method: it only draws the problem
instances the method is run on (shift vectors o, rotation matrices R,
objective ids, population sizes, dimensions) and decoded hyperparameter
vectors theta used as given inputs.  Everything the method itself draws at
run time (initial population, index draws, crossover masks) comes from the
counter-based generator that the CUDA path and the oracle each implement.

The objectives stand in for the CEC2022 suite the paper evaluates on
(Sec. IV-A), which is not available: shifted-rotated textbook functions
f(z) with z = R (x - o), o ~ U[-80, 80]^D and R a Haar-distributed
orthogonal matrix (QR of a seeded Gaussian matrix, columns sign-fixed so
that diag of the triangular factor is positive), cast to float32.  The
search box is [-100, 100]^D.

Objective ids (shared vocabulary of the C-ABI and the oracle):
  0 sphere, 1 Rosenbrock (on z + 1), 2 Rastrigin, 3 Griewank, 4 Ackley,
  5 Schwefel 1.2.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

OBJ_SPHERE, OBJ_ROSENBROCK, OBJ_RASTRIGIN, OBJ_GRIEWANK, OBJ_ACKLEY, OBJ_SCHWEFEL12, OBJ_MLP = range(7)
OBJ_NAMES = ["sphere", "rosenbrock", "rastrigin", "griewank", "ackley", "schwefel12", "mlp"]
MLP_TEACHER = 0.75  # teacher parameters ~ U[-0.75, 0.75]: hidden pre-activations of unit variance

BOX_LO, BOX_HI = -100.0, 100.0
SHIFT_LO, SHIFT_HI = -80.0, 80.0

# Outer (evolver) gene bounds for theta = (F, CR, bl, br, dn, cs); Alg. 3
# initialises the evolver inside [lb, ub].  The paper gives the domains only in
# a figure; F, CR in [0, 1], bl/br/dn in {1..4}, cs in {1..3} (Sec. III-A),
# so the floor-decoded genes live in [1, 5) and [1, 4).
OUTER_LB = np.array([0.0, 0.0, 1.0, 1.0, 1.0, 1.0], dtype=np.float32)
OUTER_UB = np.array([1.0, 1.0, 5.0, 5.0, 5.0, 4.0], dtype=np.float32)


def haar_rotation(rng: np.random.Generator, dim: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix (float64), Mezzadri's sign fix."""
    g = rng.standard_normal((dim, dim))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


@dataclass
class Problem:
    dim: int
    obj: int
    shift: np.ndarray  # float32 [dim]
    rot: np.ndarray    # float32 [dim, dim], row-major, z = rot @ (x - shift)


def make_mlp_problem(rng: np.random.Generator, hidden: int) -> Problem:
    """MLP regression objective (id 6): D = 19 hidden + 2 parameters of a
    16-hidden-2 tanh perceptron; the shift is the teacher's parameters, the
    rotation is unused (identity)."""
    dim = 19 * hidden + 2
    shift = rng.uniform(-MLP_TEACHER, MLP_TEACHER, size=dim).astype(np.float32)
    return Problem(dim=dim, obj=OBJ_MLP, shift=shift, rot=np.eye(dim, dtype=np.float32))


def make_problem(rng: np.random.Generator, dim: int, obj: int) -> Problem:
    shift = rng.uniform(SHIFT_LO, SHIFT_HI, size=dim).astype(np.float32)
    rot = haar_rotation(rng, dim).astype(np.float32)
    return Problem(dim=dim, obj=obj, shift=shift, rot=np.ascontiguousarray(rot))


def random_theta(rng: np.random.Generator, n: int) -> np.ndarray:
    """n decoded hyperparameter vectors (F, CR, bl, br, dn, cs) as float32.

    F, CR ~ U[0, 1); bl, br, dn ~ U{1..4}; cs ~ U{1..3} -- the PDE domains of
    Sec. III-A, sampled directly (no encoding step involved)."""
    th = np.empty((n, 6), dtype=np.float32)
    th[:, 0] = rng.uniform(0.0, 1.0, n)
    th[:, 1] = rng.uniform(0.0, 1.0, n)
    th[:, 2] = rng.integers(1, 5, n)
    th[:, 3] = rng.integers(1, 5, n)
    th[:, 4] = rng.integers(1, 5, n)
    th[:, 5] = rng.integers(1, 4, n)
    return th


@dataclass
class Workload:
    """A batch of inner-DE instances over a table of problems.

    inst_np[k]    population size of instance k
    inst_prob[k]  problem index of instance k (its D, objective, o, R)
    inst_group[k] MetaDE run the instance belongs to; with one-shot evaluation
                  all executors of a run share one random stream
    """
    name: str
    problems: List[Problem]
    inst_np: np.ndarray
    inst_prob: np.ndarray
    inst_group: np.ndarray
    n_groups: int
    n_out: int                       # evolver population per run (0: no outer DE)
    inner_gens: int
    outer_gens: int
    seed: int
    one_shot: int
    theta: Optional[np.ndarray] = None   # decoded theta [n_inst, 6] when given
    lo: float = BOX_LO
    hi: float = BOX_HI
    p_best_pct: int = 10
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_inst(self) -> int:
        return int(self.inst_np.shape[0])

    def dims(self) -> np.ndarray:
        return np.array([self.problems[p].dim for p in self.inst_prob], dtype=np.int32)

    def objs(self) -> np.ndarray:
        return np.array([self.problems[p].obj for p in self.inst_prob], dtype=np.int32)

    def individuals(self) -> int:
        return int(self.inst_np.sum())


def _runs(name, problems, np_per_run, n_out, inner_gens, outer_gens, seed, one_shot, notes=""):
    n_groups = len(problems)
    inst_np = np.repeat(np.asarray(np_per_run, dtype=np.int32), n_out)
    inst_prob = np.repeat(np.arange(n_groups, dtype=np.int32), n_out)
    inst_group = inst_prob.copy()
    return Workload(name=name, problems=problems, inst_np=inst_np, inst_prob=inst_prob,
                    inst_group=inst_group, n_groups=n_groups, n_out=n_out,
                    inner_gens=inner_gens, outer_gens=outer_gens, seed=seed,
                    one_shot=one_shot, notes=notes)


def tiny(problem_seed: int = 0, run_seed: int = 0) -> Workload:
    """Evolver population 8, one inner DE (NP 16, D 10, Rastrigin) per
    vector, 20 inner generations x 5 outer generations, one-shot."""
    rng = np.random.default_rng(problem_seed)
    probs = [make_problem(rng, 10, OBJ_RASTRIGIN)]
    return _runs("tiny-8x16xD10-rastrigin", probs, [16], 8, 20, 5, run_seed, 1)


def moderate(problem_seed: int = 1, run_seed: int = 0, inner_gens: int = 500) -> Workload:
    """Six MetaDE runs (one per objective): evolver population 100, inner
    population 100, D 20, 500 inner generations per meta-evaluation."""
    rng = np.random.default_rng(problem_seed)
    probs = [make_problem(rng, 20, obj) for obj in range(6)]
    return _runs("moderate-6x100x100xD20", probs, [100] * 6, 100, inner_gens, 1, run_seed, 1)


def batching(problem_seed: int = 2, run_seed: int = 0, n_inst: int = 512, inner_gens: int = 100) -> Workload:
    """512 independent inner DEs of uneven size: NP ~ U{20..400},
    D ~ U{10, 20, 50, 100}, objective ~ U{0..5}, theta sampled per instance."""
    rng = np.random.default_rng(problem_seed)
    dims = rng.choice([10, 20, 50, 100], size=n_inst)
    objs = rng.integers(0, 6, size=n_inst)
    nps = rng.integers(20, 401, size=n_inst).astype(np.int32)
    probs = [make_problem(rng, int(d), int(o)) for d, o in zip(dims, objs)]
    theta = random_theta(rng, n_inst)
    return Workload(name="batching-512-ragged", problems=probs, inst_np=nps,
                    inst_prob=np.arange(n_inst, dtype=np.int32),
                    inst_group=np.arange(n_inst, dtype=np.int32), n_groups=n_inst, n_out=0,
                    inner_gens=inner_gens, outer_gens=1, seed=run_seed, one_shot=0, theta=theta)


def precision(problem_seed: int = 3, run_seed: int = 0, n_inst: int = 64, np_: int = 512, dim: int = 1000) -> Workload:
    """64 inner DEs, NP 512, D 1000: half on Rastrigin, half on Rosenbrock
    (two problems shared by 32 executors each)."""
    rng = np.random.default_rng(problem_seed)
    probs = [make_problem(rng, dim, OBJ_RASTRIGIN), make_problem(rng, dim, OBJ_ROSENBROCK)]
    inst_prob = (np.arange(n_inst) >= n_inst // 2).astype(np.int32)
    theta = random_theta(rng, n_inst)
    return Workload(name=f"precision-{n_inst}x{np_}xD{dim}", problems=probs,
                    inst_np=np.full(n_inst, np_, dtype=np.int32), inst_prob=inst_prob,
                    inst_group=np.arange(n_inst, dtype=np.int32), n_groups=n_inst, n_out=0,
                    inner_gens=100, outer_gens=1, seed=run_seed, one_shot=0, theta=theta)


def mlp(problem_seed: int = 5, run_seed: int = 0, n_inst: int = 64, np_: int = 100, hidden: int = 80,
        n_prob: int = 4, inner_gens: int = 50) -> Workload:
    """The neuroevolution-like workload: 64 inner DEs of NP 100 on the MLP
    regression objective with h = 80 (D = 1522, the size of the paper's
    policy networks), four teacher networks shared by 16 executors each,
    random theta, box [-2, 2] (the teachers lie in [-0.75, 0.75])."""
    rng = np.random.default_rng(problem_seed)
    probs = [make_mlp_problem(rng, hidden) for _ in range(n_prob)]
    inst_prob = (np.arange(n_inst) * n_prob // n_inst).astype(np.int32)
    theta = random_theta(rng, n_inst)
    return Workload(name=f"mlp-{n_inst}x{np_}xD{19 * hidden + 2}", problems=probs,
                    inst_np=np.full(n_inst, np_, dtype=np.int32), inst_prob=inst_prob,
                    inst_group=np.arange(n_inst, dtype=np.int32), n_groups=n_inst, n_out=0,
                    inner_gens=inner_gens, outer_gens=1, seed=run_seed, one_shot=0, theta=theta, lo=-2.0, hi=2.0)


def full(problem_seed: int = 4, run_seed: int = 0, n_runs: int = 8, n_out: int = 128,
         inner_gens: int = 200, outer_gens: int = 50) -> Workload:
    """Eight MetaDE runs of 128 executors (1024 concurrent inner DEs); per run
    NP ~ U{50..200}, D ~ U{20, 50, 100, 200}, objective ~ U{0..5}."""
    rng = np.random.default_rng(problem_seed)
    dims = rng.choice([20, 50, 100, 200], size=n_runs)
    objs = rng.integers(0, 6, size=n_runs)
    nps = rng.integers(50, 201, size=n_runs)
    probs = [make_problem(rng, int(d), int(o)) for d, o in zip(dims, objs)]
    return _runs(f"full-{n_runs}x{n_out}-ragged", probs, nps, n_out, inner_gens, outer_gens, run_seed, 1)


def small_ragged(problem_seed: int = 7, run_seed: int = 0, n_inst: int = 7,
                 dims=(1, 3, 10, 17, 33, 64, 130), nps=(4, 11, 16, 37, 70, 129, 257)) -> Workload:
    """A handful of instances with ragged NP and D (not multiples of 4, 32 or
    a tile), every objective represented; used by the parity tests."""
    rng = np.random.default_rng(problem_seed)
    probs = [make_problem(rng, int(dims[k % len(dims)]), k % 6) for k in range(n_inst)]
    theta = random_theta(rng, n_inst)
    return Workload(name="small-ragged", problems=probs,
                    inst_np=np.array([nps[k % len(nps)] for k in range(n_inst)], dtype=np.int32),
                    inst_prob=np.arange(n_inst, dtype=np.int32),
                    inst_group=np.arange(n_inst, dtype=np.int32), n_groups=n_inst, n_out=0,
                    inner_gens=3, outer_gens=1, seed=run_seed, one_shot=0, theta=theta)


def random_population(rng: np.random.Generator, np_: int, dim: int,
                      lo: float = BOX_LO, hi: float = BOX_HI) -> np.ndarray:
    """A float32 population uniform in the box, for tests that start a step
    from a given state rather than from the method's own initialisation."""
    return rng.uniform(lo, hi, size=(np_, dim)).astype(np.float32)
