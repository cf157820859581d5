"""FP64 CPU oracle for the MetaDE hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``metade_oracle.c`` (plain C,
compiled for the host with gcc) through ctypes and adds nothing to its
arithmetic: the functions below marshal numpy arrays and loop over
instances.  It imports nothing from the CUDA package.

What each function follows in the paper:
  pde_step      one generation of PDE, Alg. 2 (mutation Eq. of
                Sec. III-A-2, crossovers of Sec. II-A, greedy selection)
  pde_run       a whole PDE run, Alg. 2
  init_pop      Alg. 2, initialisation (uniform in the box, evaluate)
  eval          the synthetic shifted-rotated objectives, z = R (x - o)
  outer_*       the evolver of Alg. 3 (rand/1/bin, F = 0.5, CR = 0.9,
                y initialised to +inf, floor decoding, selection)
  metade_run    Alg. 3 end to end with one-shot evaluation (Sec. III-C)
  pso_move      PSO as the evolver (supplement, comparison of evolvers)
  cso_*         CSO as the evolver (Cheng and Jin 2015; same supplement)
  nes_*         xNES as the evolver (Wierstra et al. 2014; same supplement),
                with expm_sym its matrix exponential (Jacobi eigenvectors)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "metade_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libmetade_oracle.so")
REC = 18  # int32 fields per individual in the step record

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle for the host (gcc, -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_distinct_draws.argtypes = [C.c_int, C.c_int, C.c_int, P, P]
        L.or_distinct_draws.restype = C.c_int
        L.or_objective.argtypes = [C.c_int, C.c_int, P]
        L.or_objective.restype = C.c_double
        L.or_eval.argtypes = [C.c_int, C.c_int, P, P, P]
        L.or_eval.restype = C.c_double
        L.or_init_pop.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                  C.c_double, C.c_double, P]
        L.or_eval_pop.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P]
        L.or_required_np.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_required_np.restype = C.c_int
        L.or_pde_step.argtypes = [C.c_int, C.c_int, C.c_int, P, P, C.c_double, C.c_double,
                                  C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, P, P, P,
                                  P, P, P, P, P]
        L.or_pde_step.restype = C.c_int
        L.or_best.argtypes = [C.c_int, P, P]
        L.or_best.restype = C.c_double
        L.or_pde_run.argtypes = [C.c_int, C.c_int, C.c_int, P, P, C.c_double, C.c_double,
                                 C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, P, C.c_int, P, P]
        L.or_pde_run.restype = C.c_double
        L.or_outer_init.argtypes = [C.c_int, C.c_uint64, C.c_uint32, P, P]
        L.or_outer_trial.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, P, P]
        L.or_outer_trial.restype = C.c_int
        L.or_decode.argtypes = [P, P]
        L.or_outer_select.argtypes = [C.c_int, P, P, P, P, P]
        L.or_metade_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, P, C.c_double, C.c_double,
                                    C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
        L.or_mlp_inputs.argtypes = [P]
        L.or_mlp_hidden.argtypes = [C.c_int]
        L.or_mlp_hidden.restype = C.c_int
        L.or_mlp.argtypes = [C.c_int, P, P]
        L.or_mlp.restype = C.c_double
        L.or_pso_move.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double, C.c_double,
                                  C.c_double, P, P, P, P]
        L.or_cso_move.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, P, P, P, P, P]
        L.or_cso_select.argtypes = [C.c_int, P, P, P, P, P]
        L.or_nes_init.argtypes = [P]
        L.or_nes_sample.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, P, P, P, P]
        L.or_nes_update.argtypes = [C.c_int, P, P, P]
        L.or_expm_sym.argtypes = [C.c_int, P, P]
        L.or_metade_run.restype = C.c_double
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ------------------------------------------------------------------ Philox
def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def distinct_draws(np_: int, i: int, m: int, words) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint32))
    r = np.full(max(m, 1), -1, dtype=np.int32)
    rc = lib().or_distinct_draws(np_, i, m, _p(w), _p(r))
    if rc != 0:
        raise ValueError("np too small for %d distinct draws" % m)
    return r[:m]


def required_np(bl: int, br: int, dn: int) -> int:
    return lib().or_required_np(bl, br, dn)


# -------------------------------------------------------------- objectives
def objective(obj: int, z) -> float:
    z = _f64(z)
    return lib().or_objective(obj, z.shape[0], _p(z))


def eval(obj: int, x, o, R) -> float:  # noqa: A001 - the paper's "evaluate"
    x, o, R = _f64(x), _f64(o), _f64(R)
    return lib().or_eval(obj, x.shape[0], _p(x), _p(o), _p(R))


MLP_IN, MLP_OUT, MLP_N = 16, 2, 256


def mlp_hidden(dim: int) -> int:
    """Hidden width h of the MLP objective for D = 19 h + 2 (0 if D has no such h)."""
    return lib().or_mlp_hidden(dim)


def mlp_inputs() -> np.ndarray:
    """The MLP objective's inputs, [256][16], uniform in [-1, 1]."""
    X = np.zeros((MLP_N, MLP_IN))
    lib().or_mlp_inputs(_p(X))
    return X


def mlp(theta, teacher) -> float:
    """MLP objective: mean squared difference between the outputs of the
    parameters theta and of the teacher over the inputs."""
    theta, teacher = _f64(theta), _f64(teacher)
    return lib().or_mlp(theta.shape[0], _p(theta), _p(teacher))


def eval_pop(obj: int, pop, o, R) -> np.ndarray:
    pop, o, R = _f64(pop), _f64(o), _f64(R)
    fit = np.zeros(pop.shape[0], dtype=np.float64)
    lib().or_eval_pop(pop.shape[0], pop.shape[1], obj, _p(o), _p(R), _p(pop), _p(fit))
    return fit


def init_pop(np_: int, dim: int, seed: int, stream: int, epoch: int,
             lo: float = -100.0, hi: float = 100.0) -> np.ndarray:
    pop = np.zeros((np_, dim), dtype=np.float64)
    lib().or_init_pop(np_, dim, seed, stream, epoch, lo, hi, _p(pop))
    return pop


# ---------------------------------------------------------------- PDE step
def pde_step(pop, fit, theta, obj: int, o, R, *, seed: int, stream: int, epoch: int, gen: int,
             lo: float = -100.0, hi: float = 100.0, p_best_pct: int = 10) -> Dict[str, np.ndarray]:
    """One generation on one instance; returns the new state and the record."""
    pop = _f64(pop).copy()
    fit = _f64(fit).copy()
    o, R, th = _f64(o), _f64(R), _f64(theta)
    np_, dim = pop.shape
    out = dict(trial=np.zeros((np_, dim)), ftrial=np.zeros(np_),
               accept=np.zeros(np_, dtype=np.int32), mask=np.zeros((np_, dim), dtype=np.uint8),
               rec=np.zeros((np_, REC), dtype=np.int32))
    rc = lib().or_pde_step(np_, dim, obj, _p(o), _p(R), lo, hi, seed, stream, epoch, gen,
                           p_best_pct, _p(th), _p(pop), _p(fit), _p(out["trial"]),
                           _p(out["ftrial"]), _p(out["accept"]), _p(out["mask"]), _p(out["rec"]))
    if rc != 0:
        raise ValueError("or_pde_step failed (%d)" % rc)
    out["pop"] = pop
    out["fit"] = fit
    return out


def best(fit) -> (float, int):
    fit = _f64(fit)
    bi = np.zeros(1, dtype=np.int32)
    b = lib().or_best(fit.shape[0], _p(fit), _p(bi))
    return b, int(bi[0])


def pde_run(theta, np_: int, obj: int, o, R, gens: int, *, seed: int, stream: int, epoch: int = 0,
            lo: float = -100.0, hi: float = 100.0, p_best_pct: int = 10):
    o, R, th = _f64(o), _f64(R), _f64(theta)
    dim = o.shape[0]
    pop = np.zeros((np_, dim))
    fit = np.zeros(np_)
    y = lib().or_pde_run(np_, dim, obj, _p(o), _p(R), lo, hi, seed, stream, epoch, p_best_pct,
                         _p(th), gens, _p(pop), _p(fit))
    return y, pop, fit


# ----------------------------------------------------------------- evolver
def outer_init(n_out: int, seed: int, group: int):
    pop = np.zeros((n_out, 6))
    fit = np.zeros(n_out)
    lib().or_outer_init(n_out, seed, group, _p(pop), _p(fit))
    return pop, fit


def outer_trial(pop, seed: int, group: int, gen: int) -> np.ndarray:
    pop = _f64(pop)
    trial = np.zeros_like(pop)
    if lib().or_outer_trial(pop.shape[0], seed, group, gen, _p(pop), _p(trial)) != 0:
        raise ValueError("evolver population must be >= 4")
    return trial


def decode(u) -> np.ndarray:
    u = _f64(u)
    th = np.zeros(6)
    lib().or_decode(_p(u), _p(th))
    return th


def outer_select(pop, fit, trial, meta_fit):
    pop, fit = _f64(pop).copy(), _f64(fit).copy()
    trial, meta_fit = _f64(trial), _f64(meta_fit)
    acc = np.zeros(pop.shape[0], dtype=np.int32)
    lib().or_outer_select(pop.shape[0], _p(pop), _p(fit), _p(trial), _p(meta_fit), _p(acc))
    return pop, fit, acc


def pso_move(pbest, pfit, x, v, seed: int, group: int, gen: int, w: float = 0.729, c1: float = 1.49,
             c2: float = 1.49):
    """PSO evolver move: returns the new positions and velocities (gen 0:
    x = pbest, v = 0)."""
    pbest, pfit = _f64(pbest), _f64(pfit)
    x, v = _f64(x).copy(), _f64(v).copy()
    lib().or_pso_move(pbest.shape[0], seed, group, gen, w, c1, c2, _p(pbest), _p(pfit), _p(x), _p(v))
    return x, v


def cso_move(pop, fit, v, seed: int, group: int, gen: int):
    """CSO evolver move: returns (x', v', flag) -- x' the positions to
    evaluate (losers moved, winners as they were), flag 1 for the particles
    whose evaluation replaces their position and fitness (gen 0: all)."""
    pop, fit = _f64(pop), _f64(fit)
    v = _f64(v).copy()
    xn = np.zeros_like(pop)
    flag = np.zeros(pop.shape[0], dtype=np.int32)
    lib().or_cso_move(pop.shape[0], seed, group, gen, _p(pop), _p(fit), _p(xn), _p(v), _p(flag))
    return xn, v, flag


def cso_select(pop, fit, xn, flag, meta_fit):
    pop, fit = _f64(pop).copy(), _f64(fit).copy()
    flag = np.ascontiguousarray(np.asarray(flag, dtype=np.int32))
    lib().or_cso_select(pop.shape[0], _p(pop), _p(fit), _p(_f64(xn)), _p(flag), _p(_f64(meta_fit)))
    return pop, fit


NES_STATE = 43  # mu[6], sigma, B[6][6] row-major


def nes_init() -> np.ndarray:
    st = np.zeros(NES_STATE)
    lib().or_nes_init(_p(st))
    return st


def nes_sample(st, n_out: int, seed: int, group: int, gen: int):
    """xNES samples of one generation: (s, z, clip(z)), each [n_out][6]."""
    st = _f64(st)
    s = np.zeros((n_out, 6))
    z = np.zeros((n_out, 6))
    zc = np.zeros((n_out, 6))
    lib().or_nes_sample(n_out, seed, group, gen, _p(st), _p(s), _p(z), _p(zc))
    return s, z, zc


def nes_update(st, s, meta_fit) -> np.ndarray:
    st = _f64(st).copy()
    s = _f64(s)
    lib().or_nes_update(s.shape[0], _p(st), _p(s), _p(_f64(meta_fit)))
    return st


def expm_sym(S) -> np.ndarray:
    """exp of a symmetric matrix (n <= 8) by Jacobi eigendecomposition."""
    S = _f64(S)
    E = np.zeros_like(S)
    lib().or_expm_sym(S.shape[0], _p(S), _p(E))
    return E


def metade_run(n_out: int, np_: int, obj: int, o, R, inner_gens: int, outer_gens: int, *,
               seed: int, group: int = 0, power_up: bool = False,
               lo: float = -100.0, hi: float = 100.0, p_best_pct: int = 10, evolver: int = 0):
    """evolver 0: DE/rand/1/bin (Alg. 3); 1: PSO (w = 0.729, c1 = c2 = 1.49);
    2: CSO; 3: NES (xNES)."""
    o, R = _f64(o), _f64(R)
    opop = np.zeros((n_out, 6))
    ofit = np.zeros(n_out)
    y = lib().or_metade_run(n_out, np_, o.shape[0], obj, _p(o), _p(R), lo, hi, seed, group,
                            p_best_pct, inner_gens, outer_gens, int(power_up), int(evolver), _p(opop), _p(ofit))
    return y, opop, ofit


# ----------------------------------------------------- workload-level loops
def stream_of(wl, k: int) -> int:
    """Counter word 0 of instance k: the run's shared stream under one-shot
    evaluation (Sec. III-C), the instance itself otherwise."""
    return int(wl.inst_group[k]) if wl.one_shot else int(k)


def step_workload(wl, pops: List[np.ndarray], fits: List[np.ndarray], theta: np.ndarray,
                  epoch: int, gen: int, instances=None) -> List[Dict[str, np.ndarray]]:
    """One generation of every (or the listed) instance of a workload."""
    ks = range(wl.n_inst) if instances is None else instances
    outs = []
    for k in ks:
        p = wl.problems[int(wl.inst_prob[k])]
        outs.append(pde_step(pops[k], fits[k], theta[k], p.obj, p.shift, p.rot, seed=wl.seed,
                             stream=stream_of(wl, k), epoch=epoch, gen=gen, lo=wl.lo, hi=wl.hi,
                             p_best_pct=wl.p_best_pct))
    return outs
