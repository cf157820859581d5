"""Helpers shared by the GPU parity tests: build a Batch from a synthetic
workload, feed the same state to the CUDA path and to the oracle, and
compare.  Imports the oracle (tests may) and the binding."""
from __future__ import annotations

import numpy as np

import oracle
import synth

# FP32 trial tolerance: the mutant sums at most 2 dn + 3 = 11 terms of
# magnitude <= 1100 (box 100, F <= 1, dn <= 4) with one rounding each,
# 11 * 2^-24 * 1100 < 1e-3.  Index or mask mistakes move a coordinate by
# O(1..100) and fail by orders of magnitude.
TRIAL_ATOL = 1e-3
# FP32 objective vs FP64 objective at the same float32 point.
FIT_RTOL = 1e-5


def feasible_theta(theta: np.ndarray, nps) -> np.ndarray:
    """Cap dn so that NP >= m + 1 (m = [rand used] + 2 dn) for every executor."""
    th = np.array(theta, dtype=np.float32, copy=True)
    for k, n in enumerate(nps):
        a = 1 if 1 in (int(th[k, 2]), int(th[k, 3])) else 0
        th[k, 4] = max(1, min(int(th[k, 4]), (int(n) - 1 - a) // 2))
    return th


def make_batch(wl: synth.Workload, path: int, **kw):
    import paper_2502_10470_gb300 as M
    probs = [(p.dim, p.obj, p.shift, p.rot) for p in wl.problems]
    return M.Batch(probs, wl.inst_np, wl.inst_prob, wl.inst_group, seed=wl.seed, one_shot=wl.one_shot,
                   p_best_pct=wl.p_best_pct, n_out=kw.pop("n_out", wl.n_out), path=path, lo=wl.lo, hi=wl.hi, **kw)


def random_state(wl: synth.Workload, seed: int = 0, fit_inf: bool = False):
    """float32 populations uniform in the box and float32 stored fitness
    (the oracle's FP64 value rounded), shared by both implementations."""
    rng = np.random.default_rng(seed)
    pops, fits = [], []
    for k in range(wl.n_inst):
        p = wl.problems[int(wl.inst_prob[k])]
        x = synth.random_population(rng, int(wl.inst_np[k]), p.dim, wl.lo, wl.hi)
        pops.append(x)
        if fit_inf:
            fits.append(np.full(x.shape[0], np.inf, dtype=np.float32))
        else:
            fits.append(oracle.eval_pop(p.obj, x, p.shift, p.rot).astype(np.float32))
    return pops, fits


def rel_err(a, b, floor=1.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        return np.abs(a - b) / np.maximum(np.abs(b), floor)


def z_rounding_sensitivity(obj: int, x, shift, rot, unit: float = 2.0 ** -24, acc_unit: float = 2.0 ** -24) -> np.ndarray:
    """First-order change of f when every z_j moves by its error budget
    h_j = unit * sum_c |R_jc d_c| + acc_unit * (|z_j| + sqrt(D) sum_c |R_jc d_c|):
    `unit` bounds the rounding of the products' operands (0 for float32
    operands, 2^-8 for BF16 operands, 2^-16 for split bf16x3), `acc_unit` one
    rounding of z_j plus a D-term float32 accumulation.  Measured with the
    oracle's FP64 objective by central differences."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    R = np.asarray(rot, dtype=np.float64)
    d = x - np.asarray(shift, dtype=np.float64)[None, :]
    z = d @ R.T
    D = z.shape[1]
    s1 = np.abs(d) @ np.abs(R).T
    h = unit * s1 + acc_unit * (np.abs(z) + np.sqrt(D) * s1)
    out = np.zeros(z.shape[0])
    for n in range(z.shape[0]):
        for j in range(D):
            zp, zm = z[n].copy(), z[n].copy()
            zp[j] += h[n, j]
            zm[j] -= h[n, j]
            out[n] += abs(oracle.objective(obj, zp) - oracle.objective(obj, zm)) / 2.0
    return out


def check_fitness(fv, x, prob, rtol: float, unit: float, floor: float = 0.0):
    """Fitness vs the FP64 oracle at the same float32 point: within rtol
    relative, or -- where the objective is ill-conditioned at the point --
    within rtol relative plus 4x the first-order effect of the evaluation's
    rounding budget on z (see z_rounding_sensitivity).  Returns the fraction
    of points that needed the conditioning term."""
    fv = np.asarray(fv, dtype=np.float64)
    f64 = oracle.eval_pop(prob.obj, x, prob.shift, prob.rot)
    err = np.abs(fv - f64)
    base = rtol * np.maximum(np.abs(f64), floor)
    bad = np.nonzero(err > base)[0]
    if bad.size:
        sens = z_rounding_sensitivity(prob.obj, np.asarray(x)[bad], prob.shift, prob.rot, unit=unit)
        over = err[bad] > base[bad] + 4.0 * sens
        assert not over.any(), ("fitness", prob.obj, prob.dim, err[bad][over], f64[bad][over], sens[over])
    return bad.size / max(1, fv.size)


def check_fitness_fp32(f32, x, prob, rtol: float = FIT_RTOL, floor: float = 0.0):
    """FP32 evaluation: 1e-5 relative, or the FP32 conditioning bound."""
    return check_fitness(f32, x, prob, rtol, 0.0, floor)
