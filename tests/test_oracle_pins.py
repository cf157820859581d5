"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names the passage of the paper (or the mathematical fact) it checks.
None of them needs a GPU.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_encodings.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, bl, br, dn, cs = line.split()
            rows.append((name, int(bl), int(br), int(dn), int(cs)))
    return rows


# ------------------------------------------------------------------ Philox
_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c_ptr, out_ptr, seed, N: tl.constexpr):
    o = tl.arange(0, N)
    c0 = tl.load(c_ptr + o * 4 + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + o * 4 + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + o * 4 + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + o * 4 + 3).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + o * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + o * 4 + 3, d.to(tl.int32, bitcast=True))

req = json.loads(sys.stdin.read())
res = []
for seed, ctrs in req:
    n = len(ctrs)
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32).reshape(-1))
    out = torch.zeros(n * 4, dtype=torch.int32)
    k[(1,)](c, out, seed, n)
    res.append((out.numpy().view(np.uint32).reshape(n, 4)).tolist())
print(json.dumps(res))
"""


def test_philox_matches_triton_library_philox():
    """Philox4x32-10 (SC'11) against an independent library implementation:
    Triton's tl.philox run by its CPU interpreter (key = (seed_lo, seed_hi))."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    req = []
    for seed in [0, 1, 0xFFFFFFFF, 0x123456789ABCDEF0, int(rng.integers(0, 2**63))]:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4]] + \
            rng.integers(0, 2**32, size=(13, 4), dtype=np.uint64).tolist()
        req.append((seed, ctrs))
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                          capture_output=True, text=True, env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr.strip().splitlines()[-1])
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(req, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, w in zip(ctrs, want):
            assert oracle.philox(c, key).tolist() == w


def test_philox_output_is_uniform():
    """chi-square on the top byte and on the low byte of 2^18 words; a dropped
    or mis-wired round leaves strong structure in consecutive counters."""
    words = []
    for c in range(1 << 16):
        words.extend(oracle.philox([c, 0, 7, 0], [3, 5]).tolist())
    w = np.array(words, dtype=np.uint64)
    for b in (w >> 24, w & 0xFF):
        cnt = np.bincount(b.astype(np.int64), minlength=256)
        exp = len(w) / 256
        chi2 = ((cnt - exp) ** 2 / exp).sum()
        assert chi2 < 255 + 6 * math.sqrt(2 * 255)  # ~6 sigma


# ------------------------------------------------------------ index draws
def _word_for(s, P):
    # smallest 32-bit word whose floor(w * P / 2^32) equals s
    return -(-(s << 32) // P)


@pytest.mark.parametrize("i", range(4))
def test_distinct_draws_bruteforce_np4(i):
    """Alg. 1, mutation (r1 != r2 != r3 != i): at NP = 4 the 3*2*1 draw values map
    one-to-one onto the 6 ordered triples of {0..3} \\ {i}."""
    seen = set()
    for s0 in range(3):
        for s1 in range(2):
            w = [_word_for(s0, 3), _word_for(s1, 2), _word_for(0, 1)]
            r = tuple(oracle.distinct_draws(4, i, 3, w).tolist())
            assert len(set(r)) == 3 and i not in r
            seen.add(r)
    assert len(seen) == 6


def test_distinct_draws_np10_m9_all_permutations():
    """The nine rand draws of dn = 4 with a rand base: every ordered 9-tuple
    of the other indices arises from exactly one draw vector."""
    import itertools
    i = 3
    others = [c for c in range(10) if c != i]
    seen = set()
    for svec in itertools.islice(itertools.product(*[range(9 - t) for t in range(9)]), 0, None, 7):
        w = [_word_for(s, 9 - t) for t, s in enumerate(svec)]
        r = tuple(oracle.distinct_draws(10, i, 9, w).tolist())
        assert sorted(r) == others
        seen.add(r)
    assert len(seen) == len(list(itertools.islice(
        itertools.product(*[range(9 - t) for t in range(9)]), 0, None, 7)))


def test_distinct_draws_rejects_small_np():
    with pytest.raises(ValueError):
        oracle.distinct_draws(4, 0, 4, [0, 0, 0, 0])


# -------------------------------------------------------------- objectives
def _frame(dim, seed=5):
    rng = np.random.default_rng(seed)
    R = synth.haar_rotation(rng, dim)
    o = rng.uniform(-80, 80, dim)
    return o, R


@pytest.mark.parametrize("obj", range(6))
@pytest.mark.parametrize("dim", [1, 2, 10, 33])
def test_objectives_vanish_at_shift(obj, dim):
    """f(o) = 0 for every synthetic objective (f* = 0 at z = 0)."""
    o, R = _frame(dim)
    f = oracle.eval(obj, o, o, R)
    assert abs(f) < 1e-12


def _at(obj, z, seed=5):
    z = np.asarray(z, dtype=np.float64)
    o, R = _frame(z.shape[0], seed)
    return oracle.eval(obj, o + R.T @ z, o, R)


@pytest.mark.parametrize("dim", [2, 7, 20])
def test_objective_closed_forms(dim):
    """Closed forms of the textbook objectives at simple points, reached
    through the rotation: x = o + R^T z gives R (x - o) = z."""
    e = lambda k: np.eye(dim)[k]
    assert _at(0, e(0)) == pytest.approx(1.0, abs=1e-12)
    assert _at(0, 3 * e(dim - 1)) == pytest.approx(9.0, abs=1e-12)
    # Rastrigin: z^2 - 10 cos(2 pi z) + 10
    assert _at(2, e(0)) == pytest.approx(1.0, abs=1e-10)
    assert _at(2, 0.5 * e(1 % dim)) == pytest.approx(20.25, abs=1e-10)
    # Schwefel 1.2: prefix sums of e_k are 1 from position k on
    assert _at(5, e(0)) == pytest.approx(dim, abs=1e-10)
    assert _at(5, e(dim - 1)) == pytest.approx(1.0, abs=1e-10)
    # Griewank: sum z^2/4000 - prod cos(z_j / sqrt(j)) + 1 (1-based j)
    assert _at(3, e(0)) == pytest.approx(1 / 4000 - math.cos(1.0) + 1, abs=1e-12)
    assert _at(3, e(1)) == pytest.approx(1 / 4000 - math.cos(1 / math.sqrt(2)) + 1, abs=1e-12)
    # Ackley at e_1: the cosine mean is exactly 1, leaving 20 - 20 exp(-0.2 / sqrt(D))
    assert _at(4, e(0)) == pytest.approx(20 - 20 * math.exp(-0.2 / math.sqrt(dim)), abs=1e-10)
    # Rosenbrock on y = z + 1: y = 1 - e_1 leaves the single term 100 * 1 + 1
    assert _at(1, -e(0)) == pytest.approx(101.0, abs=1e-9)


def test_rosenbrock_matches_scipy():
    """Rosenbrock on y = z + 1 equals scipy.optimize.rosen(y) (library routine)."""
    from scipy.optimize import rosen
    rng = np.random.default_rng(3)
    for dim in (2, 5, 30):
        z = rng.normal(size=dim)
        assert oracle.objective(1, z) == pytest.approx(rosen(z + 1.0), rel=1e-13)


def test_sphere_and_schwefel_match_numpy():
    rng = np.random.default_rng(4)
    z = rng.normal(size=17)
    assert oracle.objective(0, z) == pytest.approx(float(np.dot(z, z)), rel=1e-14)
    assert oracle.objective(5, z) == pytest.approx(float((np.cumsum(z) ** 2).sum()), rel=1e-13)


def test_rotation_is_R_times_d_not_transpose():
    """z = R (x - o): a cyclic permutation R (z_r = d_{r+1}) moves e_0 to the
    last coordinate, where Schwefel 1.2 scores 1; R^T would give D - 1."""
    D = 6
    R = np.zeros((D, D))
    for r in range(D):
        R[r, (r + 1) % D] = 1.0
    o = np.zeros(D)
    assert oracle.eval(5, np.eye(D)[0], o, R) == pytest.approx(1.0)
    assert oracle.eval(5, np.eye(D)[0], o, R.T) == pytest.approx(D - 1.0)


def test_haar_rotation_orthogonal():
    rng = np.random.default_rng(0)
    for dim in (1, 10, 100):
        R = synth.haar_rotation(rng, dim)
        assert np.abs(R.T @ R - np.eye(dim)).max() < 1e-12
        R32 = R.astype(np.float32).astype(np.float64)
        assert np.abs(R32.T @ R32 - np.eye(dim)).max() < 1e-6


# ------------------------------------------------------------ init / box
def test_init_uniform_in_box_and_reproducible():
    pop = oracle.init_pop(200, 13, seed=9, stream=2, epoch=0)
    assert pop.min() >= -100.0 and pop.max() < 100.0
    assert abs(pop.mean()) < 3.0 and abs(pop.std() - 200 / math.sqrt(12)) < 3.0
    np.testing.assert_array_equal(pop, oracle.init_pop(200, 13, seed=9, stream=2, epoch=0))
    assert not np.array_equal(pop, oracle.init_pop(200, 13, seed=9, stream=3, epoch=0))
    # the float32 rounding of an initial coordinate is a single rounding of lo + 200 U
    assert np.all(np.abs(pop - pop.astype(np.float32)) <= 2 ** -24 * 100)


# --------------------------------------------------- mutation / crossover
def _unit_state(npop, fit_scale=1e30, seed=0):
    """Population x_k = e_k (D = NP), so a trial's coordinates are its
    coefficients on the individuals; large distinct fitness values so that
    every trial is accepted."""
    rng = np.random.default_rng(seed)
    pop = np.eye(npop)
    fit = fit_scale * (1.0 + rng.permutation(npop))
    return pop, fit


def _step_unit(theta, npop=12, gen=0, seed=1, fit_seed=0):
    pop, fit = _unit_state(npop, seed=fit_seed)
    o = np.zeros(npop)
    R = np.eye(npop)
    out = oracle.pde_step(pop, fit, theta, 0, o, R, seed=seed, stream=0, epoch=0, gen=gen)
    return pop, fit, out


def _textbook(name, F, i, best, pbest, r, npop):
    """The classic mutation equations of Sec. II-A-1 as coefficient vectors."""
    e = np.eye(npop)
    if name == "DE/rand/1/bin":
        return e[r[0]] + F * (e[r[1]] - e[r[2]])
    if name == "DE/best/1/bin":
        return e[best] + F * (e[r[0]] - e[r[1]])
    if name == "DE/current-to-best/1/bin":
        return e[i] + F * (e[best] - e[i]) + F * (e[r[0]] - e[r[1]])
    if name == "DE/rand/2/bin":
        return e[r[0]] + F * (e[r[1]] - e[r[2]]) + F * (e[r[3]] - e[r[4]])
    if name == "DE/best/2/bin":
        return e[best] + F * (e[r[0]] - e[r[1]]) + F * (e[r[2]] - e[r[3]])
    if name == "DE/current-to-pbest/1/bin":
        return e[i] + F * (e[pbest] - e[i]) + F * (e[r[0]] - e[r[1]])
    raise KeyError(name)


@pytest.mark.parametrize("row", [r for r in table1() if r[4] == 1], ids=lambda r: r[0])
def test_table1_encodings_reduce_to_textbook_mutations(row):
    """Table I: the PDE codes reproduce the classic strategies' equations
    (Sec. II-A-1).  CR = 1 makes the trial equal the mutant."""
    name, bl, br, dn, cs = row
    F = 0.375
    npop = 12
    for gen in range(3):
        pop, fit, out = _step_unit([F, 1.0, bl, br, dn, cs], npop=npop, gen=gen)
        order = np.lexsort((np.arange(npop), fit))
        kp = max(1, -(-npop * 10 // 100))
        for i in range(npop):
            rec = out["rec"][i]
            m = rec[8]
            r = [x for x in rec[9:9 + m]]
            assert len(set(r)) == m and i not in r, "rand draws distinct and != i"
            best, pbest = rec[7], rec[6]
            assert best == order[0]
            assert pbest in order[:kp]
            want = _textbook(name, F, i, best, pbest, r, npop)
            np.testing.assert_allclose(out["trial"][i], want, atol=1e-14)


def test_current_to_rand_identity():
    """Eq. (rand/1 + arith) = Eq. (current-to-rand/1):
    x_i + K (v - x_i) = x_i + K (x_r1 - x_i) + K F (x_r2 - x_r3)."""
    F = 0.6
    npop = 12
    pop, fit, out = _step_unit([F, 0.5, 1, 1, 1, 3], npop=npop)
    e = np.eye(npop)
    for i in range(npop):
        rec = out["rec"][i]
        K = rec[5] * 2.0 ** -24
        r1, r2, r3 = rec[9], rec[10], rec[11]
        want = e[i] + K * (e[r1] - e[i]) + K * F * (e[r2] - e[r3])
        np.testing.assert_allclose(out["trial"][i], want, atol=1e-14)


@pytest.mark.parametrize("bl,br", [(b1, b2) for b1 in range(1, 5) for b2 in range(1, 5)])
@pytest.mark.parametrize("dn", [1, 2, 3, 4])
def test_all_192_strategies_affine_and_structured(bl, br, dn):
    """Sec. III-A: the mutant of every DE/bl-to-br/dn is an affine combination
    (coefficients sum to 1) of the base vectors plus dn differences of
    distinct random individuals; bl = br drops the directional term (the
    base is x_bl itself)."""
    F = 0.25
    npop = 12
    for cs in (1, 3):
        pop, fit, out = _step_unit([F, 1.0, bl, br, dn, cs], npop=npop, gen=dn)
        for i in range(npop):
            rec = out["rec"][i]
            u = out["trial"][i]
            K = rec[5] * 2.0 ** -24 if cs == 3 else 1.0
            a = 1 if 1 in (bl, br) else 0
            assert rec[8] == a + 2 * dn
            r = list(rec[9:9 + rec[8]])
            assert len(set(r)) == len(r) and i not in r
            c = np.zeros(npop)
            c[rec[0]] += 1.0
            if bl != br:
                c[rec[1]] += F
                c[rec[0]] -= F
            for q in range(dn):
                c[r[a + 2 * q]] += F
                c[r[a + 2 * q + 1]] -= F
            want = (1 - K) * np.eye(npop)[i] + K * c
            np.testing.assert_allclose(u, want, atol=1e-14)
            assert u.sum() == pytest.approx(1.0, abs=1e-13)
            base = {1: r[0] if a else None, 2: rec[7], 3: rec[6], 4: i}
            assert rec[0] == base[bl] and rec[1] == base[br]


def test_f0_cr0_trial_is_target_except_jrand():
    """F = 0 and CR = 0 with binomial crossover: the trial equals the target
    x_i except at j_rand, where it takes the base vector's coordinate."""
    rng = np.random.default_rng(8)
    pop = rng.uniform(-100, 100, (20, 9))
    fit = rng.uniform(0, 1, 20)
    o, R = _frame(9)
    for bl, br in [(1, 1), (2, 2), (4, 2), (3, 1), (2, 4)]:
        out = oracle.pde_step(pop, fit, [0.0, 0.0, bl, br, 2, 1], 2, o, R, seed=3, stream=1,
                              epoch=0, gen=5)
        for i in range(20):
            diff = np.nonzero(out["trial"][i] != pop[i])[0]
            j = out["rec"][i][2]
            assert set(diff.tolist()) <= {j}
            assert out["trial"][i][j] == pop[out["rec"][i][0]][j]
            assert out["mask"][i].sum() == 1 and out["mask"][i][j] == 1


def test_crossover_extremes():
    """CR = 1: bin and exp take the whole mutant; CR = 0: exp takes one
    coordinate (L = 1, at n); arith with any CR uses K only."""
    rng = np.random.default_rng(9)
    pop = rng.uniform(-100, 100, (16, 7))
    fit = rng.uniform(0, 1, 16)
    o, R = _frame(7)
    for cs in (1, 2):
        out = oracle.pde_step(pop, fit, [0.5, 1.0, 1, 1, 1, cs], 0, o, R, seed=1, stream=0, epoch=0, gen=0)
        assert out["mask"].all()
    out = oracle.pde_step(pop, fit, [0.5, 0.0, 1, 1, 1, 2], 0, o, R, seed=1, stream=0, epoch=0, gen=0)
    for i in range(16):
        assert out["rec"][i][4] == 1
        assert out["mask"][i].sum() == 1 and out["mask"][i][out["rec"][i][3]] == 1


def test_binomial_mask_count_distribution():
    """Eq. (bin): each coordinate other than j_rand is taken with probability
    CR, so E[#taken] = 1 + (D - 1) CR."""
    rng = np.random.default_rng(10)
    D, NP, CR = 40, 200, 0.3
    pop = rng.uniform(-100, 100, (NP, D))
    fit = rng.uniform(0, 1, NP)
    o, R = np.zeros(D), np.eye(D)
    counts = []
    for g in range(5):
        out = oracle.pde_step(pop, fit, [0.5, CR, 1, 1, 1, 1], 0, o, R, seed=2, stream=0, epoch=0, gen=g)
        counts.extend(out["mask"].sum(axis=1).tolist())
    p = math.ceil(np.float32(CR) * 2 ** 24) / 2 ** 24
    mean, n = np.mean(counts), len(counts)
    sigma = math.sqrt((D - 1) * p * (1 - p) / n)
    assert abs(mean - (1 + (D - 1) * p)) < 5 * sigma


def test_exponential_length_is_censored_geometric_and_contiguous():
    """Eq. (exp): L follows a geometric law censored at D with P(L >= k) =
    CR^(k-1), and the taken coordinates form the cyclic run n, ..., n+L-1."""
    rng = np.random.default_rng(12)
    D, NP, CR = 8, 300, 0.7
    pop = rng.uniform(-100, 100, (NP, D))
    fit = rng.uniform(0, 1, NP)
    o, R = np.zeros(D), np.eye(D)
    Ls = []
    for g in range(6):
        out = oracle.pde_step(pop, fit, [0.5, CR, 1, 1, 1, 2], 0, o, R, seed=4, stream=0, epoch=0, gen=g)
        for i in range(NP):
            L, n = out["rec"][i][4], out["rec"][i][3]
            want = np.zeros(D, dtype=np.uint8)
            want[[(n + l) % D for l in range(L)]] = 1
            np.testing.assert_array_equal(out["mask"][i], want)
            Ls.append(L)
    Ls = np.array(Ls)
    p = math.ceil(np.float32(CR) * 2 ** 24) / 2 ** 24
    for k in range(1, D + 1):
        emp = (Ls >= k).mean()
        want = p ** (k - 1)
        assert abs(emp - want) < 5 * math.sqrt(want * (1 - want) / len(Ls)) + 1e-12
    assert (Ls == D).mean() == pytest.approx(p ** (D - 1), abs=0.03)


def test_pbest_drawn_from_top_ten_percent():
    """Sec. II-A-1 (JADE): x_pbest is a random member of the top p% (10%)."""
    rng = np.random.default_rng(13)
    NP, D = 30, 5
    pop = rng.uniform(-100, 100, (NP, D))
    fit = rng.uniform(0, 1, NP)
    top = set(np.argsort(fit)[:3].tolist())  # ceil(0.1 * 30) = 3
    o, R = np.zeros(D), np.eye(D)
    seen = set()
    for g in range(4):
        out = oracle.pde_step(pop, fit, [0.5, 0.5, 4, 3, 1, 1], 0, o, R, seed=5, stream=0, epoch=0, gen=g)
        seen |= set(out["rec"][:, 6].tolist())
    assert seen == top


# --------------------------------------------------------------- selection
def test_tie_accepts_trial():
    """Alg. 1, selection: f(u) <= f(x) accepts; with F = 0 and bl = br = current
    the trial is the target itself, so every individual ties and accepts."""
    rng = np.random.default_rng(14)
    pop = rng.uniform(-100, 100, (10, 6))
    o, R = _frame(6)
    fit = oracle.eval_pop(2, pop, o, R)
    out = oracle.pde_step(pop, fit, [0.0, 0.9, 4, 4, 1, 1], 2, o, R, seed=6, stream=0, epoch=0, gen=0)
    np.testing.assert_array_equal(out["trial"], pop)
    assert out["accept"].all()


def test_generational_selection_and_monotone_best():
    """Alg. 2: the new population holds, per individual, the better of x_i and
    u_i, and the best-so-far fitness never increases."""
    p = synth.make_problem(np.random.default_rng(15), 10, synth.OBJ_RASTRIGIN)
    pop = oracle.init_pop(24, 10, seed=1, stream=0, epoch=0)
    fit = oracle.eval_pop(p.obj, pop, p.shift, p.rot)
    last = fit.min()
    for g in range(30):
        out = oracle.pde_step(pop, fit, [0.7, 0.5, 4, 2, 1, 1], p.obj, p.shift, p.rot, seed=1,
                              stream=0, epoch=0, gen=g)
        take = out["ftrial"] <= fit
        np.testing.assert_array_equal(out["accept"].astype(bool), take)
        np.testing.assert_array_equal(out["pop"], np.where(take[:, None], out["trial"], pop))
        np.testing.assert_array_equal(out["fit"], np.minimum(out["ftrial"], fit))
        assert out["fit"].min() <= last
        last = out["fit"].min()
        pop, fit = out["pop"], out["fit"]


def test_trials_clipped_to_box():
    rng = np.random.default_rng(16)
    pop = rng.uniform(90, 100, (12, 4))
    fit = np.ones(12)
    out = oracle.pde_step(pop, fit, [1.0, 1.0, 2, 4, 4, 1], 0, np.zeros(4), np.eye(4), seed=0,
                          stream=0, epoch=0, gen=0)
    assert out["trial"].max() <= 100.0 and out["trial"].min() >= -100.0


def test_rand1bin_converges_on_sphere():
    """Classic DE/rand/1/bin (F = 0.5, CR = 0.9) solves a 5-D sphere."""
    p = synth.make_problem(np.random.default_rng(17), 5, synth.OBJ_SPHERE)
    y, pop, fit = oracle.pde_run([0.5, 0.9, 1, 1, 1, 1], 40, p.obj, p.shift, p.rot, 300, seed=3, stream=0)
    assert y < 1e-6


# ----------------------------------------------------------------- evolver
def test_decode_table1_and_bounds():
    """Alg. 3, decoding: floor decoding; each Table I row decodes from any point of
    its unit cell, and the upper bound decodes to the top category."""
    for name, bl, br, dn, cs in table1():
        for frac in (0.0, 0.5, 0.999):
            th = oracle.decode([0.3, 0.8, bl + frac, br + frac, dn + frac, cs + frac])
            assert th.tolist() == [0.3, 0.8, bl, br, dn, cs]
    assert oracle.decode(synth.OUTER_UB).tolist() == [1, 1, 4, 4, 4, 3]
    assert oracle.decode(synth.OUTER_LB).tolist() == [0, 0, 1, 1, 1, 1]


def test_decode_spans_192_strategies():
    """Sec. III-A: 4 x 4 x 4 x 3 = 192 strategies DE/bl-to-br/dn/cs."""
    cells = set()
    for bl in np.arange(1.0, 5.0, 0.5):
        for br in np.arange(1.0, 5.0, 0.5):
            for dn in np.arange(1.0, 5.0, 0.5):
                for cs in np.arange(1.0, 4.0, 0.5):
                    cells.add(tuple(oracle.decode([0.5, 0.5, bl, br, dn, cs])[2:].tolist()))
    assert len(cells) == 192


def test_outer_generation0_accepts_all_and_trial_structure():
    """Alg. 3: y starts at +inf, so the first selection accepts every trial;
    trials are rand/1/bin with F = 0.5 inside [lb, ub]."""
    import itertools
    n = 8
    pop, fit = oracle.outer_init(n, seed=2, group=1)
    assert np.all(pop >= synth.OUTER_LB) and np.all(pop <= synth.OUTER_UB)
    assert np.all(np.isinf(fit))
    trial = oracle.outer_trial(pop, seed=2, group=1, gen=0)
    assert np.all(trial >= synth.OUTER_LB) and np.all(trial <= synth.OUTER_UB)
    for i in range(n):
        taken = np.nonzero(trial[i] != pop[i])[0]
        ok = False
        for r0, r1, r2 in itertools.permutations([c for c in range(n) if c != i], 3):
            v = np.clip(pop[r0] + 0.5 * (pop[r1] - pop[r2]), synth.OUTER_LB, synth.OUTER_UB)
            if np.allclose(trial[i][taken], v[taken], atol=1e-14):
                ok = True
                break
        assert ok
    meta = np.random.default_rng(0).uniform(0, 1e6, n)
    npop, nfit, acc = oracle.outer_select(pop, fit, trial, meta)
    assert acc.all()
    np.testing.assert_array_equal(npop, trial)
    np.testing.assert_array_equal(nfit, meta)


def test_metade_tiny_run_improves_meta_fitness():
    """Alg. 3 end to end at the tiny configuration: one-shot evaluation makes
    y*(theta) deterministic, so the best meta-fitness is non-increasing in the
    number of evolver generations (same seed, longer run)."""
    wl = synth.tiny()
    p = wl.problems[0]
    ys = []
    for og in (1, 2, 3):
        y, opop, ofit = oracle.metade_run(8, 16, p.obj, p.shift, p.rot, 5, og, seed=0)
        ys.append(y)
    assert ys[0] >= ys[1] >= ys[2]


# ------------------------------------------------------------ PSO evolver
# The supplement's PSO evolver (w = 0.729, c1 = c2 = 1.49).  Each pin
# switches terms off through w, c1, c2 so that a dropped, swapped or
# sign-flipped term, or the wrong global best, fails one of them.
LB = synth.OUTER_LB.astype(np.float64)
UB = synth.OUTER_UB.astype(np.float64)


def _swarm(n=8, seed=11):
    rng = np.random.default_rng(seed)
    pbest = LB + (UB - LB) * rng.random((n, 6))
    x = LB + (UB - LB) * rng.random((n, 6))
    v = 0.3 * (UB - LB) * (rng.random((n, 6)) - 0.5)
    pfit = rng.random(n) * 10
    return pbest, pfit, x, v


def test_pso_generation0_evaluates_the_initial_swarm():
    pbest, pfit, x, v = _swarm()
    xn, vn = oracle.pso_move(pbest, pfit, x, v, seed=3, group=1, gen=0)
    np.testing.assert_array_equal(xn, pbest)
    assert not vn.any()


def test_pso_inertia_only():
    """c1 = c2 = 0: the velocity only decays by w and the particle coasts."""
    pbest, pfit, x, v = _swarm()
    x = np.clip(x, LB + 0.2 * (UB - LB), UB - 0.2 * (UB - LB))
    v = 0.1 * v
    xn, vn = oracle.pso_move(pbest, pfit, x, v, seed=3, group=1, gen=4, w=0.5, c1=0.0, c2=0.0)
    np.testing.assert_allclose(vn, 0.5 * v, rtol=0, atol=1e-15)
    np.testing.assert_allclose(xn, x + 0.5 * v, rtol=0, atol=1e-15)


def test_pso_cognitive_term_pulls_toward_the_own_best():
    """w = 0, c2 = 0: v = c1 r1 (pbest - x) with r1 in [0, 1), so every
    coordinate moves toward the particle's own best and never past it."""
    pbest, pfit, x, v = _swarm()
    _, vn = oracle.pso_move(pbest, pfit, x, v, seed=5, group=2, gen=7, w=0.0, c1=1.0, c2=0.0)
    r1 = vn / (pbest - x)
    assert np.all((r1 >= 0.0) & (r1 < 1.0))
    assert np.std(r1) > 0.1                                   # one uniform per coordinate


def test_pso_social_term_pulls_toward_the_run_best():
    """w = 0, c1 = 0: v = c2 r2 (gbest - x), gbest = personal best of lowest
    fitness, ties to the lower index."""
    pbest, pfit, x, v = _swarm()
    pfit[5] = pfit[2] = pfit.min() - 1.0                      # tie: index 2 wins
    _, vn = oracle.pso_move(pbest, pfit, x, v, seed=5, group=2, gen=7, w=0.0, c1=0.0, c2=1.0)
    r2 = vn / (pbest[2] - x)
    assert np.all((r2 >= 0.0) & (r2 < 1.0))
    r1 = oracle.pso_move(pbest, pfit, x, v, seed=5, group=2, gen=7, w=0.0, c1=1.0, c2=0.0)[1] / (pbest - x)
    assert np.abs(r1 - r2).max() > 0.1                        # r1 and r2 are separate draws


def test_pso_full_update_is_the_sum_of_its_terms():
    pbest, pfit, x, v = _swarm()
    x = np.clip(x, LB + 0.3 * (UB - LB), UB - 0.3 * (UB - LB))
    v = 0.05 * v
    pbest = np.clip(pbest, LB + 0.3 * (UB - LB), UB - 0.3 * (UB - LB))
    args = dict(seed=9, group=0, gen=3)
    vw = oracle.pso_move(pbest, pfit, x, v, w=0.729, c1=0.0, c2=0.0, **args)[1]
    vc = oracle.pso_move(pbest, pfit, x, v, w=0.0, c1=1.49, c2=0.0, **args)[1]
    vs = oracle.pso_move(pbest, pfit, x, v, w=0.0, c1=0.0, c2=1.49, **args)[1]
    xn, vn = oracle.pso_move(pbest, pfit, x, v, **args)
    np.testing.assert_allclose(vn, vw + vc + vs, rtol=0, atol=1e-12)
    inside = (x + vn > LB) & (x + vn < UB)
    np.testing.assert_allclose(xn[inside], (x + vn)[inside], rtol=0, atol=1e-12)


def test_pso_positions_stay_in_the_box():
    pbest, pfit, x, v = _swarm()
    xn, _ = oracle.pso_move(pbest, pfit, x, 50.0 * v, seed=1, group=0, gen=2)
    assert np.all(xn >= LB) and np.all(xn <= UB)


def test_pso_minimises_a_sphere_in_the_evolver_box():
    """Move + Alg. 3 selection on f(x) = |x - c|^2 inside the gene box."""
    c = LB + 0.37 * (UB - LB)
    pbest, pfit = oracle.outer_init(16, seed=4, group=0)
    x = np.zeros_like(pbest)
    v = np.zeros_like(pbest)
    for g in range(120):
        x, v = oracle.pso_move(pbest, pfit, x, v, seed=4, group=0, gen=g)
        y = ((x - c) ** 2).sum(axis=1)
        pbest, pfit, _ = oracle.outer_select(pbest, pfit, x, y)
    assert pfit.min() < 1e-6


def test_pso_metade_run_meta_fitness_does_not_rise():
    wl = synth.tiny()
    p = wl.problems[0]
    y3 = oracle.metade_run(wl.n_out, 16, p.obj, p.shift, p.rot, 10, 3, seed=2, evolver=1)[0]
    y6 = oracle.metade_run(wl.n_out, 16, p.obj, p.shift, p.rot, 10, 6, seed=2, evolver=1)[0]
    assert y6 <= y3


# ------------------------------------------------------------- CSO evolver
# Competitive Swarm Optimizer (Cheng and Jin 2015) as the evolver: random
# pairs, the fitter particle of a pair is kept, the other learns from it
# (v <- r1 v + r2 (x_w - x_l), x <- x + v; swarm-mean factor phi = 0).
def _cso_partner(pop, fit, xn, flag, l):
    """The winner whose segment from x_l contains x'_l (gen-1 move, v = 0)."""
    d = xn[l] - pop[l]
    cands = []
    for w in np.flatnonzero(flag == 0):
        span = pop[w] - pop[l]
        r = np.divide(d, span, out=np.full(6, np.nan), where=span != 0)
        if np.all((span != 0) & (r >= 0) & (r < 1)):
            cands.append(int(w))
    return cands


def test_cso_generation0_evaluates_the_initial_swarm():
    pop, fit, _, _ = _swarm(9)
    xn, v, flag = oracle.cso_move(pop, fit, np.ones((9, 6)), seed=3, group=1, gen=0)
    np.testing.assert_array_equal(xn, pop)
    assert not v.any() and flag.all()


@pytest.mark.parametrize("n", [8, 9, 30])
def test_cso_losers_learn_from_their_winners(n):
    """floor(n/2) losers; a winner (and an odd particle out) is unchanged;
    with v = 0 each loser moves onto the segment toward exactly one winner,
    which is no worse than the loser; the winners found this way are
    distinct (one per pair)."""
    pop, fit, _, _ = _swarm(n, seed=n)
    xn, v, flag = oracle.cso_move(pop, fit, np.zeros((n, 6)), seed=7, group=2, gen=1)
    assert flag.sum() == n // 2
    np.testing.assert_array_equal(xn[flag == 0], pop[flag == 0])
    np.testing.assert_array_equal(v[flag == 0], 0.0)
    losers = [int(l) for l in np.flatnonzero(flag)]
    cands = {}
    for l in losers:
        np.testing.assert_allclose(v[l], xn[l] - pop[l], rtol=0, atol=1e-12)
        cands[l] = [w for w in _cso_partner(pop, fit, xn, flag, l)
                    if fit[w] < fit[l] or (fit[w] == fit[l] and w < l)]
        assert cands[l], l
    # every loser has its own winner: a perfect matching (augmenting paths)
    match = {}

    def augment(l, seen):
        for w in cands[l]:
            if w in seen:
                continue
            seen.add(w)
            if w not in match or augment(match[w], seen):
                match[w] = l
                return True
        return False

    assert all(augment(l, set()) for l in losers)


def test_cso_velocity_memory():
    """A loser's old velocity enters scaled by r1 in [0, 1): with x_w = x_l
    (identical pair) the move is r1 v exactly."""
    pop = np.tile(LB + 0.5 * (UB - LB), (2, 1))
    fit = np.array([1.0, 2.0])
    v0 = 0.1 * (UB - LB) * np.array([[1, -1, 1, -1, 1, -1], [1, 1, -1, -1, 1, 1]], dtype=float)
    xn, v, flag = oracle.cso_move(pop, fit, v0, seed=5, group=0, gen=3)
    assert flag.tolist() == [0, 1]
    r1 = v[1] / v0[1]
    assert np.all((r1 >= 0) & (r1 < 1)) and np.std(r1) > 0.05
    np.testing.assert_allclose(xn[1], pop[1] + v[1], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v[0], v0[0])


def test_cso_pairings_are_uniform():
    """m = 4 has three pairings, each with probability 1/3 under a uniform
    random permutation (Fisher-Yates); chi-square over 3000 generations."""
    # positions whose differences to the possible winners of each loser
    # differ in sign in some coordinate, so the move names the partner
    unit = np.array([[0.1] * 6, [0.7] * 6, [0.9, 0.2] * 3, [0.3, 0.8] * 3])
    pop = LB + (UB - LB) * unit
    fit = np.array([1.0, 2.0, 3.0, 4.0])
    counts = {}
    for g in range(1, 3001):
        xn, v, flag = oracle.cso_move(pop, fit, np.zeros((4, 6)), seed=11, group=0, gen=g)
        pairs = []
        for l in np.flatnonzero(flag):
            (w,) = _cso_partner(pop, fit, xn, flag, l)
            pairs.append(tuple(sorted((int(w), int(l)))))
        key = tuple(sorted(pairs))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 3
    obs = np.array(list(counts.values()), dtype=float)
    chi2 = ((obs - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 13.8                                        # p > 0.001 at 2 dof


def test_cso_select_replaces_flagged_unconditionally():
    pop, fit, _, _ = _swarm(6)
    xn = pop + 0.01
    flag = np.array([1, 0, 1, 0, 1, 0], dtype=np.int32)
    y = fit + 100.0                                           # worse, still taken
    y[4] = np.nan
    p2, f2 = oracle.cso_select(pop, fit, xn, flag, y)
    np.testing.assert_array_equal(p2[flag == 1], xn[flag == 1])
    np.testing.assert_array_equal(p2[flag == 0], pop[flag == 0])
    assert f2[0] == y[0] and f2[2] == y[2] and np.isinf(f2[4])
    np.testing.assert_array_equal(f2[flag == 0], fit[flag == 0])


def test_cso_minimises_a_sphere_in_the_evolver_box():
    c = LB + 0.37 * (UB - LB)
    pop, fit = oracle.outer_init(32, seed=4, group=0)
    v = np.zeros_like(pop)
    for g in range(300):
        xn, v, flag = oracle.cso_move(pop, fit, v, seed=4, group=0, gen=g)
        pop, fit = oracle.cso_select(pop, fit, xn, flag, ((xn - c) ** 2).sum(axis=1))
    assert fit.min() < 1e-6


# ------------------------------------------------------------- NES evolver
# xNES (Wierstra et al. 2014): the pins are the matrix exponential against
# scipy, the normal draws, the initial distribution, det B = 1 under every
# update (tr G_B = 0), and the two-sample closed form of the update.
NES_ETA = 3.0 * (3.0 + math.log(6.0)) / (5.0 * 6.0 * math.sqrt(6.0))


def test_nes_expm_matches_scipy():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(0)
    for n in (1, 2, 6):
        for _ in range(5):
            A = rng.normal(size=(n, n))
            S = 0.5 * (A + A.T)
            np.testing.assert_allclose(oracle.expm_sym(S), sl.expm(S), rtol=1e-12, atol=1e-12)


def test_nes_samples_are_standard_normal():
    stats = pytest.importorskip("scipy.stats")
    st = oracle.nes_init()
    s = np.concatenate([oracle.nes_sample(st, 500, seed=5, group=g, gen=1)[0] for g in range(4)])
    for j in range(6):
        assert stats.kstest(s[:, j], "norm").pvalue > 1e-3
    c = np.corrcoef(s.T)
    assert np.abs(c - np.eye(6)).max() < 0.06                  # independent coordinates


def test_nes_initial_distribution_and_sample_map():
    st = oracle.nes_init()
    np.testing.assert_allclose(st[:6], 0.5 * (LB + UB))
    B = st[7:].reshape(6, 6)
    np.testing.assert_allclose(st[6] * B, np.diag((UB - LB) / 4.0), atol=1e-15)
    assert abs(np.linalg.det(B) - 1.0) < 1e-12
    s, z, zc = oracle.nes_sample(st, 64, seed=2, group=0, gen=0)
    np.testing.assert_allclose(z, st[:6] + st[6] * s @ B.T, atol=1e-12)
    np.testing.assert_array_equal(zc, np.clip(z, LB, UB))


def test_nes_update_keeps_det_b_one():
    rng = np.random.default_rng(1)
    st = oracle.nes_init()
    for g in range(20):
        s, z, zc = oracle.nes_sample(st, 24, seed=3, group=0, gen=g)
        st = oracle.nes_update(st, s, rng.random(24))
        assert abs(np.linalg.det(st[7:].reshape(6, 6)) - 1.0) < 1e-9


def test_nes_two_sample_closed_form():
    """lambda = 2: utilities +1/2 (better) and -1/2 (worse), so
    mu' = mu + sigma B (s_b - s_w)/2, sigma' = sigma exp(eta (|s_b|^2 - |s_w|^2) / (4 d)),
    B' = B expm(eta/2 (G_M - G_sigma I)) with G_M = (s_b s_b^T - s_w s_w^T)/2."""
    sl = pytest.importorskip("scipy.linalg")
    st = oracle.nes_init()
    st[7:] = (st[7:].reshape(6, 6) @ sl.expm(0.1 * np.triu(np.ones((6, 6))) - 0.1 * np.tril(np.ones((6, 6))))).ravel()
    s, _, _ = oracle.nes_sample(st, 2, seed=8, group=1, gen=5)
    for y in ([1.0, 2.0], [3.0, -1.0]):
        b, w = (0, 1) if y[0] < y[1] else (1, 0)
        st2 = oracle.nes_update(st, s, np.array(y))
        B, sig = st[7:].reshape(6, 6), st[6]
        np.testing.assert_allclose(st2[:6], st[:6] + sig * B @ (s[b] - s[w]) / 2, rtol=0, atol=1e-12)
        gs = (s[b] @ s[b] - s[w] @ s[w]) / (2 * 6)
        np.testing.assert_allclose(st2[6], sig * math.exp(0.5 * NES_ETA * gs), rtol=1e-13)
        GM = 0.5 * (np.outer(s[b], s[b]) - np.outer(s[w], s[w]))
        np.testing.assert_allclose(st2[7:].reshape(6, 6), B @ sl.expm(0.5 * NES_ETA * (GM - gs * np.eye(6))),
                                   rtol=0, atol=1e-12)


def test_nes_minimises_a_sphere_in_the_evolver_box():
    c = LB + 0.37 * (UB - LB)
    st = oracle.nes_init()
    for g in range(150):
        s, z, zc = oracle.nes_sample(st, 16, seed=4, group=0, gen=g)
        st = oracle.nes_update(st, s, ((zc - c) ** 2).sum(axis=1))
    assert ((st[:6] - c) ** 2).sum() < 1e-6


def test_cso_and_nes_metade_runs():
    wl = synth.tiny()
    p = wl.problems[0]
    for ev in (2, 3):
        y, opop, ofit = oracle.metade_run(wl.n_out, 16, p.obj, p.shift, p.rot, 10, 3, seed=2, evolver=ev)
        assert np.isfinite(y) and y == ofit.min()
        assert np.all(opop >= LB) and np.all(opop <= UB)


# ------------------------------------------------------------ MLP objective
# Objective 6: a 16-h-2 tanh perceptron's parameters against a teacher (the
# shift).  The pins are symmetries and exact identities of the network, so
# a transposed weight layout, a bias outside the tanh, a wrong output index
# or a wrong normalisation fails one of them.
def _mlp_parts(th, h):
    W1 = th[:16 * h].reshape(16, h)
    b1 = th[16 * h:17 * h]
    W2 = th[17 * h:19 * h].reshape(h, 2)
    b2 = th[19 * h:]
    return W1, b1, W2, b2


def _mlp_join(W1, b1, W2, b2):
    return np.concatenate([W1.reshape(-1), b1, W2.reshape(-1), b2])


def _mlp_case(h=6, seed=5):
    rng = np.random.default_rng(seed)
    p = synth.make_mlp_problem(rng, h)
    th = rng.uniform(-1.0, 1.0, p.dim)
    return p, th


def test_mlp_dimension_rule_and_teacher_optimum():
    p, th = _mlp_case()
    assert oracle.mlp_hidden(p.dim) == 6 and oracle.mlp_hidden(p.dim + 1) == 0
    assert np.isnan(oracle.mlp(th[:-1], p.shift[:-1]))
    assert oracle.mlp(p.shift, p.shift) == 0.0
    assert oracle.eval(synth.OBJ_MLP, th, p.shift, p.rot) == oracle.mlp(th, p.shift) > 0.0


def test_mlp_inputs_are_uniform_in_the_unit_box():
    X = oracle.mlp_inputs()
    assert X.shape == (256, 16) and X.min() >= -1.0 and X.max() < 1.0
    assert abs(X.mean()) < 0.05 and abs(X.var() - 1.0 / 3.0) < 0.03
    np.testing.assert_array_equal(X, oracle.mlp_inputs())


def test_mlp_hidden_unit_permutation_and_sign_symmetry():
    p, th = _mlp_case()
    W1, b1, W2, b2 = _mlp_parts(th, 6)
    f = oracle.mlp(th, p.shift)
    perm = np.array([3, 0, 5, 1, 4, 2])
    assert np.isclose(oracle.mlp(_mlp_join(W1[:, perm], b1[perm], W2[perm], b2), p.shift), f, rtol=1e-13)
    s = np.array([1, -1, 1, -1, -1, 1.0])          # tanh is odd: flip units 1, 3, 4
    assert np.isclose(oracle.mlp(_mlp_join(W1 * s, b1 * s, W2 * s[:, None], b2), p.shift), f, rtol=1e-13)


def test_mlp_hidden_bias_enters_through_the_tanh_and_its_output_row():
    """A unit with zero input weights outputs tanh(b1_j) W2[j, :] for every
    input: moving that constant into b2 leaves f unchanged, and a unit whose
    output row is zero does not matter at all."""
    p, th = _mlp_case()
    W1, b1, W2, b2 = _mlp_parts(th, 6)
    W1[:, 2] = 0.0
    f = oracle.mlp(_mlp_join(W1, b1, W2, b2), p.shift)
    moved_b1 = b1.copy()
    moved_b1[2] = 0.0
    assert np.isclose(oracle.mlp(_mlp_join(W1, moved_b1, W2, b2 + np.tanh(b1[2]) * W2[2]), p.shift), f, rtol=1e-12)
    W2[4] = 0.0
    f0 = oracle.mlp(_mlp_join(W1, b1, W2, b2), p.shift)
    W1b, b1b = W1.copy(), b1.copy()
    W1b[:, 4] += 3.0
    b1b[4] -= 2.0
    assert oracle.mlp(_mlp_join(W1b, b1b, W2, b2), p.shift) == f0


def test_mlp_is_a_mean_of_squares_in_the_output_bias():
    """f is quadratic in each output bias with second difference 2 delta^2 /
    (number of outputs): the mean is over inputs and both outputs."""
    p, th = _mlp_case()
    d = 0.37
    for o in range(2):
        e = np.zeros(p.dim)
        e[-2 + o] = d
        second = oracle.mlp(th + e, p.shift) + oracle.mlp(th - e, p.shift) - 2.0 * oracle.mlp(th, p.shift)
        assert abs(second - d * d) < 1e-12
