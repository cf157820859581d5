"""Python binding of the MetaDE C-ABI (include/metade.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libmetade.so.  Torch tensors provide device memory and the
stream; their data pointers are passed straight through.  There is no CPU
fallback: if libmetade.so has not been built, loading it raises.

The functions keep the C names (metade_create, metade_inner_step, ...);
`Batch` is a small convenience that owns the device tensors of one batch of
executors.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmetade.so")

METADE_OK, METADE_EINVAL, METADE_ENOMEM, METADE_ECUDA, METADE_ETIMEOUT, METADE_ESTATE, METADE_EUNSUPPORTED = range(7)
METADE_FP32, METADE_BF16, METADE_FP8E4M3, METADE_BF16X3, METADE_FP64 = range(5)
EVOLVER_DE, EVOLVER_PSO, EVOLVER_CSO, EVOLVER_NES = 0, 1, 2, 3
METADE_PATH_BATCHED, METADE_PATH_PLAIN = 0, 1
REC_FIELDS = 18

EXPORTED = [
    "metade_create", "metade_destroy", "metade_layout", "metade_offsets", "metade_set_stream",
    "metade_init", "metade_inner_step", "metade_eval", "metade_eval_pop", "metade_outer_init", "metade_outer_step",
    "metade_outer_generation", "metade_draw_record", "metade_sync", "metade_plan_info",
    "metade_launch_count", "metade_strerror", "metade_plain_step_noalloc", "metade_profile",
    "metade_profile_read", "metade_autotune", "metade_wait_check", "metade_last_cuda_error",
    "metade_plain_step_noalloc_status",
]


class MetadeError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib().metade_strerror(status).decode() if _LIB is not None else str(status)
        if status == METADE_ECUDA and _LIB is not None:
            msg += " " + _lib().metade_last_cuda_error().decode()
        super().__init__("%s: %s (status %d)" % (what, msg, status))


class metade_config(C.Structure):
    _fields_ = [
        ("n_prob", C.c_int32),
        ("prob_dim", C.POINTER(C.c_int32)),
        ("prob_obj", C.POINTER(C.c_int32)),
        ("shift", C.c_void_p),
        ("rot", C.c_void_p),
        ("n_inst", C.c_int32),
        ("inst_np", C.POINTER(C.c_int32)),
        ("inst_prob", C.POINTER(C.c_int32)),
        ("inst_group", C.POINTER(C.c_int32)),
        ("lo", C.c_float),
        ("hi", C.c_float),
        ("seed", C.c_uint64),
        ("one_shot", C.c_int32),
        ("p_best_pct", C.c_int32),
        ("n_out", C.c_int32),
        ("prec", C.c_int),
        ("path", C.c_int),
        ("tie_fp64", C.c_int32),
        ("stream", C.c_void_p),
        ("evolver", C.c_int32),
        ("tc_min_dim", C.c_int32),
        ("tc_unfused", C.c_int32),
    ]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmetade.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2502_10470_gb300._build); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        P, I32, U32 = C.c_void_p, C.c_int32, C.c_uint32
        L.metade_create.argtypes = [C.POINTER(metade_config), C.POINTER(C.c_void_p)]
        L.metade_destroy.argtypes = [P]
        L.metade_destroy.restype = None
        L.metade_layout.argtypes = [P, P, P, P]
        L.metade_offsets.argtypes = [P, P, P, P]
        L.metade_set_stream.argtypes = [P, P]
        L.metade_init.argtypes = [P, P, P, U32]
        L.metade_inner_step.argtypes = [P, P, P, P, U32, U32, I32, P, P]
        L.metade_eval.argtypes = [P, P, C.c_int64, P, I32, C.c_int, P]
        L.metade_eval_pop.argtypes = [P, P, C.c_int, P]
        L.metade_outer_init.argtypes = [P, P, P]
        L.metade_outer_step.argtypes = [P, P, P, P, P, P, U32, I32]
        L.metade_outer_generation.argtypes = [P, P, P, P, P, P, P, P, P, U32, I32, I32]
        L.metade_draw_record.argtypes = [P, P, P, U32, U32, P]
        L.metade_sync.argtypes = [P]
        L.metade_plan_info.argtypes = [P, C.c_char_p, C.c_size_t]
        L.metade_launch_count.argtypes = [P]
        L.metade_launch_count.restype = C.c_int64
        L.metade_plain_step_noalloc_status.argtypes = [P]
        L.metade_plain_step_noalloc.argtypes = [P, P, P, P, P, I32, I32, I32, C.c_float, C.c_float, C.c_uint64,
                                                U32, U32, U32, I32, P]
        L.metade_profile.argtypes = [P, I32]
        L.metade_autotune.argtypes = [P, P, P, P, I32]
        L.metade_profile_read.argtypes = [P, P, P]
        L.metade_wait_check.argtypes = [I32, U32, P, P]
        L.metade_strerror.argtypes = [C.c_int]
        L.metade_strerror.restype = C.c_char_p
        L.metade_last_cuda_error.argtypes = []
        L.metade_last_cuda_error.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("metade_destroy", "metade_launch_count", "metade_strerror", "metade_last_cuda_error"):
                getattr(L, name).restype = C.c_int
        _LIB = L
    return _LIB


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(status: int, what: str):
    if status != METADE_OK:
        raise MetadeError(status, what)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


# ---------------------------------------------------------------- C names
def metade_create(prob_dim, prob_obj, shift, rot, inst_np, inst_prob, inst_group=None, *, lo=-100.0, hi=100.0,
                  seed=0, one_shot=0, p_best_pct=10, n_out=0, prec=METADE_FP32, path=METADE_PATH_BATCHED,
                  tie_fp64=0, stream=None, evolver=EVOLVER_DE, tc_min_dim=0, tc_unfused=0) -> int:
    """shift/rot: device float32 tensors (concatenated o_p and row-major R_p)."""
    pd, po, nps, ip = _i32(prob_dim), _i32(prob_obj), _i32(inst_np), _i32(inst_prob)
    ig = _i32(inst_group) if inst_group is not None else None
    cfg = metade_config()
    cfg.n_prob = len(pd)
    cfg.prob_dim = _i32p(pd)
    cfg.prob_obj = _i32p(po)
    cfg.shift = _ptr(shift)
    cfg.rot = _ptr(rot)
    cfg.n_inst = len(nps)
    cfg.inst_np = _i32p(nps)
    cfg.inst_prob = _i32p(ip)
    cfg.inst_group = _i32p(ig) if ig is not None else None
    cfg.lo, cfg.hi = lo, hi
    cfg.seed = seed
    cfg.one_shot = int(one_shot)
    cfg.p_best_pct = p_best_pct
    cfg.n_out = n_out
    cfg.prec = prec
    cfg.path = path
    cfg.tie_fp64 = int(tie_fp64)
    cfg.stream = stream
    cfg.evolver = int(evolver)
    cfg.tc_min_dim = int(tc_min_dim)
    cfg.tc_unfused = int(tc_unfused)
    out = C.c_void_p()
    _check(_lib().metade_create(C.byref(cfg), C.byref(out)), "metade_create")
    return out.value


def metade_destroy(ctx: int) -> None:
    _lib().metade_destroy(ctx)


def metade_layout(ctx: int):
    pf, ni, ng = C.c_int64(), C.c_int64(), C.c_int32()
    _check(_lib().metade_layout(ctx, C.byref(pf), C.byref(ni), C.byref(ng)), "metade_layout")
    return pf.value, ni.value, ng.value


def metade_offsets(ctx: int, n_inst: int):
    po = np.zeros(n_inst, dtype=np.int64)
    fo = np.zeros(n_inst, dtype=np.int64)
    dp = np.zeros(n_inst, dtype=np.int32)
    _check(_lib().metade_offsets(ctx, po.ctypes.data, fo.ctypes.data, dp.ctypes.data), "metade_offsets")
    return po, fo, dp


def metade_set_stream(ctx: int, stream) -> None:
    _check(_lib().metade_set_stream(ctx, stream), "metade_set_stream")


def metade_init(ctx: int, pop, fit, epoch: int = 0) -> None:
    _check(_lib().metade_init(ctx, _ptr(pop), _ptr(fit), epoch), "metade_init")


def metade_inner_step(ctx: int, pop, fit, theta, epoch: int, gen0: int, n_gens: int, best_f=None, best_i=None) -> None:
    _check(_lib().metade_inner_step(ctx, _ptr(pop), _ptr(fit), _ptr(theta), epoch, gen0, n_gens, _ptr(best_f),
                                    _ptr(best_i)), "metade_inner_step")


def metade_eval(ctx: int, x, n: int, inst, ldx: int, prec: int, f_out) -> None:
    """Caller-given points: x [n][ldx] float32, inst [n] int32 executor ids."""
    _check(_lib().metade_eval(ctx, _ptr(x), int(n), _ptr(inst), int(ldx), prec, _ptr(f_out)), "metade_eval")


def metade_eval_pop(ctx: int, pop, prec: int, f_out) -> None:
    """Every population row, in the fitness layout."""
    _check(_lib().metade_eval_pop(ctx, _ptr(pop), prec, _ptr(f_out)), "metade_eval_pop")


def metade_outer_init(ctx: int, opop, ofit) -> None:
    _check(_lib().metade_outer_init(ctx, _ptr(opop), _ptr(ofit)), "metade_outer_init")


def metade_outer_step(ctx: int, opop, ofit, trial, theta, meta_fit, outer_gen: int, phase: int) -> None:
    _check(_lib().metade_outer_step(ctx, _ptr(opop), _ptr(ofit), _ptr(trial), _ptr(theta), _ptr(meta_fit),
                                    outer_gen, phase), "metade_outer_step")


def metade_outer_generation(ctx: int, opop, ofit, trial, theta, pop, fit, best_f, best_i, outer_gen: int,
                            n_inner_gens: int, use_graph: bool = True) -> None:
    _check(_lib().metade_outer_generation(ctx, _ptr(opop), _ptr(ofit), _ptr(trial), _ptr(theta), _ptr(pop),
                                          _ptr(fit), _ptr(best_f), _ptr(best_i), outer_gen, n_inner_gens,
                                          int(use_graph)), "metade_outer_generation")


def metade_draw_record(ctx: int, fit, theta, epoch: int, gen: int, rec) -> None:
    _check(_lib().metade_draw_record(ctx, _ptr(fit), _ptr(theta), epoch, gen, _ptr(rec)), "metade_draw_record")


def metade_sync(ctx: int) -> int:
    """Returns the sticky device status (0 = ok) after waiting for the stream."""
    return _lib().metade_sync(ctx)


def metade_plan_info(ctx: int) -> str:
    buf = C.create_string_buffer(1 << 16)
    _check(_lib().metade_plan_info(ctx, buf, len(buf)), "metade_plan_info")
    return buf.value.decode()


def metade_launch_count(ctx: int) -> int:
    return _lib().metade_launch_count(ctx)


def metade_plain_step_noalloc(pop, fit, theta, shift, rot, np_: int, dim: int, obj: int, lo: float, hi: float,
                              seed: int, stream_id: int, epoch: int, gen: int, p_best_pct: int = 10,
                              stream=None) -> int:
    """One plain generation of one executor with no allocation; returns the status."""
    return _lib().metade_plain_step_noalloc(_ptr(pop), _ptr(fit), _ptr(theta), _ptr(shift), _ptr(rot), np_, dim,
                                            obj, lo, hi, seed, stream_id, epoch, gen, p_best_pct, stream)


def metade_plain_step_noalloc_status() -> int:
    """0 if the last allocation-free generation on this device ran, 1 if its theta skipped it (waits)."""
    v = C.c_int32(0)
    _check(_lib().metade_plain_step_noalloc_status(C.byref(v)), "metade_plain_step_noalloc_status")
    return int(v.value)


def metade_autotune(ctx: int, pop, fit, theta, n_gens: int = 3) -> None:
    _check(_lib().metade_autotune(ctx, _ptr(pop), _ptr(fit), _ptr(theta), n_gens), "metade_autotune")


PROFILE_KINDS = ["fused_small", "fused_general", "tc_gemm", "tc_generation", "fused_tile_stream", "fused_tile",
                 "mlp_generations", "tc_prologue", "tc_trial", "tc_select", "tc_ties", "tc_sel", "near_ties"]


def metade_profile(ctx: int, enable) -> None:
    """enable: 0 off, 1 (or True) events around every launch, n > 1 around
    the tensor-core kernels of one generation in n."""
    _check(_lib().metade_profile(ctx, int(enable)), "metade_profile")


def metade_profile_read(ctx: int):
    """{kind: (milliseconds, launches)} since the last read."""
    ms = np.zeros(len(PROFILE_KINDS), dtype=np.float64)
    n = np.zeros(len(PROFILE_KINDS), dtype=np.int64)
    _check(_lib().metade_profile_read(ctx, ms.ctypes.data, n.ctypes.data), "metade_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROFILE_KINDS)}


def metade_wait_check(arrive: bool, rounds: int = 0):
    """The tensor-core pipeline's bounded mbarrier wait on its own: returns
    (status, completed, seconds); status METADE_ETIMEOUT when the wait gave up."""
    done = C.c_int32(0)
    sec = C.c_double(0.0)
    st = _lib().metade_wait_check(int(arrive), int(rounds), C.byref(done), C.byref(sec))
    return int(st), int(done.value), float(sec.value)


def metade_strerror(status: int) -> str:
    return _lib().metade_strerror(status).decode()


# ------------------------------------------------------------ convenience
def trial_shape(evolver: int, n_groups: int, n_out: int):
    """Shape of the evolver's `trial` buffer (float32): DE [n][6], PSO [n][12]
    (position, velocity), CSO [n][13] (position, velocity, flag) with
    n = n_groups * n_out; NES [n_groups][12 n_out + 96] (samples, then the
    search distribution as doubles)."""
    if evolver == EVOLVER_NES:
        return (n_groups, 12 * n_out + 96)
    return (n_groups * n_out, {EVOLVER_PSO: 12, EVOLVER_CSO: 13}.get(evolver, 6))


class Batch:
    """Device tensors and a context for one batch of executors.

    problems: sequence of (dim, obj, shift[dim] float32, rot[dim, dim] float32)
    """

    def __init__(self, problems: Sequence, inst_np, inst_prob, inst_group=None, *, seed=0, one_shot=0,
                 p_best_pct=10, n_out=0, path=METADE_PATH_BATCHED, prec=METADE_FP32, lo=-100.0, hi=100.0,
                 tie_fp64=0, device="cuda", stream=None, evolver=EVOLVER_DE, tc_min_dim=0, tc_unfused=0):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        dims = [int(p[0]) for p in problems]
        objs = [int(p[1]) for p in problems]
        shift = np.concatenate([np.asarray(p[2], dtype=np.float32).reshape(-1) for p in problems])
        rot = np.concatenate([np.asarray(p[3], dtype=np.float32).reshape(-1) for p in problems])
        self.shift_d = torch.from_numpy(shift).to(self.device)
        self.rot_d = torch.from_numpy(rot).to(self.device)
        self.inst_np = _i32(inst_np)
        self.inst_prob = _i32(inst_prob)
        self.n_inst = len(self.inst_np)
        self.n_out = n_out
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = stream
        self.ctx = metade_create(dims, objs, self.shift_d, self.rot_d, self.inst_np, self.inst_prob, inst_group,
                                 lo=lo, hi=hi, seed=seed, one_shot=one_shot, p_best_pct=p_best_pct, n_out=n_out,
                                 prec=prec, path=path, tie_fp64=tie_fp64, stream=stream, evolver=evolver,
                                 tc_min_dim=tc_min_dim, tc_unfused=tc_unfused)
        self.dims = np.array([dims[p] for p in self.inst_prob], dtype=np.int32)
        self.pop_floats, self.n_indiv, self.n_groups = metade_layout(self.ctx)
        self.pop_off, self.fit_off, self.dpad = metade_offsets(self.ctx, self.n_inst)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.pop = torch.zeros(max(self.pop_floats, 1), **f32)
        self.fit = torch.zeros(max(self.n_indiv, 1), **f32)
        self.best_f = torch.zeros(max(self.n_inst, 1), **f32)
        self.best_i = torch.zeros(max(self.n_inst, 1), dtype=torch.int32, device=self.device)
        self.theta = torch.zeros((max(self.n_inst, 1), 6), **f32)
        if n_out:
            self.opop = torch.zeros((self.n_groups * n_out, 6), **f32)
            self.ofit = torch.zeros(self.n_groups * n_out, **f32)
            # DE: the trial vectors; PSO: position then velocity of every particle
            self.trial = torch.zeros(trial_shape(evolver, self.n_groups, n_out), **f32)

    def close(self):
        if self.ctx:
            metade_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # marshalling between the padded device layout and per-executor arrays
    def set_population(self, pops, fits=None):
        buf = np.zeros(max(self.pop_floats, 1), dtype=np.float32)
        for k, p in enumerate(pops):
            p = np.asarray(p, dtype=np.float32)
            n, d = p.shape
            view = buf[self.pop_off[k]:self.pop_off[k] + n * self.dpad[k]].reshape(n, self.dpad[k])
            view[:, :d] = p
        self.pop.copy_(self.torch.from_numpy(buf))
        if fits is not None:
            f = np.concatenate([np.asarray(x, dtype=np.float32) for x in fits]) if self.n_inst else np.zeros(1)
            self.fit[:len(f)].copy_(self.torch.from_numpy(f.astype(np.float32)))

    def get_population(self):
        buf = self.pop.cpu().numpy()
        fit = self.fit.cpu().numpy()
        pops, fits = [], []
        for k in range(self.n_inst):
            n, dp, d = int(self.inst_np[k]), int(self.dpad[k]), int(self.dims[k])
            pops.append(buf[self.pop_off[k]:self.pop_off[k] + n * dp].reshape(n, dp)[:, :d].copy())
            fits.append(fit[self.fit_off[k]:self.fit_off[k] + n].copy())
        return pops, fits

    def set_theta(self, theta):
        self.theta.copy_(self.torch.from_numpy(np.asarray(theta, dtype=np.float32).reshape(-1, 6)))

    def sync(self):
        s = metade_sync(self.ctx)
        if s != METADE_OK:
            raise MetadeError(s, "device status")

    def run_metade(self, outer_gens: int, inner_gens: int, power_up: bool = False, use_graph: bool = True):
        """Alg. 3: evolver initialisation, then `outer_gens` evolver generations
        (trials and decoding, executor runs, selection), each one call of
        metade_outer_generation.  With power_up the last generation gives the
        executors 5x the inner generations (Sec. III-D).  Returns the evolver
        population [n_groups, n_out, 6] and fitness [n_groups, n_out]."""
        if not self.n_out:
            raise MetadeError(METADE_ESTATE, "run_metade needs an evolver (n_out > 0)")
        metade_outer_init(self.ctx, self.opop, self.ofit)
        for g in range(outer_gens):
            n = 5 * inner_gens if (power_up and g == outer_gens - 1) else inner_gens
            metade_outer_generation(self.ctx, self.opop, self.ofit, self.trial, self.theta, self.pop, self.fit,
                                    self.best_f, self.best_i, g, n, use_graph)
        self.sync()
        return (self.opop.cpu().numpy().reshape(self.n_groups, self.n_out, 6),
                self.ofit.cpu().numpy().reshape(self.n_groups, self.n_out))
