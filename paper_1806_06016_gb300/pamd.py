"""ctypes binding of libpamd (include/pamd.h), one Python function per C entry point.

Argument marshalling only: every step of the method runs in the CUDA
library.  If the library is missing the functions raise ``RuntimeError``;
there is no CPU fallback.  Device memory and the CUDA stream can come from
PyTorch (``torch_options``); PyTorch is not otherwise used.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpamd.so")

PAMD_OK = 0
PAMD_EINVAL, PAMD_ENOMEM, PAMD_ECUDA, PAMD_ETIMEOUT = -1, -2, -3, -4
PAMD_ENONFINITE, PAMD_ESTATE, PAMD_EUNSUPPORTED = -5, -6, -7
PAMD_PREC_MIXED, PAMD_PREC_FP64 = 0, 1
PAMD_RESAMPLE_MULTINOMIAL, PAMD_RESAMPLE_SYSTEMATIC = 0, 1
PAMD_RESAMPLE_NEAREST, PAMD_RESAMPLE_POISSON = 2, 3
PAMD_EPOPSIZE = -8
PAMD_PAIRS_AUTO, PAMD_PAIRS_SCALAR, PAMD_PAIRS_PACKED = 0, 1, 2
PAMD_MAX_ATOMS = 256

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class PamdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pamd error {code}: {msg}")
        self.code = code


class PamdTopology(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int32),
        ("mass", C.c_void_p), ("charge", C.c_void_p), ("sigma", C.c_void_p),
        ("epsilon", C.c_void_p), ("x0", C.c_void_p),
        ("n_bonds", C.c_int32), ("bond", C.c_void_p), ("bond_r0", C.c_void_p), ("bond_k", C.c_void_p),
        ("n_angles", C.c_int32), ("angle", C.c_void_p), ("angle_t0", C.c_void_p), ("angle_k", C.c_void_p),
        ("n_dihedrals", C.c_int32), ("dihedral", C.c_void_p), ("dih_n", C.c_void_p),
        ("dih_k", C.c_void_p), ("dih_phase", C.c_void_p),
        ("n_excl", C.c_int32), ("excl", C.c_void_p),
        ("n_pair14", C.c_int32), ("pair14", C.c_void_p),
        ("scale14_lj", C.c_double), ("scale14_coul", C.c_double),
    ]


class PamdOptions(C.Structure):
    _fields_ = [
        ("gamma_per_ps", C.c_double),
        ("precision", C.c_int32),
        ("lanes_per_replica", C.c_int32),
        ("warps_per_block", C.c_int32),
        ("mol_id", C.c_int32),
        ("autotune", C.c_int32),
        ("replicas_per_lane", C.c_int32),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_user", C.c_void_p),
        ("stream", C.c_void_p),
        ("resample_rule", C.c_int32),
        ("pair_arith", C.c_int32),
    ]


class PamdTune(C.Structure):
    _fields_ = [("lanes_per_replica", C.c_int32), ("atoms_per_lane", C.c_int32),
                ("warps_per_block", C.c_int32), ("replicas_per_lane", C.c_int32),
                ("from_cache", C.c_int32), ("ms", C.c_double), ("pair_arith", C.c_int32),
                ("pad_", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class PamdObs(C.Structure):
    _fields_ = [
        ("T", C.c_double), ("lnQ", C.c_double), ("sum_lnQ", C.c_double),
        ("e_pot", C.c_double), ("e_pot_se", C.c_double), ("e_kin", C.c_double),
        ("e_kin_se", C.c_double), ("t_meas", C.c_double),
        ("rg", C.c_double), ("rg_se", C.c_double), ("rg2", C.c_double), ("rg2_se", C.c_double),
        ("n_families", C.c_int64), ("max_copies", C.c_int32), ("pad_", C.c_int32),
        ("R_live", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


EXPORTS = [
    "pamd_options_default", "pamd_init", "pamd_init_batch", "pamd_batch_size", "pamd_batch_sub",
    "pamd_reset", "pamd_propagate", "pamd_resample", "pamd_observables",
    "pamd_anneal", "pamd_get_state", "pamd_set_state", "pamd_forces", "pamd_get_counters",
    "pamd_set_counters", "pamd_autotune", "pamd_get_shape", "pamd_population_size", "pamd_fp32_peak", "pamd_fp32_peak_threads", "pamd_resample_counts_noalloc", "pamd_info", "pamd_launch_count", "pamd_sync", "pamd_destroy",
    "pamd_last_error",
    # learned surrogate (include/pamd_mlp.h), wrapped in surrogate.py
    "pamd_gemm_bf16", "pamd_gemm_bf16_time", "pamd_mlp_create", "pamd_mlp_info", "pamd_mlp_set_params",
    "pamd_mlp_get_params", "pamd_mlp_fit_normalization", "pamd_mlp_energy_forces",
    "pamd_mlp_loss_grads", "pamd_mlp_get_grads", "pamd_mlp_adam_step", "pamd_set_force_model",
    "pamd_mlp_sync", "pamd_mlp_launch_count", "pamd_mlp_destroy", "pamd_mlp_save", "pamd_mlp_load",
    "pamd_checkpoint", "pamd_restore",
    # multiple-histogram reweighting (include/pamd_wham.h)
    "pamd_record_energies", "pamd_wham",
    # temperature schedules from the overlap condition (include/pamd_adaptive.h)
    "pamd_overlap_temperature", "pamd_next_temperature", "pamd_anneal_adaptive",
]

class PamdWhamArgs(C.Structure):
    _fields_ = [("E", C.c_void_p), ("n_temps", C.c_int32), ("R", C.c_int64), ("T", C.c_void_p),
                ("n_bins", C.c_int32), ("e_min", C.c_double), ("e_max", C.c_double),
                ("lnZ_init", C.c_void_p), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("n_eval", C.c_int32), ("T_eval", C.c_void_p), ("stream", C.c_void_p)]


class PamdWhamResult(C.Structure):
    _fields_ = [("lnZ", C.c_void_p), ("ln_g", C.c_void_p), ("hist", C.c_void_p),
                ("lnZ_eval", C.c_void_p), ("e_mean_eval", C.c_void_p), ("e_var_eval", C.c_void_p),
                ("e_min", C.c_double), ("bin_width", C.c_double), ("iterations", C.c_int32),
                ("max_delta", C.c_double)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libpamd.so (built by ``paper_1806_06016_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libpamd.so not built ({p}); run paper_1806_06016_gb300.build.build()")
        lib = C.CDLL(p)
        P, I32, I64, U32, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        sig = {
            "pamd_options_default": (None, [C.POINTER(PamdOptions)]),
            "pamd_init": (C.c_int, [C.POINTER(P), C.POINTER(PamdTopology), I64, D, U64,
                                    C.POINTER(PamdOptions)]),
            "pamd_init_batch": (C.c_int, [C.POINTER(P), I32, C.POINTER(PamdTopology), P, P, U64,
                                          C.POINTER(PamdOptions)]),
            "pamd_batch_size": (I32, [P]),
            "pamd_batch_sub": (P, [P, I32]),
            "pamd_reset": (C.c_int, [P, D, U64]),
            "pamd_propagate": (C.c_int, [P, I32, D, D]),
            "pamd_resample": (C.c_int, [P, D, D, P, P]),
            "pamd_observables": (C.c_int, [P, D, C.POINTER(PamdObs)]),
            "pamd_anneal": (C.c_int, [P, I32, P, I32, D, I32, C.POINTER(PamdObs)]),
            "pamd_get_state": (C.c_int, [P, P, P, P, P]),
            "pamd_set_state": (C.c_int, [P, P, P, P, P]),
            "pamd_forces": (C.c_int, [P, P, P]),
            "pamd_get_counters": (C.c_int, [P, C.POINTER(U32), C.POINTER(U32), C.POINTER(D)]),
            "pamd_set_counters": (C.c_int, [P, U32, U32, D]),
            "pamd_autotune": (C.c_int, [P, I32, C.POINTER(PamdTune)]),
            "pamd_get_shape": (C.c_int, [P, C.POINTER(PamdTune)]),
            "pamd_population_size": (C.c_int, [P, C.POINTER(I64), C.POINTER(I64)]),
            "pamd_fp32_peak": (C.c_int, [I32, I32, I32, P, P, C.POINTER(D), C.POINTER(D)]),
            "pamd_fp32_peak_threads": (I32, []),
            "pamd_resample_counts_noalloc": (C.c_int, [P, I64, D, D, U64, U32, I32, P, P, P, P]),
            "pamd_info": (C.c_int, [P, C.POINTER(I64), C.POINTER(I32), C.POINTER(I32),
                                    C.POINTER(I32), C.POINTER(I32)]),
            "pamd_launch_count": (I64, [P]),
            "pamd_sync": (C.c_int, [P]),
            "pamd_destroy": (None, [P]),
            "pamd_last_error": (C.c_char_p, []),
            # learned surrogate (pamd_mlp.h)
            "pamd_gemm_bf16": (C.c_int, [P, P, P, I32, I32, I32, I32, I32, I32, P]),
            "pamd_gemm_bf16_time": (C.c_int, [P, P, P, I32, I32, I32, I32, I32, I32, I32, P,
                                              C.POINTER(C.c_float)]),
            "pamd_mlp_create": (C.c_int, [C.POINTER(P), I32, I32, U64, P]),
            "pamd_mlp_info": (C.c_int, [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]),
            "pamd_mlp_set_params": (C.c_int, [P, P]),
            "pamd_mlp_get_params": (C.c_int, [P, P]),
            "pamd_mlp_fit_normalization": (C.c_int, [P, P, P, I64]),
            "pamd_mlp_energy_forces": (C.c_int, [P, P, I64, P, P]),
            "pamd_mlp_loss_grads": (C.c_int, [P, P, P, P, P, I64, D, C.POINTER(D)]),
            "pamd_mlp_get_grads": (C.c_int, [P, P]),
            "pamd_mlp_adam_step": (C.c_int, [P, D, D, D, D]),
            "pamd_set_force_model": (C.c_int, [P, P]),
            "pamd_mlp_sync": (C.c_int, [P]),
            "pamd_mlp_launch_count": (I64, [P]),
            "pamd_mlp_destroy": (None, [P]),
            "pamd_mlp_save": (C.c_int, [P, C.c_char_p]),
            "pamd_mlp_load": (C.c_int, [C.POINTER(P), C.c_char_p, P]),
            "pamd_checkpoint": (C.c_int, [P, C.c_char_p]),
            "pamd_restore": (C.c_int, [P, C.c_char_p]),
            "pamd_record_energies": (C.c_int, [P, P, I32]),
            "pamd_wham": (C.c_int, [C.POINTER(PamdWhamArgs), C.POINTER(PamdWhamResult)]),
            "pamd_overlap_temperature": (C.c_int, [P, I64, D, D, D, C.POINTER(D), C.POINTER(D), P]),
            "pamd_next_temperature": (C.c_int, [P, D, D, D, C.POINTER(D), C.POINTER(D)]),
            "pamd_anneal_adaptive": (C.c_int, [P, D, D, D, I32, D, I32, I32, C.POINTER(PamdObs), P,
                                               C.POINTER(I32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _check(rc):
    if rc != PAMD_OK:
        msg = load().pamd_last_error().decode(errors="replace")
        raise PamdError(rc, msg)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _TopologyArgs:
    """Keeps the numpy arrays behind a PamdTopology alive for the duration of a call."""

    def __init__(self, top):
        a = top.arrays()
        self._a = a
        self.s = PamdTopology(
            top.n_atoms, _ptr(a["mass"]), _ptr(a["charge"]), _ptr(a["sigma"]), _ptr(a["epsilon"]),
            _ptr(a["x0"]),
            len(a["bond"]), _ptr(a["bond"]), _ptr(a["bond_r0"]), _ptr(a["bond_k"]),
            len(a["angle"]), _ptr(a["angle"]), _ptr(a["angle_t0"]), _ptr(a["angle_k"]),
            len(a["dihedral"]), _ptr(a["dihedral"]), _ptr(a["dih_n"]), _ptr(a["dih_k"]),
            _ptr(a["dih_phase"]),
            len(a["excl"]), _ptr(a["excl"]), len(a["pair14"]), _ptr(a["pair14"]),
            float(top.scale14_lj), float(top.scale14_coul),
        )


def pamd_options_default() -> PamdOptions:
    o = PamdOptions()
    load().pamd_options_default(C.byref(o))
    return o


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on the current device."""

    def __init__(self):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream()
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, _user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _free(self, ptr, _user):
        self.torch.cuda.caching_allocator_delete(ptr)


_keepalive: dict[int, object] = {}


def torch_options(gamma_per_ps: float = 1.0, **kw) -> PamdOptions:
    """Options whose device memory and stream come from PyTorch: the caching
    allocator and torch's current stream.  If that stream is the legacy
    default stream (handle 0) the library uses a stream of its own, which is
    not ordered with torch's work; make a side stream current first to share
    one stream with torch."""
    o = pamd_options_default()
    o.gamma_per_ps = gamma_per_ps
    for k, v in kw.items():
        setattr(o, k, v)
    al = _TorchAllocator()
    o.dev_alloc = al.alloc
    o.dev_free = al.free
    o.stream = al.stream.cuda_stream
    o._allocator = al  # keeps the callbacks alive with the options object
    return o


def pamd_init(top, R: int, T0: float, seed: int, options: PamdOptions | None = None):
    lib = load()
    ctx = C.c_void_p()
    ta = _TopologyArgs(top)
    opt = options if options is not None else pamd_options_default()
    _check(lib.pamd_init(C.byref(ctx), C.byref(ta.s), int(R), float(T0), int(seed), C.byref(opt)))
    _keepalive[ctx.value] = getattr(opt, "_allocator", None)
    return ctx


def pamd_init_batch(tops, R, T0, seed: int, options: PamdOptions | None = None):
    """Batch context over several molecules (one persistent launch per propagate)."""
    lib = load()
    n = len(tops)
    args = [_TopologyArgs(t) for t in tops]
    arr = (PamdTopology * n)(*[a.s for a in args])
    Rv = np.ascontiguousarray(R, dtype=np.int64)
    Tv = np.ascontiguousarray(T0, dtype=np.float64)
    ctx = C.c_void_p()
    opt = options if options is not None else pamd_options_default()
    _check(lib.pamd_init_batch(C.byref(ctx), n, arr, _ptr(Rv), _ptr(Tv), int(seed), C.byref(opt)))
    _keepalive[ctx.value] = getattr(opt, "_allocator", None)
    return ctx


def pamd_batch_size(ctx) -> int:
    return int(load().pamd_batch_size(ctx))


def pamd_batch_sub(ctx, m: int):
    """Context of molecule m of a batch (owned by the batch)."""
    h = load().pamd_batch_sub(ctx, int(m))
    if not h:
        raise PamdError(PAMD_EINVAL, pamd_last_error())
    return C.c_void_p(h)


def pamd_reset(ctx, T0: float, seed: int) -> None:
    _check(load().pamd_reset(ctx, float(T0), int(seed)))


def pamd_propagate(ctx, theta: int, dt_ps: float, T: float) -> None:
    _check(load().pamd_propagate(ctx, int(theta), float(dt_ps), float(T)))


def pamd_resample(ctx, T_prev: float, T_next: float, want_copies: bool = True):
    """Returns (copies[R] int32 or None, lnQ); for a batch context lnQ is a
    list over molecules and copies spans all molecules in order."""
    R = pamd_info(ctx)["R"]
    nb = pamd_batch_size(ctx)
    cnt = np.zeros(R, np.int32) if want_copies else None
    lnq = np.zeros(max(nb, 1))
    _check(load().pamd_resample(ctx, float(T_prev), float(T_next), _ptr(cnt), _ptr(lnq)))
    return cnt, (list(lnq) if nb > 0 else float(lnq[0]))


def pamd_observables(ctx, T: float):
    """dict, or a list of dicts (one per molecule) for a batch context."""
    nb = pamd_batch_size(ctx)
    out = (PamdObs * max(nb, 1))()
    _check(load().pamd_observables(ctx, float(T), out))
    return [o.as_dict() for o in out] if nb > 0 else out[0].as_dict()


def pamd_anneal(ctx, temps, theta: int, dt_ps: float, resample: bool = True):
    """Per-temperature observables: a list of dicts, or for a batch context a
    list (per temperature) of lists (per molecule)."""
    t = np.ascontiguousarray(temps, dtype=np.float64)
    K = len(t) - 1
    nb = pamd_batch_size(ctx)
    M = max(nb, 1)
    out = (PamdObs * ((K + 1) * M))()
    _check(load().pamd_anneal(ctx, K, _ptr(t), int(theta), float(dt_ps), int(bool(resample)), out))
    if nb > 0:
        return [[out[i * M + m].as_dict() for m in range(M)] for i in range(K + 1)]
    return [o.as_dict() for o in out]


def pamd_info(ctx) -> dict:
    R, n, L, B, rpb = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().pamd_info(ctx, C.byref(R), C.byref(n), C.byref(L), C.byref(B), C.byref(rpb)))
    return {"R": R.value, "n_atoms": n.value, "lanes_per_replica": L.value,
            "atoms_per_lane": B.value, "replicas_per_block": rpb.value}


def pamd_get_state(ctx, positions=True, velocities=True, energies=True, families=True):
    """(x[R,N,3], v[R,N,3], E[R], fam[R]); parts not asked for are None."""
    info = pamd_info(ctx)
    R, N = info["R"], info["n_atoms"]
    x = np.zeros((R, N, 3)) if positions else None
    v = np.zeros((R, N, 3)) if velocities else None
    E = np.zeros(R) if energies else None
    fam = np.zeros(R, np.int32) if families else None
    _check(load().pamd_get_state(ctx, _ptr(x), _ptr(v), _ptr(E), _ptr(fam)))
    return x, v, E, fam


def pamd_set_state(ctx, x, v, E=None, fam=None) -> None:
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    E = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
    fam = None if fam is None else np.ascontiguousarray(fam, dtype=np.int32)
    info = pamd_info(ctx)
    shape = (info["R"], info["n_atoms"], 3)
    if x.shape != shape or v.shape != shape:
        raise ValueError(f"x and v must have shape {shape}")
    _check(load().pamd_set_state(ctx, _ptr(x), _ptr(v), _ptr(E), _ptr(fam)))


def pamd_forces(ctx):
    """(F[R,N,3], E[R]) of the current population."""
    info = pamd_info(ctx)
    f = np.zeros((info["R"], info["n_atoms"], 3)); E = np.zeros(info["R"])
    _check(load().pamd_forces(ctx, _ptr(f), _ptr(E)))
    return f, E


def pamd_get_counters(ctx):
    s, r, q = C.c_uint32(), C.c_uint32(), C.c_double()
    _check(load().pamd_get_counters(ctx, C.byref(s), C.byref(r), C.byref(q)))
    return s.value, r.value, q.value


def pamd_set_counters(ctx, step: int, resample_index: int, sum_lnQ: float) -> None:
    _check(load().pamd_set_counters(ctx, int(step), int(resample_index), float(sum_lnQ)))


def pamd_fp32_peak(packed: bool, iters: int = 20000, reps: int = 100, stream: int = 0) -> dict:
    """FP32 FMA throughput of the current device (include/pamd_bench.h):
    {"tflops", "ms"} of `reps` timed launches, scalar or packed FP32x2."""
    import torch
    n = load().pamd_fp32_peak_threads()
    if n <= 0:
        raise PamdError(PAMD_ECUDA, "no CUDA device")
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    tf, ms = C.c_double(), C.c_double()
    _check(load().pamd_fp32_peak(1 if packed else 0, int(iters), int(reps), C.c_void_p(stream or None),
                                 C.c_void_p(out.data_ptr()), C.byref(tf), C.byref(ms)))
    return {"tflops": tf.value, "ms": ms.value}


def pamd_population_size(ctx) -> tuple:
    """(live population size, capacity)."""
    live, cap = C.c_int64(), C.c_int64()
    _check(load().pamd_population_size(ctx, C.byref(live), C.byref(cap)))
    return live.value, cap.value


def pamd_get_shape(ctx) -> dict:
    t = PamdTune()
    _check(load().pamd_get_shape(ctx, C.byref(t)))
    return t.as_dict()


def pamd_autotune(ctx, theta_probe: int = 20) -> dict:
    t = PamdTune()
    _check(load().pamd_autotune(ctx, int(theta_probe), C.byref(t)))
    return t.as_dict()


def pamd_resample_counts_noalloc(E_dev: int, R: int, T_prev: float, T_next: float, seed: int,
                                 resample_index: int, counts_dev: int, lnQ_dev: int = 0,
                                 mol_id: int = 0, stream: int = 0, status_dev: int = 0) -> None:
    """Copy counts and ln Q from device energies into device outputs without
    allocating (pointers are device addresses, e.g. ``tensor.data_ptr()``);
    status_dev (int32) receives 0 or PAMD_ENONFINITE."""
    _check(load().pamd_resample_counts_noalloc(
        C.c_void_p(E_dev), int(R), float(T_prev), float(T_next), int(seed), int(resample_index),
        int(mol_id), C.c_void_p(counts_dev), C.c_void_p(lnQ_dev or None),
        C.c_void_p(status_dev or None), C.c_void_p(stream or None)))


def pamd_record_energies(ctx, E_dev: int, rows: int) -> None:
    """Record the energies pamd_anneal measures into device memory [rows][R]
    float64 at address E_dev (e.g. ``tensor.data_ptr()``); rows = 0 stops."""
    _check(load().pamd_record_energies(ctx, C.c_void_p(E_dev or None), int(rows)))


def pamd_wham(E_dev: int, n_temps: int, R: int, T, n_bins: int, e_range=None, lnZ_init=None,
              max_iter: int = 100, tol: float = 1e-10, T_eval=None, stream: int = 0,
              want_hist: bool = False) -> dict:
    """Histograms and self-consistency sweeps of the device energies E_dev
    ([n_temps][R] float64, row i sampled at T[i]); results as numpy arrays."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    Te = None if T_eval is None else np.ascontiguousarray(np.atleast_1d(T_eval), dtype=np.float64)
    z0 = None if lnZ_init is None else np.ascontiguousarray(lnZ_init, dtype=np.float64)
    ne = 0 if Te is None else len(Te)
    lo, hi = (0.0, 0.0) if e_range is None else (float(e_range[0]), float(e_range[1]))
    a = PamdWhamArgs(C.c_void_p(E_dev), int(n_temps), int(R), _ptr(T), int(n_bins), lo, hi, _ptr(z0),
                     int(max_iter), float(tol), ne, _ptr(Te), C.c_void_p(stream or None))
    lnZ = np.zeros(n_temps)
    ln_g = np.zeros(n_bins)
    hist = np.zeros((n_temps, n_bins), np.uint32) if want_hist else None
    ev = np.zeros((3, max(ne, 1)))
    r = PamdWhamResult(_ptr(lnZ), _ptr(ln_g), _ptr(hist), _ptr(ev[0]) if ne else None,
                       _ptr(ev[1]) if ne else None, _ptr(ev[2]) if ne else None)
    _check(load().pamd_wham(C.byref(a), C.byref(r)))
    out = {"lnZ": lnZ, "ln_g": ln_g, "e_min": r.e_min, "bin_width": r.bin_width,
           "iterations": r.iterations, "max_delta": r.max_delta}
    if want_hist:
        out["hist"] = hist
    if ne:
        out["lnZ_eval"], out["e_mean_eval"], out["e_var_eval"] = ev[0].copy(), ev[1].copy(), ev[2].copy()
    return out


def pamd_overlap_temperature(E_dev: int, R: int, T_prev: float, T_final: float, alpha_target: float,
                             stream: int = 0):
    """(T_next, overlap at T_next) from R device energies (address E_dev)."""
    t, a = C.c_double(), C.c_double()
    _check(load().pamd_overlap_temperature(C.c_void_p(E_dev), int(R), float(T_prev), float(T_final),
                                           float(alpha_target), C.byref(t), C.byref(a),
                                           C.c_void_p(stream or None)))
    return t.value, a.value


def pamd_next_temperature(ctx, T_prev: float, T_final: float, alpha_target: float):
    """(T_next, overlap at T_next) for the context's current population."""
    t, a = C.c_double(), C.c_double()
    _check(load().pamd_next_temperature(ctx, float(T_prev), float(T_final), float(alpha_target),
                                        C.byref(t), C.byref(a)))
    return t.value, a.value


def pamd_anneal_adaptive(ctx, T0: float, T_final: float, alpha_target: float, theta: int, dt_ps: float,
                         max_steps: int, resample: bool = True):
    """(per-temperature observable dicts, temperatures) of an anneal whose
    temperatures follow the overlap condition."""
    obs = (PamdObs * (max_steps + 1))()
    temps = np.zeros(max_steps + 1)
    n = C.c_int32()
    _check(load().pamd_anneal_adaptive(ctx, float(T0), float(T_final), float(alpha_target), int(theta),
                                       float(dt_ps), int(max_steps), int(bool(resample)), obs, _ptr(temps),
                                       C.byref(n)))
    return [obs[i].as_dict() for i in range(n.value)], temps[: n.value].copy()


def pamd_checkpoint(ctx, path: str) -> None:
    _check(load().pamd_checkpoint(ctx, os.fsencode(path)))


def pamd_restore(ctx, path: str) -> None:
    _check(load().pamd_restore(ctx, os.fsencode(path)))


def pamd_launch_count(ctx) -> int:
    return int(load().pamd_launch_count(ctx))


def pamd_sync(ctx) -> None:
    _check(load().pamd_sync(ctx))


def pamd_destroy(ctx) -> None:
    if ctx is None or not ctx.value:
        return
    load().pamd_destroy(ctx)
    _keepalive.pop(ctx.value, None)


def pamd_last_error() -> str:
    return load().pamd_last_error().decode(errors="replace")


class Population:
    """A PAMD population on the GPU (R replicas of one molecule)."""

    def __init__(self, top, R: int, T0: float, seed: int, options: PamdOptions | None = None):
        self.top = top
        self.ctx = pamd_init(top, R, T0, seed, options)
        self.R = R

    def reset(self, T0, seed):
        pamd_reset(self.ctx, T0, seed)

    def propagate(self, theta, dt_ps, T):
        pamd_propagate(self.ctx, theta, dt_ps, T)

    def resample(self, T_prev, T_next, want_copies=True):
        return pamd_resample(self.ctx, T_prev, T_next, want_copies)

    def observables(self, T):
        return pamd_observables(self.ctx, T)

    def anneal(self, temps, theta, dt_ps, resample=True):
        return pamd_anneal(self.ctx, temps, theta, dt_ps, resample)

    def state(self):
        return pamd_get_state(self.ctx)

    def set_state(self, x, v, E=None, fam=None):
        pamd_set_state(self.ctx, x, v, E, fam)

    def forces(self):
        return pamd_forces(self.ctx)

    def info(self):
        return pamd_info(self.ctx)

    def checkpoint(self, path):
        pamd_checkpoint(self.ctx, path)

    def restore(self, path):
        pamd_restore(self.ctx, path)

    def autotune(self, theta_probe=20):
        return pamd_autotune(self.ctx, theta_probe)

    def close(self):
        if self.ctx is not None:
            pamd_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
