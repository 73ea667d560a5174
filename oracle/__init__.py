"""FP64 CPU oracle for population-annealing MD -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import this
package.  It loads ``liborc_pamd.so`` built from ``pamd_oracle.c`` with gcc
(contraction off, no fast-math, so x86-64 and aarch64 give the same bits) and
wraps it with numpy-friendly functions.  It shares no code with the CUDA
library.

Functions without an independent pin are listed as "parity unpinned" in the
C file's header; at present every exported function is pinned by a test in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pamd_oracle.c")
_HDR = os.path.join(_HERE, "pamd_oracle.h")
_LIB = os.path.join(_HERE, "liborc_pamd.so")
_lock = threading.Lock()
_lib = None

PURPOSE_NOISE, PURPOSE_INIT, PURPOSE_RESAMPLE = 0, 1, 2
NBINS = 64
KB = 0.008314462618


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its sources."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcTopology(C.Structure):
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


class OrcObs(C.Structure):
    _fields_ = [
        ("T", C.c_double), ("lnQ", C.c_double), ("sum_lnQ", C.c_double),
        ("e_pot", C.c_double), ("e_pot_se", C.c_double), ("e_kin", C.c_double),
        ("e_kin_se", C.c_double), ("t_meas", C.c_double),
        ("rg", C.c_double), ("rg_se", C.c_double), ("rg2", C.c_double), ("rg2_se", C.c_double),
        ("n_families", C.c_int64), ("max_copies", C.c_int32), ("pad_", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P, I32, I64, U32, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
        TP = C.POINTER(OrcTopology)
        sig = {
            "orc_philox4x32_10": (None, [P, P, P]),
            "orc_normal3": (None, [U64, U32, U32, U32, U32, P]),
            "orc_exp_det": (D, [D]),
            "orc_dihedral_angle": (D, [P, P, P, P]),
            "orc_energy_forces": (D, [TP, P, P, P]),
            "orc_init": (None, [TP, I64, D, U64, I32, P, P, P]),
            "orc_propagate": (None, [TP, I64, P, P, P, I32, D, D, D, U64, U32, I32, I32]),
            "orc_propagate_slots": (None, [TP, I64, P, P, P, P, I32, D, D, D, U64, U32, I32, I32]),
            "orc_energies": (None, [TP, I64, P, P]),
            "orc_weight_shift": (I32, [I64]),
            "orc_resample_weights": (D, [P, I64, D, D, P]),
            "orc_ancestor": (I64, [P, I64, U64]),
            "orc_resample_uniform": (U64, [U64, U32, U32, I32]),
            "orc_multinomial_counts": (None, [P, I64, U64, U32, I32, P]),
            "orc_gather": (None, [TP, I64, P, P, P, P, P, D, P, P, P, P]),
            "orc_kinetic": (D, [TP, P]),
            "orc_rgyr": (D, [TP, P]),
            "orc_observables": (None, [TP, I64, P, P, P, P, C.POINTER(OrcObs)]),
            "orc_anneal": (C.c_int, [TP, I64, I32, P, I32, D, D, U64, I32, I32, I32,
                                     C.POINTER(OrcObs), P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Topo:
    """Keeps the numpy arrays of a ``pamd_inputs.Topology`` alive behind an OrcTopology."""

    def __init__(self, top):
        self.top = top
        self.n = top.n_atoms
        self._a = top.arrays()
        a = self._a
        self.s = OrcTopology(
            top.n_atoms, _p(a["mass"]), _p(a["charge"]), _p(a["sigma"]), _p(a["epsilon"]), _p(a["x0"]),
            len(a["bond"]), _p(a["bond"]), _p(a["bond_r0"]), _p(a["bond_k"]),
            len(a["angle"]), _p(a["angle"]), _p(a["angle_t0"]), _p(a["angle_k"]),
            len(a["dihedral"]), _p(a["dihedral"]), _p(a["dih_n"]), _p(a["dih_k"]), _p(a["dih_phase"]),
            len(a["excl"]), _p(a["excl"]), len(a["pair14"]), _p(a["pair14"]),
            float(top.scale14_lj), float(top.scale14_coul),
        )

    @property
    def ref(self):
        return C.byref(self.s)


def _topo(top):
    return top if isinstance(top, Topo) else Topo(top)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


# ---------------------------------------------------------------- wrappers

def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def normal3(seed, atom, slot, step, purpose):
    z = np.zeros(3)
    _load().orc_normal3(seed, atom, slot, step, purpose, _p(z))
    return z


def exp_det(x):
    lib = _load()
    return np.array([lib.orc_exp_det(float(v)) for v in np.ravel(x)]).reshape(np.shape(x))


def dihedral_angle(xi, xj, xk, xl):
    a = [_f64(v, (3,)) for v in (xi, xj, xk, xl)]
    return _load().orc_dihedral_angle(*[_p(v) for v in a])


def energy_forces(top, x):
    """(E, F[N,3], terms[5]) for one configuration x[N,3]."""
    t = _topo(top)
    x = _f64(x, (t.n, 3))
    f = np.zeros((t.n, 3))
    terms = np.zeros(5)
    e = _load().orc_energy_forces(t.ref, _p(x), _p(f), _p(terms))
    return e, f, terms


def init(top, R, T0, seed, mol=0):
    t = _topo(top)
    x = np.zeros((R, t.n, 3))
    v = np.zeros((R, t.n, 3))
    fam = np.zeros(R, np.int32)
    _load().orc_init(t.ref, R, T0, seed, mol, _p(x), _p(v), _p(fam))
    return x, v, fam


def propagate(top, x, v, theta, dt, T, gamma, seed, step0, mol=0, n_threads=None, slots=None):
    """theta MD steps on copies of x, v; returns (x, v, E).  ``slots`` gives the
    replica slot (noise counter) of each row; default: the row index."""
    t = _topo(top)
    x = _f64(x).copy()
    v = _f64(v).copy()
    R = x.shape[0]
    E = np.zeros(R)
    nt = n_threads or os.cpu_count() or 1
    sl = None if slots is None else np.ascontiguousarray(slots, dtype=np.int64)
    _load().orc_propagate_slots(t.ref, R, _p(sl), _p(x), _p(v), _p(E), theta, dt, T, gamma, seed,
                                step0, mol, nt)
    return x, v, E


def energies(top, x):
    t = _topo(top)
    x = _f64(x)
    E = np.zeros(x.shape[0])
    _load().orc_energies(t.ref, x.shape[0], _p(x), _p(E))
    return E


def weight_shift(R):
    return _load().orc_weight_shift(R)


def resample_weights(E, T_prev, T_next):
    """(lnQ, W[u64])."""
    E = _f64(E)
    W = np.zeros(len(E), np.uint64)
    lnq = _load().orc_resample_weights(_p(E), len(E), T_prev, T_next, _p(W))
    return lnq, W


def ancestor(C_incl, t):
    c = np.ascontiguousarray(C_incl, dtype=np.uint64)
    return _load().orc_ancestor(_p(c), len(c), int(t))


def resample_uniform(seed, k, temp_index, mol=0):
    return _load().orc_resample_uniform(seed, k, temp_index, mol)


def multinomial_counts(W, seed, temp_index, mol=0):
    W = np.ascontiguousarray(W, dtype=np.uint64)
    cnt = np.zeros(len(W), np.int32)
    _load().orc_multinomial_counts(_p(W), len(W), seed, temp_index, mol, _p(cnt))
    return cnt


def gather(top, counts, x, v, fam, E, vscale):
    t = _topo(top)
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    x = _f64(x); v = _f64(v); E = _f64(E)
    fam = np.ascontiguousarray(fam, dtype=np.int32)
    x2 = np.zeros_like(x); v2 = np.zeros_like(v); f2 = np.zeros_like(fam); E2 = np.zeros_like(E)
    _load().orc_gather(t.ref, len(counts), _p(counts), _p(x), _p(v), _p(fam), _p(E), vscale,
                       _p(x2), _p(v2), _p(f2), _p(E2))
    return x2, v2, f2, E2


def kinetic(top, v):
    t = _topo(top)
    return _load().orc_kinetic(t.ref, _p(_f64(v, (t.n, 3))))


def rgyr(top, x):
    t = _topo(top)
    return _load().orc_rgyr(t.ref, _p(_f64(x, (t.n, 3))))


def observables(top, x, v, fam, E):
    t = _topo(top)
    o = OrcObs()
    x = _f64(x); v = _f64(v); E = _f64(E)
    fam = np.ascontiguousarray(fam, dtype=np.int32)
    _load().orc_observables(t.ref, x.shape[0], _p(x), _p(v), _p(fam), _p(E), C.byref(o))
    return o.as_dict()


def anneal(top, R, temps, theta, dt, gamma, seed, mol=0, resample=True, n_threads=None):
    """Whole PAMD run; returns (list of per-temperature observable dicts, x, v, fam, E)."""
    t = _topo(top)
    temps = _f64(temps)
    K = len(temps) - 1
    out = (OrcObs * (K + 1))()
    x = np.zeros((R, t.n, 3)); v = np.zeros((R, t.n, 3))
    fam = np.zeros(R, np.int32); E = np.zeros(R)
    nt = n_threads or os.cpu_count() or 1
    rc = _load().orc_anneal(t.ref, R, K, _p(temps), theta, dt, gamma, seed, mol, int(bool(resample)),
                            nt, out, _p(x), _p(v), _p(fam), _p(E))
    if rc != 0:
        raise MemoryError("oracle anneal: allocation failed")
    return [o.as_dict() for o in out], x, v, fam, E
