"""Binding of the learned energy surrogate (include/pamd_mlp.h).

Argument marshalling only: features, the dense layers, forces, the
force-matching loss and its gradient and Adam run in libpamd's kernels.
PyTorch provides device memory and the stream; ``SurrogateEnergy`` is the
torch.autograd.Function whose backward is the library's force kernel.
"""
from __future__ import annotations

import ctypes as C
import functools
import os

import numpy as np

from . import pamd as _p


class PamdMlpParams(C.Structure):
    _fields_ = [("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_double), ("mu", C.c_void_p), ("sd", C.c_void_p),
                ("mu_E", C.c_double), ("sigma_E", C.c_double)]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the surrogate runs on the GPU only; no CUDA device is visible")
    return torch


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def gemm_bf16(A, B):
    """C = A @ B.T on the tensor cores: A [M, K], B [N, K] bf16 CUDA tensors -> FP32 [M, N]."""
    torch = _torch()
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _p._check(_p.load().pamd_gemm_bf16(_dptr(A), _dptr(B), _dptr(out), M, N, K, K, K, N,
                                       _stream_handle(torch)))
    return out


def gemm_bf16_time(A, B, reps: int = 10):
    """Mean device time (ms) of `reps` back-to-back tensor-core launches of A @ B.T,
    bracketed by CUDA events on torch's current stream."""
    torch = _torch()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    ms = C.c_float(0.0)
    _p._check(_p.load().pamd_gemm_bf16_time(_dptr(A), _dptr(B), _dptr(out), M, N, K, K, K, N, reps,
                                            _stream_handle(torch), C.byref(ms)))
    return ms.value


class MLP:
    """An MLP energy surrogate over inverse pair distances (2 SiLU layers).

    The model's kernels run on a stream of its own; every call orders it after
    the work already queued on torch's current stream, and the current stream
    after the model's work, so tensors can be passed in and used as usual.
    """

    def __init__(self, n_atoms: int, hidden: int = 512, seed: int = 0):
        torch = _torch()
        self._torch = torch
        self._lib = _p.load()
        self._stream = torch.cuda.Stream()
        h = C.c_void_p()
        _p._check(self._lib.pamd_mlp_create(C.byref(h), n_atoms, hidden, seed,
                                            C.c_void_p(self._stream.cuda_stream)))
        self._h = h
        self.n_atoms, self.hidden = n_atoms, hidden
        self.n_pairs = n_atoms * (n_atoms - 1) // 2

    def _call(self, fn, *args):
        cur = self._torch.cuda.current_stream()
        self._stream.wait_stream(cur)
        try:
            _p._check(fn(self._h, *args))
        finally:
            cur.wait_stream(self._stream)

    # ---------------------------------------------------------------- params
    def _struct(self, arrays):
        s = PamdMlpParams()
        for k in ("W1", "b1", "W2", "b2", "w3", "mu", "sd"):
            a = arrays.get(k)
            setattr(s, k, None if a is None else a.ctypes.data_as(C.c_void_p))
        return s

    def _empty(self):
        H, P = self.hidden, self.n_pairs
        return {"W1": np.zeros((H, P), np.float32), "b1": np.zeros(H, np.float32),
                "W2": np.zeros((H, H), np.float32), "b2": np.zeros(H, np.float32),
                "w3": np.zeros(H, np.float32), "mu": np.zeros(P, np.float32),
                "sd": np.zeros(P, np.float32)}

    def get_params(self) -> dict:
        a = self._empty()
        s = self._struct(a)
        self._call(self._lib.pamd_mlp_get_params, C.byref(s))
        a.update(b3=s.b3, mu_E=s.mu_E, sigma_E=s.sigma_E)
        return a

    def set_params(self, p: dict) -> None:
        a = {k: (None if p.get(k) is None else np.ascontiguousarray(p[k], dtype=np.float32))
             for k in ("W1", "b1", "W2", "b2", "w3", "mu", "sd")}
        s = self._struct(a)
        s.b3 = float(p.get("b3", 0.0))
        s.mu_E = float(p.get("mu_E", 0.0))
        s.sigma_E = float(p.get("sigma_E", 1.0))
        self._call(self._lib.pamd_mlp_set_params, C.byref(s))

    def get_grads(self) -> dict:
        a = self._empty()
        a["mu"] = a["sd"] = None
        s = self._struct(a)
        self._call(self._lib.pamd_mlp_get_grads, C.byref(s))
        a["b3"] = s.b3
        return {k: v for k, v in a.items() if v is not None}

    # ------------------------------------------------------------- compute
    def _check_x(self, x):
        torch = self._torch
        assert x.is_cuda and x.dtype == torch.float32 and x.shape[1:] == (self.n_atoms, 3)
        return x.contiguous()

    def fit_normalization(self, x, E) -> None:
        x = self._check_x(x)
        E = E.contiguous()
        self._call(self._lib.pamd_mlp_fit_normalization, _dptr(x), _dptr(E), x.shape[0])

    def energy_forces(self, x, forces: bool = True):
        """(E [M] float64, F [M, N, 3] float32 or None) of positions x [M, N, 3]."""
        torch = self._torch
        x = self._check_x(x)
        E = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        F = torch.empty_like(x) if forces else None
        self._call(self._lib.pamd_mlp_energy_forces, _dptr(x), x.shape[0], _dptr(E), _dptr(F))
        return E, F

    def loss_grads(self, x, E, F, idx=None, lam: float = 1.0, sync: bool = True):
        x = self._check_x(x)
        M = x.shape[0] if idx is None else idx.shape[0]
        loss = C.c_double(0.0)
        E, F = E.contiguous(), F.contiguous()
        self._call(self._lib.pamd_mlp_loss_grads, _dptr(x), _dptr(E), _dptr(F), _dptr(idx), M, lam,
                   C.byref(loss) if sync else None)
        return loss.value if sync else None

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._call(self._lib.pamd_mlp_adam_step, lr, beta1, beta2, eps)

    def sync(self) -> None:
        self._call(self._lib.pamd_mlp_sync)

    def launch_count(self) -> int:
        return int(self._lib.pamd_mlp_launch_count(self._h))

    def train(self, x, E, F, *, epochs: int, batch: int = 1024, lam: float = 1.0,
              lr: float = 1e-3, lr_final: float | None = None, seed: int = 0,
              report_every: int = 200):
        """Minibatch Adam over the dataset (x [n, N, 3], E [n], F [n, N, 3] on the device).

        The learning rate decays geometrically from lr to lr_final over all
        steps.  Returns the losses of every ``report_every``-th step.
        """
        torch = self._torch
        n = x.shape[0]
        steps_per_epoch = n // batch
        total = epochs * steps_per_epoch
        rng = np.random.default_rng(seed)
        lr_final = lr if lr_final is None else lr_final
        decay = (lr_final / lr) ** (1.0 / max(1, total - 1))
        hist, step = [], 0
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(x.device)
            for b in range(steps_per_epoch):
                idx = perm[b * batch:(b + 1) * batch]
                want = report_every and step % report_every == 0
                loss = self.loss_grads(x, E, F, idx=idx, lam=lam, sync=bool(want))
                if want:
                    hist.append((step, loss))
                self.adam_step(lr * decay ** step)
                step += 1
        self.sync()
        return hist

    def save(self, path: str) -> None:
        self._call(self._lib.pamd_mlp_save, os.fsencode(path))

    @classmethod
    def load(cls, path: str) -> "MLP":
        """A model read from a file written by ``save``."""
        self = cls.__new__(cls)
        torch = _torch()
        self._torch = torch
        self._lib = _p.load()
        self._stream = torch.cuda.Stream()
        h = C.c_void_p()
        _p._check(self._lib.pamd_mlp_load(C.byref(h), os.fsencode(path), C.c_void_p(self._stream.cuda_stream)))
        self._h = h
        n = C.c_int32(); npairs = C.c_int32(); hid = C.c_int32()
        _p._check(self._lib.pamd_mlp_info(h, C.byref(n), C.byref(npairs), C.byref(hid)))
        self.n_atoms, self.hidden, self.n_pairs = n.value, hid.value, npairs.value
        return self

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pamd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def attach(ctx, model: MLP | None) -> None:
    """Use ``model`` (None: the exact force field) for a population's forces."""
    _p._check(_p.load().pamd_set_force_model(ctx, None if model is None else model._h))


@functools.lru_cache(maxsize=None)
def _autograd_function():
    torch = _torch()

    class SurrogateEnergy(torch.autograd.Function):
        """E(x) of the surrogate; the backward pass is the library's force kernel."""

        @staticmethod
        def forward(ctx, x, model):
            E, _ = model.energy_forces(x.detach(), forces=False)
            ctx.save_for_backward(x.detach())
            ctx.model = model
            return E

        @staticmethod
        def backward(ctx, gE):
            (x,) = ctx.saved_tensors
            _, F = ctx.model.energy_forces(x, forces=True)
            # dE/dx = -F, scaled by the incoming gradient
            return -(gE.to(F.dtype)[:, None, None] * F), None

    return SurrogateEnergy


def surrogate_energy(x, model: MLP):
    """Differentiable surrogate energy of positions x [M, N, 3] (float32, CUDA)."""
    return _autograd_function().apply(x, model)


def harvest(top, R: int, temps, theta: int, dt_ps: float, seed: int, options=None, model=None):
    """(x [n, N, 3] float32, E [n] float64, F [n, N, 3] float32) sampled from an anneal.

    One population of R replicas is annealed through ``temps``; after the
    theta steps at every temperature the whole population is recorded with
    its exact energies and forces.  With ``model`` the population is driven
    by that surrogate (it samples the surrogate's distribution) and every
    recorded configuration is labelled by the exact force field of a second
    population of the same size.
    """
    xs, Es, Fs = [], [], []
    label = _p.Population(top, R, temps[0], seed, options) if model is not None else None
    try:
        with _p.Population(top, R, temps[0], seed, options) as pop:
            if model is not None:
                attach(pop.ctx, model)
            for i, T in enumerate(temps):
                if i:
                    pop.resample(temps[i - 1], T, want_copies=False)
                pop.propagate(theta, dt_ps, T)
                x, v, _, _ = pop.state()
                if label is not None:
                    label.set_state(x, v)
                    f, E = label.forces()
                else:
                    f, E = pop.forces()
                xs.append(x.astype(np.float32))
                Fs.append(f.astype(np.float32))
                Es.append(E.copy())
    finally:
        if label is not None:
            label.close()
    return np.concatenate(xs), np.concatenate(Es), np.concatenate(Fs)
