"""Thin Python binding of the C ABI in include/gda.h (argument marshalling only).

Every computation runs in libgda.so's CUDA kernels.  Loading fails loudly if
the library has not been built (`python -m paper_1807_00699_gb300._build` or
`__graft_entry__.build()`); there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgda.so")

ISING, XY = 0, 1
EULER, RK4 = 0, 1
FP32, BF16, FP8, SPARSE = 0, 1, 2, 3
GD, GDMOD = 0, 1  # coupling feedback (gda_coupling_mode)
AUTO, PER_STEP, RESIDENT, PAIR, STREAM, STREAM_PAIR, RESIDENT_PAIR = 0, 1, 2, 3, 4, 5, 6

STATUS = {0: "GDA_OK", 1: "GDA_ERR_INVALID", 2: "GDA_ERR_CUDA", 3: "GDA_ERR_OOM", 4: "GDA_ERR_DIVERGED",
          5: "GDA_ERR_TIMEOUT", 6: "GDA_ERR_UNSUPPORTED", 7: "GDA_ERR_STATE"}

# Every symbol include/gda.h declares, with its ctypes signature.
_D = ct.POINTER(ct.c_double)
_F = ct.POINTER(ct.c_float)
_VP = ct.c_void_p


class Params(ct.Structure):
    """gda_params (include/gda.h)."""
    _fields_ = [("integ", ct.c_int32), ("prec", ct.c_int32), ("dt", ct.c_double), ("eps", ct.c_double),
                ("rho_th", ct.c_double), ("gamma0", ct.c_double), ("beta0", ct.c_double),
                ("eps_hat", ct.c_double), ("noise_D", ct.c_double), ("noise_decay", ct.c_int32),
                ("energy_every", ct.c_int32), ("seed", ct.c_uint64), ("init_mode", ct.c_int32),
                ("schedule", ct.c_int32), ("init_amp", ct.c_double), ("coupling", ct.c_int32),
                ("withhold_flag", ct.c_int32), ("gamma_c", ct.c_double), ("q", ct.c_int32),
                ("reserved2", ct.c_int32), ("hq", ct.c_double), ("wait_s", ct.c_double)]


SIGNATURES = {
    "gda_default_params": (None, [ct.POINTER(Params)]),
    "gda_create": (ct.c_int, [_D, _D, ct.c_int32, ct.c_int32, ct.POINTER(_VP)]),
    "gda_load": (ct.c_int, [_VP, _D, _D]),
    "gda_load_dev": (ct.c_int, [_VP, _VP, _VP]),
    "gda_set_stream": (ct.c_int, [_VP, _VP]),
    "gda_run": (ct.c_int, [_VP, ct.POINTER(Params), ct.c_int32, ct.c_int64]),
    "gda_sync": (ct.c_int, [_VP]),
    "gda_energy": (ct.c_int, [_VP, _D]),
    "gda_energy_dev": (ct.c_int, [_VP, _VP]),
    "gda_best": (ct.c_int, [_VP, _D, ct.POINTER(ct.c_int32), _VP]),
    "gda_get_state": (ct.c_int, [_VP, _F, _F, _F, ct.POINTER(ct.c_int64)]),
    "gda_set_state": (ct.c_int, [_VP, _F, _F, _F, ct.c_int32, ct.c_int64]),
    "gda_best_seen": (ct.c_int, [_VP, _D, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int64), _VP]),
    "gda_trace": (ct.c_int, [_VP, ct.POINTER(ct.c_int64), _D, ct.POINTER(ct.c_int32), ct.c_int32,
                             ct.POINTER(ct.c_int32)]),
    "gda_trace_energy": (ct.c_int, [_VP, ct.c_int32, ct.c_int32, _D]),
    "gda_coupling": (ct.c_int, [_VP, ct.c_int32, ct.c_int32, _F, _F]),
    "gda_profile": (ct.c_int, [_VP, ct.c_int32]),
    "gda_profile_read": (ct.c_int, [_VP, ct.POINTER(ct.c_uint64), ct.c_int32, ct.POINTER(ct.c_int32)]),
    "gda_energy_noalloc": (ct.c_int, [_VP, _VP, ct.c_int32, ct.c_int32, _VP, ct.c_int32, _VP, _VP]),
    "gda_features": (ct.c_int, [_VP, _VP]),
    "gda_set_init_base": (ct.c_int, [_VP, _VP, ct.c_int32]),
    "gda_mlp_forward": (ct.c_int, [_VP, _VP, ct.c_int32, _VP, _VP, _VP]),
    "gda_mlp_backward": (ct.c_int, [_VP, _VP, _VP, _VP, ct.c_int32, _VP, _VP]),
    "gda_proposal_loss": (ct.c_int, [_VP, _VP, _VP, _VP, _VP, ct.c_int32, ct.c_float, _VP, _VP, _VP]),
    "gda_proposal_head": (ct.c_int, [_VP, ct.c_int32, ct.c_int32, ct.c_double, _VP, _VP, _VP]),
    "gda_adam_step": (ct.c_int, [_VP, _VP, _VP, _VP, ct.c_int32, ct.c_float, ct.c_float, ct.c_float, ct.c_float,
                                 ct.c_int32, _VP]),
    "gda_batch_create": (ct.c_int, [ct.c_int32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                                    ct.POINTER(_VP), ct.POINTER(_VP), ct.c_uint64, ct.POINTER(_VP)]),
    "gda_batch_set_stream": (ct.c_int, [_VP, _VP]),
    "gda_batch_set_tile": (ct.c_int, [_VP, ct.c_int32]),
    "gda_batch_set_schedule": (ct.c_int, [_VP, ct.c_int32]),
    "gda_batch_run": (ct.c_int, [_VP, ct.POINTER(Params), ct.c_int64]),
    "gda_batch_set_params": (ct.c_int, [_VP, ct.c_int32, ct.POINTER(Params)]),
    "gda_batch_set_init_base": (ct.c_int, [_VP, ct.c_int32, _VP, ct.c_int32]),
    "gda_batch_launch_mode": (ct.c_int32, [_VP]),
    "gda_batch_best": (ct.c_int, [_VP, _D, ct.POINTER(ct.c_int32)]),
    "gda_batch_get_state": (ct.c_int, [_VP, ct.c_int32, _F, _F, _F]),
    "gda_batch_last_error": (ct.c_char_p, [_VP]),
    "gda_batch_destroy": (None, [_VP]),
    "gda_kernel_launches": (ct.c_int64, [_VP]),
    "gda_last_error": (ct.c_char_p, [_VP]),
    "gda_status_string": (ct.c_char_p, [ct.c_int]),
    "gda_destroy": (None, [_VP]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ct.CDLL:
    """Loads libgda.so and binds every declared symbol (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GdaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(ct.POINTER(typ))


def default_params(**kw) -> Params:
    p = Params()
    load_library().gda_default_params(ct.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Solver:
    """One gda_ctx: an N-spin instance on the current CUDA device."""

    def __init__(self, J: np.ndarray, g: np.ndarray | None = None, model: int = ISING, stream=None):
        lib = load_library()
        self._lib = lib
        J = np.ascontiguousarray(J, dtype=np.float64)
        if J.ndim != 2 or J.shape[0] != J.shape[1]:
            raise ValueError("J must be square")
        self.N = J.shape[0]
        self.model = model
        gp = None
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64)
            gp = _ptr(g, ct.c_double)
        h = _VP()
        st = lib.gda_create(_ptr(J, ct.c_double), gp, self.N, model, ct.byref(h))
        if st != 0:
            raise GdaError(st, "gda_create failed")
        self._h = h
        self.R = 0
        if stream is not None:
            self.set_stream(stream)

    # -- helpers
    def _check(self, st: int):
        if st != 0:
            raise GdaError(st, self._lib.gda_last_error(self._h).decode())

    @property
    def width(self) -> int:
        return 2 if self.model == XY else 1

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.gda_set_stream(self._h, _VP(handle or 0)))

    def load(self, J: np.ndarray, g: np.ndarray | None = None):
        J = np.ascontiguousarray(J, dtype=np.float64)
        gp = None if g is None else _ptr(np.ascontiguousarray(g, dtype=np.float64), ct.c_double)
        self._check(self._lib.gda_load(self._h, _ptr(J, ct.c_double), gp))

    def load_dev(self, J_ptr: int, g_ptr: int | None = None):
        self._check(self._lib.gda_load_dev(self._h, _VP(J_ptr), _VP(g_ptr or 0)))

    def run(self, params: Params, R: int, steps: int):
        self._check(self._lib.gda_run(self._h, ct.byref(params), int(R), int(steps)))
        self.R = int(R)

    def sync(self):
        self._check(self._lib.gda_sync(self._h))

    def energy(self) -> np.ndarray:
        E = np.empty(self.R, dtype=np.float64)
        self._check(self._lib.gda_energy(self._h, _ptr(E, ct.c_double)))
        return E

    def energy_dev(self, E_ptr: int):
        self._check(self._lib.gda_energy_dev(self._h, _VP(E_ptr)))

    def best(self, with_cfg: bool = True):
        """(E, r, cfg): cfg int8 spins (Ising) or float64 theta (XY)."""
        E = ct.c_double()
        r = ct.c_int32()
        cfg = None
        cp = None
        if with_cfg:
            cfg = np.empty(self.N, dtype=np.float64 if self.model == XY else np.int8)
            cp = cfg.ctypes.data_as(_VP)
        self._check(self._lib.gda_best(self._h, ct.byref(E), ct.byref(r), cp))
        return E.value, r.value, cfg

    def best_seen(self, with_cfg: bool = True):
        """(E, r, step, cfg) of the lowest tracked energy any restart reached
        (gda_best_seen): the configuration kept at that step, in FP64."""
        E = ct.c_double()
        r = ct.c_int32()
        st = ct.c_int64()
        cfg = None
        cp = None
        if with_cfg:
            cfg = np.empty(self.N, dtype=np.float64 if self.model == XY else np.int8)
            cp = cfg.ctypes.data_as(_VP)
        self._check(self._lib.gda_best_seen(self._h, ct.byref(E), ct.byref(r), ct.byref(st), cp))
        return E.value, r.value, st.value, cfg

    def get_state(self):
        R, N, W = self.R, self.N, self.width
        psi = np.empty(R * N * W, dtype=np.float32)
        gam = np.empty(R * N, dtype=np.float32)
        beta = np.empty(R, dtype=np.float32)
        step = ct.c_int64()
        self._check(self._lib.gda_get_state(self._h, _ptr(psi, ct.c_float), _ptr(gam, ct.c_float),
                                            _ptr(beta, ct.c_float), ct.byref(step)))
        psi = psi.reshape(R, N, W)
        psi = psi[..., 0] + 1j * psi[..., 1] if W == 2 else psi[..., 0]
        return psi, gam.reshape(R, N), beta, step.value

    def set_state(self, psi: np.ndarray, gamma: np.ndarray | None = None, beta: np.ndarray | None = None,
                  step: int = 0):
        psi = np.asarray(psi)
        R = psi.shape[0]
        if self.model == XY:
            flat = np.stack([psi.real, psi.imag], axis=-1).astype(np.float32).ravel()
        else:
            flat = np.ascontiguousarray(psi, dtype=np.float32).ravel()
        gp = None if gamma is None else _ptr(np.ascontiguousarray(gamma, dtype=np.float32), ct.c_float)
        bp = None if beta is None else _ptr(np.ascontiguousarray(beta, dtype=np.float32), ct.c_float)
        self._check(self._lib.gda_set_state(self._h, _ptr(flat, ct.c_float), gp, bp, R, int(step)))
        self.R = R

    def trace(self, cap: int = 65536):
        steps = np.empty(cap, dtype=np.int64)
        E = np.empty(cap, dtype=np.float64)
        r = np.empty(cap, dtype=np.int32)
        n = ct.c_int32()
        self._check(self._lib.gda_trace(self._h, _ptr(steps, ct.c_int64), _ptr(E, ct.c_double),
                                        _ptr(r, ct.c_int32), cap, ct.byref(n)))
        m = min(n.value, cap)
        return steps[:m], E[:m], r[:m]

    def trace_energy(self, first: int = 0, count: int | None = None) -> np.ndarray:
        """FP64 energies of the configurations the trace names (gda_trace_energy):
        entry k is the lowest-tracked restart as it was at trace step k."""
        if count is None:
            count = len(self.trace()[0]) - first
        E = np.empty(max(count, 0), dtype=np.float64)
        self._check(self._lib.gda_trace_energy(self._h, int(first), int(count), _ptr(E, ct.c_double)))
        return E

    def coupling(self, X: np.ndarray, prec: int = FP32) -> np.ndarray:
        """Y = J0 X (the coupling product alone) for X of shape (R, N)."""
        X = np.asarray(X)
        R = X.shape[0]
        if self.model == XY:
            flat = np.stack([X.real, X.imag], axis=-1).astype(np.float32).ravel()
        else:
            flat = np.ascontiguousarray(X, dtype=np.float32).ravel()
        Y = np.empty_like(flat)
        self._check(self._lib.gda_coupling(self._h, prec, R, _ptr(flat, ct.c_float), _ptr(Y, ct.c_float)))
        self.R = R
        Y = Y.reshape(R, self.N, self.width)
        return Y[..., 0] + 1j * Y[..., 1] if self.model == XY else Y[..., 0]

    def profile(self, enable: bool = True):
        self._check(self._lib.gda_profile(self._h, 1 if enable else 0))

    def profile_read(self, cap_ctas: int = 4096) -> np.ndarray:
        """(ctas, 8) uint64 nanosecond stamps of the last tensor-core step launch."""
        buf = np.zeros(cap_ctas * 8, dtype=np.uint64)
        n = ct.c_int32()
        self._check(self._lib.gda_profile_read(self._h, _ptr(buf, ct.c_uint64), cap_ctas, ct.byref(n)))
        return buf[: n.value * 8].reshape(n.value, 8)

    def set_init_base(self, base: np.ndarray):
        """Per-spin base amplitude [N] (real or complex) for init_mode 3."""
        base = np.asarray(base)
        if self.model == XY:
            flat = np.stack([base.real, base.imag], axis=-1).astype(np.float32).ravel()
        else:
            flat = np.ascontiguousarray(base.real, dtype=np.float32)
        self._check(self._lib.gda_set_init_base(self._h, flat.ctypes.data_as(_VP), 0))

    def set_init_base_dev(self, base_ptr: int):
        """init_mode 3 base amplitudes from a device buffer in
        gda_set_init_base's layout (e.g. gda_proposal_head's output)."""
        self._check(self._lib.gda_set_init_base(self._h, _VP(base_ptr), 1))

    def features(self, F_ptr: int):
        """Per-spin features [N][8] into a device buffer (see gda_features)."""
        self._check(self._lib.gda_features(self._h, _VP(F_ptr)))

    def kernel_launches(self) -> int:
        return int(self._lib.gda_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gda_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GOLDEN64 = 0x9E3779B97F4A7C15


class Batch:
    """A gda_batch: many instances stepped together (BF16 Euler)."""

    def __init__(self, instances, seed: int = 0, stream=None):
        """instances: list of (J, g or None, model, R)."""
        lib = load_library()
        self._lib = lib
        n = len(instances)
        self.N = [int(np.asarray(J).shape[0]) for J, _, _, _ in instances]
        self.model = [int(m) for _, _, m, _ in instances]
        self.R = [int(r) for _, _, _, r in instances]
        self._Js = [np.ascontiguousarray(J, dtype=np.float64) for J, _, _, _ in instances]
        self._gs = [None if g is None else np.ascontiguousarray(g, dtype=np.float64) for _, g, _, _ in instances]
        Jp = (_VP * n)(*[a.ctypes.data for a in self._Js])
        gp = (_VP * n)(*[0 if a is None else a.ctypes.data for a in self._gs])
        arr = lambda v: (ct.c_int32 * n)(*v)  # noqa: E731
        h = _VP()
        st = lib.gda_batch_create(n, arr(self.N), arr(self.model), arr(self.R), Jp, gp, seed & (2 ** 64 - 1),
                                  ct.byref(h))
        if st != 0:
            raise GdaError(st, "gda_batch_create failed")
        self._h = h
        self.n = n
        self.seed = seed
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            self._check(lib.gda_batch_set_stream(h, _VP(handle or 0)))

    def instance_seed(self, k: int) -> int:
        return (self.seed + k * GOLDEN64) & (2 ** 64 - 1)

    def _check(self, st):
        if st != 0:
            raise GdaError(st, self._lib.gda_batch_last_error(self._h).decode())

    def set_tile(self, bn: int):
        self._check(self._lib.gda_batch_set_tile(self._h, bn))

    def set_schedule(self, schedule: int):
        """RESIDENT: one persistent launch per 100 steps; PER_STEP: one launch per step."""
        self._check(self._lib.gda_batch_set_schedule(self._h, schedule))

    def run(self, params: Params, steps: int):
        self._check(self._lib.gda_batch_run(self._h, ct.byref(params), int(steps)))

    def set_params(self, k: int, params: Params | None):
        """Instance k's own eps, rho_th, beta0, eps_hat (None: follow each run's)."""
        self._check(self._lib.gda_batch_set_params(self._h, int(k), None if params is None else ct.byref(params)))

    def set_init_base(self, k: int, base: np.ndarray | None):
        """Per-spin base amplitudes [N_k] (real or complex) of instance k for init_mode 3."""
        if base is None:
            self._check(self._lib.gda_batch_set_init_base(self._h, int(k), None, 0))
            return
        base = np.asarray(base)
        if self.model[k] == XY:
            flat = np.stack([base.real, base.imag], axis=-1).astype(np.float32).ravel()
        else:
            flat = np.ascontiguousarray(base.real, dtype=np.float32)
        self._check(self._lib.gda_batch_set_init_base(self._h, int(k), flat.ctypes.data_as(_VP), 0))

    def set_init_base_dev(self, k: int, base_ptr: int):
        """Instance k's init_mode 3 base amplitudes from a device buffer."""
        self._check(self._lib.gda_batch_set_init_base(self._h, int(k), _VP(base_ptr), 1))

    def launch_mode(self) -> int:
        """1: chunks replay a captured CUDA graph; 0: direct launches."""
        return int(self._lib.gda_batch_launch_mode(self._h))

    def best(self):
        E = np.empty(self.n, dtype=np.float64)
        r = np.empty(self.n, dtype=np.int32)
        self._check(self._lib.gda_batch_best(self._h, _ptr(E, ct.c_double), _ptr(r, ct.c_int32)))
        return E, r

    def get_state(self, k: int):
        N, R, W = self.N[k], self.R[k], 2 if self.model[k] == XY else 1
        psi = np.empty(R * N * W, dtype=np.float32)
        gam = np.empty(R * N, dtype=np.float32)
        beta = np.empty(R, dtype=np.float32)
        self._check(self._lib.gda_batch_get_state(self._h, k, _ptr(psi, ct.c_float), _ptr(gam, ct.c_float),
                                                  _ptr(beta, ct.c_float)))
        psi = psi.reshape(R, N, W)
        psi = psi[..., 0] + 1j * psi[..., 1] if W == 2 else psi[..., 0]
        return psi, gam.reshape(R, N), beta

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gda_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
