"""ctypes binding of libolb.so (include/olb.h).  Argument marshalling only:
every step of the method runs in the library's CUDA kernels.

Importing this module loads ``_build/libolb.so`` and raises ImportError if it
is missing (build it with ``python -m paper_1702_01690_gb300.build``); there
is no CPU fallback.  PyTorch supplies the CUDA stream of a context and, via
the allocator hook, its device memory (torch's caching allocator).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"libolb.so not built ({LIB}); run python -m paper_1702_01690_gb300.build")

_lib = ctypes.CDLL(LIB)

OK = 0
ERR_ARG, ERR_CFL, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_STATE, ERR_NOMEM = -1, -2, -3, -4, -5, -6, -7
SIDE_PERIODIC, SIDE_DIFFUSE, SIDE_SPECULAR, SIDE_SPECULAR_DIFFUSE = 0, 1, 2, 3
FP64, FP32_KAHAN = 0, 1
WENO_JS, WENO_LEARNED = 0, 1
MLP_PARAMS = 1347

SYMBOLS = ("olb_set_allocator", "olb_create", "olb_destroy", "olb_init_fields",
           "olb_init_fields_device", "olb_step", "olb_step_async", "olb_get_status",
           "olb_moments", "olb_moments_device", "olb_get_populations",
           "olb_set_populations", "olb_status_string", "olb_profile", "olb_totals", "olb_step_totals", "olb_set_tile", "olb_get_tile", "olb_step_static",
           "olb_batch_create", "olb_batch_destroy", "olb_batch_init_fields", "olb_batch_step",
           "olb_batch_step_async", "olb_batch_get_status", "olb_batch_moments",
           "olb_batch_get_populations", "olb_batch_set_tile", "olb_batch_get_tile",
           "olb_batch_autotune", "olb_batch_profile", "olb_mlp_forward", "olb_mlp_grad",
           "olb_mlp_train", "olb_set_weno_mlp")


class Params(ctypes.Structure):
    """Mirror of olb_params."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("ds", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("sigma", ctypes.c_double),
                ("Tw", ctypes.c_double * 2), ("uw", ctypes.c_double * 2),
                ("side_x", ctypes.c_int), ("side_y", ctypes.c_int),
                ("precision", ctypes.c_int), ("weno_mode", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib.olb_set_allocator.argtypes = [ALLOC_FN, FREE_FN, _VP]
_lib.olb_set_allocator.restype = ctypes.c_int
_lib.olb_create.argtypes = [ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]
_lib.olb_create.restype = ctypes.c_int
_lib.olb_destroy.argtypes = [_VP]
_lib.olb_destroy.restype = None
for _n in ("olb_init_fields", "olb_init_fields_device", "olb_moments", "olb_moments_device"):
    getattr(_lib, _n).argtypes = [_VP, _VP, _VP, _VP, _VP]
    getattr(_lib, _n).restype = ctypes.c_int
for _n in ("olb_step", "olb_step_async"):
    getattr(_lib, _n).argtypes = [_VP, ctypes.c_int]
    getattr(_lib, _n).restype = ctypes.c_int
_lib.olb_get_status.argtypes = [_VP]
_lib.olb_get_status.restype = ctypes.c_int
for _n in ("olb_get_populations", "olb_set_populations"):
    getattr(_lib, _n).argtypes = [_VP, _VP]
    getattr(_lib, _n).restype = ctypes.c_int
_lib.olb_profile.argtypes = [_VP, ctypes.c_int, _VP, _VP]
_lib.olb_totals.argtypes = [_VP, _VP]
_lib.olb_totals.restype = ctypes.c_int
_lib.olb_step_totals.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
_lib.olb_step_totals.restype = ctypes.c_int
_lib.olb_set_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.olb_set_tile.restype = ctypes.c_int
_lib.olb_get_tile.argtypes = [_VP, _VP, _VP, _VP]
_lib.olb_get_tile.restype = ctypes.c_int
_lib.olb_profile.restype = ctypes.c_int
_lib.olb_step_static.argtypes = [ctypes.POINTER(Params), _VP, _VP, ctypes.c_int]
_lib.olb_step_static.restype = ctypes.c_int
STATIC_MAX_NODES = 16384
_lib.olb_batch_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int, _VP, ctypes.POINTER(_VP)]
_lib.olb_batch_create.restype = ctypes.c_int
_lib.olb_batch_destroy.argtypes = [_VP]
_lib.olb_batch_destroy.restype = None
_lib.olb_batch_init_fields.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]
_lib.olb_batch_init_fields.restype = ctypes.c_int
_lib.olb_batch_moments.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP, _VP]
_lib.olb_batch_moments.restype = ctypes.c_int
for _n in ("olb_batch_step", "olb_batch_step_async"):
    getattr(_lib, _n).argtypes = [_VP, ctypes.c_int]
    getattr(_lib, _n).restype = ctypes.c_int
_lib.olb_batch_get_status.argtypes = [_VP, _VP]
_lib.olb_batch_get_status.restype = ctypes.c_int
_lib.olb_batch_get_populations.argtypes = [_VP, ctypes.c_int, _VP]
_lib.olb_batch_get_populations.restype = ctypes.c_int
_lib.olb_batch_set_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.olb_batch_set_tile.restype = ctypes.c_int
for _n in ("olb_batch_get_tile",):
    getattr(_lib, _n).argtypes = [_VP, _VP, _VP, _VP]
    getattr(_lib, _n).restype = ctypes.c_int
_lib.olb_batch_autotune.argtypes = [_VP, ctypes.c_int, _VP, _VP, _VP]
_lib.olb_batch_autotune.restype = ctypes.c_int
_lib.olb_batch_profile.argtypes = [_VP, ctypes.c_int, _VP]
_lib.olb_batch_profile.restype = ctypes.c_int
_lib.olb_mlp_forward.argtypes = [_VP, _VP, ctypes.c_int, _VP, _VP]
_lib.olb_mlp_forward.restype = ctypes.c_int
_lib.olb_mlp_grad.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP]
_lib.olb_mlp_grad.restype = ctypes.c_int
_lib.olb_mlp_train.argtypes = [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                               _VP, _VP]
_lib.olb_mlp_train.restype = ctypes.c_int
_lib.olb_set_weno_mlp.argtypes = [_VP, _VP]
_lib.olb_set_weno_mlp.restype = ctypes.c_int
_lib.olb_status_string.argtypes = [ctypes.c_int]
_lib.olb_status_string.restype = ctypes.c_char_p


class OlbError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


def status_string(code: int) -> str:
    return _lib.olb_status_string(int(code)).decode()


def _check(code: int, what: str) -> int:
    if code != OK:
        raise OlbError(code, what)
    return code


def library():
    return _lib


# ------------------------------------------------------------ torch allocator hook
_hook_refs = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching
    allocator (applies to contexts created afterwards)."""
    global _hook_refs
    if not enable:
        _check(_lib.olb_set_allocator(ALLOC_FN(0), FREE_FN(0), None), "olb_set_allocator")
        _hook_refs = None
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(_lib.olb_set_allocator(refs[0], refs[1], None), "olb_set_allocator")
    _hook_refs = refs


# ------------------------------------------------------------ marshalling helpers

def _host_ptr(a):
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_VP)


def _dev_ptr(t):
    assert t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
    return _VP(t.data_ptr())


def params_from(run, precision: int = FP64, weno_mode: int = WENO_JS) -> Params:
    """Params from any object with the fields of inputs.RunParams."""
    p = Params()
    p.nx, p.ny = int(run.nx), int(run.ny)
    p.ds, p.dt, p.tau = float(run.ds), float(run.dt), float(run.tau)
    p.a, p.b, p.sigma = float(run.a), float(run.b), float(run.sigma)
    p.Tw[0], p.Tw[1] = float(run.Tw[0]), float(run.Tw[1])
    p.uw[0], p.uw[1] = float(run.uw[0]), float(run.uw[1])
    p.side_x, p.side_y = int(run.side_x), int(run.side_y)
    p.precision = int(precision)
    p.weno_mode = int(weno_mode)
    return p


class Context:
    """One olb_ctx.  Fields are (ny, nx) float64 arrays: numpy arrays go
    through the host entry points, CUDA tensors through the device ones."""

    def __init__(self, params: Params, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.nx, self.ny = params.nx, params.ny
        self.params = params
        h = _VP()
        _check(_lib.olb_create(ctypes.byref(params), _VP(stream.cuda_stream), ctypes.byref(h)),
               "olb_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.olb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_fields(self, n, ux, uy, T):
        arrs = (n, ux, uy, T)
        if isinstance(n, np.ndarray):
            arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.ny, self.nx) for a in arrs]
            _check(_lib.olb_init_fields(self._h, *[_host_ptr(a) for a in arrs]), "olb_init_fields")
        else:
            _check(_lib.olb_init_fields_device(self._h, *[_dev_ptr(a) for a in arrs]),
                   "olb_init_fields_device")

    def step(self, nsteps: int = 1) -> int:
        return _check(_lib.olb_step(self._h, int(nsteps)), "olb_step")

    def step_async(self, nsteps: int = 1) -> None:
        _check(_lib.olb_step_async(self._h, int(nsteps)), "olb_step_async")

    def status(self) -> int:
        return _lib.olb_get_status(self._h)

    def moments(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        _check(_lib.olb_moments(self._h, *[_host_ptr(a) for a in out]), "olb_moments")
        return tuple(out)

    def moments_device(self, out=None):
        import torch
        if out is None:
            out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        _check(_lib.olb_moments_device(self._h, *[_dev_ptr(a) for a in out]), "olb_moments_device")
        return tuple(out)

    def profile(self, nsteps: int):
        """Mean device ms per launch of the stage kernel and the launch count."""
        ms = np.zeros(1)
        cnt = np.zeros(1, dtype=np.int32)
        _check(_lib.olb_profile(self._h, int(nsteps), ms.ctypes.data_as(_VP), cnt.ctypes.data_as(_VP)),
               "olb_profile")
        return {"stage_ms": float(ms[0]), "stage_launches": int(cnt[0])}

    def totals(self) -> np.ndarray:
        """Mass, momentum (x, y) and particle kinetic energy summed over the
        grid (times ds^2), computed on the GPU in FP64."""
        out = np.zeros(4)
        _check(_lib.olb_totals(self._h, out.ctypes.data_as(_VP)), "olb_totals")
        return out

    def step_totals(self, nsteps: int, every: int) -> np.ndarray:
        """Advance nsteps steps, recording the four sums of totals() after
        every `every` steps: array [nsteps // every][4]."""
        out = np.zeros((max(int(nsteps) // int(every), 0), 4))
        _check(_lib.olb_step_totals(self._h, int(nsteps), int(every), out.ctypes.data_as(_VP)), "olb_step_totals")
        return out

    def set_tile(self, tx: int, ty: int, kp: int) -> None:
        _check(_lib.olb_set_tile(self._h, int(tx), int(ty), int(kp)), "olb_set_tile")

    def get_tile(self):
        v = [ctypes.c_int() for _ in range(3)]
        _check(_lib.olb_get_tile(self._h, *[ctypes.byref(x) for x in v]), "olb_get_tile")
        return tuple(x.value for x in v)

    def get_populations(self) -> np.ndarray:
        out = np.zeros((25, self.ny, self.nx))
        _check(_lib.olb_get_populations(self._h, _host_ptr(out)), "olb_get_populations")
        return out

    def set_weno_mlp(self, theta) -> None:
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32).reshape(MLP_PARAMS))
        _check(_lib.olb_set_weno_mlp(self._h, th.ctypes.data_as(_VP)), "olb_set_weno_mlp")

    def set_populations(self, f) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(25, self.ny, self.nx)
        _check(_lib.olb_set_populations(self._h, _host_ptr(f)), "olb_set_populations")


def create(run, precision: int = FP64, stream=None, weno_mode: int = WENO_JS) -> Context:
    return Context(params_from(run, precision, weno_mode), stream)


# ------------------------------------------------------------ learned weights
def _f32_dev(t, shape=None):
    import torch
    t = torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
    if shape is not None:
        assert tuple(t.shape) == tuple(shape), (t.shape, shape)
    return t


def mlp_forward(theta, x):
    """Weights [n][3] of normalised stencils x [n][5] (CUDA tensors)."""
    import torch
    theta = _f32_dev(theta, (MLP_PARAMS,))
    x = _f32_dev(x)
    w = torch.empty((x.shape[0], 3), dtype=torch.float32, device="cuda")
    _check(_lib.olb_mlp_forward(_VP(theta.data_ptr()), _VP(x.data_ptr()), int(x.shape[0]), _VP(w.data_ptr()),
                                _VP(torch.cuda.current_stream().cuda_stream)), "olb_mlp_forward")
    return w


def mlp_grad(theta, x, gn, tn):
    """(mean loss, gradient) on the device for samples x [n][5], gn [n][3], tn [n]."""
    import torch
    theta = _f32_dev(theta, (MLP_PARAMS,))
    x, gn, tn = _f32_dev(x), _f32_dev(gn), _f32_dev(tn)
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(_lib.olb_mlp_grad(_VP(theta.data_ptr()), _VP(x.data_ptr()), _VP(gn.data_ptr()), _VP(tn.data_ptr()),
                             int(x.shape[0]), _VP(grad.data_ptr()), _VP(loss.data_ptr()),
                             _VP(torch.cuda.current_stream().cuda_stream)), "olb_mlp_grad")
    return float(loss.item()), grad


def mlp_train(theta, x, gn, tn, epochs: int, batch: int = 4096, lr: float = 1e-3):
    """Train theta (CUDA float32 tensor, updated in place); returns the loss
    history per epoch."""
    import torch
    assert theta.is_cuda and theta.dtype == torch.float32 and theta.numel() == MLP_PARAMS
    x, gn, tn = _f32_dev(x), _f32_dev(gn), _f32_dev(tn)
    hist = np.zeros(int(epochs), dtype=np.float32)
    _check(_lib.olb_mlp_train(_VP(theta.data_ptr()), _VP(x.data_ptr()), _VP(gn.data_ptr()), _VP(tn.data_ptr()),
                              int(x.shape[0]), int(epochs), int(batch), ctypes.c_float(lr),
                              _VP(torch.cuda.current_stream().cuda_stream), hist.ctypes.data_as(_VP)),
           "olb_mlp_train")
    return hist


class Batch:
    """One olb_batch: independent runs of uneven sizes advanced together."""

    def __init__(self, runs, precision: int = FP64, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        plist = [params_from(r, precision) for r in runs]
        arr = (Params * len(plist))(*plist)
        self.shapes = [(p.ny, p.nx) for p in plist]
        h = _VP()
        _check(_lib.olb_batch_create(arr, len(plist), _VP(stream.cuda_stream), ctypes.byref(h)),
               "olb_batch_create")
        self._h = h

    @property
    def count(self) -> int:
        return len(self.shapes)

    def close(self):
        if getattr(self, "_h", None):
            _lib.olb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, run: int, n, ux, uy, T):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shapes[run]) for a in (n, ux, uy, T)]
        _check(_lib.olb_batch_init_fields(self._h, int(run), *[_host_ptr(a) for a in arrs]),
               "olb_batch_init_fields")

    def step(self, nsteps: int = 1) -> int:
        return _check(_lib.olb_batch_step(self._h, int(nsteps)), "olb_batch_step")

    def step_async(self, nsteps: int = 1) -> None:
        _check(_lib.olb_batch_step_async(self._h, int(nsteps)), "olb_batch_step_async")

    def status(self):
        per = np.zeros(self.count, dtype=np.int32)
        rc = _lib.olb_batch_get_status(self._h, per.ctypes.data_as(_VP))
        return rc, per

    def moments(self, run: int):
        out = [np.zeros(self.shapes[run]) for _ in range(4)]
        _check(_lib.olb_batch_moments(self._h, int(run), *[_host_ptr(a) for a in out]), "olb_batch_moments")
        return tuple(out)

    def get_populations(self, run: int) -> np.ndarray:
        out = np.zeros((25,) + self.shapes[run])
        _check(_lib.olb_batch_get_populations(self._h, int(run), _host_ptr(out)), "olb_batch_get_populations")
        return out

    def set_tile(self, tx: int, ty: int, kp: int) -> None:
        _check(_lib.olb_batch_set_tile(self._h, int(tx), int(ty), int(kp)), "olb_batch_set_tile")

    def get_tile(self):
        v = [ctypes.c_int() for _ in range(3)]
        _check(_lib.olb_batch_get_tile(self._h, *[ctypes.byref(x) for x in v]), "olb_batch_get_tile")
        return tuple(x.value for x in v)

    def autotune(self, nsteps: int = 3):
        v = [ctypes.c_int() for _ in range(3)]
        _check(_lib.olb_batch_autotune(self._h, int(nsteps), *[ctypes.byref(x) for x in v]), "olb_batch_autotune")
        return tuple(x.value for x in v)

    def profile(self, nsteps: int) -> float:
        ms = ctypes.c_double()
        _check(_lib.olb_batch_profile(self._h, int(nsteps), ctypes.byref(ms)), "olb_batch_profile")
        return ms.value
