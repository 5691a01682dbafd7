"""FP64 CPU oracle for the off-lattice Boltzmann step of arXiv:1702.01690.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_1702_01690_gb300``)
and neither imports the other.

The arithmetic lives in ``olb_oracle.c`` (plain C, FP64, compiled without
FMA contraction or fast-math); this module only builds it with gcc and
marshals numpy arrays through ctypes.  ``maxwell.py`` and ``analytic.py``
hold closed-form physics used as pins (Maxwell equal-area construction,
linearised shear-wave decay).

Parity status of each oracle function (what pins it, see tests/test_oracle_*):
  orc_quadrature, orc_hermite  -- numpy's Gauss-HermiteE rule, He_5(R)=0,
                                  W_q = Q!/He_6(R_q)^2 (Table trots)
  orc_g, orc_feq               -- Gaussian moments of orders 0..4
  orc_dp_line                  -- analytic p-derivative of w*P(p), P cubic
  orc_moments_node             -- moments of f^eq reproduce (n, u, T)
  orc_grad_stencil             -- exactness on degree<=6 polynomials; 1-D
                                  reduction printed in Sec. 4
  orc_glap_stencil             -- same, for grad(Laplacian)
  orc_weno5                    -- Table tab:weno, exactness on quadratics,
                                  5th-order linear limit, convergence on sines
  orc_weno5_learned, mlp.py    -- mlp.grad against central finite differences;
                                  the C forward against mlp.py; Table tab:weno
                                  wherever an indicator vanishes
  orc_step                     -- conservation of mass; rest state is a fixed
                                  point; shear-wave decay rate (Eq. shear_sol);
                                  self-convergence order in ds; n_w zero net flux
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "olb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile olb_oracle.c into oracle/_build/liborc.so (gcc, -O2, OpenMP).

    No FMA contraction and no fast-math, so that the oracle rounds every
    operation as written."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("ds", ctypes.c_double), ("dt", ctypes.c_double),
                ("tau", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("sigma", ctypes.c_double),
                ("Tw", ctypes.c_double * 2), ("uw", ctypes.c_double * 2),
                ("side_x", ctypes.c_int), ("side_y", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)


def _declare(L):
    """Argument and result types of the oracle's exported calls."""
    L.orc_hermite.restype = ctypes.c_double
    L.orc_hermite.argtypes = [ctypes.c_int, ctypes.c_double]
    L.orc_quadrature.argtypes = [_D, _D]
    L.orc_g.restype = ctypes.c_double
    L.orc_g.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.orc_feq.argtypes = [ctypes.c_double] * 4 + [_D]
    L.orc_dp_line.argtypes = [_D, _D]
    L.orc_moments_node.argtypes = [_D, _D]
    L.orc_pw.restype = ctypes.c_double
    L.orc_pw.argtypes = [ctypes.c_double] * 4
    L.orc_grad_stencil.argtypes = [_D]
    L.orc_glap_stencil.argtypes = [_D]
    L.orc_weno5.restype = ctypes.c_double
    L.orc_weno5.argtypes = [_D, _D]
    L.orc_create.restype = ctypes.c_void_p
    L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
    L.orc_destroy.argtypes = [ctypes.c_void_p]
    L.orc_init.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
    L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_get_f.argtypes = [ctypes.c_void_p, _D]
    L.orc_set_f.argtypes = [ctypes.c_void_p, _D]
    L.orc_get_moments.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
    L.orc_eval.argtypes = [ctypes.c_void_p, _D, _D, _D]
    L.orc_weno5_learned.restype = ctypes.c_double
    L.orc_weno5_learned.argtypes = [_D, _D, _D]
    L.orc_set_mlp.argtypes = [ctypes.c_void_p, _D]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_max_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
    return _lib


def source() -> str:
    """Text of olb_oracle.c."""
    with open(_SRC) as fh:
        return fh.read()


def load_variant(text: str, directory: str):
    """Compile a modified copy `text` of olb_oracle.c (single-threaded, same
    rounding flags) into `directory` and return the loaded library, for tests
    that plant a mistake in the oracle and check that a pin catches it.  Pass
    it to Oracle(..., library=...)."""
    src = os.path.join(directory, "variant.c")
    out = os.path.join(directory, "libvariant.so")
    with open(src, "w") as fh:
        fh.write(text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", out, src, "-lm"], check=True, capture_output=True)
    return _declare(ctypes.CDLL(out))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- pieces

def quadrature():
    R = np.zeros(5)
    W = np.zeros(5)
    lib().orc_quadrature(_p(R), _p(W))
    return R, W


def hermite(l: int, x: float) -> float:
    return lib().orc_hermite(int(l), float(x))


def g(k: int, u: float, T: float) -> float:
    return lib().orc_g(int(k), float(u), float(T))


def feq(n, ux, uy, T) -> np.ndarray:
    out = np.zeros(25)
    lib().orc_feq(float(n), float(ux), float(uy), float(T), _p(out))
    return out


def dp_line(line) -> np.ndarray:
    line = _f64(line)
    out = np.zeros(5)
    lib().orc_dp_line(_p(line), _p(out))
    return out


def moments_node(f25) -> np.ndarray:
    f25 = _f64(f25)
    out = np.zeros(4)
    lib().orc_moments_node(_p(f25), _p(out))
    return out


def pw(n, T, a, b) -> float:
    return lib().orc_pw(float(n), float(T), float(a), float(b))


def grad_stencil() -> np.ndarray:
    out = np.zeros(49)
    lib().orc_grad_stencil(_p(out))
    return out.reshape(7, 7)


def glap_stencil() -> np.ndarray:
    out = np.zeros(49)
    lib().orc_glap_stencil(_p(out))
    return out.reshape(7, 7)


def weno5(v, return_weights: bool = False):
    v = _f64(v)
    w = np.zeros(3)
    val = lib().orc_weno5(_p(v), _p(w))
    return (val, w) if return_weights else val


def weno5_learned(theta, v, return_weights: bool = False):
    theta = _f64(theta)
    v = _f64(v)
    w = np.zeros(3)
    val = lib().orc_weno5_learned(_p(theta), _p(v), _p(w))
    return (val, w) if return_weights else val


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------- solver

class Oracle:
    """FP64 reference solver: same semantics as the library's olb_* calls.

    Fields are [ny][nx] float64; populations are exchanged as [25][ny][nx]."""

    def __init__(self, nx, ny, ds, dt, tau, a=9.0 / 8.0, b=1.0 / 3.0,
                 sigma=1e-4, Tw=(1.0, 1.0), uw=(0.0, 0.0), side_x=0,
                 side_y=0, library=None):
        self._lib = library if library is not None else lib()
        self.nx, self.ny = int(nx), int(ny)
        p = OrcParams()
        p.nx, p.ny = self.nx, self.ny
        p.ds, p.dt, p.tau = float(ds), float(dt), float(tau)
        p.a, p.b, p.sigma = float(a), float(b), float(sigma)
        p.Tw[0], p.Tw[1] = float(Tw[0]), float(Tw[1])
        p.uw[0], p.uw[1] = float(uw[0]), float(uw[1])
        p.side_x, p.side_y = int(side_x), int(side_y)
        self._params = p
        h = self._lib.orc_create(ctypes.byref(p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self):
        return (self.ny, self.nx)

    def init_fields(self, n, ux, uy, T):
        arrs = [_f64(x).reshape(self._shape()) for x in (n, ux, uy, T)]
        self._lib.orc_init(self._h, *[_p(a) for a in arrs])

    def step(self, nsteps: int = 1):
        self._lib.orc_step(self._h, int(nsteps))

    def set_mlp(self, theta=None):
        """Learned WENO weights with parameters theta (None: Jiang-Shu)."""
        if theta is None:
            self._lib.orc_set_mlp(self._h, None)
        else:
            self._mlp = _f64(theta)
            self._lib.orc_set_mlp(self._h, _p(self._mlp))

    def moments(self):
        out = [np.zeros(self._shape()) for _ in range(4)]
        self._lib.orc_get_moments(self._h, *[_p(a) for a in out])
        return tuple(out)

    def get_populations(self) -> np.ndarray:
        out = np.zeros((25,) + self._shape())
        self._lib.orc_get_f(self._h, _p(out))
        return out

    def set_populations(self, f) -> None:
        f = _f64(f).reshape((25,) + self._shape())
        self._lib.orc_set_f(self._h, _p(f))

    def evaluate(self):
        """L[f] ([25][ny][nx]) and the stage fields of the current f:
        dict with n, ux, uy, T, dp, Fx, Fy ([ny][nx]) and nw ([2][ny])."""
        L = np.zeros((25,) + self._shape())
        f7 = np.zeros((7,) + self._shape())
        nw = np.zeros((2, self.ny))
        self._lib.orc_eval(self._h, _p(L), _p(f7), _p(nw))
        names = ("n", "ux", "uy", "T", "dp", "Fx", "Fy")
        out = {k: f7[i] for i, k in enumerate(names)}
        out["nw"] = nw
        out["L"] = L
        return out
