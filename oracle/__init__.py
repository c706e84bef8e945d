"""FP64 CPU oracle of the SPH timestep (arXiv 1905.03344, Sec. 3).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this package.  The CUDA library and
its binding never do, and this package never imports them.

Thin ctypes wrappers over sph_oracle.c; every array is float64 (int64/int32
for lists) and C-contiguous.  See sph_oracle.c for the formulas and the
readings (R1..R18) each function follows.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)


class OrcParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("n_target", ctypes.c_double),
                ("courant", ctypes.c_double), ("dt_growth", ctypes.c_double),
                ("av_alpha", ctypes.c_double), ("av_beta", ctypes.c_double),
                ("av_eps", ctypes.c_double), ("lz", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("adapt_h", ctypes.c_int32),
                ("use_grid", ctypes.c_int32), ("grad_h", ctypes.c_int32), ("pad", ctypes.c_int32)]


class OrcState(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(k, _D) for k in (
        "x", "y", "z", "vx", "vy", "vz", "m", "h", "u", "du_prev", "axp", "ayp", "azp",
        "rho", "P", "c", "ax", "ay", "az", "du")] + [
        ("nown", _I32), ("nnz", ctypes.c_int64), ("dt", ctypes.c_double),
        ("dt_prev", ctypes.c_double), ("step", ctypes.c_int64)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_sigma_w.restype = ctypes.c_double
        L.orc_w.restype = ctypes.c_double
        L.orc_w.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_gradw_fac.restype = ctypes.c_double
        L.orc_gradw_fac.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_pair_in.restype = ctypes.c_int
        L.orc_pair_in.argtypes = [ctypes.c_double] * 9
        for name in ("orc_neighbors_brute", "orc_neighbors_grid"):
            f = getattr(L, name)
            f.restype = ctypes.c_int64
            f.argtypes = [ctypes.c_int64, _D, _D, _D, _D, ctypes.c_double, _I64, _I32, _I32,
                          ctypes.c_int64, ctypes.c_int]
        L.orc_density.restype = None
        L.orc_density.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_double, _I64, _I32,
                                  _D, ctypes.c_int]
        L.orc_eos.restype = None
        L.orc_eos.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _D, _D]
        L.orc_momentum_energy.restype = None
        L.orc_momentum_energy.argtypes = ([ctypes.c_int64] + [_D] * 11 +
                                          [ctypes.c_double] * 4 + [_I64, _I32] + [_D] * 7 +
                                          [ctypes.c_int])
        L.orc_omega.restype = None
        L.orc_omega.argtypes = [ctypes.c_int64] + [_D] * 6 + [ctypes.c_double, _I64, _I32, _D, ctypes.c_int]
        L.orc_dwdh.restype = ctypes.c_double
        L.orc_dwdh.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_courant.restype = ctypes.c_double
        L.orc_courant.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double]
        L.orc_conserved.restype = None
        L.orc_conserved.argtypes = [ctypes.c_int64] + [_D] * 8
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.POINTER(OrcParams), ctypes.POINTER(OrcState), ctypes.c_int]
        L.orc_set_kernel.restype = ctypes.c_int
        L.orc_set_kernel.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_sinc_bn.restype = ctypes.c_double
        L.orc_sinc_bn.argtypes = [ctypes.c_int]
        L.orc_kernel_bn.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sigma_w():
    return lib().orc_sigma_w()


KERNELS = {"wendland": 0, "sinc": 1}


def set_kernel(kind="wendland", n=6):
    """Selects the kernel of every later call: "wendland" (Eq. 2) or "sinc"
    with index n (the Sinc family of Sec. 3)."""
    if lib().orc_set_kernel(KERNELS[kind], int(n)) != 0:
        raise ValueError("unsupported kernel %s/%d" % (kind, n))


class kernel:
    """with oracle.kernel("sinc", 6): ... -- the kernel for the block, then Wendland."""

    def __init__(self, kind="wendland", n=6):
        self.kind, self.n = kind, n

    def __enter__(self):
        set_kernel(self.kind, self.n)
        return self

    def __exit__(self, *exc):
        set_kernel("wendland")
        return False


def sinc_bn(n):
    """B_n of the Sinc kernel (normalisation by composite Simpson)."""
    return lib().orc_sinc_bn(int(n))


def w(r, h):
    """Wendland kernel value (Eq. 2 with 1/h^3), scalar."""
    return lib().orc_w(float(r), float(h))


def gradw_fac(r, h):
    """f with grad_i W(r_ij, h) = -f (x_i - x_j), scalar."""
    return lib().orc_gradw_fac(float(r), float(h))


def pair_in(pi, pj, hi, hj, lz=1.0):
    """(in N(i), r^2 < 4 h_i^2) for two points, exact FP64 predicate."""
    f = lib().orc_pair_in(float(pi[0]), float(pi[1]), float(pi[2]), float(hi),
                          float(pj[0]), float(pj[1]), float(pj[2]), float(hj), float(lz))
    return bool(f & 1), bool(f & 2)


@dataclass
class Neighbors:
    off: np.ndarray   # int64[n+1]
    col: np.ndarray   # int32[nnz], ascending within each row
    nown: np.ndarray  # int32[n], n_i = #{j : r^2 < 4 h_i^2}

    def rows(self):
        return [self.col[self.off[i]:self.off[i + 1]] for i in range(len(self.off) - 1)]


def neighbors(x, y, z, h, lz=1.0, method="auto", nthreads=1):
    x, y, z, h = map(_f64, (x, y, z, h))
    n = len(x)
    if method == "auto":
        method = "grid" if n > 5000 else "brute"
    f = lib().orc_neighbors_grid if method == "grid" else lib().orc_neighbors_brute
    off = np.zeros(n + 1, dtype=np.int64)
    nown = np.zeros(max(n, 1), dtype=np.int32)
    nnz = f(n, _d(x), _d(y), _d(z), _d(h), lz, off.ctypes.data_as(_I64), None,
            nown.ctypes.data_as(_I32), 0, nthreads)
    if nnz < 0:
        raise RuntimeError("oracle neighbour count failed (%d)" % nnz)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    r = f(n, _d(x), _d(y), _d(z), _d(h), lz, off.ctypes.data_as(_I64), col.ctypes.data_as(_I32),
          nown.ctypes.data_as(_I32), nnz, nthreads)
    if r != nnz:
        raise RuntimeError("oracle neighbour fill failed (%d)" % r)
    return Neighbors(off, col[:nnz], nown[:n])


def density(x, y, z, m, h, nb, lz=1.0, nthreads=1):
    x, y, z, m, h = map(_f64, (x, y, z, m, h))
    rho = np.zeros(len(x))
    lib().orc_density(len(x), _d(x), _d(y), _d(z), _d(m), _d(h), lz,
                      nb.off.ctypes.data_as(_I64), nb.col.ctypes.data_as(_I32), _d(rho), nthreads)
    return rho


def eos(rho, u, gamma=5.0 / 3.0):
    rho, u = _f64(rho), _f64(u)
    P = np.zeros(len(rho))
    c = np.zeros(len(rho))
    lib().orc_eos(len(rho), _d(rho), _d(u), gamma, _d(P), _d(c))
    return P, c


def momentum_energy(x, y, z, vx, vy, vz, m, h, rho, P, c, nb, lz=1.0, alpha=1.0, beta=2.0,
                    eps=0.01, nthreads=1, omega=None):
    """Returns (ax, ay, az, du, sa, sdu); sa/sdu are the term-magnitude sums.
    With omega (from omega()), the grad-h form (R20)."""
    arrs = list(map(_f64, (x, y, z, vx, vy, vz, m, h, rho, P, c)))
    n = len(arrs[0])
    outs = [np.zeros(n) for _ in range(6)]
    om = _f64(omega) if omega is not None else None
    lib().orc_momentum_energy(n, *[_d(a) for a in arrs], lz, alpha, beta, eps,
                              nb.off.ctypes.data_as(_I64), nb.col.ctypes.data_as(_I32),
                              _d(om) if om is not None else None,
                              *[_d(o) for o in outs], nthreads)
    return tuple(outs)


def omega(x, y, z, m, h, rho, nb, lz=1.0, nthreads=1):
    """Grad-h factor Omega_i = 1 + h_i/(3 rho_i) sum_j m_j dW_ij(h_i)/dh_i (R20)."""
    arrs = list(map(_f64, (x, y, z, m, h, rho)))
    n = len(arrs[0])
    out = np.zeros(n)
    lib().orc_omega(n, *[_d(a) for a in arrs], lz, nb.off.ctypes.data_as(_I64),
                    nb.col.ctypes.data_as(_I32), _d(out), nthreads)
    return out


def dwdh(r, h):
    """dW/dh at fixed r for the current kernel."""
    return lib().orc_dwdh(float(r), float(h))


def courant(h, c, C=0.2):
    h, c = _f64(h), _f64(c)
    return lib().orc_courant(len(h), _d(h), _d(c), C)


def conserved(x, y, vx, vy, vz, m, u):
    """(M, Px, Py, Pz, Lz, Ekin, Eint), compensated FP64 sums."""
    arrs = list(map(_f64, (x, y, vx, vy, vz, m, u)))
    out = np.zeros(7)
    lib().orc_conserved(len(arrs[0]), *[_d(a) for a in arrs], _d(out))
    return out


STATE_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "m", "h", "u", "du_prev", "axp", "ayp", "azp")
OUT_FIELDS = ("rho", "P", "c", "ax", "ay", "az", "du")


class Sim:
    """Oracle simulation state; step() advances one timestep in place."""

    def __init__(self, fields, gamma=5.0 / 3.0, n_target=100.0, courant=0.2, dt_growth=1.1,
                 av_alpha=1.0, av_beta=2.0, av_eps=0.01, lz=1.0, adapt_h=True, dt_fixed=0.0,
                 use_grid=-1, nthreads=1, kernel="wendland", kernel_n=6, grad_h=False):
        n = len(fields["x"])
        self.n = n
        self.arr = {}
        for k in STATE_FIELDS:
            if k in ("du_prev", "axp", "ayp", "azp"):
                self.arr[k] = _f64(fields.get(k, np.zeros(n))).copy()
            else:
                self.arr[k] = _f64(fields[k]).copy()
        for k in OUT_FIELDS:
            self.arr[k] = np.zeros(n)
        self.arr["nown"] = np.zeros(max(n, 1), dtype=np.int32)
        self.params = OrcParams(gamma, n_target, courant, dt_growth, av_alpha, av_beta, av_eps,
                                lz, dt_fixed, int(bool(adapt_h)), int(use_grid), int(bool(grad_h)), 0)
        self.st = OrcState()
        self.st.n = n
        for k in STATE_FIELDS + OUT_FIELDS:
            setattr(self.st, k, _d(self.arr[k]))
        self.st.nown = self.arr["nown"].ctypes.data_as(_I32)
        self.st.nnz = 0
        self.st.dt = 0.0
        self.st.dt_prev = 0.0
        self.st.step = 0
        self.nthreads = nthreads
        self.kernel = (kernel, kernel_n)

    def step(self, nsteps=1):
        with kernel(*self.kernel):
            for _ in range(nsteps):
                r = lib().orc_step(ctypes.byref(self.params), ctypes.byref(self.st), self.nthreads)
                if r != 0:
                    raise RuntimeError("oracle step failed")
        return self

    def __getitem__(self, k):
        if k == "nown":
            return self.arr["nown"][: self.n]
        return self.arr[k]

    @property
    def dt(self):
        return self.st.dt

    @property
    def step_count(self):
        return self.st.step

    @property
    def nnz(self):
        return self.st.nnz

    def conserved(self):
        a = self.arr
        return conserved(a["x"], a["y"], a["vx"], a["vy"], a["vz"], a["m"], a["u"])


def omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or os.cpu_count() or 1
