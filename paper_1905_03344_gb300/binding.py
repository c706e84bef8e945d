"""Python binding of the C ABI in include/sph.h (libsph_gb300.so).

Argument marshalling only: every step of the SPH timestep runs in the CUDA
kernels behind the C ABI.  Functions carry the names of the C entry points;
`SPH` is a small object wrapper over one context.  Device arrays are torch
CUDA tensors (float64 / int64 / int32, contiguous); host arrays are numpy.

The library must be built first (`python -m paper_1905_03344_gb300.build` or
`__graft_entry__.build()`); there is no CPU fallback: a missing library or a
missing GPU raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_EOVERFLOW, SPH_ENONFINITE, SPH_ETIMEOUT, SPH_ESTATE = range(8)
SPH_FP64, SPH_MIXED = 0, 1
SPH_KERNEL_WENDLAND, SPH_KERNEL_SINC = 0, 1
SPH_PAIRS_LISTS, SPH_PAIRS_FUSED, SPH_PAIRS_AUTO = 0, 1, 2
PAIR_MODES = {"lists": SPH_PAIRS_LISTS, "fused": SPH_PAIRS_FUSED, "auto": SPH_PAIRS_AUTO}

FIELDS = ["x", "y", "z", "vx", "vy", "vz", "m", "h", "u", "du_prev", "axp", "ayp", "azp",
          "rho", "P", "c", "ax", "ay", "az", "du", "nown", "nnb"]
FIELD = {k: i for i, k in enumerate(FIELDS)}
PHASES = ["bbox", "keys", "sort", "gather", "nb_reset", "nb", "density", "momentum", "update"]


class SphConfig(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("kernel", ctypes.c_int32), ("kernel_n", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("n_target", ctypes.c_double),
                ("courant", ctypes.c_double), ("dt_growth", ctypes.c_double),
                ("av_alpha", ctypes.c_double), ("av_beta", ctypes.c_double),
                ("av_eps", ctypes.c_double), ("lz", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("adapt_h", ctypes.c_int32), ("grad_h", ctypes.c_int32),
                ("threads_per_particle", ctypes.c_int32), ("pair_mode", ctypes.c_int32),
                ("cell_factor", ctypes.c_double), ("list_skin", ctypes.c_double),
                ("max_particles", ctypes.c_int64), ("max_pairs", ctypes.c_int64),
                ("max_patches", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("pair_bins", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p)]


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


STATUS_NAMES = {0: "SPH_OK", 1: "SPH_EINVAL", 2: "SPH_ENOMEM", 3: "SPH_ECUDA",
                4: "SPH_EOVERFLOW", 5: "SPH_ENONFINITE", 6: "SPH_ETIMEOUT", 7: "SPH_ESTATE"}

# exported symbols and their (restype, argtypes); the test suite checks this
# list against include/sph.h
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_ST = ctypes.c_int
SIGNATURES = {
    "sph_config_default": (None, [ctypes.POINTER(SphConfig)]),
    "sph_create": (_ST, [ctypes.POINTER(SphConfig), ctypes.POINTER(_P)]),
    "sph_destroy": (None, [_P]),
    "sph_last_error": (ctypes.c_char_p, [_P]),
    "sph_status_string": (ctypes.c_char_p, [_ST]),
    "sph_set_particles": (_ST, [_P, _I64] + [_P] * 9 + [ctypes.c_int]),
    "sph_set_patches": (_ST, [_P, _I32, _P]),
    "sph_find_neighbors": (_ST, [_P]),
    "sph_get_neighbors": (_ST, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                               ctypes.POINTER(_I64)]),
    "sph_copy_neighbors": (_ST, [_P, _P, _P, _P, ctypes.c_int]),
    "sph_density": (_ST, [_P]),
    "sph_momentum_energy": (_ST, [_P]),
    "sph_step": (_ST, [_P, _I32, ctypes.POINTER(_D)]),
    "sph_conserved": (_ST, [_P, _I32, _P]),
    "sph_get_field": (_ST, [_P, _I32, _P, ctypes.c_int]),
    "sph_get_dt": (_ST, [_P, _I32, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "sph_get_state": (_ST, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "sph_set_state": (_ST, [_P, _P, ctypes.c_size_t]),
    "sph_autotune": (_ST, [_P]),
    "sph_get_tuning": (_ST, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_D)]),
    "sph_get_pair_mode": (_ST, [_P, ctypes.POINTER(_I32)]),
    "sph_get_density_tpp": (_ST, [_P, ctypes.POINTER(_I32)]),
    "sph_get_pair_bins": (_ST, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "sph_get_list_rebuilds": (_ST, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "sph_set_profiling": (_ST, [_P, ctypes.c_int]),
    "sph_get_profile": (_ST, [_P, _P, _P, _I32]),
    "sph_get_launch_count": (_ST, [_P, ctypes.POINTER(_I64)]),
    "sph_get_nnz": (_ST, [_P, ctypes.POINTER(_I64)]),
    "sph_get_pair_count": (_ST, [_P, ctypes.POINTER(_I64), ctypes.c_int]),
    "sph_conserved_noalloc": (_ST, [_I64] + [_P] * 8 + [_P]),
    "sph_noalloc_last_error": (ctypes.c_char_p, []),
    "sph_fma_peak": (_ST, [_I32, _P, _P]),
    "sph_fma_peak_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path():
    return _build.LIB


def lib():
    """Loads libsph_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libsph_gb300.so is not built (%s); run __graft_entry__.build() or "
                              "python -m paper_1905_03344_gb300.build" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx, st):
    if st != SPH_OK:
        msg = lib().sph_last_error(ctx)
        raise SphError(st, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous)."""
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data), 0


# ---- entry points (same names as the C ABI) ---------------------------------
def sph_config_default():
    c = SphConfig()
    lib().sph_config_default(ctypes.byref(c))
    return c


def sph_create(cfg=None):
    if cfg is None:
        cfg = sph_config_default()
    h = ctypes.c_void_p()
    st = lib().sph_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != SPH_OK:
        raise SphError(st, lib().sph_last_error(None).decode())
    return h


def sph_destroy(ctx):
    lib().sph_destroy(ctx)


def _f64_buffer(a, n, what, exact=True):
    """Checks that a (a torch tensor or numpy array) is a contiguous float64
    buffer of n elements (at least n when exact is False), on the current
    device if it is a CUDA tensor; returns (pointer, on_device).  Nothing is
    passed to the library before these checks: a wrong dtype or length would
    let it read or write past the buffer."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64:
            raise ValueError("%s must be float64, not %s" % (what, a.dtype))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % what)
        size = a.numel()
        if a.is_cuda and a.device.index != torch.cuda.current_device():
            raise ValueError("%s is on cuda:%d, the current device is cuda:%d"
                             % (what, a.device.index, torch.cuda.current_device()))
    else:
        if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be a contiguous float64 array" % what)
        size = a.size
    if (size != n) if exact else (size < n):
        raise ValueError("%s has %d elements, %s %d expected" % (what, size, "" if exact else "at least", n))
    return _ptr(a)


def sph_set_particles(ctx, fields):
    """fields: dict with x y z vx vy vz m h u, each float64 of length n (all
    torch CUDA tensors on the current device, all host tensors, or array-likes
    converted to float64 numpy arrays)."""
    names = ["x", "y", "z", "vx", "vy", "vz", "m", "h", "u"]
    missing = [k for k in names if k not in fields]
    if missing:
        raise ValueError("sph_set_particles: missing fields %s" % missing)
    arrs = [fields[k] if hasattr(fields[k], "data_ptr") else np.ascontiguousarray(fields[k], dtype=np.float64)
            for k in names]
    n = len(arrs[0])
    ptrs = []
    dev = None
    for k, a in zip(names, arrs):
        p, d = _f64_buffer(a, n, "sph_set_particles: " + k)
        dev = d if dev is None else dev
        if d != dev:
            raise ValueError("sph_set_particles: fields must all be device tensors or all host buffers")
        ptrs.append(p)
    _check(ctx, lib().sph_set_particles(ctx, n, *ptrs, dev))


def sph_set_patches(ctx, offsets):
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(ctx, lib().sph_set_patches(ctx, len(o) - 1, ctypes.c_void_p(o.ctypes.data)))


def sph_find_neighbors(ctx):
    _check(ctx, lib().sph_find_neighbors(ctx))


def sph_get_nnz(ctx):
    v = ctypes.c_int64()
    _check(ctx, lib().sph_get_nnz(ctx, ctypes.byref(v)))
    return v.value


def sph_get_neighbors(ctx):
    """Borrowed device pointers (off, col, perm, nnz) as integers."""
    o, c, p = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    nnz = ctypes.c_int64()
    _check(ctx, lib().sph_get_neighbors(ctx, ctypes.byref(o), ctypes.byref(c), ctypes.byref(p),
                                        ctypes.byref(nnz)))
    return o.value, c.value, p.value, nnz.value


def sph_copy_neighbors(ctx, n, device=None):
    """(off int64[n+1], col int32[nnz], perm int32[n]) as torch tensors on
    `device`, or numpy arrays when device is None."""
    nnz = sph_get_nnz(ctx)
    if device is None:
        off = np.zeros(n + 1, dtype=np.uint64)
        col = np.zeros(max(nnz, 1), dtype=np.uint32)
        perm = np.zeros(max(n, 1), dtype=np.uint32)
        _check(ctx, lib().sph_copy_neighbors(ctx, ctypes.c_void_p(off.ctypes.data),
                                             ctypes.c_void_p(col.ctypes.data),
                                             ctypes.c_void_p(perm.ctypes.data), 0))
        return off.astype(np.int64), col[:nnz].astype(np.int64), perm[:n].astype(np.int64)
    import torch
    off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    col = torch.zeros(max(nnz, 1), dtype=torch.int32, device=device)
    perm = torch.zeros(max(n, 1), dtype=torch.int32, device=device)
    _check(ctx, lib().sph_copy_neighbors(ctx, ctypes.c_void_p(off.data_ptr()),
                                         ctypes.c_void_p(col.data_ptr()),
                                         ctypes.c_void_p(perm.data_ptr()), 1))
    return off, col[:nnz], perm[:n]


def sph_density(ctx):
    _check(ctx, lib().sph_density(ctx))


def sph_momentum_energy(ctx):
    _check(ctx, lib().sph_momentum_energy(ctx))


def sph_step(ctx, nsteps=1):
    dt = ctypes.c_double()
    _check(ctx, lib().sph_step(ctx, int(nsteps), ctypes.byref(dt)))
    return dt.value


def sph_conserved(ctx, patch=-1):
    out = np.zeros(7)
    _check(ctx, lib().sph_conserved(ctx, int(patch), ctypes.c_void_p(out.ctypes.data)))
    return out


def sph_get_field(ctx, field, n, out=None):
    """Field (name or SPH_FIELD_* index) in original order.  With out (a
    float64 torch CUDA tensor or numpy array of length n) fills it; otherwise
    returns a new numpy array."""
    f = FIELD[field] if isinstance(field, str) else int(field)
    if out is not None:
        p, d = _f64_buffer(out, n, "sph_get_field: out", exact=False)
        _check(ctx, lib().sph_get_field(ctx, f, p, d))
        return out
    res = np.zeros(max(n, 1))
    p, d = _ptr(res)
    _check(ctx, lib().sph_get_field(ctx, f, p, d))
    return res[:n]


def sph_get_dt(ctx, patch=0):
    dt, dtp, step = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(ctx, lib().sph_get_dt(ctx, int(patch), ctypes.byref(dt), ctypes.byref(dtp),
                                 ctypes.byref(step)))
    return dt.value, dtp.value, step.value


def sph_state_bytes(ctx):
    """Size of the checkpoint of the current state."""
    nb = ctypes.c_size_t()
    _check(ctx, lib().sph_get_state(ctx, None, ctypes.byref(nb)))
    return nb.value


def _host_buffer(buf):
    """(pointer, size in bytes) of a host uint8 buffer: a CPU torch tensor
    (pinned memory makes the copies fast) or a numpy array."""
    if hasattr(buf, "data_ptr"):
        if buf.is_cuda or not buf.is_contiguous():
            raise ValueError("state buffer: a contiguous host tensor")
        return ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()
    if not buf.flags["C_CONTIGUOUS"]:
        raise ValueError("state buffer: a contiguous array")
    return ctypes.c_void_p(buf.ctypes.data), buf.nbytes


def sph_get_state(ctx, out=None):
    """The checkpoint as bytes, or, with out (a host uint8 tensor or array of
    at least sph_state_bytes(ctx) bytes), written into out; returns its size
    then."""
    if out is not None:
        p, size = _host_buffer(out)
        nb = ctypes.c_size_t(size)
        _check(ctx, lib().sph_get_state(ctx, p, ctypes.byref(nb)))
        return nb.value
    nb = ctypes.c_size_t(sph_state_bytes(ctx))
    buf = ctypes.create_string_buffer(nb.value)
    _check(ctx, lib().sph_get_state(ctx, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(nb)))
    return buf.raw[: nb.value]


def sph_set_state(ctx, blob, nbytes=None):
    """Restores a checkpoint: bytes, or a host uint8 tensor or array holding
    nbytes (default: all of it) of one."""
    if isinstance(blob, (bytes, bytearray)):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(ctx, lib().sph_set_state(ctx, ctypes.cast(buf, ctypes.c_void_p), len(blob)))
        return
    p, size = _host_buffer(blob)
    _check(ctx, lib().sph_set_state(ctx, p, size if nbytes is None else int(nbytes)))


def sph_autotune(ctx):
    _check(ctx, lib().sph_autotune(ctx))


def sph_get_pair_mode(ctx):
    """"lists" or "fused": how the pair sums currently find their pairs."""
    m = ctypes.c_int32()
    _check(ctx, lib().sph_get_pair_mode(ctx, ctypes.byref(m)))
    return "fused" if m.value == SPH_PAIRS_FUSED else "lists"


def sph_get_pair_bins(ctx):
    """(density, momentum): list words per lane of the row-length bins of each
    pair sum, 0 where the sum runs with uniform lanes per particle."""
    d, m = ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, lib().sph_get_pair_bins(ctx, ctypes.byref(d), ctypes.byref(m)))
    return d.value, m.value


def sph_get_density_tpp(ctx):
    """Lanes per particle of the density sum."""
    v = ctypes.c_int32()
    _check(ctx, lib().sph_get_density_tpp(ctx, ctypes.byref(v)))
    return v.value


def sph_get_list_rebuilds(ctx):
    """Candidate supersets built so far (list_skin > 0)."""
    v = ctypes.c_int64()
    _check(ctx, lib().sph_get_list_rebuilds(ctx, ctypes.byref(v)))
    return v.value


def sph_get_tuning(ctx):
    t, f = ctypes.c_int32(), ctypes.c_double()
    _check(ctx, lib().sph_get_tuning(ctx, ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def sph_set_profiling(ctx, enable):
    _check(ctx, lib().sph_set_profiling(ctx, int(bool(enable))))


def sph_get_profile(ctx):
    ms = np.zeros(len(PHASES))
    ln = np.zeros(len(PHASES), dtype=np.int64)
    _check(ctx, lib().sph_get_profile(ctx, ctypes.c_void_p(ms.ctypes.data),
                                      ctypes.c_void_p(ln.ctypes.data), len(PHASES)))
    return {k: (float(ms[i]), int(ln[i])) for i, k in enumerate(PHASES)}


def sph_get_launch_count(ctx):
    v = ctypes.c_int64()
    _check(ctx, lib().sph_get_launch_count(ctx, ctypes.byref(v)))
    return v.value


def sph_get_pair_count(ctx, reset=False):
    v = ctypes.c_int64()
    _check(ctx, lib().sph_get_pair_count(ctx, ctypes.byref(v), int(bool(reset))))
    return v.value


def _noalloc_args(fields, out):
    """Checks the arguments of sph_conserved_noalloc without touching the
    device: seven float64 fields of one length n, a float64 out of at least 7
    elements, all contiguous CUDA tensors on the current device.  Returns the
    field tensors in the C ABI's order and n."""
    names = ["x", "y", "vx", "vy", "vz", "m", "u"]
    missing = [k for k in names if k not in fields]
    if missing:
        raise ValueError("sph_conserved_noalloc: missing fields %s" % missing)
    arrs = [fields[k] for k in names]
    import torch
    for k, a in zip(names + ["out"], arrs + [out]):
        if not isinstance(a, torch.Tensor):
            raise ValueError("sph_conserved_noalloc: %s must be a torch tensor" % k)
        if a.dtype != torch.float64:
            raise ValueError("sph_conserved_noalloc: %s must be float64, not %s" % (k, a.dtype))
    n = arrs[0].numel()
    for k, a in zip(names, arrs):
        if a.numel() != n:
            raise ValueError("sph_conserved_noalloc: %s has %d elements, x has %d" % (k, a.numel(), n))
    if out.numel() < 7:
        raise ValueError("sph_conserved_noalloc: out must hold 7 elements, it has %d" % out.numel())
    for k, a in zip(names + ["out"], arrs + [out]):
        if not (a.is_cuda and a.is_contiguous()):
            raise ValueError("sph_conserved_noalloc: %s must be a contiguous CUDA tensor" % k)
    dev = torch.cuda.current_device()
    for k, a in zip(names + ["out"], arrs + [out]):
        if a.device.index != dev:
            raise ValueError("sph_conserved_noalloc: %s is on cuda:%d, the current device is cuda:%d"
                             % (k, a.device.index, dev))
    return arrs, n


def sph_conserved_noalloc(fields, out, stream=None):
    """Conserved sums (M, Px, Py, Pz, Lz, Ekin, Eint) of device arrays without
    any allocation: fields holds x y vx vy vz m u as float64 CUDA tensors of
    equal length on the current device, out is a float64 CUDA tensor of at
    least 7 elements; asynchronous on stream (a CUDA stream handle or None).
    Calls whose kernels overlap on the GPU race on the library's one scratch
    array."""
    arrs, n = _noalloc_args(fields, out)
    st = lib().sph_conserved_noalloc(n, *[ctypes.c_void_p(a.data_ptr()) for a in arrs],
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream or 0))
    if st != SPH_OK:
        raise SphError(st, lib().sph_noalloc_last_error().decode())


def sph_fma_peak(precision="mixed", stream=None):
    """FP32 (precision "mixed") or FP64 ("fp64") fused multiply-add rate of the
    current device in FLOP/s, measured by the library's FMA-chain kernel."""
    v = ctypes.c_double()
    st = lib().sph_fma_peak(SPH_FP64 if precision == "fp64" else SPH_MIXED, ctypes.byref(v),
                            ctypes.c_void_p(stream or 0))
    if st != SPH_OK:
        raise SphError(st, lib().sph_fma_peak_last_error().decode())
    return v.value


# ---- object wrapper -----------------------------------------------------------
class SPH:
    """One library context.  Example::

        sim = SPH(max_particles=8000, precision="fp64")
        sim.set_particles(fields)          # dict of numpy arrays or CUDA tensors
        sim.step(10)
        rho = sim.field("rho")
    """

    def __init__(self, max_particles, precision="mixed", max_patches=1, stream=None, **kw):
        cfg = sph_config_default()
        cfg.precision = SPH_FP64 if precision == "fp64" else SPH_MIXED
        if isinstance(kw.get("kernel"), str):
            kw["kernel"] = {"wendland": SPH_KERNEL_WENDLAND, "sinc": SPH_KERNEL_SINC}[kw["kernel"]]
        if isinstance(kw.get("pair_mode"), str):
            kw["pair_mode"] = PAIR_MODES[kw["pair_mode"]]
        cfg.max_particles = int(max_particles)
        cfg.max_patches = int(max_patches)
        if stream is not None:
            cfg.cuda_stream = stream
        for k, v in kw.items():
            if not hasattr(cfg, k):
                raise TypeError("unknown config field %s" % k)
            setattr(cfg, k, v)
        self.cfg = cfg
        self.ctx = sph_create(cfg)
        self.n = 0

    def close(self):
        if self.ctx:
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, fields):
        sph_set_particles(self.ctx, fields)
        self.n = len(fields["x"])

    def set_patches(self, offsets):
        sph_set_patches(self.ctx, offsets)

    def find_neighbors(self):
        sph_find_neighbors(self.ctx)

    def neighbors(self, device=None):
        return sph_copy_neighbors(self.ctx, self.n, device)

    def density(self):
        sph_density(self.ctx)

    def momentum_energy(self):
        sph_momentum_energy(self.ctx)

    def step(self, nsteps=1):
        return sph_step(self.ctx, nsteps)

    def conserved(self, patch=-1):
        return sph_conserved(self.ctx, patch)

    def field(self, name, out=None):
        return sph_get_field(self.ctx, name, self.n, out)

    def dt(self, patch=0):
        return sph_get_dt(self.ctx, patch)

    def get_state(self, out=None):
        return sph_get_state(self.ctx, out)

    def state_bytes(self):
        return sph_state_bytes(self.ctx)

    def set_state(self, blob, nbytes=None):
        sph_set_state(self.ctx, blob, nbytes)
        import struct
        if isinstance(blob, (bytes, bytearray)):
            head = bytes(blob[:24])
        elif hasattr(blob, "numpy"):
            head = blob[:24].numpy().tobytes()
        else:
            head = blob[:24].tobytes()
        self.n = struct.unpack_from("<q", head, 16)[0]

    def autotune(self):
        sph_autotune(self.ctx)
        return sph_get_tuning(self.ctx)

    def pair_mode(self):
        return sph_get_pair_mode(self.ctx)

    def pair_bins(self):
        return sph_get_pair_bins(self.ctx)

    def list_rebuilds(self):
        return sph_get_list_rebuilds(self.ctx)

    def profile(self, enable=None):
        if enable is not None:
            sph_set_profiling(self.ctx, enable)
            return None
        return sph_get_profile(self.ctx)

    def launches(self):
        return sph_get_launch_count(self.ctx)

    def pair_count(self, reset=False):
        return sph_get_pair_count(self.ctx, reset)
