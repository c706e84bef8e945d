"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
put its outputs in the oracle's layout.  Imports nothing from oracle/."""
import numpy as np


def lists_to_original(off, col, perm, n):
    """CSR in sorted order (rows = sorted particles, cols = sorted indices)
    -> CSR in original order with ascending columns (the oracle's layout)."""
    off = np.asarray(off, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    perm = np.asarray(perm, dtype=np.int64)
    counts = np.diff(off)
    row_o = np.repeat(perm[:n], counts)
    col_o = perm[col] if len(col) else col
    order = np.lexsort((col_o, row_o))
    off_o = np.zeros(n + 1, dtype=np.int64)
    off_o[1:] = np.cumsum(np.bincount(row_o, minlength=n))
    return off_o, col_o[order].astype(np.int32)


def normwise(g, o):
    """max_i |g - o| / max_i |o| (the tolerance norm of reading R16)."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    d = np.abs(o).max()
    return float(np.abs(g - o).max() / d) if d > 0 else float(np.abs(g - o).max())


def normwise_vec(g3, o3):
    """Vector field: max over components of max_i |g - o| / max_i |o_i| (Euclidean
    magnitude).  A component that vanishes by symmetry (a_z, v_z on the
    z-periodic patch) is rounding noise on both sides; it is measured against
    the field's magnitude, not against its own noise."""
    G = np.stack([np.asarray(a, dtype=np.float64) for a in g3])
    O = np.stack([np.asarray(a, dtype=np.float64) for a in o3])
    d = np.sqrt((O ** 2).sum(axis=0)).max()
    e = np.abs(G - O).max()
    return float(e / d) if d > 0 else float(e)


def scaled(g, o, scale):
    """max_i |g - o| / scale_i, scale = the sum of the term magnitudes."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    s = np.maximum(np.asarray(scale, dtype=np.float64), 1e-300)
    return float((np.abs(g - o) / s).max())


def zdist(a, b, lz=1.0):
    d = np.asarray(a) - np.asarray(b)
    return np.abs(d - lz * np.round(d / lz))


CONSERVED = ("M", "Px", "Py", "Pz", "Lz", "Ekin", "Eint")


def conserved_scales(x, y, vx, vy, vz, m, u):
    """For each of the 7 conserved sums (M, P, L_z, E_kin, E_int), the sum of
    its terms' magnitudes: the natural scale of its rounding error (P of the
    square patch is zero by symmetry, so a relative error of P itself is
    undefined).  The components of P share the scale sum m |v| (the vector's
    magnitude, as for vector fields in the tolerance norm): v_z of the
    z-periodic patch is itself rounding noise."""
    x, y, vx, vy, vz, m, u = (np.asarray(a, dtype=np.float64) for a in (x, y, vx, vy, vz, m, u))
    pv = (m * np.sqrt(vx * vx + vy * vy + vz * vz)).sum()
    return np.array([m.sum(), pv, pv, pv,
                     (m * (np.abs(x * vy) + np.abs(y * vx))).sum(),
                     (0.5 * m * (vx * vx + vy * vy + vz * vz)).sum(), (m * np.abs(u)).sum()])


def conserved_errors(g, o, scales):
    """{name: |g - o| / scale} for the 7 conserved sums."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    return {k: float(abs(g[q] - o[q]) / max(scales[q], 1e-300)) for q, k in enumerate(CONSERVED)}
