"""Seeded synthetic inputs: the rotating square patch of Sec. 4 and its variants.

This module only builds particle arrays (numpy, float64).  It holds none of the
timestep's arithmetic and imports neither the CUDA library nor the oracle, so
both can be fed the same inputs.

Square patch (Sec. 4, Eq. 3 and the pressure series that follows it):
  * a 2D layer of n x n particles, copied n times along z, periodic in z;
    lattice positions -1/2 + (i + 1/2)/n per axis (reading R14);
  * rigid rotation v_x = omega y, v_y = -omega x, omega = 5 (Eq. 3);
  * initial pressure from the incompressible Poisson solution, summed over odd
    m, n only (the printed m, n = 0 terms divide by zero), second sine taken
    in y, coordinates measured from the patch corner, truncated at
    m, n <= 199 (reading R12);
  * a constant offset P_off = rho0 c0^2 / gamma with c0 = 10 omega L / sqrt(2)
    keeps the pressure positive (reading R13); u = P / ((gamma - 1) rho0);
  * m = rho0 / n^3, h0 = eta dx with eta = (3*100/(4 pi))^(1/3) / 2, i.e. 100
    lattice neighbours inside 2h (reading R14).
"""
import math

import numpy as np

ETA = 0.5 * (3.0 * 100.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
GAMMA = 5.0 / 3.0


def pressure_series(x, y, omega=5.0, rho0=1.0, L=1.0, nmax=199):
    """P0(x, y) of the rotating square patch, zero on the patch edges.

    P0 = rho sum_{m,n odd} -32 omega^2 / (m n pi^2 [(m pi/L)^2 + (n pi/L)^2])
         * sin(m pi x*/L) sin(n pi y*/L),   x* = x + L/2, y* = y + L/2.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    k = np.arange(1, nmax + 1, 2, dtype=np.float64)          # odd m, n
    coef = -32.0 * omega ** 2 / (np.outer(k, k) * math.pi ** 2 *
                                 ((k[:, None] * math.pi / L) ** 2 + (k[None, :] * math.pi / L) ** 2))
    out = np.empty(np.broadcast(x, y).shape)
    xf, yf, of = np.broadcast_to(x, out.shape).ravel(), np.broadcast_to(y, out.shape).ravel(), out.ravel()
    chunk = 1 << 16
    for s in range(0, xf.size, chunk):
        sx = np.sin(np.outer(xf[s:s + chunk] + 0.5 * L, k) * (math.pi / L))
        sy = np.sin(np.outer(yf[s:s + chunk] + 0.5 * L, k) * (math.pi / L))
        of[s:s + chunk] = np.einsum("pm,mn,pn->p", sx, coef, sy, optimize=True)
    return rho0 * out


def pressure_offset(omega=5.0, rho0=1.0, L=1.0, gamma=GAMMA):
    """P_off = rho0 c0^2 / gamma, c0 = 10 omega L / sqrt(2) (reading R13)."""
    c0 = 10.0 * omega * L / math.sqrt(2.0)
    return rho0 * c0 * c0 / gamma


def lattice_1d(n, L=1.0):
    return -0.5 * L + (np.arange(n, dtype=np.float64) + 0.5) * (L / n)


def square_patch(n, omega=5.0, rho0=1.0, L=1.0, gamma=GAMMA, nmax=199):
    """n^3 particles; x fastest, then y, then z.  Returns a dict of float64 arrays."""
    g = lattice_1d(n, L)
    dx = L / n
    # the initial state depends on (x, y) only: evaluate the series on one layer
    X2, Y2 = np.meshgrid(g, g, indexing="xy")                 # [iy, ix]
    P2 = pressure_series(X2, Y2, omega, rho0, L, nmax) + pressure_offset(omega, rho0, L, gamma)
    x = np.tile(X2.ravel(), n)
    y = np.tile(Y2.ravel(), n)
    z = np.repeat(g, n * n)
    P = np.tile(P2.ravel(), n)
    N = n ** 3
    return {
        "x": x, "y": y, "z": z,
        "vx": omega * y, "vy": -omega * x, "vz": np.zeros(N),
        "m": np.full(N, rho0 * L ** 3 / N),
        "h": np.full(N, ETA * dx),
        "u": P / ((gamma - 1.0) * rho0),
    }


def irregular_patch(n=159, sigma=0.3, mass_sigma=0.5, omega=5.0, rho0=1.0, L=1.0, gamma=GAMMA,
                    seed_pos=1, seed_mass=2, nmax=199):
    """Jittered lattice with log-normal masses (neighbour counts spread ~50-400).

    positions += N(0, (sigma dx)^2) per axis (seed_pos), z wrapped into
    [-1/2, 1/2); m = m0 exp(N(0, mass_sigma^2)) (seed_mass);
    h = h0 (m/m0)^(1/3); velocity and pressure from the patch formulas at the
    jittered positions.
    """
    g = lattice_1d(n, L)
    dx = L / n
    N = n ** 3
    x = np.tile(np.tile(g, n), n)
    y = np.tile(np.repeat(g, n), n)
    z = np.repeat(g, n * n)
    rng = np.random.default_rng(seed_pos)
    x = x + rng.normal(0.0, sigma * dx, N)
    y = y + rng.normal(0.0, sigma * dx, N)
    z = z + rng.normal(0.0, sigma * dx, N)
    z = z - L * np.floor(z / L + 0.5)
    z[z >= 0.5 * L] -= L
    m0 = rho0 * L ** 3 / N
    m = m0 * np.exp(np.random.default_rng(seed_mass).normal(0.0, mass_sigma, N))
    h = ETA * dx * (m / m0) ** (1.0 / 3.0)
    P = pressure_series(x, y, omega, rho0, L, nmax) + pressure_offset(omega, rho0, L, gamma)
    return {"x": x, "y": y, "z": z, "vx": omega * y, "vy": -omega * x, "vz": np.zeros(N),
            "m": m, "h": h, "u": P / ((gamma - 1.0) * rho0)}


def batch_patches(count=64, lo=10, hi=60, wlo=2.0, whi=8.0, seed=0, nmax=199):
    """Independent square patches, each in its own unit box.

    edges = rng.integers(lo, hi + 1, count), omega = rng.uniform(wlo, whi, count)
    with rng = default_rng(seed).  Returns (fields, offsets[count+1], edges, omegas).
    """
    rng = np.random.default_rng(seed)
    edges = rng.integers(lo, hi + 1, count)
    omegas = rng.uniform(wlo, whi, count)
    parts = [square_patch(int(e), float(w), nmax=nmax) for e, w in zip(edges, omegas)]
    fields = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    offsets = np.zeros(count + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([int(e) ** 3 for e in edges])
    return fields, offsets, edges, omegas


def random_cloud(n, seed=0, box=1.0, h_lo=0.04, h_hi=0.09, vscale=1.0, u_lo=1.0, u_hi=2.0,
                 lz=1.0):
    """Uniform random positions (z in [-lz/2, lz/2)), random h, v, m, u.

    Used by the tests for states where the artificial viscosity is active and
    neighbour sets are irregular.
    """
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5 * box, 0.5 * box, n)
    y = rng.uniform(-0.5 * box, 0.5 * box, n)
    z = rng.uniform(-0.5 * lz, 0.5 * lz, n)
    return {"x": x, "y": y, "z": z,
            "vx": rng.normal(0, vscale, n), "vy": rng.normal(0, vscale, n),
            "vz": rng.normal(0, vscale, n),
            "m": rng.uniform(0.5, 1.5, n) / max(n, 1), "h": rng.uniform(h_lo, h_hi, n),
            "u": rng.uniform(u_lo, u_hi, n)}


def config_patch(name):
    """Named workloads: 'c1' 20^3, 'c2' 100^3, 'c3' 200^3, 'c5' irregular 159^3."""
    name = name.lower()
    if name == "c1":
        return square_patch(20)
    if name == "c2":
        return square_patch(100)
    if name == "c3":
        return square_patch(200)
    if name == "c5":
        return irregular_patch(159)
    raise ValueError(name)
