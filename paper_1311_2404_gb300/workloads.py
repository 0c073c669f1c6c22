"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: geometry masks and initial
macroscopic fields.  It contains none of the lattice Boltzmann arithmetic and
imports neither the CUDA binding nor the CPU oracle, so both sides can be fed
identical inputs from it.

Seeds follow one convention: NumPy PCG64(1311) for geometry, PCG64(2404) for
turbulence phases, PCG64(512) for the batched ensemble.

All arrays are C-ordered with x fastest: scalar fields [nz, ny, nx], vector
fields [D, nz, ny, nx], masks uint8 [nz, ny, nx] with 0 = fluid, 1 = solid.
"""
from __future__ import annotations

import math
import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# Taylor-Green vortex (Sec. 3.7, Eq. taylor_green)
# --------------------------------------------------------------------------
def taylor_green(n: int, u0: float = 0.05, nz: int | None = None, rho0: float = 1.0,
                 D: int = 3):
    """2D Taylor-Green vortex with wavenumber k = 2 pi / n on an n x n plane,
    extruded along z (nz planes; D = 2 gives nz = 1).

        u_x = -u0 cos(kx) sin(ky),   u_y = u0 sin(kx) cos(ky),   u_z = 0
        p   = -(rho0 u0^2 / 4)(cos 2kx + cos 2ky),   rho = rho0 + 3 p

    (the pressure line of Eq. taylor_green is garbled in print; this is the
    incompressible Navier-Stokes pressure of the printed velocity field, with
    rho = rho0 + p / c_s^2, c_s^2 = 1/3).  Returns (rho, u) in float64."""
    if D == 2:
        nz = 1
    elif nz is None:
        nz = n
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")      # [ny, nx]
    ux = -u0 * np.cos(k * X) * np.sin(k * Y)
    uy = u0 * np.sin(k * X) * np.cos(k * Y)
    p = -(rho0 * u0 * u0 / 4.0) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho2 = rho0 + 3.0 * p
    rho = np.broadcast_to(rho2, (nz, n, n)).copy()
    u = np.zeros((D, nz, n, n))
    u[0] = ux
    u[1] = uy
    return rho, u


# --------------------------------------------------------------------------
# Channels
# --------------------------------------------------------------------------
def channel_mask(nx: int, ny: int, nz: int = 1) -> np.ndarray:
    """Solid rows y = 0 and y = ny - 1 (periodic in x, and in z when nz > 1)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[:, 0, :] = 1
    m[:, ny - 1, :] = 1
    return m


def duct_with_spheres(nx: int = 512, ny: int = 256, nz: int = 256,
                      solid_fraction: float = 0.20, rmin: float = 4.0,
                      rmax: float = 12.0, seed: int = 1311):
    """Duct periodic in x (streamwise) with one-node solid walls on the y and
    z faces, filled with random spheres (radius ~ U[rmin, rmax], centre ~
    U(box), overlaps allowed) until the solid voxel fraction, walls included,
    reaches solid_fraction.  A node is solid when |x - c| <= r (periodic in x).
    Returns (mask, n_spheres)."""
    rng = _rng(seed)
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    m[:, 0, :] = 1
    m[:, ny - 1, :] = 1
    m[0, :, :] = 1
    m[nz - 1, :, :] = 1
    total = m.size
    nsolid = int(m.sum(dtype=np.int64))
    nsph = 0
    while nsolid < solid_fraction * total:
        r = rng.uniform(rmin, rmax)
        c = rng.uniform((0.0, 0.0, 0.0), (nx, ny, nz))
        ri = int(math.ceil(r))
        zs = np.arange(max(0, int(c[2]) - ri), min(nz, int(c[2]) + ri + 2))
        ys = np.arange(max(0, int(c[1]) - ri), min(ny, int(c[1]) + ri + 2))
        xs = np.arange(int(c[0]) - ri, int(c[0]) + ri + 2)
        dz = (zs - c[2])[:, None, None]
        dy = (ys - c[1])[None, :, None]
        dx = (xs - c[0])[None, None, :]
        inside = (dx * dx + dy * dy + dz * dz) <= r * r
        xw = np.mod(xs, nx)
        sub = m[np.ix_(zs, ys, xw)]
        newly = inside & (sub == 0)
        nsolid += int(newly.sum())
        sub[inside] = 1
        m[np.ix_(zs, ys, xw)] = sub
        nsph += 1
    return m, nsph


# --------------------------------------------------------------------------
# Decaying turbulence initial field
# --------------------------------------------------------------------------
def turbulence(n: int = 256, k0: float = 4.0, u_rms: float = 0.04, seed: int = 2404):
    """Random-phase solenoidal velocity on a periodic n^3 box with energy
    spectrum E(k) ~ k^4 exp(-2 (k/k0)^2): white noise filtered by
    sqrt(E(k) / (4 pi k^2)) (Nyquist modes dropped), projected onto
    divergence-free fields, scaled so
    that the per-component rms sqrt(<|u|^2>/3) equals u_rms.  rho = 1.
    Returns (rho, u) in float64."""
    rng = _rng(seed)
    kk = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(kk, kk, np.fft.rfftfreq(n, d=1.0 / n) * 1.0, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    kmag = np.sqrt(k2)
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = np.where(k2 > 0, np.sqrt(kmag ** 4 * np.exp(-2.0 * (kmag / k0) ** 2)
                                       / (4 * np.pi * k2)), 0.0)
    # drop the Nyquist planes, whose real-valued modes cannot hold a projected
    # (complex) solenoidal component
    half = n // 2
    amp[(np.abs(kx) == half) | (np.abs(ky) == half) | (np.abs(kz) == half)] = 0.0
    uh = []
    for _ in range(3):
        w = rng.standard_normal((n, n, n))
        uh.append(np.fft.rfftn(w) * amp)
    with np.errstate(divide="ignore", invalid="ignore"):
        kdotu = (kx * uh[0] + ky * uh[1] + kz * uh[2]) / np.where(k2 > 0, k2, 1.0)
    uh = [uh[0] - kx * kdotu, uh[1] - ky * kdotu, uh[2] - kz * kdotu]
    u = np.stack([np.fft.irfftn(c, s=(n, n, n), axes=(0, 1, 2)) for c in uh])   # [3, z, y, x]
    u -= u.mean(axis=(1, 2, 3), keepdims=True)
    rms = math.sqrt(float((u * u).sum(axis=0).mean()) / 3.0)
    u *= u_rms / rms
    rho = np.ones((n, n, n))
    return rho, u


# --------------------------------------------------------------------------
# Lid-driven cavity (Sec. 5.1 validation; the benchmark shape of Sec. 4)
# --------------------------------------------------------------------------
def ldc_mask(n: int = 254, D: int = 3) -> np.ndarray:
    """Cubic (square for D = 2) cavity of n nodes per side: solid walls
    (mask 1) on every face except the top (y = n - 1), whose interior nodes
    are boundary nodes of condition 0 (mask 2), the moving lid; the lid's
    edge nodes belong to the side walls.  [nz, ny, nx] uint8."""
    nz = n if D == 3 else 1
    m = np.zeros((nz, n, n), dtype=np.uint8)
    m[:, :, 0] = 1
    m[:, :, n - 1] = 1
    m[:, 0, :] = 1
    if D == 3:
        m[0] = 1
        m[n - 1] = 1
    lid = m[:, n - 1, :]
    lid[lid == 0] = 2
    return m


def ldc_tau(n: int, re: float = 1000.0, u_lid: float = 0.05) -> float:
    """Relaxation time for Re = u_lid L / nu, L = n - 2 fluid nodes across."""
    return 0.5 + 3.0 * u_lid * (n - 2) / re


# --------------------------------------------------------------------------
# Kida vortex (Sec. 5.2)
# --------------------------------------------------------------------------
def kida(n: int = 256, u0: float = 0.05, rho0: float = 1.0):
    """Kida's initial field on an n^3 periodic box of face 2 pi (node i at
    x = 2 pi i / n):

        u_x = u0 sin x (cos 3y cos z - cos y cos 3z)
        u_y = u0 sin y (cos 3z cos x - cos z cos 3x)
        u_z = u0 sin z (cos 3x cos y - cos x cos 3y)

    with uniform density rho0 (the free decay starts from this velocity field;
    Sec. 5.2 runs it at u0 = 0.05).  Returns (rho [n,n,n], u [3,n,n,n]) in
    float64."""
    c = 2.0 * math.pi * np.arange(n) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u = np.empty((3, n, n, n))
    u[0] = u0 * np.sin(x) * (np.cos(3 * y) * np.cos(z) - np.cos(y) * np.cos(3 * z))
    u[1] = u0 * np.sin(y) * (np.cos(3 * z) * np.cos(x) - np.cos(z) * np.cos(3 * x))
    u[2] = u0 * np.sin(z) * (np.cos(3 * x) * np.cos(y) - np.cos(x) * np.cos(3 * y))
    return np.full((n, n, n), rho0), u


# --------------------------------------------------------------------------
# Batched ensemble of D2Q9 channels with a cylinder
# --------------------------------------------------------------------------
def batch_channel_specs(ndom: int = 512, nmin: int = 64, nmax: int = 1024,
                        u_max: float = 0.05, seed: int = 512):
    """Parameters of ndom independent D2Q9 channels: nx, ny ~ U{nmin..nmax},
    tau ~ U[0.52, 0.9], one cylinder of radius U[0.05, 0.15] ny centred at
    (nx/4, ny/2 + U[-0.05, 0.05] ny), walls at y = 0 and ny - 1, periodic x,
    body force g = 8 nu u_max / H^2 along x (H = ny - 2 fluid rows,
    nu = (2 tau - 1)/6), sized so the empty channel would peak near u_max."""
    rng = _rng(seed)
    specs = []
    for d in range(ndom):
        nx = int(rng.integers(nmin, nmax + 1))
        ny = int(rng.integers(nmin, nmax + 1))
        tau = float(rng.uniform(0.52, 0.9))
        r = float(rng.uniform(0.05, 0.15)) * ny
        cx = nx / 4.0
        cy = ny / 2.0 + float(rng.uniform(-0.05, 0.05)) * ny
        nu = (2.0 * tau - 1.0) / 6.0
        H = ny - 2
        g = 8.0 * nu * u_max / (H * H)
        specs.append(dict(nx=nx, ny=ny, tau=tau, radius=r, cx=cx, cy=cy, gx=g))
    return specs


def batch_channel_mask(spec) -> np.ndarray:
    """uint8 [1, ny, nx] mask of one channel spec (walls + cylinder)."""
    nx, ny = spec["nx"], spec["ny"]
    m = channel_mask(nx, ny, 1)
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    dx = x - spec["cx"]
    dx = dx - nx * np.round(dx / nx)          # periodic in x
    inside = dx * dx + (y - spec["cy"]) ** 2 <= spec["radius"] ** 2
    m[0][inside] = 1
    return m


# --------------------------------------------------------------------------
# Generic perturbed states for parity tests
# --------------------------------------------------------------------------
def random_state(nx: int, ny: int, nz: int, D: int, u_amp: float = 0.05,
                 rho_amp: float = 0.02, seed: int = 1311):
    """Smooth-ish random rho, u: a few random Fourier modes per field."""
    rng = _rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def field(amp):
        out = np.zeros((nz, ny, nx))
        for _ in range(4):
            kx = rng.integers(0, 3) * 2 * np.pi / nx
            ky = rng.integers(0, 3) * 2 * np.pi / ny
            kz = (rng.integers(0, 3) * 2 * np.pi / nz) if nz > 1 else 0.0
            ph = rng.uniform(0, 2 * np.pi)
            out += np.cos(kx * x + ky * y + kz * z + ph)
        out += 0.25 * rng.standard_normal((nz, ny, nx))
        return amp * out / max(1e-30, np.abs(out).max())

    rho = 1.0 + field(rho_amp)
    u = np.stack([field(u_amp) for _ in range(D)])
    return rho, u


# --------------------------------------------------------------------------
# Synthetic training pairs for the alpha surrogate's training throughput
# --------------------------------------------------------------------------
def mlp_pairs(n: int = 1 << 20, seed: int = 1393):
    """n (features, alpha) pairs shaped like the ELBM kernel's: 8 FP32
    features of the spreads the invariants take (the fifth, eps, positive
    and small) and alpha near 2 varying smoothly with them.  A throughput
    workload: the values carry no physics."""
    rng = _rng(seed)
    X = rng.standard_normal((n, 8)) * np.array([1.0, 2.0, 3.0, 4.0, 1e-2, 2.0, 2.0, 1.0])
    X[:, 4] = np.abs(X[:, 4]) + 1e-3
    alpha = 2.0 + 0.5 * X[:, 4] * (np.tanh(X[:, 0]) + 0.3 * X[:, 1])
    return X.astype(np.float32), alpha
