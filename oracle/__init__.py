"""FP64 CPU oracle of the lattice Boltzmann stream-and-collide step.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library.  It shares no code,
table or constant with the CUDA path.

Contents:
  lbm_oracle.c   the oracle proper (plain C, FP64, node by node; AB pull)
  np_oracle.py   a second, independent NumPy formulation (push streaming with
                 np.roll) used to pin the C oracle's streaming and walls
  mlp_oracle.py  FP64 forward / backward / Adam of the alpha surrogate

The C file is compiled by build() with plain flags (-O2, no fast-math, no FP
contraction) into oracle/_lib/liboracle.so and loaded with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

# model / alpha-mode codes of the oracle's parameter block
BGK, MRT, ELBM, REG, SMAG = 0, 1, 2, 3, 4
NEWTON, SERIES_GUARDED, MLP_GUARDED, FIXED2, ROOT_GUARDED = 0, 1, 2, 3, 4
# per-node alpha outcomes
AL_CONV, AL_SKIP, AL_CLAMP, AL_NOCONV, AL_FIXED, AL_GUARDED = range(6)

# d'Humieres et al. (2002) D3Q19 rates: conserved moments 0, shear moments
# (3pxx, pww, pxy, pyz, pxz) 1/tau, the rest their stabilising values.
def default_mrt_rates(tau: float) -> np.ndarray:
    w = 1.0 / tau
    s = np.zeros(19)
    s[1] = 1.19
    s[2] = 1.4
    s[4] = s[6] = s[8] = 1.2
    s[9] = s[11] = s[13] = s[14] = s[15] = w
    s[10] = s[12] = 1.4
    s[16] = s[17] = s[18] = 1.98
    return s


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("D", ctypes.c_int), ("model", ctypes.c_int), ("alpha_mode", ctypes.c_int),
        ("max_iter", ctypes.c_int), ("feq_variant", ctypes.c_int),
        ("nthreads", ctypes.c_int), ("guard_steps", ctypes.c_int),
        ("tau", ctypes.c_double), ("force", ctypes.c_double * 3),
        ("s", ctypes.c_double * 19), ("tol", ctypes.c_double),
        ("skip_eps", ctypes.c_double), ("guard_tol", ctypes.c_double),
        ("mlp", ctypes.POINTER(ctypes.c_double)),
        ("smag_cs", ctypes.c_double),
        ("q", ctypes.c_int),
        ("bc_kind", ctypes.c_int * 15), ("bc_method", ctypes.c_int * 15),
        ("bc_normal", ctypes.c_int * 15), ("bc_val", (ctypes.c_double * 3) * 15),
    ]


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into oracle/_lib/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        PP = ctypes.POINTER(OracleParams)
        L.oracle_lattice.argtypes = [ctypes.c_int, ip, dp, ip]
        L.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.oracle_mrt_matrix.argtypes = [dp, dp]
        L.oracle_collide.argtypes = [PP, dp, dp, dp, dp]
        L.oracle_elbm_g.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
        L.oracle_elbm_alpha.argtypes = [PP, dp, dp, dp]
        L.oracle_elbm_features.argtypes = [ctypes.c_int, dp, dp, dp, dp]
        L.oracle_mlp_guess.argtypes = [dp, dp]
        L.oracle_mlp_guess.restype = ctypes.c_double
        L.oracle_series_root_guess.argtypes = [dp, ctypes.c_double]
        L.oracle_series_root_guess.restype = ctypes.c_double
        L.oracle_init.argtypes = [PP, dp, dp, dp]
        L.oracle_bc_node.argtypes = [PP, ctypes.c_int, dp]
        L.oracle_run.argtypes = [PP, dp, dp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                 dp, dp, dp, dp]
        L.oracle_max_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def Q_of(D: int) -> int:
    """Velocities of a lattice code: 2 / 9 D2Q9, 3 / 19 D3Q19, 15 D3Q15, 27 D3Q27."""
    return {2: 9, 9: 9, 3: 19, 19: 19, 15: 15, 27: 27}[D]


def dim_of(code: int) -> int:
    return 2 if code in (2, 9) else 3


def lattice(D: int):
    """(e [Q,3] int, w [Q], opp [Q]) in the oracle's enumeration order."""
    Q = Q_of(D)
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib().oracle_lattice(D, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                         opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e, w, opp


def feq(D: int, rho: float, u, kind: int = 0) -> np.ndarray:
    """kind 0 polynomial, 1 entropic product, 2 entropic with moments restored."""
    uu = np.zeros(3)
    uu[:len(u)] = u
    out = np.zeros(Q_of(D))
    r = lib().oracle_feq(D, kind, float(rho), _dp(uu), _dp(out))
    assert r == 0
    return out


def mrt_matrix():
    M = np.zeros((19, 19))
    Mi = np.zeros((19, 19))
    lib().oracle_mrt_matrix(_dp(M), _dp(Mi))
    return M, Mi


def make_params(nx=1, ny=1, nz=1, D=3, model=BGK, tau=0.6, force=(0.0, 0.0, 0.0),
                s=None, alpha_mode=NEWTON, max_iter=20, feq_variant=0, tol=1e-12,
                skip_eps=1e-3, guard_tol=1e-6, guard_steps=2, mlp=None, nthreads=0,
                smag_cs=0.1, q=0):
    """D is the dimension or a lattice code (15, 19, 27 for D3Q15/19/27)."""
    if D in (9, 15, 19, 27):
        q = D
        D = dim_of(D)
    p = OracleParams()
    p.nx, p.ny, p.nz, p.D, p.model = nx, ny, nz, D, model
    p.q = q
    p.alpha_mode, p.max_iter, p.feq_variant = alpha_mode, max_iter, feq_variant
    p.nthreads, p.guard_steps = nthreads, guard_steps
    p.tau = tau
    for a in range(3):
        p.force[a] = float(force[a]) if a < len(force) else 0.0
    ss = default_mrt_rates(tau) if s is None else np.asarray(s, dtype=np.float64)
    for k in range(19):
        p.s[k] = float(ss[k])
    p.tol, p.skip_eps, p.guard_tol = tol, skip_eps, guard_tol
    p.smag_cs = smag_cs
    if mlp is not None:
        arr = np.ascontiguousarray(mlp, dtype=np.float64)
        p._mlp_keep = arr  # keep alive with the struct
        p.mlp = _dp(arr)
    return p


# boundary-condition codes: kinds, methods, inward normals (+-1 x, +-2 y, +-3 z)
BC_VELOCITY, BC_PRESSURE = 1, 2
BC_EQUILIBRIUM, BC_ZOUHE, BC_REGULARIZED = 0, 1, 2


def set_bc(p: OracleParams, k: int, kind: int, method: int, normal: int, value) -> None:
    """Condition k, used by mask code 2 + k: value is the velocity (kind
    BC_VELOCITY) or [rho] (BC_PRESSURE)."""
    p.bc_kind[k], p.bc_method[k], p.bc_normal[k] = kind, method, normal
    val = list(value) + [0.0] * (3 - len(value))
    for a in range(3):
        p.bc_val[k][a] = float(val[a])


def bc_node(p: OracleParams, k: int, f) -> np.ndarray:
    """Condition k applied to one node's post-streaming populations."""
    ff = np.array(f, dtype=np.float64)
    r = lib().oracle_bc_node(ctypes.byref(p), int(k), _dp(ff))
    assert r == 0
    return ff


def collide(p: OracleParams, f) -> tuple:
    """One node: returns (f_post, rho, v[3], info): info = [alpha, evals,
    status, |g|/a2] for ELBM, info[0] = total relaxation time for SMAG."""
    ff = np.array(f, dtype=np.float64)
    rho = np.zeros(1)
    v = np.zeros(3)
    info = np.zeros(4)
    r = lib().oracle_collide(ctypes.byref(p), _dp(ff), _dp(rho), _dp(v), _dp(info))
    assert r == 0
    return ff, rho[0], v, info


def elbm_g(D, f, fe, alpha):
    g = np.zeros(1)
    gp = np.zeros(1)
    lib().oracle_elbm_g(D, _dp(np.ascontiguousarray(f, dtype=np.float64)),
                        _dp(np.ascontiguousarray(fe, dtype=np.float64)), float(alpha),
                        _dp(g), _dp(gp))
    return g[0], gp[0]


def elbm_alpha(p: OracleParams, f, fe):
    out = np.zeros(4)
    lib().oracle_elbm_alpha(ctypes.byref(p), _dp(np.ascontiguousarray(f, dtype=np.float64)),
                            _dp(np.ascontiguousarray(fe, dtype=np.float64)), _dp(out))
    return out


def elbm_features(D, f, fe):
    feat = np.zeros(8)
    ak = np.zeros(7)
    lib().oracle_elbm_features(D, _dp(np.ascontiguousarray(f, dtype=np.float64)),
                               _dp(np.ascontiguousarray(fe, dtype=np.float64)),
                               _dp(feat), _dp(ak))
    return feat, ak


def mlp_guess(P, feat) -> float:
    return lib().oracle_mlp_guess(_dp(np.ascontiguousarray(P, dtype=np.float64)),
                                  _dp(np.ascontiguousarray(feat, dtype=np.float64)))


def series_root_guess(ak, A1) -> float:
    """Root of g(alpha)/alpha with g's alpha-series truncated after a_6 (ak =
    a_0..a_6, A1 = A + a_1): the guess of alpha mode ROOT_GUARDED."""
    return lib().oracle_series_root_guess(_dp(np.ascontiguousarray(ak, dtype=np.float64)),
                                          float(A1))


def init(p: OracleParams, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
    """F [Q, nz, ny, nx] = f_eq(rho, u); rho [nz,ny,nx], u [D,nz,ny,nx]."""
    D = p.D
    N = p.nx * p.ny * p.nz
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(D * N)
    F = np.zeros((Q_of(p.q or D), p.nz, p.ny, p.nx))
    r = lib().oracle_init(ctypes.byref(p), _dp(rho), _dp(u), _dp(F))
    assert r == 0
    return F


def run(p: OracleParams, F: np.ndarray, nsteps: int, mask: np.ndarray | None = None,
        want_alpha: bool = False):
    """Advance F in place by nsteps.  Returns (rho, u, alpha|None, stats)."""
    D = p.D
    N = p.nx * p.ny * p.nz
    assert F.shape == (Q_of(p.q or D), p.nz, p.ny, p.nx) and F.dtype == np.float64
    assert F.flags.c_contiguous
    tmp = np.empty_like(F)
    rho = np.zeros((p.nz, p.ny, p.nx))
    u = np.zeros((D, p.nz, p.ny, p.nx))
    alpha = np.zeros((p.nz, p.ny, p.nx)) if want_alpha else None
    stats = np.zeros(6)
    mptr = None
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(N)
        mptr = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    r = lib().oracle_run(ctypes.byref(p), _dp(F), _dp(tmp), mptr, int(nsteps), _dp(rho),
                         _dp(u), _dp(alpha) if alpha is not None else None, _dp(stats))
    assert r == 0
    return rho, u, alpha, stats


def max_threads(nthreads: int = 0) -> int:
    return lib().oracle_max_threads(nthreads)


def kinetic_energy_enstrophy(v: np.ndarray):
    """E = (1/2V) sum |v|^2 and Omega = (1/2V) sum |curl v|^2 of a periodic
    velocity field v [D, nz, ny, nx] (lattice units, D = 2 or 3), the
    vorticity by second-order central differences (Sec. 5.2, Kida vortex
    diagnostics); a 2-D field has only the z component of the vorticity.
    FP64, whole-array NumPy."""
    v = np.asarray(v, dtype=np.float64)

    def d(f, axis):          # axis 0: z, 1: y, 2: x of a [nz, ny, nx] field
        return 0.5 * (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis))

    vx, vy = v[0], v[1]
    vz = v[2] if v.shape[0] == 3 else np.zeros_like(vx)
    wz = d(vy, 2) - d(vx, 1)
    if v.shape[0] == 3:
        wx = d(vz, 1) - d(vy, 0)
        wy = d(vx, 0) - d(vz, 2)
    else:
        wx = wy = np.zeros_like(vx)
    V = vx.size
    E = 0.5 * (vx * vx + vy * vy + vz * vz).sum() / V
    Om = 0.5 * (wx * wx + wy * wy + wz * wz).sum() / V
    return E, Om
