"""FP64 CPU oracle of the boosted-frame PIC step — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline``
leg and ``--impl reference`` arm) may import this package.  The product path
(``paper_2411_04703_gb300``) never imports it and shares no code with it: the C
source ``pic_oracle.c`` is a plain restatement of the paper's method in double
precision (see its header for the passage each function follows).

This module only builds the C library with gcc and marshals numpy arrays through
ctypes.
"""
from __future__ import annotations

import math
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, PML, OPEN = 0, 1, 2
LAB, BOOSTED = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
FIELD_NAMES = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]

# Layout of the moments vector written by osim_moments.
MOMENT_NAMES = [
    "count", "sum_w", "charge", "mean_x", "mean_y", "mean_z", "rms_x", "rms_y", "rms_z",
    "mean_ux", "mean_uy", "mean_uz", "mean_gamma", "rel_energy_spread", "emit_nx",
    "emit_ny", "bunching", "kinetic_energy", "mean_t", "field_energy",
]


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into a shared library (gcc, FP64, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    # OpenMP only serves the multi-threaded timing of the particle loop (osim_set_threads); a
    # compiler without it builds the serial library
    if subprocess.run(cmd[:-4] + ["-fopenmp"] + cmd[-4:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, d, i, l = C.c_void_p, C.c_double, C.c_int, C.c_long
            P = C.POINTER
            pd, pi, pl = P(C.c_double), P(C.c_int), P(C.c_long)
            sig = {
                "osim_create": (vp, [i, i, i, d, d, d, d, d, pi, i, i, i, d]),
                "osim_destroy": (None, [vp]),
                "osim_beta": (d, [vp]),
                "osim_add_species": (i, [vp, d, d, i, l]),
                "osim_load": (l, [vp, i, l, pd, pd, pd, i, pd, i]),
                "osim_set_state": (None, [vp, i, l, pd, pd, pd, pl]),
                "osim_set_next_id": (None, [vp, i, l]),
                "osim_set_time": (None, [vp, l, l, l]),
                "osim_get_time": (None, [vp, pl]),
                "osim_count": (l, [vp, i]),
                "osim_get_particles": (None, [vp, i, pd, pd, pd, pl]),
                "osim_set_field": (None, [vp, i, pd]),
                "osim_get_field": (None, [vp, i, pd]),
                "osim_set_external": (None, [vp, i, d, d, d, d, d]),
                "osim_external_at": (None, [vp, d, d, d, pd, pd]),
                "osim_undulator_Ax": (d, [vp, d, d]),
                "osim_set_plasma": (None, [vp, i, i, pi, pi, i, pd, pd, i]),
                "osim_step": (None, [vp, l]),
                "osim_fdtd": (None, [vp]),
                "osim_dropped": (l, [vp]),
                "osim_rho": (None, [vp, pd]),
                "osim_divE": (None, [vp, pd]),
                "osim_deposit_one": (None, [vp, d, pd, pd]),
                "osim_gather_at": (None, [vp, pd, pd]),
                "osim_moments": (None, [vp, i, i, d, pd]),
                "oracle_boris": (None, [d, d, pd, pd, pd]),
                "oracle_vay": (None, [d, d, pd, pd, pd]),
                "osim_set_pusher": (None, [vp, i]),
                "osim_set_threads": (i, [vp, i]),
                "osim_set_gather": (None, [vp, i]),
                "osim_set_ion_ramp": (None, [vp, i, d]),
                "osim_snapshot_begin": (None, [vp, i, d]),
                "osim_snapshot_get": (l, [vp, pd, P(C.c_ubyte)]),
                "osim_snapshot_n": (l, [vp]),
                "osim_snapshot_moments": (None, [vp, d, pd]),
                "oracle_field_transform": (None, [pd, pd, d, pd, pd]),
                "oracle_lab_to_boosted": (None, [d, pd, pd, pd, pd]),
                "oracle_boosted_to_lab": (None, [d, pd, d, pd, pd, pd, pd]),
                "oracle_tile_sort": (None, [l, pd, pi, pi, pl, pl]),
                "oracle_resonant_wavelength": (d, [d, d, d]),
                "oracle_doppler_rrf": (d, [d, d]),
                "oracle_beam_elongation": (d, [d, d]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _pl(a):
    return a.ctypes.data_as(C.POINTER(C.c_long))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- single-step helpers

def resolution_factor(L_wind: float, n_cells: int, gamma_R: float) -> float:
    """Relativistic resolution factor R_RF = (8 L_wind / N) sqrt((1 - beta_R)/(1 + beta_R))
    (Eq. Rrf1), written as the formula reads."""
    bR = math.sqrt(1.0 - 1.0 / (gamma_R * gamma_R))
    return 8.0 * L_wind / n_cells * math.sqrt((1.0 - bR) / (1.0 + bR))


def vay(qm: float, dt: float, E, B, u):
    """One Vay push of momentum u (copied) in E, B; returns the new momentum."""
    u = np.array(u, dtype=np.float64)
    lib().oracle_vay(qm, dt, _pd(_f64(E)), _pd(_f64(B)), _pd(u))
    return u


def boris(qm: float, dt: float, E, B, u):
    u = _f64(u).copy()
    lib().oracle_boris(qm, dt, _pd(_f64(E)), _pd(_f64(B)), _pd(u))
    return u


def field_transform(E, B, beta: float):
    Ep, Bp = np.zeros(3), np.zeros(3)
    lib().oracle_field_transform(_pd(_f64(E)), _pd(_f64(B)), beta, _pd(Ep), _pd(Bp))
    return Ep, Bp


def lab_to_boosted(gamma_R: float, x, u):
    xp, up = np.zeros(3), np.zeros(3)
    lib().oracle_lab_to_boosted(gamma_R, _pd(_f64(x)), _pd(_f64(u)), _pd(xp), _pd(up))
    return xp, up


def boosted_to_lab(gamma_R: float, xp, tp: float, up):
    x, u, t = np.zeros(3), np.zeros(3), np.zeros(1)
    lib().oracle_boosted_to_lab(gamma_R, _pd(_f64(xp)), tp, _pd(_f64(up)), _pd(x), _pd(t), _pd(u))
    return x, float(t[0]), u


def resonant_wavelength(lambda_u: float, K: float, gamma_B: float) -> float:
    return lib().oracle_resonant_wavelength(lambda_u, K, gamma_B)


def doppler_rrf(lam: float, gamma_R: float) -> float:
    return lib().oracle_doppler_rrf(lam, gamma_R)


def beam_elongation(gamma_B: float, gamma_R: float) -> float:
    return lib().oracle_beam_elongation(gamma_B, gamma_R)


def tile_sort(X: np.ndarray, grid, tile):
    """Stable sort of particles (grid coordinates X, shape (n, 3)) by the tile-major cell +
    octant key; returns (order, keys)."""
    Xc = _f64(X).reshape(-1, 3)
    n = Xc.shape[0]
    order = np.zeros(n, np.int64)
    keys = np.zeros(n, np.int64)
    g = np.ascontiguousarray(grid, dtype=np.int32)
    t = np.ascontiguousarray(tile, dtype=np.int32)
    lib().oracle_tile_sort(n, _pd(Xc), _pi(g), _pi(t), _pl(order), _pl(keys))
    return order, keys


class Sim:
    """FP64 oracle simulation.  Same semantics as the C-ABI of the CUDA path."""

    def __init__(self, grid, d, dt, gamma_R, bc=((0, 0), (0, 0), (0, 0)), pml=0, order=1,
                 moving_window=False, window_v=0.0):
        self.L = lib()
        self.grid = tuple(int(v) for v in grid)
        self.d = tuple(float(v) for v in d)
        self.dt = float(dt)
        self.gamma_R = float(gamma_R)
        self.order = int(order)
        bc6 = np.array([bc[0][0], bc[0][1], bc[1][0], bc[1][1], bc[2][0], bc[2][1]], np.int32)
        self.h = self.L.osim_create(*self.grid, *self.d, self.dt, self.gamma_R, _pi(bc6), int(pml),
                                    self.order, int(bool(moving_window)), float(window_v))
        self.beta_R = self.L.osim_beta(self.h)
        self.species = []

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.osim_destroy(h)
            self.h = None

    @property
    def ncell(self):
        return self.grid[0] * self.grid[1] * self.grid[2]

    def add_species(self, q, m, frozen=False, capacity=1024):
        sid = self.L.osim_add_species(self.h, float(q), float(m), int(bool(frozen)), int(capacity))
        assert sid >= 0
        self.species.append(sid)
        return sid

    def load(self, sid, x, u, w=None, frame=LAB, origin=(0.0, 0.0, 0.0), match_undulator=False):
        x = _f64(x).reshape(3, -1)
        u = _f64(u).reshape(3, -1)
        n = x.shape[1]
        wp = _pd(_f64(w)) if w is not None else None
        org = _f64(origin)
        return self.L.osim_load(self.h, sid, n, _pd(x), _pd(u), wp, int(frame), _pd(org),
                                int(bool(match_undulator)))

    def set_state(self, sid, X, U, W, ids):
        """X, U as (n, 3) arrays in grid cells / momentum; W (n,); ids (n,)."""
        X = _f64(X).reshape(-1, 3)
        U = _f64(U).reshape(-1, 3)
        W = _f64(W)
        ids = np.ascontiguousarray(ids, np.int64)
        self.L.osim_set_state(self.h, sid, X.shape[0], _pd(X), _pd(U), _pd(W), _pl(ids))

    def set_next_id(self, sid, nxt):
        self.L.osim_set_next_id(self.h, sid, int(nxt))

    def set_time(self, step, shifts=0, m_last=0):
        self.L.osim_set_time(self.h, int(step), int(shifts), int(m_last))

    def time(self):
        out = np.zeros(3, np.int64)
        self.L.osim_get_time(self.h, _pl(out))
        return tuple(int(v) for v in out)

    def count(self, sid):
        return self.L.osim_count(self.h, sid)

    def particles(self, sid):
        n = self.count(sid)
        X = np.zeros((max(n, 1), 3))
        U = np.zeros((max(n, 1), 3))
        W = np.zeros(max(n, 1))
        ids = np.zeros(max(n, 1), np.int64)
        self.L.osim_get_particles(self.h, sid, _pd(X), _pd(U), _pd(W), _pl(ids))
        return X[:n], U[:n], W[:n], ids[:n]

    def field(self, which):
        out = np.zeros(self.ncell)
        self.L.osim_get_field(self.h, int(which), _pd(out))
        return out.reshape(self.grid[2], self.grid[1], self.grid[0])

    def set_field(self, which, arr):
        a = _f64(arr).reshape(-1)
        assert a.size == self.ncell
        self.L.osim_set_field(self.h, int(which), _pd(a))

    def set_external(self, K, lambda_u, phase=0.0, z_start=-np.inf, ramp=-1.0, kind=1):
        self.L.osim_set_external(self.h, int(kind), float(K), float(lambda_u), float(phase),
                                 float(z_start), float(ramp))

    def external_at(self, zp, tp, y=0.0):
        """RRF external field at RRF z' (absolute), time t' and y from the undulator axis."""
        E, B = np.zeros(3), np.zeros(3)
        self.L.osim_external_at(self.h, float(y), float(zp), float(tp), _pd(E), _pd(B))
        return E, B

    def undulator_Ax(self, zlab, y=0.0):
        return self.L.osim_undulator_Ax(self.h, float(y), float(zlab))

    def set_plasma(self, sp_e, sp_i, ppc, xrange, z_nodes, n_nodes, fill=True):
        ppc = np.ascontiguousarray(ppc, np.int32)
        xr = np.ascontiguousarray(xrange, np.int32)
        zn = _f64(z_nodes)
        dn = _f64(n_nodes)
        self.L.osim_set_plasma(self.h, sp_e, sp_i, _pi(ppc), _pi(xr), zn.size, _pd(zn), _pd(dn),
                               int(bool(fill)))

    def step(self, n=1):
        self.L.osim_step(self.h, int(n))

    def set_threads(self, n):
        """Threads of the particle loop (timing only; 1, the default, is the serial reference
        loop).  Returns the number used (1 without OpenMP)."""
        return self.L.osim_set_threads(self.h, int(n))

    def snapshot_begin(self, sid, t_lab):
        """Arm a lab-frame snapshot of species sid at lab time t_lab (time-skew reconstruction)."""
        self.L.osim_snapshot_begin(self.h, int(sid), float(t_lab))

    def snapshot(self):
        """(records [n_ids, 7]: lab x, y, z, u_x, u_y, u_z, w; state [n_ids]: 0 pending, 1 recorded,
        2 missed) by particle id."""
        n = self.L.osim_snapshot_n(self.h)
        rec = np.zeros((max(n, 1), 7))
        st = np.zeros(max(n, 1), np.uint8)
        self.L.osim_snapshot_get(self.h, _pd(rec), st.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return rec[:n], st[:n]

    def snapshot_moments(self, k=0.0):
        out = np.zeros(len(MOMENT_NAMES))
        self.L.osim_snapshot_moments(self.h, float(k), _pd(out))
        return dict(zip(MOMENT_NAMES, out.tolist()))

    def set_ion_ramp(self, sid, T):
        """Artificial ions compensating species sid now, faded linearly over T (T <= 0: none)."""
        self.L.osim_set_ion_ramp(self.h, int(sid), float(T))

    def set_gather(self, gather):
        """0: momentum-conserving gather (default), 1: energy-conserving."""
        self.L.osim_set_gather(self.h, int(gather))

    def set_pusher(self, pusher):
        """0: Boris (default), 1: Vay."""
        self.L.osim_set_pusher(self.h, int(pusher))

    def fdtd(self):
        self.L.osim_fdtd(self.h)

    def dropped(self):
        return self.L.osim_dropped(self.h)

    def rho(self):
        out = np.zeros(self.ncell)
        self.L.osim_rho(self.h, _pd(out))
        return out.reshape(self.grid[2], self.grid[1], self.grid[0])

    def divE(self):
        out = np.zeros(self.ncell)
        self.L.osim_divE(self.h, _pd(out))
        return out.reshape(self.grid[2], self.grid[1], self.grid[0])

    def deposit_one(self, qw, X0, X1):
        self.L.osim_deposit_one(self.h, float(qw), _pd(_f64(X0)), _pd(_f64(X1)))
        return [self.field(JX), self.field(JY), self.field(JZ)]

    def gather_at(self, X):
        out = np.zeros(6)
        self.L.osim_gather_at(self.h, _pd(_f64(X)), _pd(out))
        return out

    def moments(self, sid, frame=0, k=0.0):
        out = np.zeros(len(MOMENT_NAMES))
        self.L.osim_moments(self.h, sid, int(frame), float(k), _pd(out))
        return dict(zip(MOMENT_NAMES, out.tolist()))
