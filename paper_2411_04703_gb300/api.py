"""Thin ctypes binding of the gbpic C-ABI (include/gbpic.h).

Argument marshalling only: every step of the PIC path runs in the CUDA kernels of
``libgbpic.so``.  PyTorch supplies device memory (its caching allocator, through the
``pic_device`` callbacks) and the CUDA stream.  There is no CPU fallback: if the
library or a GPU is missing, constructing :class:`Sim` raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

PIC_OK = 0
PIC_BC_PERIODIC, PIC_BC_PML, PIC_BC_OPEN = 0, 1, 2
PIC_FRAME_LAB, PIC_FRAME_BOOSTED = 0, 1
PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO = range(10)
PIC_EXT_NONE, PIC_EXT_PLANAR_UNDULATOR, PIC_EXT_PLANAR_UNDULATOR_3D = 0, 1, 2
PIC_GATHER_MOMENTUM, PIC_GATHER_ENERGY = 0, 1
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_ALLOC", -4: "PIC_ERR_STATE",
          -5: "PIC_ERR_DEVICE", -6: "PIC_ERR_CAPACITY"}
MOMENT_NAMES = [
    "count", "sum_w", "charge", "mean_x", "mean_y", "mean_z", "rms_x", "rms_y", "rms_z",
    "mean_ux", "mean_uy", "mean_uz", "mean_gamma", "rel_energy_spread", "emit_nx",
    "emit_ny", "bunching", "kinetic_energy", "mean_t", "field_energy",
]


PIC_PUSHER_BORIS, PIC_PUSHER_VAY = 0, 1


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class pic_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class pic_boundaries(C.Structure):
    _fields_ = [("face", (C.c_int * 2) * 3), ("pml_cells", C.c_int), ("moving_window", C.c_int),
                ("window_v", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class pic_device(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p), ("stream", C.c_void_p),
                ("device", C.c_int)]


class pic_tuning(C.Structure):
    _fields_ = [("tile", C.c_int * 3), ("sort_every", C.c_int), ("margin", C.c_int)]


class pic_species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("frozen", C.c_int), ("capacity", C.c_int64),
                ("origin", C.c_double * 3), ("match_undulator", C.c_int)]


class pic_external(C.Structure):
    _fields_ = [("type", C.c_int), ("K", C.c_double), ("lambda_u", C.c_double), ("phase", C.c_double),
                ("z_start", C.c_double), ("ramp_len", C.c_double)]


class pic_plasma(C.Structure):
    _fields_ = [("ppc", C.c_int * 3), ("x_range", C.c_int * 4), ("n_nodes", C.c_int),
                ("z_nodes", C.POINTER(C.c_double)), ("density", C.POINTER(C.c_double)),
                ("capacity", C.c_int64)]


class pic_trace(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("events", C.c_int64 * 8), ("kernels", C.c_int64), ("fallback", C.c_int64)]


TRACE_CLASSES = ["sort", "push", "push_frozen", "fields", "window", "inject", "other", "unused"]


class pic_adjoint_seed(C.Structure):
    _fields_ = [("species_id", C.c_int), ("k_bunch", C.c_double)]


class pic_grads(C.Structure):
    _fields_ = [("loss", C.c_double), ("dL_dK", C.c_double), ("n_profile", C.c_int),
                ("dL_dprofile", C.c_double * 64)]


class pic_moments(C.Structure):
    _fields_ = [("v", C.c_double * 20)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib(build_if_missing: bool = True):
    """Load libgbpic.so (building it with nvcc when missing or stale) and set signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"gbpic CUDA library missing at {path}; run build()")
        L = C.CDLL(path)
        vp, i, i64, d, sz = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
        P = C.POINTER
        sigs = {
            "pic_create": [P(vp), pic_grid, P(d), d, d, P(pic_boundaries), i, P(pic_device)],
            "pic_create_batch": [P(vp), i, pic_grid, P(d), d, d, P(pic_boundaries), i, P(pic_device)],
            "pic_load_species_batch": [vp, P(pic_species), P(i64), vp, vp, vp, i, P(i)],
            "pic_set_external_field_batch": [vp, P(pic_external)],
            "pic_set_plasma_batch": [vp, P(pic_plasma), P(d), P(i), P(i)],
            "pic_get_moments_run": [vp, i, i, i, d, P(pic_moments)],
            "pic_autotune": [vp, i, P(i)],
            "pic_autotune_tiles": [vp, P(i), i, i, P(i), P(i)],
            "pic_use_graphs": [vp, i],
            "pic_set_pusher": [vp, i],
            "pic_set_gather": [vp, i],
            "pic_set_ion_ramp": [vp, i, d],
            "pic_lab_snapshot": [vp, i, d],
            "pic_lab_snapshot_read": [vp, vp, vp, i64, P(i64), P(i64)],
            "pic_lab_snapshot_moments": [vp, d, P(pic_moments)],
            "pic_resolution_factor": [vp, d, P(d), P(i)],
            "pic_resonant_wavenumber": [d, d, d, d, i, P(d)],
            "pic_checkpoint": [vp, i],
            "pic_backward": [vp, P(pic_adjoint_seed), P(pic_grads)],
            "pic_set_tuning": [vp, P(pic_tuning)],
            "pic_load_species": [vp, P(pic_species), i64, vp, vp, vp, i, P(i)],
            "pic_set_external_field": [vp, P(pic_external)],
            "pic_set_plasma": [vp, P(pic_plasma), P(i), P(i)],
            "pic_step": [vp, i64],
            "pic_sync": [vp],
            "pic_sort": [vp],
            "pic_get_fields": [vp, i, vp, sz],
            "pic_set_fields": [vp, i, vp, sz],
            "pic_get_particles": [vp, i, i64, P(i64), vp, vp, vp, vp, vp],
            "pic_get_moments": [vp, i, i, d, P(pic_moments)],
            "pic_get_time": [vp, P(i64)],
            "pic_get_count": [vp, i, P(i64)],
            "pic_destroy": [vp],
            "pic_trace_enable": [vp, i],
            "pic_trace_read": [vp, P(pic_trace)],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.pic_last_error.argtypes = [vp]
        L.pic_last_error.restype = C.c_char_p
        _lib = L
        return L


def _ptr(a) -> Optional[int]:
    """Raw address of a numpy array or torch tensor (host or device), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


def _f64_c(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    return a.contiguous()


class Sim:
    """One boosted-frame PIC simulation on one GPU (a ``pic_ctx``)."""

    def __init__(self, grid, d, dt, gamma_R, bc=((0, 0), (0, 0), (0, 0)), pml=0, order=1,
                 moving_window=False, window_v=0.0, device=0, stream=None, tuning=None,
                 torch_allocator=True, runs=1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gbpic needs a CUDA GPU (no CPU fallback)")
        self.L = lib()
        self.runs = int(runs)
        self.run_grid = tuple(int(v) for v in grid)
        # an ensemble stacks its runs along z: the context's grid has runs * nz rows
        self.grid = (self.run_grid[0], self.run_grid[1], self.run_grid[2] * self.runs)
        self.d = tuple(float(v) for v in d)
        self.dt = float(dt)
        self.gamma_R = float(gamma_R)
        self.order = int(order)
        self.device = int(device)
        torch.cuda.set_device(self.device)
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
            if stream.cuda_stream == 0:
                # the legacy null stream cannot be handed over (NULL means "make your own" in
                # the C-ABI); use a dedicated torch stream so torch events see the work
                stream = torch.cuda.Stream(self.device)
        self.stream = stream
        dev = pic_device()
        dev.device = self.device
        dev.stream = C.c_void_p(stream.cuda_stream)
        self._cb = None
        if torch_allocator:
            live = {}

            def _alloc(nbytes, user):
                try:
                    p = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
                    live[p] = nbytes
                    return p
                except Exception:
                    return None

            def _free(ptr, nbytes, user):
                if ptr in live:
                    del live[ptr]
                    torch.cuda.caching_allocator_delete(ptr)

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free), live)
            dev.alloc, dev.free = self._cb[0], self._cb[1]
        b = pic_boundaries()
        for dd in range(3):
            b.face[dd][0], b.face[dd][1] = int(bc[dd][0]), int(bc[dd][1])
        b.pml_cells = int(pml)
        b.moving_window = int(bool(moving_window))
        b.window_v = float(window_v)
        h = C.c_void_p()
        darr = (C.c_double * 3)(*self.d)
        r = self.L.pic_create_batch(C.byref(h), self.runs, pic_grid(*self.run_grid), darr, self.dt, self.gamma_R,
                                    C.byref(b), self.order, C.byref(dev))
        if r != PIC_OK:
            raise PicError(r, self.L.pic_last_error(None).decode())
        self.h = h
        self._dev = dev
        if tuning is not None:
            t = pic_tuning()
            for dd in range(3):
                t.tile[dd] = int(tuning.get("tile", (8, 8, 8))[dd])
            t.sort_every = int(tuning.get("sort_every", 8))
            t.margin = int(tuning.get("margin", 1))
            self._check(self.L.pic_set_tuning(self.h, C.byref(t)))

    # ------------------------------------------------------------------ plumbing
    def _check(self, r):
        if r != PIC_OK:
            raise PicError(r, self.L.pic_last_error(self.h).decode())
        return r

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ncell(self):
        return self.grid[0] * self.grid[1] * self.grid[2]

    # ------------------------------------------------------------------ set-up
    def load_species(self, q, m, x=None, u=None, w=None, frame=PIC_FRAME_LAB, origin=(0.0, 0.0, 0.0),
                     capacity=0, frozen=False, match_undulator=False):
        """x, u: (3, n) FP64 (numpy, or torch on host or device); w: (n,) or None."""
        n = 0 if x is None else int(x.shape[1])
        xs = _f64_c(x) if n else None
        us = _f64_c(u) if n else None
        ws = _f64_c(w) if (n and w is not None) else None
        sp = pic_species(float(q), float(m), int(bool(frozen)), int(max(capacity, n, 1)),
                         (C.c_double * 3)(*[float(v) for v in origin]), int(bool(match_undulator)))
        sid = C.c_int()
        self._check(self.L.pic_load_species(self.h, C.byref(sp), n, _ptr(xs), _ptr(us), _ptr(ws),
                                            int(frame), C.byref(sid)))
        return sid.value

    def load_species_batch(self, q, m, n_run, x, u, w=None, frame=PIC_FRAME_LAB, origin=(0.0, 0.0, 0.0),
                           capacity=0, frozen=False, match_undulator=False):
        """Ensemble load: n_run[r] particles into run r; x, u: (3, sum n_run) FP64, run-major."""
        counts = np.ascontiguousarray(n_run, np.int64)
        assert counts.size == self.runs
        n = int(counts.sum())
        xs, us = _f64_c(x), _f64_c(u)
        ws = _f64_c(w) if w is not None else None
        sp = pic_species(float(q), float(m), int(bool(frozen)), int(max(capacity, n, 1)),
                         (C.c_double * 3)(*[float(v) for v in origin]), int(bool(match_undulator)))
        sid = C.c_int()
        self._check(self.L.pic_load_species_batch(self.h, C.byref(sp), counts.ctypes.data_as(C.POINTER(C.c_int64)),
                                                  _ptr(xs), _ptr(us), _ptr(ws), int(frame), C.byref(sid)))
        return sid.value

    def set_external_field_batch(self, K_run, lambda_u, phase=0.0, kind=PIC_EXT_PLANAR_UNDULATOR):
        arr = (pic_external * self.runs)(*[pic_external(int(kind), float(k), float(lambda_u), float(phase),
                                                        -math.inf, -1.0) for k in K_run])
        self._check(self.L.pic_set_external_field_batch(self.h, arr))

    def set_plasma_batch(self, ppc, x_range, z_nodes, density, density_scale, capacity=0):
        zn = np.ascontiguousarray(z_nodes, np.float64)
        dn = np.ascontiguousarray(density, np.float64)
        sc = np.ascontiguousarray(density_scale, np.float64)
        assert sc.size == self.runs
        p = pic_plasma((C.c_int * 3)(*ppc), (C.c_int * 4)(*x_range), int(zn.size),
                       zn.ctypes.data_as(C.POINTER(C.c_double)), dn.ctypes.data_as(C.POINTER(C.c_double)),
                       int(capacity))
        e, i = C.c_int(), C.c_int()
        self._check(self.L.pic_set_plasma_batch(self.h, C.byref(p), sc.ctypes.data_as(C.POINTER(C.c_double)),
                                                C.byref(e), C.byref(i)))
        return e.value, i.value

    def get_moments_run(self, sid, run, frame=PIC_FRAME_BOOSTED, k_bunch=0.0):
        m = pic_moments()
        self._check(self.L.pic_get_moments_run(self.h, int(sid), int(run), int(frame), float(k_bunch), C.byref(m)))
        return dict(zip(MOMENT_NAMES, list(m.v)))

    def set_external_field(self, K, lambda_u, phase=0.0, z_start=-math.inf, ramp_len=-1.0,
                           kind=PIC_EXT_PLANAR_UNDULATOR):
        f = pic_external(int(kind), float(K), float(lambda_u), float(phase), float(z_start), float(ramp_len))
        self._check(self.L.pic_set_external_field(self.h, C.byref(f)))

    def set_plasma(self, ppc, x_range, z_nodes, density, capacity=0):
        zn = np.ascontiguousarray(z_nodes, np.float64)
        dn = np.ascontiguousarray(density, np.float64)
        p = pic_plasma((C.c_int * 3)(*ppc), (C.c_int * 4)(*x_range), int(zn.size),
                       zn.ctypes.data_as(C.POINTER(C.c_double)), dn.ctypes.data_as(C.POINTER(C.c_double)),
                       int(capacity))
        e, i = C.c_int(), C.c_int()
        self._check(self.L.pic_set_plasma(self.h, C.byref(p), C.byref(e), C.byref(i)))
        return e.value, i.value

    # ------------------------------------------------------------------ stepping
    def step(self, n=1):
        self._check(self.L.pic_step(self.h, int(n)))

    def checkpoint(self, every_k):
        """Start recording for the adjoint: checkpoints now and every every_k steps."""
        self._check(self.L.pic_checkpoint(self.h, int(every_k)))

    def backward(self, species_id, k_bunch):
        """Gradient of the boosted-frame bunching factor of a species at the current step with
        respect to K and the plasma profile nodes: {loss, dL_dK, dL_dprofile}."""
        seed = pic_adjoint_seed(int(species_id), float(k_bunch))
        g = pic_grads()
        self._check(self.L.pic_backward(self.h, C.byref(seed), C.byref(g)))
        return {"loss": g.loss, "dL_dK": g.dL_dK, "dL_dprofile": np.array(g.dL_dprofile[:g.n_profile])}

    def resolution_factor(self, lambda_lab):
        """(R_RF, R_RF < lambda_lab) of the grid (Eq. Rrf1)."""
        r, ok = C.c_double(), C.c_int()
        self._check(self.L.pic_resolution_factor(self.h, float(lambda_lab), C.byref(r), C.byref(ok)))
        return r.value, bool(ok.value)

    def lab_snapshot(self, species_id, t_lab):
        """Arm the lab-frame snapshot of a species at lab time t_lab (NaN disarms)."""
        self._check(self.L.pic_lab_snapshot(self.h, int(species_id), float(t_lab)))

    def lab_snapshot_read(self):
        """(records [n_ids, 7]: lab x, y, z, u_x, u_y, u_z, w; states [n_ids]: 0 pending,
        1 recorded, 2 missed) by particle id."""
        n, m = C.c_int64(), C.c_int64()
        self._check(self.L.pic_lab_snapshot_read(self.h, None, None, 0, C.byref(n), None))
        rec = np.zeros((max(n.value, 1), 7))
        st = np.zeros(max(n.value, 1), np.uint8)
        self._check(self.L.pic_lab_snapshot_read(self.h, rec.ctypes.data, st.ctypes.data, n.value, C.byref(n),
                                                 C.byref(m)))
        return rec[:n.value], st[:n.value]

    def lab_snapshot_moments(self, k_bunch=0.0):
        m = pic_moments()
        self._check(self.L.pic_lab_snapshot_moments(self.h, float(k_bunch), C.byref(m)))
        return dict(zip(MOMENT_NAMES, list(m.v)))

    def set_ion_ramp(self, species_id, T_ion):
        """Artificial ions compensating species_id now, faded linearly over T_ion (<= 0: none)."""
        self._check(self.L.pic_set_ion_ramp(self.h, int(species_id), float(T_ion)))

    def set_gather(self, gather):
        """PIC_GATHER_MOMENTUM (0, default) or PIC_GATHER_ENERGY (1)."""
        self._check(self.L.pic_set_gather(self.h, int(gather)))

    def set_pusher(self, pusher):
        """PIC_PUSHER_BORIS (0, default) or PIC_PUSHER_VAY (1)."""
        self._check(self.L.pic_set_pusher(self.h, int(pusher)))

    def use_graphs(self, on=True):
        """Replay captured step sequences (CUDA graphs) where the step allows it."""
        self._check(self.L.pic_use_graphs(self.h, int(bool(on))))

    def autotune(self, max_sort_every=16):
        """Pick the sort cadence by timed trials (advances the simulation); returns it."""
        out = C.c_int()
        self._check(self.L.pic_autotune(self.h, int(max_sort_every), C.byref(out)))
        return out.value

    def autotune_tiles(self, tiles=((8, 8, 8), (8, 8, 4), (8, 4, 4), (4, 4, 4)), max_sort_every=16):
        """Pick the tile size (from `tiles`, the first the reference) and then the sort cadence by
        timed trials (advances the simulation); returns (tile, sort_every)."""
        flat = (C.c_int * (3 * len(tiles)))(*[int(v) for t in tiles for v in t])
        tout, sout = (C.c_int * 3)(), C.c_int()
        self._check(self.L.pic_autotune_tiles(self.h, flat, len(tiles), int(max_sort_every), tout, C.byref(sout)))
        return tuple(int(v) for v in tout), sout.value

    def sync(self):
        self._check(self.L.pic_sync(self.h))

    def sort(self):
        self._check(self.L.pic_sort(self.h))

    # ------------------------------------------------------------------ getters
    def get_field(self, which, out=None):
        """Grid component as (nz, ny, nx) float32: numpy by default, or into `out`
        (a numpy array or a CUDA tensor of ncell floats)."""
        if out is None:
            out = np.empty((self.grid[2], self.grid[1], self.grid[0]), np.float32)
        self._check(self.L.pic_get_fields(self.h, int(which), _ptr(out), self.ncell))
        return out

    def set_field(self, which, src):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, np.float32)
        self._check(self.L.pic_set_fields(self.h, int(which), _ptr(src), self.ncell))

    def get_count(self, sid):
        n = C.c_int64()
        self._check(self.L.pic_get_count(self.h, int(sid), C.byref(n)))
        return n.value

    def get_particles(self, sid):
        n = self.get_count(sid)
        cap = max(n, 1)
        cell = np.zeros((3, cap), np.int32)
        off = np.zeros((3, cap), np.float32)
        u = np.zeros((3, cap), np.float32)
        w = np.zeros(cap, np.float32)
        ids = np.zeros(cap, np.int64)
        nn = C.c_int64()
        self._check(self.L.pic_get_particles(self.h, int(sid), cap, C.byref(nn), _ptr(cell), _ptr(off),
                                             _ptr(u), _ptr(w), _ptr(ids)))
        k = nn.value
        return {"cell": cell[:, :k].T.copy(), "off": off[:, :k].T.copy(), "u": u[:, :k].T.copy(),
                "w": w[:k].copy(), "id": ids[:k].copy()}

    def get_moments(self, sid, frame=PIC_FRAME_BOOSTED, k_bunch=0.0):
        m = pic_moments()
        self._check(self.L.pic_get_moments(self.h, int(sid), int(frame), float(k_bunch), C.byref(m)))
        return dict(zip(MOMENT_NAMES, list(m.v)))

    def trace_enable(self, on=True):
        self._check(self.L.pic_trace_enable(self.h, int(bool(on))))

    def trace_read(self):
        t = pic_trace()
        self._check(self.L.pic_trace_read(self.h, C.byref(t)))
        return {"ms": {TRACE_CLASSES[k]: t.ms[k] for k in range(7)},
                "events": {TRACE_CLASSES[k]: int(t.events[k]) for k in range(7)},
                "kernels": int(t.kernels), "fallback": int(t.fallback)}

    def get_time(self):
        out = (C.c_int64 * 3)()
        self._check(self.L.pic_get_time(self.h, out))
        return tuple(int(v) for v in out)


def resonant_wavenumber(lambda_u: float, K: float, gamma_B: float, gamma_R: float = 1.0,
                        frame: int = PIC_FRAME_LAB) -> float:
    """FEL resonant wavenumber of Eq. RadLambda (pic_resonant_wavenumber): the lab value, or its
    image in the frame of Lorentz factor gamma_R (frame=PIC_FRAME_BOOSTED)."""
    L = lib()
    k = C.c_double()
    r = L.pic_resonant_wavenumber(float(K), float(lambda_u), float(gamma_B), float(gamma_R), int(frame), C.byref(k))
    if r != 0:
        raise PicError(r, L.pic_last_error(None).decode())
    return k.value


def from_workload(w, device=0, stream=None, tuning=None, beam=True, beam_arrays=None):
    """Create a Sim for a workload of :mod:`paper_2411_04703_gb300.workloads` and load its
    undulator, plasma and (seeded) beam.  Returns (sim, species ids dict)."""
    from . import workloads as W
    t = tuning if tuning is not None else {"tile": w.tile, "sort_every": w.sort_every, "margin": 1}
    sim = Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
              moving_window=w.moving_window, window_v=w.window_v, device=device, stream=stream,
              tuning=t)
    ids = {}
    if w.undulator is not None:
        un = w.undulator
        sim.set_external_field(un.K, un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
    if w.plasma is not None:
        p = w.plasma
        ids["plasma_e"], ids["plasma_i"] = sim.set_plasma(p.ppc, p.xrange, p.z_nodes, p.n_nodes)
    if beam and w.beam is not None:
        if beam_arrays is None:
            beam_arrays = W.sample_beam(w)
        x, u, wt = beam_arrays
        b = w.beam
        ids["beam"] = sim.load_species(b.q, b.m, x, u, wt, frame=PIC_FRAME_LAB, origin=b.origin,
                                       match_undulator=bool(w.undulator is not None and w.undulator.match))
    return sim, ids


def from_ensemble(e, device=0, stream=None, tuning=None, beam=True):
    """Create an ensemble Sim for a :class:`workloads.Ensemble` (runs stacked along z) and load
    every run's undulator K, plasma density and seeded beam.  Returns (sim, species ids dict)."""
    from . import workloads as W
    b = e.base
    t = tuning if tuning is not None else {"tile": b.tile, "sort_every": b.sort_every, "margin": 1}
    sim = Sim(b.grid, b.d, b.dt, b.gamma_R, bc=b.bc, pml=b.pml, order=b.order, device=device, stream=stream,
              tuning=t, runs=e.runs)
    ids = {}
    if b.undulator is not None:
        sim.set_external_field_batch(e.K, b.undulator.lambda_u, b.undulator.phase)
    if b.plasma is not None:
        p = b.plasma
        ids["plasma_e"], ids["plasma_i"] = sim.set_plasma_batch(p.ppc, p.xrange, p.z_nodes, p.n_nodes, e.dens_scale)
    if beam and b.beam is not None:
        parts = [W.sample_beam(W.ensemble_run(e, r)) for r in range(e.runs)]
        x = np.concatenate([q[0] for q in parts], axis=1)
        u = np.concatenate([q[1] for q in parts], axis=1)
        wt = np.concatenate([q[2] for q in parts])
        ids["beam"] = sim.load_species_batch(b.beam.q, b.beam.m, [q[0].shape[1] for q in parts], x, u, wt,
                                             frame=PIC_FRAME_LAB, origin=b.beam.origin,
                                             match_undulator=bool(b.undulator is not None and b.undulator.match))
    return sim, ids


def rrf_resonant_wavenumber(w) -> float:
    """The boosted-frame image of the lab resonant wavenumber of workload ``w`` (its undulator's
    K and period, the beam's gamma, the frame's gamma_R), from pic_resonant_wavenumber."""
    un = w.undulator
    return resonant_wavenumber(un.lambda_u, un.K, w.beam.gamma, w.gamma_R, PIC_FRAME_BOOSTED)


_BUNCHING_FN = None


def _bunching_fn():
    global _BUNCHING_FN
    if _BUNCHING_FN is not None:
        return _BUNCHING_FN
    import copy

    import torch

    class BunchingLoss(torch.autograd.Function):
        """Forward: run the workload with (K, profile) and return the bunching factor; backward:
        the gradients pic_backward computed during the forward, times the incoming gradient."""

        @staticmethod
        def forward(ctx, K, profile, w, species, every, k_bunch, device):
            nodes = tuple(float(v) for v in profile.detach().to("cpu", torch.float64).reshape(-1).tolist())
            if w.plasma is None or len(nodes) != len(w.plasma.z_nodes):
                raise ValueError("profile needs one density per plasma profile node of the workload")
            wk = copy.deepcopy(w)
            wk.plasma.n_nodes = nodes
            sim, ids = from_workload(wk, device=device)
            try:
                un = wk.undulator
                sim.set_external_field(float(K), un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
                sim.checkpoint(every)
                sim.step(wk.steps)
                g = sim.backward(ids[species], k_bunch)
            finally:
                sim.close()
            ctx.meta = (K.dtype, K.device, profile.dtype, profile.device, profile.shape)
            ctx.save_for_backward(torch.tensor(float(g["dL_dK"]), dtype=torch.float64),
                                  torch.tensor(np.asarray(g["dL_dprofile"], np.float64)))
            return torch.tensor(float(g["loss"]), dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            dK, dP = ctx.saved_tensors
            kt, kd, pt, pd, ps = ctx.meta
            grad = grad.to("cpu", torch.float64)
            return ((grad * dK).to(kd, kt), (grad * dP).reshape(ps).to(pd, pt),
                    None, None, None, None, None)

    _BUNCHING_FN = BunchingLoss
    return BunchingLoss


def bunching_loss(w, K, profile, species="beam", checkpoint_every=10, k_bunch=None, device=0):
    """Differentiable loss for torch: the boosted-frame bunching factor of ``species`` after
    ``w.steps`` steps of workload ``w``, run with undulator strength ``K`` and plasma profile node
    densities ``profile`` (lab, units of n_n, one per node of ``w.plasma.z_nodes``).

    ``K`` (0-d) and ``profile`` are tensors; ``loss.backward()`` gives their gradients from
    pic_backward (checkpoints every ``checkpoint_every`` steps, segment recompute, adjoint sweep).
    K enters through the undulator field seen during the steps; the beam is loaded matched to
    ``w.undulator.K`` and held fixed.  ``k_bunch`` defaults to the boosted-frame image of the
    resonant wavenumber at ``w.undulator.K`` (fixed, so it carries no gradient).  The forward runs
    the whole simulation on the GPU; only the loss and the gradients come back.
    """
    kb = rrf_resonant_wavenumber(w) if k_bunch is None else float(k_bunch)
    return _bunching_fn().apply(K, profile, w, species, int(checkpoint_every), kb, device)
