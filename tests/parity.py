"""Helpers for the GPU-vs-oracle parity tests (imported by tests/ and __graft_entry__.smoke()).

The CUDA path is driven through its C-ABI binding; the FP64 oracle is loaded with the
GPU's exact state (cell + float offset widened to FP64, float momenta, weights, ids and
fields), so that one step of each starts from an identical state.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2411_04703_gb300 import api

SPECIES_QM = {"plasma_e": (-1.0, 1.0, False), "plasma_i": (1.0, 1836.15267343, True)}


def species_params(w, name):
    if name == "beam":
        return w.beam.q, w.beam.m, False
    return SPECIES_QM[name]


def plasma_next_id(w, m_last):
    p = w.plasma
    lo = 1 if w.order == 1 else 2
    m_first = math.ceil(p.ppc[2] * lo - 0.5)
    per_plane = (p.xrange[1] - p.xrange[0]) * (p.xrange[3] - p.xrange[2]) * p.ppc[0] * p.ppc[1]
    return (m_last - m_first + 1) * per_plane


def oracle_from_gpu(w, sim, ids, fields=True):
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order,
                   moving_window=w.moving_window, window_v=w.window_v)
    oid = {}
    for name, sid in sorted(ids.items(), key=lambda kv: kv[1]):
        q, m, frozen = species_params(w, name)
        oid[name] = o.add_species(q, m, frozen=frozen, capacity=1024)
        P = sim.get_particles(sid)
        X = P["cell"].astype(np.float64) + P["off"].astype(np.float64)
        o.set_state(oid[name], X, P["u"].astype(np.float64), P["w"].astype(np.float64), P["id"])
    if w.undulator is not None:
        un = w.undulator
        o.set_external(un.K, un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
    step, shifts, m_last = sim.get_time()
    if w.plasma is not None:
        p = w.plasma
        o.set_plasma(oid["plasma_e"], oid["plasma_i"], p.ppc, p.xrange, p.z_nodes, p.n_nodes, fill=False)
        nxt = plasma_next_id(w, m_last)
        o.set_next_id(oid["plasma_e"], nxt)
        o.set_next_id(oid["plasma_i"], nxt)
    o.set_time(step, shifts, m_last)
    if fields:
        for c in range(6):
            o.set_field(c, sim.get_field(c).astype(np.float64))
    return o, oid


def rel_err(g, r):
    den = np.max(np.abs(r))
    if den == 0:
        return float(np.max(np.abs(g)))
    return float(np.max(np.abs(g - r)) / den)


def compare_species(w, sim, sid, o, osid, tie=1e-5):
    """Match particles by id; returns a dict of parity figures."""
    P = sim.get_particles(sid)
    X, U, Wt, ids = o.particles(osid)
    gi = np.argsort(P["id"], kind="stable")
    oi = np.argsort(ids, kind="stable")
    gid, oidv = P["id"][gi], ids[oi]
    common, ga, oa = np.intersect1d(gid, oidv, return_indices=True)
    only_gpu = len(gid) - len(common)
    only_oracle = len(oidv) - len(common)
    cg = P["cell"][gi][ga].astype(np.int64)
    Xg = cg + P["off"][gi][ga].astype(np.float64)
    Xo = X[oi][oa]
    co = np.floor(Xo).astype(np.int64)
    n = np.array(w.grid)
    frac = Xo - np.floor(Xo)
    is_tie = np.any(np.minimum(frac, 1 - frac) < tie, axis=1)
    cell_mismatch = int(np.sum(np.any(cg != co, axis=1) & ~is_tie))
    dX = Xg - Xo
    for dd in range(3):
        if w.bc[dd][0] == 0:
            dX[:, dd] = (dX[:, dd] + n[dd] / 2) % n[dd] - n[dd] / 2
    Ug = P["u"][gi][ga].astype(np.float64)
    Uo = U[oi][oa]
    out = {
        "n": len(common), "only_gpu": only_gpu, "only_oracle": only_oracle,
        "ties": int(np.sum(is_tie)), "cell_mismatch": cell_mismatch,
        "pos_abs_err": float(np.max(np.abs(dX))) if len(common) else 0.0,
        "u_rel_err": max(rel_err(Ug[:, c], Uo[:, c]) for c in range(3)) if len(common) else 0.0,
        # per particle |u_gpu - u_ref| / |u_ref|: the per-component figure above is ill-conditioned
        # for a component that is the residual of cancelling forces (a lab-static plasma electron
        # in the undulator: E'_x = -beta_R B'_y and v_z = -beta_R cancel exactly)
        "u_vec_rel_err": float(np.max(np.linalg.norm(Ug - Uo, axis=1) /
                                      np.maximum(np.linalg.norm(Uo, axis=1), 1e-300))) if len(common) else 0.0,
    }
    return out


def compare_fields(sim, o, comps=range(9)):
    names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]
    return {names[c]: rel_err(sim.get_field(c).astype(np.float64), o.field(c)) for c in comps}


def run_particles(sim, sid, run, nzr):
    """GPU particles of one run of an ensemble, cells in the run's own coordinates."""
    P = sim.get_particles(sid)
    k = P["cell"][:, 2]
    m = (k >= run * nzr) & (k < (run + 1) * nzr)
    out = {key: v[m].copy() for key, v in P.items()}
    out["cell"][:, 2] -= run * nzr
    return out


def oracle_from_gpu_run(e, sim, ids, run, fields=True):
    """FP64 oracle of run `run` of an ensemble, loaded with that run's exact GPU state."""
    from paper_2411_04703_gb300 import workloads as W
    w = W.ensemble_run(e, run)
    nzr = w.grid[2]
    o = oracle.Sim(w.grid, w.d, w.dt, w.gamma_R, bc=w.bc, pml=w.pml, order=w.order)
    oid = {}
    for name, sid in sorted(ids.items(), key=lambda kv: kv[1]):
        q, m, frozen = species_params(w, name)
        oid[name] = o.add_species(q, m, frozen=frozen, capacity=1024)
        P = run_particles(sim, sid, run, nzr)
        X = P["cell"].astype(np.float64) + P["off"].astype(np.float64)
        o.set_state(oid[name], X, P["u"].astype(np.float64), P["w"].astype(np.float64), P["id"])
    if w.undulator is not None:
        un = w.undulator
        o.set_external(un.K, un.lambda_u, un.phase, un.z_start, un.ramp, kind=un.kind)
    step, shifts, m_last = sim.get_time()
    if w.plasma is not None:
        p = w.plasma
        o.set_plasma(oid["plasma_e"], oid["plasma_i"], p.ppc, p.xrange, p.z_nodes, p.n_nodes, fill=False)
    o.set_time(step, shifts, m_last)
    if fields:
        for c in range(6):
            o.set_field(c, sim.get_field(c)[run * nzr:(run + 1) * nzr].astype(np.float64))
    return o, oid


def compare_species_run(e, sim, sid, o, osid, run):
    """compare_species for one run of an ensemble."""
    from paper_2411_04703_gb300 import workloads as W
    w = W.ensemble_run(e, run)

    class _View:
        def get_particles(self, _sid):
            return run_particles(sim, sid, run, w.grid[2])

    return compare_species(w, _View(), sid, o, osid)


def compare_fields_run(sim, o, run, nzr, comps=range(9), j_scale=0.0, dt=0.0):
    """Per-component relative errors of one run; with j_scale, J components are measured against
    max(max|J_ref|, j_scale) and E, B components against max(max|F_ref|, dt j_scale): E^{n+1} takes
    dt J, and B^{n+1} takes (dt/2) curl of that, which is smaller for dt < dx (see current_scale)."""
    names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]
    out = {}
    for c in comps:
        g = sim.get_field(c)[run * nzr:(run + 1) * nzr].astype(np.float64)
        floor = j_scale if c >= 6 else dt * j_scale
        out[names[c]] = rel_err_scaled(g, o.field(c), floor)
    return out


def current_scale(w, parts):
    """Largest current density one species carries in one cell, max over species of
    max_cell sum_p |q w_p v_p| / V (parts: {name: GPU particle dict}).  The reference scale of a
    current component that is the residual of opposite species' currents (a neutral drifting
    plasma's electron and ion currents cancel), and, times dt, of the field it drives."""
    V = w.d[0] * w.d[1] * w.d[2]
    nx, ny, nz = w.grid
    best = 0.0
    for name, P in parts.items():
        q = species_params(w, name)[0]
        if len(P["id"]) == 0:
            continue
        u = P["u"].astype(np.float64)
        g = np.sqrt(1.0 + np.sum(u * u, axis=1))
        cell = P["cell"].astype(np.int64)
        lin = (cell[:, 2] * ny + cell[:, 1]) * nx + cell[:, 0]
        for c in range(3):
            j = np.bincount(lin, weights=np.abs(q * P["w"].astype(np.float64) * u[:, c] / g), minlength=nx * ny * nz)
            best = max(best, float(np.max(j)) / V)
    return best


def rel_err_scaled(g, r, floor):
    den = max(float(np.max(np.abs(r))), floor)
    return float(np.max(np.abs(g - r)) / den) if den > 0 else float(np.max(np.abs(g)))
