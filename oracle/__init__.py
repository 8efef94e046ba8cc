"""FP64 CPU oracle of the column-generation VMAT optimiser (ctypes over vmat_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product path never does.  It
shares no code with the CUDA library.  See vmat_oracle.c for the equations
each routine follows (Eq. 1 cost, Eq. 2 smoothing, Eq. 3 model, Sec. 2.2
pricing and master problem).

Every routine here is pinned by tests against something other than itself
(closed forms, brute force, an independent solver, invariants), except the
whole-plan result of the column-generation loop, whose parity is unpinned:
column generation with one aperture per beam is a heuristic for the
non-convex joint problem and the paper prints no plan values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_i64 = ctypes.c_int64
_c_i32 = ctypes.c_int
_c_d = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile vmat_oracle.c into liboracle.so (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        sig = {
            "vo_F": (_c_d, [_c_d, _c_d, _c_d, _c_d]),
            "vo_dF": (_c_d, [_c_d, _c_d, _c_d, _c_d]),
            "vo_voxel_cost": (_c_d, [_c_i64, _p, _p, _p, _p, _p]),
            "vo_voxel_dcost": (None, [_c_i64, _p, _p, _p, _p, _p, _p]),
            "vo_G": (_c_d, [_c_i32, _p, _p, _c_i32]),
            "vo_dG": (None, [_c_i32, _p, _p, _c_i32, _p]),
            "vo_dose": (None, [_c_i64, _c_i64, _p, _p, _p, _p, _p]),
            "vo_price": (None, [_c_i64, ctypes.c_int32, _p, _p, _p, _p, _p, _p]),
            "vo_aperture_fluence": (None, [_c_i32, _c_i32, _c_i32, _p, _p, _p, _p]),
            "vo_aperture_adjoint": (None, [_c_i32, _c_i32, _c_i32, _p, _p, _p, _p]),
            "vo_aperture_dose": (None, [_c_i64, _c_i32, _c_i32, _p, _p, _p, _c_i32, _p, _p, _p]),
            "vo_leaf_limits": (None, [_c_i32] * 5 + [_p, _p, _p, _c_i32, _p, _p, _p, _p]),
            "vo_row_scan": (_c_i32, [_c_i32, _p, _c_i32, _c_i32, _c_i32, _c_i32, _p, _p, _p]),
            "vo_row_scan_f32": (_c_i32, [_c_i32, _p, _c_i32, _c_i32, _c_i32, _c_i32, _p, _p, _p]),
            "vo_pricing": (_c_i32, [_c_i32] * 5 + [_p, _p, _p, _p, _c_i32, _p, _p, _p, _p, _p, _p, _p, _p]),
            "vo_line_search": (_c_d, [_c_i64, _p, _p, _p, _p, _p, _p, _c_d, _c_d, _c_d]),
            "vo_master": (_c_i32, [_c_i64, _c_i32, _p, _p, _c_i32, _p, _c_i32, _c_d, _p, _p, _p,
                                   _p, _c_d, _c_d, _c_i32, _p, _p, _p]),
            "vo_dvh": (None, [_c_i64, _p, _p, _c_i32, _c_d, _c_i32, _p]),
            "vo_colgen": (_c_i32, [_c_i64, _c_i32, _c_i32, _c_i32, _p, _p, _p, _p, _p, _p, _p,
                                   _p, _c_d, _c_i32, _c_i32, _c_i32, _c_d, _c_i32, _p, _p, _p,
                                   _c_i32, _c_i32] + [_p] * 14),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- Eq. 1 / Eq. 2
def voxel_cost(z, sid, T, alpha, beta) -> float:
    """sum_j F(z_j), Eq. 1."""
    z, T, alpha, beta = _f64(z), _f64(T), _f64(alpha), _f64(beta)
    sid = np.ascontiguousarray(sid, dtype=np.uint8)
    return lib().vo_voxel_cost(z.size, _ptr(z), _ptr(sid), _ptr(T), _ptr(alpha), _ptr(beta))


def voxel_dcost(z, sid, T, alpha, beta) -> np.ndarray:
    """F'(z_j) per voxel, Eq. 1."""
    z, T, alpha, beta = _f64(z), _f64(T), _f64(alpha), _f64(beta)
    sid = np.ascontiguousarray(sid, dtype=np.uint8)
    out = np.empty_like(z)
    lib().vo_voxel_dcost(z.size, _ptr(z), _ptr(sid), _ptr(T), _ptr(alpha), _ptr(beta), _ptr(out))
    return out


def G(theta, y, cyclic=True) -> float:
    """Dose-rate smoothing term, Eq. 2 (ring if cyclic)."""
    theta, y = _f64(theta), _f64(y)
    return lib().vo_G(y.size, _ptr(theta), _ptr(y), int(cyclic))


def dG(theta, y, cyclic=True) -> np.ndarray:
    theta, y = _f64(theta), _f64(y)
    out = np.empty_like(y)
    lib().vo_dG(y.size, _ptr(theta), _ptr(y), int(cyclic), _ptr(out))
    return out


# ---------------------------------------------------------------- dose / price
def dose(prob, x) -> np.ndarray:
    """z = D^T x (z_j = sum_i D_ij x_i), Sec. 2.1."""
    x = _f64(x)
    z = np.empty(prob.n_vox)
    lib().vo_dose(prob.n_beamlets, prob.n_vox, _ptr(prob.row_ptr), _ptr(prob.vox_idx),
                  _ptr(prob.val), _ptr(x), _ptr(z))
    return z


def price(prob, f, mask=None) -> np.ndarray:
    """g_i = sum_j D_ij f_j; beams with mask[k] == 0 are left at 0."""
    f = _f64(f)
    cfg = prob.cfg
    g = np.zeros(prob.n_beamlets)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    lib().vo_price(prob.n_beamlets, cfg.n_rows * cfg.n_cols, _ptr(prob.row_ptr),
                   _ptr(prob.vox_idx), _ptr(prob.val), _ptr(f), _ptr(m), _ptr(g))
    return g


def aperture_fluence(cfg, l, r, y) -> np.ndarray:
    l = np.ascontiguousarray(l, dtype=np.int16)
    r = np.ascontiguousarray(r, dtype=np.int16)
    y = _f64(y)
    x = np.empty(cfg.n_beamlets)
    lib().vo_aperture_fluence(cfg.n_angles, cfg.n_rows, cfg.n_cols, _ptr(l), _ptr(r), _ptr(y), _ptr(x))
    return x


def aperture_adjoint(cfg, l, r, g) -> np.ndarray:
    l = np.ascontiguousarray(l, dtype=np.int16)
    r = np.ascontiguousarray(r, dtype=np.int16)
    g = _f64(g)
    out = np.empty(cfg.n_angles)
    lib().vo_aperture_adjoint(cfg.n_angles, cfg.n_rows, cfg.n_cols, _ptr(l), _ptr(r), _ptr(g), _ptr(out))
    return out


def aperture_dose(prob, k, l, r) -> np.ndarray:
    """Column k of the aperture-dose matrix: sum over open beamlets of D_i,: ."""
    cfg = prob.cfg
    l = np.ascontiguousarray(l, dtype=np.int16)
    r = np.ascontiguousarray(r, dtype=np.int16)
    col = np.empty(prob.n_vox)
    lib().vo_aperture_dose(prob.n_vox, cfg.n_rows, cfg.n_cols, _ptr(prob.row_ptr),
                           _ptr(prob.vox_idx), _ptr(prob.val), int(k), _ptr(l), _ptr(r), _ptr(col))
    return col


# ---------------------------------------------------------------- pricing
def leaf_limits(N, R, C, s, cyclic, occ, lleaf, rleaf, k):
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    lleaf = np.ascontiguousarray(lleaf, dtype=np.int16)
    rleaf = np.ascontiguousarray(rleaf, dtype=np.int16)
    out = np.zeros((4, R), dtype=np.int32)
    lib().vo_leaf_limits(N, R, C, s, int(cyclic), _ptr(occ), _ptr(lleaf), _ptr(rleaf), int(k),
                         _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _ptr(out[3]))
    return out  # rows: Llo, Lhi, Rlo, Rhi


def row_scan(g, Llo, Lhi, Rlo, Rhi, f32=False):
    """(value, l, r) of the single left-to-right pass, or None if infeasible."""
    C = len(g)
    l = ctypes.c_int()
    r = ctypes.c_int()
    if f32:
        gg = np.ascontiguousarray(g, dtype=np.float32)
        v = ctypes.c_float()
        rc = lib().vo_row_scan_f32(C, _ptr(gg), Llo, Lhi, Rlo, Rhi, ctypes.byref(v), ctypes.byref(l), ctypes.byref(r))
    else:
        gg = _f64(g)
        v = ctypes.c_double()
        rc = lib().vo_row_scan(C, _ptr(gg), Llo, Lhi, Rlo, Rhi, ctypes.byref(v), ctypes.byref(l), ctypes.byref(r))
    return None if rc != 0 else (v.value, l.value, r.value)


def pricing(cfg, occ, lleaf, rleaf, g, f32=False, N=None, R=None, C=None, s=None, cyclic=None,
            offset=None):
    """Pricing subproblem over beams without an aperture (Sec. 2.2).
    offset [N]: added to each beam's aperture price (None: the beamlet sum
    alone); smoothing_offset() gives the one of the exact reduced cost.
    Returns dict(k, l, r, p, p2, row_margin) or raises on failure."""
    N = cfg.n_angles if N is None else N
    R = cfg.n_rows if R is None else R
    C = cfg.n_cols if C is None else C
    s = cfg.max_leaf_step if s is None else s
    cyclic = cfg.cyclic if cyclic is None else cyclic
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    lleaf = np.ascontiguousarray(lleaf, dtype=np.int16)
    rleaf = np.ascontiguousarray(rleaf, dtype=np.int16)
    g = _f64(g)
    k = ctypes.c_int()
    lo = np.zeros(R, dtype=np.int16)
    ro = np.zeros(R, dtype=np.int16)
    p = ctypes.c_double()
    p2 = ctypes.c_double()
    rm = ctypes.c_double()
    res = np.zeros(2)
    off = None if offset is None else _f64(offset)
    if off is not None and off.size != N:
        raise ValueError("offset must have one value per beam")
    rc = lib().vo_pricing(N, R, C, s, int(cyclic), _ptr(occ), _ptr(lleaf), _ptr(rleaf), _ptr(g),
                          int(f32), ctypes.byref(k), _ptr(lo), _ptr(ro), ctypes.byref(p),
                          ctypes.byref(p2), ctypes.byref(rm), _ptr(off), _ptr(res))
    if rc != 0:
        raise RuntimeError(f"oracle pricing failed: {rc}")
    return dict(k=k.value, l=lo, r=ro, p=p.value, p2=p2.value, row_margin=rm.value,
                f32_res=res[0], row_res=res[1])


def smoothing_offset(theta, y, gamma, cyclic=True) -> np.ndarray:
    """gamma * dG/dy at y (Eq. 2): for a beam without an aperture (y_k = 0)
    the smoothing part of the derivative of Eq. 3 along its new column."""
    return gamma * dG(theta, y, cyclic)


# ---------------------------------------------------------------- master
def line_search(z, w, sid, T, alpha, beta, gdot, Gd, gamma) -> float:
    z, w, T, alpha, beta = _f64(z), _f64(w), _f64(T), _f64(alpha), _f64(beta)
    sid = np.ascontiguousarray(sid, dtype=np.uint8)
    return lib().vo_line_search(z.size, _ptr(z), _ptr(w), _ptr(sid), _ptr(T), _ptr(alpha),
                                _ptr(beta), gdot, Gd, gamma)


def master(M, col_beam, theta, sid, T, alpha, beta, gamma, cyclic, y0, eps=1e-8, max_iter=100000,
           rho_ref=0.0):
    """Projected-gradient master problem.  M: [ncol, V] columns; col_beam[q]
    is the beam of column q; y0 [N] warm start.  Stops at
    rho <= eps*max(rho_start, rho_ref).  Returns dict(y, z, cost, rho, rho0,
    iters, status)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    ncol, V = M.shape
    col_beam = np.ascontiguousarray(col_beam, dtype=np.int32)
    theta, T, alpha, beta = _f64(theta), _f64(T), _f64(alpha), _f64(beta)
    sid = np.ascontiguousarray(sid, dtype=np.uint8)
    y = _f64(y0).copy()
    z = np.empty(V)
    out = np.zeros(4)
    st = lib().vo_master(V, ncol, _ptr(M), _ptr(col_beam), y.size, _ptr(theta), int(cyclic),
                         gamma, _ptr(sid), _ptr(T), _ptr(alpha), _ptr(beta), eps, rho_ref, max_iter,
                         _ptr(y), _ptr(z), _ptr(out))
    return dict(y=y, z=z, cost=out[0], rho=out[1], rho0=out[2], iters=int(out[3]), status=st)


# ---------------------------------------------------------------- column generation
def colgen(prob, n_iter=None, eps=None, max_iter=100000, forced=None, f32_pricing=False,
           price_smoothing=False):
    """Column generation (Sec. 2.2, Fig. 1) from an empty plan.
    forced: optional (k [n_iter], l [n_iter, R], r [n_iter, R]) to replay.
    price_smoothing: price each beam by the exact reduced cost (beamlet sum
    plus gamma dG/dy_k at the current y) instead of the beamlet sum alone.
    Returns a dict of per-iteration records and the final plan."""
    cfg = prob.cfg
    N, R, C = cfg.n_angles, cfg.n_rows, cfg.n_cols
    n_iter = cfg.iterations if n_iter is None else n_iter
    eps = cfg.kkt_eps if eps is None else eps
    rec = dict(k=np.zeros(n_iter, np.int32), p=np.zeros(n_iter), margin=np.zeros(n_iter),
               row_margin=np.zeros(n_iter), f32_res=np.zeros(n_iter), row_res=np.zeros(n_iter),
               cost=np.zeros(n_iter), rho=np.zeros(n_iter),
               iters=np.zeros(n_iter, np.int32), status=np.zeros(n_iter, np.int32))
    y = np.zeros(N)
    z = np.zeros(prob.n_vox)
    lleaf = np.zeros(N * R, np.int16)
    rleaf = np.zeros(N * R, np.int16)
    fk = fl = fr = None
    if forced is not None:
        fk = np.ascontiguousarray(forced[0], dtype=np.int32)
        fl = np.ascontiguousarray(forced[1], dtype=np.int16)
        fr = np.ascontiguousarray(forced[2], dtype=np.int16)
    T, alpha, beta, theta = _f64(prob.T), _f64(prob.alpha), _f64(prob.beta), _f64(prob.theta_deg)
    rc = lib().vo_colgen(
        prob.n_vox, N, R, C, _ptr(prob.row_ptr), _ptr(prob.vox_idx), _ptr(prob.val),
        _ptr(prob.struct_id), _ptr(T), _ptr(alpha), _ptr(beta), _ptr(theta), cfg.gamma,
        int(cfg.cyclic), cfg.max_leaf_step, n_iter, eps, max_iter, _ptr(fk), _ptr(fl), _ptr(fr),
        int(f32_pricing), int(price_smoothing), _ptr(rec["k"]), _ptr(rec["p"]), _ptr(rec["margin"]),
        _ptr(rec["row_margin"]), _ptr(rec["f32_res"]), _ptr(rec["row_res"]), _ptr(rec["cost"]), _ptr(rec["rho"]), _ptr(rec["iters"]),
        _ptr(rec["status"]), _ptr(y), _ptr(z), _ptr(lleaf), _ptr(rleaf))
    if rc != 0:
        raise RuntimeError(f"oracle colgen failed: {rc}")
    rec.update(y=y, z=z, lleaf=lleaf, rleaf=rleaf)
    return rec


# ---------------------------------------------------------------- plan evaluation (Fig. 2)
def dvh(z, sid, n_struct, dose_max, n_bins) -> np.ndarray:
    """Dose-volume histogram counts [n_struct, n_bins] of the dose z: voxel j
    of structure sid[j] in bin b when b*w <= z_j < (b+1)*w, w =
    dose_max/n_bins (doses >= dose_max in the last bin, < 0 in the first)."""
    z = _f64(z)
    sid = np.ascontiguousarray(sid, dtype=np.uint8)
    if sid.size != z.size or (sid.size and int(sid.max()) >= n_struct):
        raise ValueError("sid must give every voxel a structure < n_struct")
    if not (dose_max > 0) or n_bins < 1:
        raise ValueError("dose_max > 0 and n_bins >= 1 required")
    out = np.zeros((n_struct, n_bins), np.int64)
    lib().vo_dvh(z.size, _ptr(z), _ptr(sid), int(n_struct), float(dose_max), int(n_bins), _ptr(out))
    return out


# ---------------------------------------------------------------- dose-rate feasibility (Sec. 3)
def rate_violation(theta, y, max_rate, cyclic=True) -> float:
    """Largest dose-rate variation over neighbouring beams, |y_k' - y_k| / gap
    (gap in degrees, the wrap pair included on a ring), minus max_rate."""
    theta, y = _f64(theta), _f64(y)
    n = y.size
    if n < 2:
        return -float(max_rate)
    worst = -np.inf
    pairs = [(k, k + 1) for k in range(n - 1)] + ([(n - 1, 0)] if cyclic else [])
    for k, kp in pairs:
        gap = theta[kp] - theta[k] if kp > k else theta[0] + 360.0 - theta[n - 1]
        worst = max(worst, abs(y[kp] - y[k]) / gap - max_rate)
    return float(worst)


def dose_rate_feasibility(prob, col_beam, lleaf, rleaf, y0, max_rate, gamma_factor=2.0,
                          max_rounds=20, eps=1e-8, rho_ref=0.0, max_iter=100000):
    """Sec. 3, final step: the smoothing term of Eq. 2 is a soft penalty; to
    meet a hard limit on the dose-rate variation the weight gamma is raised
    and the intensities of the final apertures re-optimised (master problem,
    warm start from the last y) until the plan is feasible.  Each round
    multiplies gamma by gamma_factor.  Returns dict(y, gamma, rounds,
    violation, cost, G) with cost = Eq. 3 at the end (final gamma) and G the
    smoothing term of each round's solution (round 0: the starting y)."""
    cfg = prob.cfg
    R = cfg.n_rows
    col_beam = np.asarray(col_beam, dtype=np.int32)
    M = np.array([aperture_dose(prob, k, lleaf[k * R:(k + 1) * R], rleaf[k * R:(k + 1) * R])
                  for k in col_beam])
    theta = prob.theta_deg
    gamma = cfg.gamma
    y = _f64(y0).copy()
    v = rate_violation(theta, y, max_rate, cfg.cyclic)
    Gs = [G(theta, y, cfg.cyclic)]
    rounds = 0
    while v > 0.0 and rounds < max_rounds:
        gamma *= gamma_factor
        rounds += 1
        res = master(M, col_beam, theta, prob.struct_id, prob.T, prob.alpha, prob.beta, gamma,
                     cfg.cyclic, y, eps=eps, max_iter=max_iter, rho_ref=rho_ref)
        y = res["y"]
        v = rate_violation(theta, y, max_rate, cfg.cyclic)
        Gs.append(G(theta, y, cfg.cyclic))
    z = M.T @ y[col_beam]
    cost = voxel_cost(z, prob.struct_id, prob.T, prob.alpha, prob.beta) + gamma * G(theta, y, cfg.cyclic)
    return dict(y=y, gamma=gamma, rounds=rounds, violation=v, cost=cost, G=np.array(Gs))
