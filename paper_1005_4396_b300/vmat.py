"""Python binding of libvmat (include/vmat.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module passes
torch tensors' device pointers and host numpy arrays through ctypes.  There is
no CPU fallback: if libvmat.so is missing or no CUDA device is present,
loading fails with an error.

Module-level functions carry the C names (vmat_create, vmat_dose, ...);
`Plan` wraps one context for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvmat.so")

VMAT_OK, VMAT_EINVAL, VMAT_ENOMEM, VMAT_ECUDA, VMAT_ENOTCONV, VMAT_ETIMEOUT, VMAT_ESTATE = range(7)
VMAT_F64, VMAT_F32, VMAT_F16, VMAT_BF16 = range(4)
DTYPES = {"f32": VMAT_F32, "f16": VMAT_F16, "bf16": VMAT_BF16}
STATUS_NAMES = ["VMAT_OK", "VMAT_EINVAL", "VMAT_ENOMEM", "VMAT_ECUDA", "VMAT_ENOTCONV",
                "VMAT_ETIMEOUT", "VMAT_ESTATE"]

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double


class VmatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class vmat_problem(ctypes.Structure):
    _fields_ = [("n_vox", _i32), ("n_angles", _i32), ("n_rows", _i32), ("n_cols", _i32),
                ("theta_deg", _p), ("struct_id", _p), ("n_struct", _i32), ("T", _p),
                ("alpha", _p), ("beta", _p), ("gamma", _d), ("cyclic", _i32),
                ("max_leaf_step", _i32), ("nnz", _i64), ("row_ptr", _p), ("vox_idx", _p),
                ("val_dtype", ctypes.c_int), ("val", _p)]


class vmat_info(ctypes.Structure):
    _fields_ = [("n_vox", _i32), ("n_active", _i32), ("n_angles", _i32), ("n_rows", _i32),
                ("n_cols", _i32), ("n_beamlets", _i64), ("nnz", _i64), ("n_columns", _i32),
                ("device_bytes", _i64), ("d_dtype", ctypes.c_int), ("master_grid", _i32),
                ("master_block", _i32), ("n_launches", _i64), ("master_ms", _d * 4),
                ("master_syncs", _i64), ("master_wait_ms", _d), ("master_pg_iters", _i64), ("master_rejected", _i64), ("subtile_voxels", _i32),
                ("n_subtiles", _i32), ("tile_entries", _i64 * 2), ("price_calls", _i64 * 2),
                ("price_live_entries", _i64)]


class vmat_column(ctypes.Structure):
    _fields_ = [("angle", _i32), ("price", _d), ("runner_up", _d), ("l", _p), ("r", _p)]


class vmat_colgen_opts(ctypes.Structure):
    _fields_ = [("n_iters", _i32), ("master_max_iters", _i32), ("kkt_tol", _d),
                ("forced_angle", _p), ("forced_l", _p), ("forced_r", _p)]


class vmat_colgen_result(ctypes.Structure):
    _fields_ = [("angle_order", _p), ("l", _p), ("r", _p), ("y", _p), ("price", _p),
                ("runner_up", _p), ("cost", _p), ("kkt", _p), ("master_iters", _p),
                ("phase_ms", _p), ("col_subtiles", _p), ("priced_angle", _p), ("priced_l", _p),
                ("priced_r", _p)]


EXPORTS = {
    "vmat_create": [ctypes.POINTER(vmat_problem), ctypes.c_int, _p, ctypes.POINTER(_p)],
    "vmat_destroy": [_p],
    "vmat_last_error": [_p],
    "vmat_get_info": [_p, ctypes.POINTER(vmat_info)],
    "vmat_dose": [_p, _p, _p, _p, _p],
    "vmat_price": [_p, _p, _p, _p],
    "vmat_pricing_select": [_p, _p, ctypes.POINTER(vmat_column)],
    "vmat_add_column": [_p, ctypes.POINTER(vmat_column)],
    "vmat_master_step": [_p, _i32, _d, _d, _p, _p, _p, _p],
    "vmat_plan_dose": [_p, _p],
    "vmat_reset": [_p],
    "vmat_colgen_run": [_p, ctypes.POINTER(vmat_colgen_opts), ctypes.POINTER(vmat_colgen_result)],
    "vmat_dose_batch32": [_p, _p, _p, _p, _p],
    "vmat_price_batch32": [_p, _p, _p, _p],
    "vmat_selftest_grid_wait": [_p, _i32, _d],
    "vmat_set_profiling": [_p, _i32],
    "vmat_dose_cost_noalloc": [_i32, _p, _p, _p, _p, _p, _p, _i32, _p, _p, _p, _p],
    "vmat_aperture_fluence_batch32": [_p, _p, _p, _p, _p],
    "vmat_aperture_adjoint_batch32": [_p, _p, _p, _p, _p, _p, _p],
    "vmat_smoothing_batch32": [_p, _p, _p, _p],
    "vmat_aperture_dose_cost_batch32": [_p, _p, _p, _p, _p, _p, _p, _p],
    "vmat_set_master_budget": [_p, _i32],
    "vmat_batch_create": [_p, _i32, _p, ctypes.POINTER(_p)],
    "vmat_batch_destroy": [_p],
    "vmat_batch_last_error": [_p],
    "vmat_batch_configure": [_p, _i32],
    "vmat_batch_tune": [_p, _i32, _i32, _d, _p, _p],
    "vmat_batch_colgen_run": [_p, _i32, _d, _p, _p, _p],
    "vmat_list_schedule": [_i32, _p, _p, _i32, _p, _p, _p, _p],
    "vmat_set_master_method": [_p, _i32],
    "vmat_set_price_smoothing": [_p, _i32],
    "vmat_set_price_path": [_p, _i32],
    "vmat_set_master_precision": [_p, _i32],
    "vmat_dvh": [_p, _p, _d, _i32, _p],
    "vmat_dose_rate_feasibility": [_p, _d, _d, _i32, _i32, _d, _p, _p, _p, _p, _p],
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libvmat.so and declare its entry points (no CUDA call is made)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libvmat.so not built ({path}); run python -m paper_1005_4396_b300.build")
        L = ctypes.CDLL(path)
        for name, args in EXPORTS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in ("vmat_destroy", "vmat_batch_destroy") else (
                ctypes.c_char_p if name in ("vmat_last_error", "vmat_batch_last_error") else ctypes.c_int)
        _lib = L
    return _lib


def _ptr(t):
    """Device pointer of a torch tensor / host pointer of a numpy array / None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _check(ctx, status):
    if status != VMAT_OK:
        msg = load_library().vmat_last_error(ctx)
        raise VmatError(status, msg.decode() if msg else "")


def _require_cuda(t, dtype, numel, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.numel() == numel):
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of {numel} elements")


# ---------------------------------------------------------------- C-named calls
def vmat_create(prob, dtype="f32", stream=None, val_f32=False):
    """Create a context from an inputs.Problem; returns (ctx handle, keepalive)."""
    L = load_library()
    theta = np.ascontiguousarray(prob.theta_deg, dtype=np.float64)
    sid = np.ascontiguousarray(prob.struct_id, dtype=np.uint8)
    T = np.ascontiguousarray(prob.T, dtype=np.float64)
    al = np.ascontiguousarray(prob.alpha, dtype=np.float64)
    be = np.ascontiguousarray(prob.beta, dtype=np.float64)
    rp = np.ascontiguousarray(prob.row_ptr, dtype=np.int64)
    vx = np.ascontiguousarray(prob.vox_idx, dtype=np.int32)
    if val_f32:
        val = np.ascontiguousarray(prob.val, dtype=np.float32)
        vdt = VMAT_F32
    else:
        val = np.ascontiguousarray(prob.val, dtype=np.float64)
        vdt = VMAT_F64
    cfg = prob.cfg
    P = vmat_problem(sid.size, cfg.n_angles, cfg.n_rows, cfg.n_cols, theta.ctypes.data,
                     sid.ctypes.data, T.size, T.ctypes.data, al.ctypes.data, be.ctypes.data,
                     cfg.gamma, int(cfg.cyclic), int(cfg.max_leaf_step), int(rp[-1]),
                     rp.ctypes.data, vx.ctypes.data, vdt, val.ctypes.data)
    h = _p()
    st = L.vmat_create(ctypes.byref(P), DTYPES[dtype], stream, ctypes.byref(h))
    if st != VMAT_OK:
        raise VmatError(st, L.vmat_last_error(None).decode())
    return h


def vmat_create_raw(P: vmat_problem, dtype=VMAT_F32, stream=None):
    L = load_library()
    h = _p()
    st = L.vmat_create(ctypes.byref(P), dtype, stream, ctypes.byref(h))
    if st != VMAT_OK:
        raise VmatError(st, L.vmat_last_error(None).decode())
    return h


def vmat_destroy(ctx):
    load_library().vmat_destroy(ctx)


def vmat_get_info(ctx) -> dict:
    inf = vmat_info()
    _check(ctx, load_library().vmat_get_info(ctx, ctypes.byref(inf)))
    out = {k: getattr(inf, k) for k, _ in vmat_info._fields_}
    out["master_ms"] = list(out["master_ms"])
    out["tile_entries"] = list(out["tile_entries"])
    out["price_calls"] = list(out["price_calls"])
    return out


def vmat_dose(ctx, x, z=None, fprime=None, want_cost=True):
    c = ctypes.c_double()
    _check(ctx, load_library().vmat_dose(ctx, _ptr(x), _ptr(z), _ptr(fprime),
                                         ctypes.byref(c) if want_cost else None))
    return c.value if want_cost else None


def vmat_price(ctx, f, g, mask=None):
    _check(ctx, load_library().vmat_price(ctx, _ptr(f), _ptr(mask), _ptr(g)))


def vmat_pricing_select(ctx, g, n_rows):
    l = np.zeros(n_rows, np.int16)
    r = np.zeros(n_rows, np.int16)
    col = vmat_column(0, 0.0, 0.0, l.ctypes.data, r.ctypes.data)
    _check(ctx, load_library().vmat_pricing_select(ctx, _ptr(g), ctypes.byref(col)))
    return dict(k=col.angle, p=col.price, p2=col.runner_up, l=l, r=r)


def vmat_add_column(ctx, k, l, r):
    l = np.ascontiguousarray(l, dtype=np.int16)
    r = np.ascontiguousarray(r, dtype=np.int16)
    col = vmat_column(int(k), 0.0, 0.0, l.ctypes.data, r.ctypes.data)
    _check(ctx, load_library().vmat_add_column(ctx, ctypes.byref(col)))


def vmat_master_step(ctx, max_iters, kkt_tol, rho_ref=0.0, y=None):
    """y: numpy float64 [N] warm start, updated in place (None: keep the context's y)."""
    cost, kkt, its = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    st = load_library().vmat_master_step(ctx, int(max_iters), float(kkt_tol), float(rho_ref),
                                         _ptr(y), ctypes.byref(cost), ctypes.byref(kkt),
                                         ctypes.byref(its))
    out = dict(cost=cost.value, kkt=kkt.value, iters=its.value, status=st)
    if st not in (VMAT_OK, VMAT_ENOTCONV):
        _check(ctx, st)
    return out


def vmat_plan_dose(ctx, z):
    _check(ctx, load_library().vmat_plan_dose(ctx, _ptr(z)))


def vmat_reset(ctx):
    _check(ctx, load_library().vmat_reset(ctx))


def vmat_colgen_run(ctx, N, R, n_iters, master_max_iters=100000, kkt_tol=1e-6, forced=None,
                    allow_notconv=False):
    fa = fl = fr = None
    if forced is not None:
        fa = np.ascontiguousarray(forced[0], dtype=np.int32)
        fl = np.ascontiguousarray(forced[1], dtype=np.int16)
        fr = np.ascontiguousarray(forced[2], dtype=np.int16)
    opts = vmat_colgen_opts(int(n_iters), int(master_max_iters), float(kkt_tol), _ptr(fa),
                            _ptr(fl), _ptr(fr))
    n = max(int(n_iters), 1)
    out = dict(k=np.zeros(n, np.int32), lleaf=np.zeros(N * R, np.int16),
               rleaf=np.zeros(N * R, np.int16), y=np.zeros(N), p=np.zeros(n), p2=np.zeros(n),
               cost=np.zeros(n), rho=np.zeros(n), iters=np.zeros(n, np.int32),
               phase_ms=np.zeros((n, 4)), col_subtiles=np.zeros(n, np.int32),
               priced_k=np.zeros(n, np.int32), priced_l=np.zeros((n, R), np.int16),
               priced_r=np.zeros((n, R), np.int16))
    res = vmat_colgen_result(*[out[k].ctypes.data for k in
                               ("k", "lleaf", "rleaf", "y", "p", "p2", "cost", "rho", "iters",
                                "phase_ms", "col_subtiles", "priced_k", "priced_l", "priced_r")])
    st = load_library().vmat_colgen_run(ctx, ctypes.byref(opts), ctypes.byref(res))
    out["status"] = st
    if st != VMAT_OK and not (allow_notconv and st == VMAT_ENOTCONV):
        _check(ctx, st)
    if n_iters == 0:
        for k in ("k", "p", "p2", "cost", "rho", "iters", "phase_ms", "col_subtiles", "priced_k",
                  "priced_l", "priced_r"):
            out[k] = out[k][:0]
    return out


def vmat_dose_batch32(ctx, X, Z, fprime=None, want_cost=True):
    c = (ctypes.c_double * 32)()
    _check(ctx, load_library().vmat_dose_batch32(ctx, _ptr(X), _ptr(Z), _ptr(fprime),
                                                 c if want_cost else None))
    return np.array(c[:]) if want_cost else None


def vmat_price_batch32(ctx, Fp, G, w=None):
    _check(ctx, load_library().vmat_price_batch32(ctx, _ptr(Fp), _ptr(w), _ptr(G)))


def vmat_dose_cost_noalloc(n_vox, row_ptr, beamlet, val, x, struct_id, params, n_struct,
                           z=None, fprime=None, cost=None, stream=None):
    """Dose + voxel cost with no device allocation by the library (tensors
    are the caller's; see include/vmat.h).  Enqueued on `stream`."""
    st = load_library().vmat_dose_cost_noalloc(
        int(n_vox), _ptr(row_ptr), _ptr(beamlet), _ptr(val), _ptr(x), _ptr(struct_id),
        _ptr(params), int(n_struct), _ptr(z), _ptr(fprime), _ptr(cost), stream)
    if st != VMAT_OK:
        raise VmatError(st, load_library().vmat_last_error(None).decode())


def vmat_aperture_fluence_batch32(ctx, l, r, Y, X):
    _check(ctx, load_library().vmat_aperture_fluence_batch32(ctx, _ptr(l), _ptr(r), _ptr(Y), _ptr(X)))


def vmat_aperture_adjoint_batch32(ctx, l, r, GX, GY, Y=None, w=None):
    _check(ctx, load_library().vmat_aperture_adjoint_batch32(ctx, _ptr(l), _ptr(r), _ptr(GX),
                                                             _ptr(Y), _ptr(w), _ptr(GY)))


def vmat_aperture_dose_cost_batch32(ctx, l, r, Y, X, Z, fprime=None):
    """Eq. 3 cost [32] (float64) of 32 intensity vectors Y [N, 32] on the
    apertures l, r; fills X = A Y, Z = D^T X and F'(Z) (if given)."""
    cost = np.zeros(32)
    _check(ctx, load_library().vmat_aperture_dose_cost_batch32(ctx, _ptr(l), _ptr(r), _ptr(Y), _ptr(X),
                                                               _ptr(Z), _ptr(fprime), cost.ctypes.data))
    return cost


def vmat_smoothing_batch32(ctx, Y, dG=None):
    g = (ctypes.c_double * 32)()
    _check(ctx, load_library().vmat_smoothing_batch32(ctx, _ptr(Y), g, _ptr(dG)))
    return np.array(g[:])


def vmat_set_profiling(ctx, on):
    _check(ctx, load_library().vmat_set_profiling(ctx, int(on)))


def vmat_selftest_grid_wait(ctx, skip_one, wait_seconds):
    """Status of the bounded-wait self-test (VMAT_ETIMEOUT expected with skip_one)."""
    return load_library().vmat_selftest_grid_wait(ctx, int(skip_one), float(wait_seconds))


# ---------------------------------------------------------------- convenience
class Plan:
    """One library context over a planning problem (inputs.Problem)."""

    def __init__(self, prob, dtype="f32", val_f32=False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1005_4396_b300.vmat needs a CUDA device")
        self.prob = prob
        self.cfg = prob.cfg
        self.stream = torch.cuda.current_stream()
        self.ctx = vmat_create(prob, dtype, ctypes.c_void_p(self.stream.cuda_stream), val_f32)
        self.info = vmat_get_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            vmat_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # tensors -------------------------------------------------------
    def _t(self, n, dtype=None):
        import torch
        return torch.empty(n, dtype=dtype or torch.float32, device="cuda")

    def dose(self, x):
        import torch
        _require_cuda(x, torch.float32, self.cfg.n_beamlets, "x")
        z = self._t(self.prob.n_vox)
        fp = self._t(self.prob.n_vox)
        cost = vmat_dose(self.ctx, x, z, fp)
        return z, fp, cost

    def price(self, f, mask=None):
        import torch
        _require_cuda(f, torch.float32, self.prob.n_vox, "f")
        g = torch.zeros(self.cfg.n_beamlets, dtype=torch.float32, device="cuda")
        m = None
        if mask is not None:
            m = torch.as_tensor(np.asarray(mask, dtype=np.uint8), device="cuda")
        vmat_price(self.ctx, f, g, m)
        return g

    def pricing_select(self, g):
        import torch
        _require_cuda(g, torch.float32, self.cfg.n_beamlets, "g")
        return vmat_pricing_select(self.ctx, g, self.cfg.n_rows)

    def add_column(self, k, l, r):
        vmat_add_column(self.ctx, k, l, r)

    def master_step(self, max_iters=100000, kkt_tol=1e-6, rho_ref=0.0, y=None):
        return vmat_master_step(self.ctx, max_iters, kkt_tol, rho_ref, y)

    def plan_dose(self):
        z = self._t(self.prob.n_vox)
        vmat_plan_dose(self.ctx, z)
        return z

    def reset(self):
        vmat_reset(self.ctx)

    def dvh(self, z, dose_max, n_bins=1000):
        import torch
        _require_cuda(z, torch.float32, self.prob.n_vox, "z")
        return vmat_dvh(self.ctx, z, self.prob.T.size, dose_max, n_bins)

    def dose_rate_feasibility(self, max_rate, **kw):
        return vmat_dose_rate_feasibility(self.ctx, self.cfg.n_angles, max_rate, **kw)

    def set_master_method(self, method):
        """'pg' (the paper's gradient projection, default) or 'newton'."""
        vmat_set_master_method(self.ctx, method)

    def set_master_precision(self, extended=True):
        vmat_set_master_precision(self.ctx, extended)

    def set_price_smoothing(self, on=True):
        """Price beams by the exact reduced cost (beamlet sum + gamma dG/dy_k)
        instead of the beamlet sum alone (the default, as in the paper)."""
        vmat_set_price_smoothing(self.ctx, on)

    def set_price_path(self, path="auto"):
        """How the FP32 prices g = D f are formed: 'auto' (default), 'rows'
        (beamlet-major row products) or 'live' (voxel-major rows of the
        voxels with f != 0, fixed-point sums)."""
        vmat_set_price_path(self.ctx, PRICE_PATHS[path])

    def set_profiling(self, on=True):
        vmat_set_profiling(self.ctx, on)

    def launches(self):
        return vmat_get_info(self.ctx)["n_launches"]

    def colgen_run(self, n_iters=None, master_max_iters=100000, kkt_tol=None, forced=None,
                   allow_notconv=False):
        n_iters = self.cfg.iterations if n_iters is None else n_iters
        kkt_tol = self.cfg.kkt_eps if kkt_tol is None else kkt_tol
        return vmat_colgen_run(self.ctx, self.cfg.n_angles, self.cfg.n_rows, n_iters,
                               master_max_iters, kkt_tol, forced, allow_notconv)

    def dose_batch32(self, X, want_fprime=True):
        import torch
        _require_cuda(X, torch.float32, self.cfg.n_beamlets * 32, "X")
        Z = self._t(self.prob.n_vox * 32)
        Fp = self._t(self.prob.n_vox * 32) if want_fprime else None
        cost = vmat_dose_batch32(self.ctx, X, Z, Fp)
        return Z, Fp, cost

    def price_batch32(self, Fp, w=None):
        import torch
        _require_cuda(Fp, torch.float32, self.prob.n_vox * 32, "Fp")
        G = self._t(self.cfg.n_beamlets * 32)
        vmat_price_batch32(self.ctx, Fp, G, w)
        return G


VMAT_MASTER_PROJECTED_GRADIENT = 0
VMAT_MASTER_PROJECTED_NEWTON = 1
MASTER_METHODS = {"pg": VMAT_MASTER_PROJECTED_GRADIENT, "newton": VMAT_MASTER_PROJECTED_NEWTON}


def vmat_set_master_method(ctx, method):
    _check(ctx, load_library().vmat_set_master_method(ctx, int(MASTER_METHODS.get(method, method))))


def vmat_set_master_precision(ctx, extended):
    _check(ctx, load_library().vmat_set_master_precision(ctx, int(bool(extended))))


def vmat_set_price_smoothing(ctx, on):
    _check(ctx, load_library().vmat_set_price_smoothing(ctx, int(bool(on))))


PRICE_PATHS = {"auto": 0, "rows": 1, "live": 2}


def vmat_set_price_path(ctx, path):
    _check(ctx, load_library().vmat_set_price_path(ctx, int(path)))


def vmat_dose_rate_feasibility(ctx, n_angles, max_rate, gamma_factor=2.0, max_rounds=20,
                               master_max_iters=100000, kkt_tol=1e-6, allow_infeasible=False):
    """Sec. 3 final step: raise gamma and re-optimise y until every neighbour
    pair has |dy|/gap <= max_rate.  Returns dict(y, gamma, rounds, violation,
    cost, status)."""
    y = np.zeros(n_angles)
    g, v, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    r = ctypes.c_int32()
    st = load_library().vmat_dose_rate_feasibility(ctx, float(max_rate), float(gamma_factor),
                                                   int(max_rounds), int(master_max_iters),
                                                   float(kkt_tol), y.ctypes.data, ctypes.byref(g),
                                                   ctypes.byref(r), ctypes.byref(v), ctypes.byref(c))
    if st != VMAT_OK and not (allow_infeasible and st == VMAT_ENOTCONV):
        _check(ctx, st)
    return dict(y=y, gamma=g.value, rounds=r.value, violation=v.value, cost=c.value, status=st)


def vmat_dvh(ctx, z, n_struct, dose_max, n_bins=1000):
    """Per-structure dose histogram counts [n_struct, n_bins] of the device dose z."""
    counts = np.zeros(n_struct * n_bins, np.int64)
    _check(ctx, load_library().vmat_dvh(ctx, _ptr(z), float(dose_max), int(n_bins), counts.ctypes.data))
    return counts.reshape(n_struct, n_bins)


def vmat_set_master_budget(ctx, max_ctas):
    _check(ctx, load_library().vmat_set_master_budget(ctx, int(max_ctas)))


def _result_arrays(N, R, n):
    out = dict(k=np.zeros(n, np.int32), lleaf=np.zeros(N * R, np.int16),
               rleaf=np.zeros(N * R, np.int16), y=np.zeros(N), p=np.zeros(n), p2=np.zeros(n),
               cost=np.zeros(n), rho=np.zeros(n), iters=np.zeros(n, np.int32),
               phase_ms=np.zeros((n, 4)), col_subtiles=np.zeros(n, np.int32))
    res = vmat_colgen_result(*[out[k].ctypes.data for k in
                               ("k", "lleaf", "rleaf", "y", "p", "p2", "cost", "rho", "iters",
                                "phase_ms", "col_subtiles")])
    return out, res


def vmat_list_schedule(budget, est, sms, want_tokens=False):
    """The batch's list schedule (host only): returns (order, deps, tokens)
    with deps[p] the plans plan p waits for and tokens [n, sms] bool or None."""
    budget = np.ascontiguousarray(budget, dtype=np.int32)
    est = np.ascontiguousarray(est, dtype=np.float64)
    n = budget.size
    order = np.zeros(n, np.int32)
    ndep = np.zeros(n, np.int32)
    deps = np.zeros(n * n, np.int32)
    tokens = np.zeros(n * sms, np.uint8) if want_tokens else None
    st = load_library().vmat_list_schedule(n, _ptr(budget), _ptr(est), int(sms), _ptr(order),
                                           _ptr(ndep), _ptr(deps), _ptr(tokens))
    if st != VMAT_OK:
        raise VmatError(st, "vmat_list_schedule: bad sizes")
    dl = [deps[p * n:p * n + ndep[p]].tolist() for p in range(n)]
    return order, dl, (tokens.reshape(n, sms).astype(bool) if want_tokens else None)


class Batch:
    """Many plans at once: per-plan SM budgets, a list schedule of which plans
    run side by side, one CUDA graph per run.  While a Plan is in a batch its
    context runs on a stream of the batch."""

    def __init__(self, plans):
        import torch
        self.plans = list(plans)
        arr = (_p * len(self.plans))(*[p.ctx for p in self.plans])
        h = _p()
        L = load_library()
        st = L.vmat_batch_create(arr, len(self.plans),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                 ctypes.byref(h))
        if st != VMAT_OK:
            raise VmatError(st, L.vmat_last_error(None).decode())
        self.h = h

    def _chk(self, st, ok=(VMAT_OK,)):
        if st not in ok:
            raise VmatError(st, load_library().vmat_batch_last_error(self.h).decode())
        return st

    def configure(self, share):
        self._chk(load_library().vmat_batch_configure(self.h, int(share)))

    def tune(self, trial_iters=20, master_max_iters=100000, kkt_tol=1e-6):
        share = ctypes.c_int32()
        ms = np.zeros(4)
        self._chk(load_library().vmat_batch_tune(self.h, int(trial_iters), int(master_max_iters),
                                                 float(kkt_tol), ctypes.byref(share),
                                                 ms.ctypes.data))
        return share.value, dict(zip((1, 2, 3, 4), ms.tolist()))

    def run(self, master_max_iters=100000, kkt_tol=1e-6):
        outs, ress = [], []
        for p in self.plans:
            o, r = _result_arrays(p.cfg.n_angles, p.cfg.n_rows, p.cfg.n_angles)
            outs.append(o)
            ress.append(r)
        res_arr = (vmat_colgen_result * len(ress))(*ress)
        plan_ms = np.zeros(len(self.plans))
        total = ctypes.c_double()
        st = load_library().vmat_batch_colgen_run(self.h, int(master_max_iters), float(kkt_tol),
                                                  res_arr, plan_ms.ctypes.data, ctypes.byref(total))
        self._chk(st)
        return outs, plan_ms, total.value

    def close(self):
        if getattr(self, "h", None):
            load_library().vmat_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
