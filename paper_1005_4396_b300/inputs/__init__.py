"""Seeded synthetic VMAT planning problems (phantom, structures, D).

This module produces the inputs that both the oracle and the CUDA path
consume.  It holds none of the optimisation method's arithmetic: it only lays
out voxels, assigns each voxel a structure (prescription T_j and weights
alpha_j, beta_j of Eq. 1), lists the gantry angles theta_k (Sec. 2.1) and
computes a stand-in dose-deposition matrix D_ij with a parallel-ray model
(the paper's D comes from a separate dose engine, Sec. 2.1).

Workloads (shapes follow the paper's prostate and head-and-neck cases of
Table 1, rescaled to B300-sized problems):
  tiny      32x32x8 grid at 4 mm, 36 angles, 10x10 MLC            (cfg "tiny")
  prostate  128x128x64 grid at 3 mm, 180 angles, 40x40 MLC        (cfg "prostate")
  headneck  160x160x96 grid at 2.5 mm, 180 angles, 60x40 MLC      (cfg "headneck")
plus small custom grids for tests.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from . import rng

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libphantom.so")


# --------------------------------------------------------------------------
# configuration
# --------------------------------------------------------------------------
@dataclass
class Structure:
    """One region of interest.  kind: 'ellipsoid' (params cx,cy,cz,ax,ay,az),
    'cylz' (cx,cy,radius,z0,z1) or 'box' (x0,x1,y0,y1,z0,z1); mm."""
    name: str
    kind: str
    params: Tuple[float, ...]
    T: float
    alpha: float
    beta: float


@dataclass
class PlanConfig:
    name: str
    nx: int
    ny: int
    nz: int
    h: float                      # voxel pitch, mm
    body: Tuple                   # ('box',) or ('ellcyl', ax, ay)
    structures: List[Structure]   # highest priority first
    tissue: Tuple[float, float, float] = (0.6, 0.0, 0.05)  # (T, alpha, beta)
    n_angles: int = 36
    n_rows: int = 10
    n_cols: int = 10
    w_row: float = 10.0
    w_col: float = 10.0
    sigma: float = 4.0
    mu: float = 0.005
    cutoff: float = 1e-3
    gamma: float = 0.1
    cyclic: bool = True
    max_leaf_step: int = 3
    n_iter: Optional[int] = None  # column-generation iterations (default N)
    kkt_eps: float = 1e-8
    round_f32: bool = False       # D values rounded to FP32-representable doubles
    seed: int = 0

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_beamlets(self) -> int:
        return self.n_angles * self.n_rows * self.n_cols

    @property
    def iterations(self) -> int:
        return self.n_angles if self.n_iter is None else self.n_iter

    def theta_deg(self) -> np.ndarray:
        """N uniformly spaced angles over one 360 degree arc, sorted from 0."""
        return np.arange(self.n_angles, dtype=np.float64) * (360.0 / self.n_angles)


def tiny_config(**kw) -> PlanConfig:
    """32x32x8 grid at 4 mm; centred ellipsoid target, posterior spherical OAR."""
    c = PlanConfig(
        name="tiny", nx=32, ny=32, nz=8, h=4.0, body=("box",),
        structures=[
            Structure("target", "ellipsoid", (0, 0, 0, 24, 20, 12), 1.0, 1.0, 1.0),
            Structure("oar", "ellipsoid", (0, 20, 0, 12, 12, 12), 0.5, 0.0, 0.5),
        ],
        tissue=(0.6, 0.0, 0.05), n_angles=36, n_rows=10, n_cols=10,
        w_row=10.0, w_col=10.0, sigma=4.0, gamma=0.1, cyclic=True,
        max_leaf_step=3, kkt_eps=1e-8, seed=0)
    return dataclasses.replace(c, **kw)


def prostate_config(**kw) -> PlanConfig:
    """128x128x64 grid at 3 mm; target, rectum, bladder in an elliptic body."""
    c = PlanConfig(
        name="prostate", nx=128, ny=128, nz=64, h=3.0, body=("ellcyl", 180.0, 110.0),
        structures=[
            Structure("target", "ellipsoid", (0, 0, 0, 30, 25, 30), 1.0, 1.0, 1.0),
            Structure("rectum", "cylz", (0, 37, 12, -30, 30), 0.6, 0.0, 0.5),
            Structure("bladder", "ellipsoid", (0, -35, 35, 35, 30, 25), 0.6, 0.0, 0.5),
        ],
        tissue=(0.6, 0.0, 0.05), n_angles=180, n_rows=40, n_cols=40,
        w_row=10.0, w_col=5.0, sigma=3.0, gamma=0.1, cyclic=True,
        max_leaf_step=1, kkt_eps=1e-6, round_f32=True, seed=1)
    return dataclasses.replace(c, **kw)


def headneck_config(**kw) -> PlanConfig:
    """160x160x96 grid at 2.5 mm; two targets and five OARs in a neck-sized body."""
    c = PlanConfig(
        name="headneck", nx=160, ny=160, nz=96, h=2.5, body=("ellcyl", 90.0, 80.0),
        structures=[
            Structure("ptv1", "ellipsoid", (0, 0, 0, 30, 25, 30), 1.0, 1.0, 1.0),
            Structure("ptv2", "ellipsoid", (0, 0, 0, 45, 40, 50), 0.85, 1.0, 1.0),
            Structure("cord", "cylz", (0, 35, 6, -120, 120), 0.65, 0.0, 5.0),
            Structure("brainstem", "ellipsoid", (0, 30, 55, 12, 12, 12), 0.6, 0.0, 1.0),
            Structure("parotid_l", "ellipsoid", (-45, 5, 0, 15, 12, 20), 0.4, 0.0, 0.5),
            Structure("parotid_r", "ellipsoid", (45, 5, 0, 15, 12, 20), 0.4, 0.0, 0.5),
            Structure("mandible", "box", (-50, 50, -50, -40, -20, 0), 0.7, 0.0, 0.2),
        ],
        tissue=(0.6, 0.0, 0.05), n_angles=180, n_rows=60, n_cols=40,
        w_row=5.0, w_col=5.0, sigma=2.5, gamma=0.1, cyclic=True,
        max_leaf_step=1, kkt_eps=1e-6, round_f32=True, seed=2)
    return dataclasses.replace(c, **kw)


def small_config(nx=20, ny=18, nz=6, n_angles=12, n_rows=6, n_cols=8, **kw) -> PlanConfig:
    """A tiny-style problem with free sizes (ragged, non-power-of-two by default)."""
    base = tiny_config()
    c = dataclasses.replace(
        base, name="small", nx=nx, ny=ny, nz=nz, n_angles=n_angles, n_rows=n_rows,
        n_cols=n_cols, w_row=base.h * nz / max(n_rows - 2, 1), w_col=base.h * nx / (n_cols + 2),
        structures=[
            Structure("target", "ellipsoid", (0, 0, 0, 0.3 * nx * base.h, 0.25 * ny * base.h,
                                                 0.35 * nz * base.h), 1.0, 1.0, 1.0),
            Structure("oar", "ellipsoid", (0, 0.3 * ny * base.h, 0, 0.15 * nx * base.h,
                                              0.15 * ny * base.h, 0.4 * nz * base.h), 0.5, 0.0, 0.5),
        ])
    return dataclasses.replace(c, **kw)


def asym_config(nx=20, ny=18, nz=6, n_angles=12, n_rows=6, n_cols=8, **kw) -> PlanConfig:
    """small_config with the target and the organ at risk moved off the
    grid's symmetry planes, and D rounded to FP32-representable values.  On
    the centred phantoms opposite beams see mirror images of one another and
    their prices tie exactly; here no two beams or leaf intervals tie, so a
    whole plan's decisions can be compared one by one."""
    base = small_config(nx=nx, ny=ny, nz=nz, n_angles=n_angles, n_rows=n_rows, n_cols=n_cols)
    h = base.h
    c = dataclasses.replace(
        base, name="asym", round_f32=True,
        structures=[
            Structure("target", "ellipsoid", (0.13 * nx * h, -0.07 * ny * h, 0.05 * nz * h,
                                                 0.27 * nx * h, 0.22 * ny * h, 0.33 * nz * h),
                      1.0, 1.0, 1.0),
            Structure("oar", "ellipsoid", (-0.12 * nx * h, 0.27 * ny * h, -0.04 * nz * h,
                                              0.14 * nx * h, 0.16 * ny * h, 0.38 * nz * h),
                      0.5, 0.0, 0.5),
        ])
    return dataclasses.replace(c, **kw)


CONFIGS = {"tiny": tiny_config, "prostate": prostate_config, "headneck": headneck_config}


def batch_configs(seeds=range(10, 26), scale=1.0):
    """Independent plans of uneven size, one per seed: beams N in {90, 120,
    150, 180}, MLC 40x40 or 60x40, prostate- or head-and-neck-like
    structures, grid voxel count V_target in [200k, 2.4M] (x scale) reached by
    changing the voxel pitch over the same field of view."""
    out = []
    for seed in seeds:
        u = rng.uniform(seed, 4)
        N = (90, 120, 150, 180)[int(u[0] * 4)]
        rows = 40 if u[1] < 0.5 else 60
        hn = u[2] >= 0.5
        vt = (200e3 + u[3] * (2.4e6 - 200e3)) * scale
        base = headneck_config() if hn else prostate_config()
        v0 = base.nx * base.ny * base.nz
        f = (vt / v0) ** (1.0 / 3.0)
        nx, ny, nz = (max(8, int(round(base.nx * f))), max(8, int(round(base.ny * f))),
                      max(4, int(round(base.nz * f))))
        h = base.h * base.nx / nx
        w_row = base.w_row * base.n_rows / rows if not hn else base.w_row
        out.append(dataclasses.replace(
            base, name=f"plan{seed}{'-hn' if hn else '-pr'}", nx=nx, ny=ny, nz=nz, h=h,
            n_angles=N, n_rows=rows, w_row=w_row, seed=seed))
    return out


# --------------------------------------------------------------------------
# problem
# --------------------------------------------------------------------------
@dataclass
class Problem:
    cfg: PlanConfig
    theta_deg: np.ndarray       # [N] float64
    struct_id: np.ndarray       # [V] uint8 (0 = outside body, 1 = tissue, 2.. = structures)
    T: np.ndarray               # [n_struct] float64
    alpha: np.ndarray
    beta: np.ndarray
    row_ptr: np.ndarray         # [B+1] int64, beamlet-major CSR of D
    vox_idx: np.ndarray         # [nnz] int32, ascending within each row
    val: np.ndarray             # [nnz] float64
    struct_names: List[str] = field(default_factory=list)

    @property
    def n_vox(self):
        return self.struct_id.shape[0]

    @property
    def n_beamlets(self):
        return self.row_ptr.shape[0] - 1

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def voxel_params(self):
        """Per-voxel (T_j, alpha_j, beta_j) as float64 arrays."""
        s = self.struct_id
        return self.T[s], self.alpha[s], self.beta[s]


def voxel_centres(cfg: PlanConfig):
    x = (np.arange(cfg.nx) - 0.5 * (cfg.nx - 1)) * cfg.h
    y = (np.arange(cfg.ny) - 0.5 * (cfg.ny - 1)) * cfg.h
    z = (np.arange(cfg.nz) - 0.5 * (cfg.nz - 1)) * cfg.h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")  # flat index (iz*ny+iy)*nx+ix
    return X.ravel(), Y.ravel(), Z.ravel()


def _in_body(cfg, X, Y):
    if cfg.body[0] == "box":
        return np.ones(X.shape, dtype=bool)
    ax, ay = cfg.body[1], cfg.body[2]
    return (X / ax) ** 2 + (Y / ay) ** 2 <= 1.0


def _in_structure(s: Structure, X, Y, Z):
    p = s.params
    if s.kind == "ellipsoid":
        cx, cy, cz, ax, ay, az = p
        return ((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 + ((Z - cz) / az) ** 2 <= 1.0
    if s.kind == "cylz":
        cx, cy, rad, z0, z1 = p
        return ((X - cx) ** 2 + (Y - cy) ** 2 <= rad * rad) & (Z >= z0) & (Z <= z1)
    if s.kind == "box":
        x0, x1, y0, y1, z0, z1 = p
        return (X >= x0) & (X <= x1) & (Y >= y0) & (Y <= y1) & (Z >= z0) & (Z <= z1)
    raise ValueError(s.kind)


def structure_map(cfg: PlanConfig):
    X, Y, Z = voxel_centres(cfg)
    body = _in_body(cfg, X, Y)
    sid = np.where(body, 1, 0).astype(np.uint8)
    for n, s in reversed(list(enumerate(cfg.structures))):  # highest priority written last
        sid[body & _in_structure(s, X, Y, Z)] = 2 + n
    T = np.array([0.0, cfg.tissue[0]] + [s.T for s in cfg.structures])
    alpha = np.array([0.0, cfg.tissue[1]] + [s.alpha for s in cfg.structures])
    beta = np.array([0.0, cfg.tissue[2]] + [s.beta for s in cfg.structures])
    names = ["air", "tissue"] + [s.name for s in cfg.structures]
    return sid, T, alpha, beta, names


# --------------------------------------------------------------------------
# the D generator (C, OpenMP)
# --------------------------------------------------------------------------
class _Spec(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("h", ctypes.c_double),
        ("body_kind", ctypes.c_int32), ("body_ax", ctypes.c_double), ("body_ay", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("theta_deg", ctypes.POINTER(ctypes.c_double)),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("w_row", ctypes.c_double), ("w_col", ctypes.c_double),
        ("sigma", ctypes.c_double), ("mu", ctypes.c_double), ("cutoff", ctypes.c_double),
        ("round_f32", ctypes.c_int32),
    ]


def build_native(force: bool = False) -> str:
    """Compile phantom.c into libphantom.so beside it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "phantom.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-std=c11", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _native():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_native())
        _lib.ph_count.restype = ctypes.c_int64
        _lib.ph_count.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p]
        _lib.ph_fill.restype = ctypes.c_int
        _lib.ph_fill.argtypes = [ctypes.POINTER(_Spec), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return _lib


def dose_matrix(cfg: PlanConfig):
    """Beamlet-major CSR (row_ptr, vox_idx, val) of the stand-in D."""
    lib = _native()
    theta = np.ascontiguousarray(cfg.theta_deg())
    spec = _Spec(cfg.nx, cfg.ny, cfg.nz, cfg.h,
                 0 if cfg.body[0] == "box" else 1,
                 0.0 if cfg.body[0] == "box" else cfg.body[1],
                 0.0 if cfg.body[0] == "box" else cfg.body[2],
                 cfg.n_angles, theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 cfg.n_rows, cfg.n_cols, cfg.w_row, cfg.w_col,
                 cfg.sigma, cfg.mu, cfg.cutoff, 1 if cfg.round_f32 else 0)
    B = cfg.n_beamlets
    counts = np.zeros(B, dtype=np.int64)
    nnz = lib.ph_count(ctypes.byref(spec), counts.ctypes.data)
    row_ptr = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    assert row_ptr[-1] == nnz
    vox = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    if lib.ph_fill(ctypes.byref(spec), row_ptr.ctypes.data, vox.ctypes.data, val.ctypes.data) != 0:
        raise RuntimeError("phantom: fill pass disagrees with count pass")
    return row_ptr, vox, val


def make_problem(cfg: PlanConfig) -> Problem:
    sid, T, alpha, beta, names = structure_map(cfg)
    row_ptr, vox, val = dose_matrix(cfg)
    return Problem(cfg=cfg, theta_deg=cfg.theta_deg(), struct_id=sid, T=T, alpha=alpha,
                   beta=beta, row_ptr=row_ptr, vox_idx=vox, val=val, struct_names=names)


# --------------------------------------------------------------------------
# random inputs (fluence batches, intensities, feasible apertures)
# --------------------------------------------------------------------------
def fluence_batch(seed: int, n_beamlets: int, batch: int) -> np.ndarray:
    """[batch, B] float32 fluence vectors, U(0,1)."""
    return rng.uniform(seed, batch * n_beamlets).astype(np.float32).reshape(batch, n_beamlets)


def random_apertures(seed: int, cfg: PlanConfig, stream: int = 1):
    """Seeded leaf pairs l <= r in [0, C] for every (angle, row): [N*R] int16 each.
    Apertures respect the leaf-travel limit of cfg.max_leaf_step between
    neighbouring angles by construction (a bounded random walk around the arc)."""
    N, R, C, s = cfg.n_angles, cfg.n_rows, cfg.n_cols, cfg.max_leaf_step
    u = rng.uniform(seed * 1000 + stream, 2 * N * R).reshape(N, R, 2)
    l = np.zeros((N, R), dtype=np.int64)
    r = np.zeros((N, R), dtype=np.int64)
    for row in range(R):
        a, b = C // 4, C - C // 4
        for k in range(N):
            if k > 0:
                a = a + int(np.floor(u[k, row, 0] * (2 * s + 1))) - s
                b = b + int(np.floor(u[k, row, 1] * (2 * s + 1))) - s
            a = min(max(a, 0), C)
            b = min(max(b, 0), C)
            if a > b:
                a = b = (a + b) // 2
            l[k, row], r[k, row] = a, b
    return l.astype(np.int16).ravel(), r.astype(np.int16).ravel()


# --------------------------------------------------------------------------
# coarse voxels for unspecified tissue (Sec. 3)
# --------------------------------------------------------------------------
@dataclass
class CoarseProblem:
    """A problem whose unspecified-tissue voxels are merged in 2x2x2 blocks.
    fine_to: [V_fine] index of each fine voxel's voxel in `prob`; weight:
    [V] fine voxels represented (1 for kept voxels, 1..8 for merged
    tissue).  Volume weighting rides on the structures: a merged voxel of
    weight w gets a structure with (T, w alpha, w beta) of tissue, so that
    Eq. 1 summed over the coarse voxels counts every fine voxel once."""
    prob: Problem
    fine_to: np.ndarray
    weight: np.ndarray


def coarse_tissue(prob: Problem, tissue_sid: int = 1) -> CoarseProblem:
    """Merge the tissue voxels (structure `tissue_sid`) of each 2x2x2 block of
    the grid into one voxel whose D row is the mean of its members' rows (a
    member with no entry counts as 0); every other voxel is kept.  Kept
    voxels come first in grid order, then one voxel per block with tissue,
    in block order."""
    cfg = prob.cfg
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    V = prob.n_vox
    j = np.arange(V)
    ix, iy, iz = j % nx, (j // nx) % ny, j // (nx * ny)
    bx, by = (nx + 1) // 2, (ny + 1) // 2
    block = ((iz // 2) * by + iy // 2) * bx + ix // 2
    tissue = prob.struct_id == tissue_sid
    kept = np.flatnonzero(~tissue)
    fine_to = np.empty(V, np.int64)
    fine_to[kept] = np.arange(kept.size)
    ublocks, binv, bcount = np.unique(block[tissue], return_inverse=True, return_counts=True)
    fine_to[tissue] = kept.size + binv
    Vc = kept.size + ublocks.size
    weight = np.ones(Vc, np.int64)
    weight[kept.size:] = bcount
    # structures: the original ones, then tissue with weight 2..8 (weight 1 keeps tissue_sid)
    n_s = prob.T.size
    sid = np.empty(Vc, np.uint8)
    sid[:kept.size] = prob.struct_id[kept]
    wc = weight[kept.size:]
    sid[kept.size:] = np.where(wc == 1, tissue_sid, n_s + wc - 2).astype(np.uint8)
    ws = np.arange(2, 9)
    T = np.concatenate([prob.T, np.full(7, prob.T[tissue_sid])])
    alpha = np.concatenate([prob.alpha, ws * prob.alpha[tissue_sid]])
    beta = np.concatenate([prob.beta, ws * prob.beta[tissue_sid]])
    names = list(prob.struct_names) + [f"tissue x{w}" for w in ws]
    # D rows: map voxels, scale merged entries by 1/weight, sum duplicates per row
    B = prob.n_beamlets
    rows = np.repeat(np.arange(B, dtype=np.int64), np.diff(prob.row_ptr))
    cols = fine_to[prob.vox_idx]
    vals = prob.val / weight[cols]
    key = rows * Vc + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    first = np.concatenate([[True], key[1:] != key[:-1]])
    starts = np.flatnonzero(first)
    vals = np.add.reduceat(vals, starts)
    key = key[starts]
    rows, cols = key // Vc, key % Vc
    row_ptr = np.zeros(B + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=B), out=row_ptr[1:])
    coarse = Problem(cfg=cfg, theta_deg=prob.theta_deg, struct_id=sid, T=T, alpha=alpha, beta=beta,
                     row_ptr=row_ptr, vox_idx=cols.astype(np.int32), val=vals, struct_names=names)
    return CoarseProblem(prob=coarse, fine_to=fine_to, weight=weight)
