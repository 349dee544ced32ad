"""FP64 CPU oracle of the TaylorGrid method (arXiv 2402.14415).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The oracle shares no code
with the CUDA library; it is plain C (``tg_oracle.c``) compiled with gcc and
called through ctypes with numpy arrays.

Parity unpinned: the full multi-step fit trajectories (atomics change the FP32
summation order on the GPU, and the sign of the L1 residual amplifies it); they
are compared step by step and by their final error against the analytic SDF.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libtg_oracle.so")
_lib = None
_lock = threading.Lock()

_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction). Returns the .so path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            L.tgo_num_coefs.argtypes = [i32, i32]; L.tgo_num_coefs.restype = i32
            L.tgo_locate.argtypes = [i32, i32, _f32p, _i32p, _f64p]
            L.tgo_eval_cell.argtypes = [i32, i32, i32, i32, _f64p, _i32p, _f64p, _f64p, _f64p]
            L.tgo_query.argtypes = [i32, i32, i32, i32, _f64p, i64, _f32p, _f64p, _f64p, _i32p, _f64p]
            L.tgo_query_backward.argtypes = [i32, i32, i32, i32, i64, _f32p, _f64p, _f64p, _f64p, _f64p]
            L.tgo_query_absscale.argtypes = [i32, i32, i32, i32, _f64p, i64, _f32p, _f64p]
            L.tgo_query_gradscale.argtypes = [i32, i32, i32, i32, _f64p, i64, _f32p, _f64p]
            L.tgo_adam.argtypes = [i64, _f64p, _f64p, _f64p, _f64p, f64, f64, f64, f64, i64, i32]
            L.tgo_adam_lazy.argtypes = [i64, _f64p, _f64p, _f64p, _f64p, f64, f64, f64, f64, i64, i32]
            L.tgo_bf16_round.argtypes = [f64]; L.tgo_bf16_round.restype = f64
            L.tgo_sdf_union.argtypes = [i32, _f32p, i32, _f32p, _f64p]; L.tgo_sdf_union.restype = f64
            L.tgo_sdf_step.argtypes = [i32, i32, _f64p, i64, _f32p, i32, _f32p, i32, _f32p, f64, f64, _f64p, _f64p]
            L.tgo_adaptive_weight1.argtypes = [f64, f64]; L.tgo_adaptive_weight1.restype = f64
            L.tgo_tv.argtypes = [i32, i32, _f64p, f64, _f64p]; L.tgo_tv.restype = f64
            L.tgo_resample.argtypes = [i32, i32, i32, _f64p, i32, i32, _f64p]
            L.tgo_uniform.argtypes = [u64, u64, u64]; L.tgo_uniform.restype = f64
            L.tgo_marching_tets.argtypes = [i32, _f64p, f64, _f64p, i64]; L.tgo_marching_tets.restype = i64
            L.tgo_sample_mesh.argtypes = [i64, _f32p, i64, u64, u64, _f64p]
            L.tgo_ray_box.argtypes = [_f64p, _f64p, _f64p, _f64p]; L.tgo_ray_box.restype = i32
            L.tgo_render.argtypes = [i32, i32, _f64p, i32, _f64p, i64, i32, _f32p, _f32p, u64, u64, f64,
                                     _f64p, _f32p, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.tgo_render_blobs.argtypes = [i32, _f64p, _f64p, _f64p, _f64p, i64, _f32p, _f32p, i32, f64, _f64p]
            _lib = L
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def num_coefs(dim: int, order: int) -> int:
    return lib().tgo_num_coefs(dim, order)


def set_threads(n: int) -> None:
    """Limit the OpenMP threads of later oracle calls (must be set before the first call)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


def locate(dim: int, res: int, pts: np.ndarray):
    pts = _c(pts, np.float32).reshape(-1, dim)
    cells = np.zeros((pts.shape[0], dim), np.int32)
    ts = np.zeros((pts.shape[0], dim), np.float64)
    for n in range(pts.shape[0]):
        lib().tgo_locate(dim, res, _p(pts[n], _f32p), _p(cells[n], _i32p), _p(ts[n], _f64p))
    return cells, ts


def query(dim, res, order, C, coefs, pts, want_grad=True, want_cells=False):
    """Values (N, C), world-unit spatial gradients (N, C, dim), cells (N, dim), t (N, dim)."""
    coefs = _c(coefs, np.float64)
    pts = _c(pts, np.float32).reshape(-1, dim)
    N = pts.shape[0]
    out = np.zeros((N, C)); gx = np.zeros((N, C, dim)) if want_grad else None
    cells = np.zeros((N, dim), np.int32) if want_cells else None
    ts = np.zeros((N, dim)) if want_cells else None
    lib().tgo_query(dim, res, order, C, _p(coefs, _f64p), N, _p(pts, _f32p), _p(out, _f64p),
                    _p(gx, _f64p), _p(cells, _i32p), _p(ts, _f64p))
    return out, gx, cells, ts


def query_backward(dim, res, order, C, pts, dL_df, dL_dgx=None, want_abs=False):
    pts = _c(pts, np.float32).reshape(-1, dim)
    N = pts.shape[0]
    K = num_coefs(dim, order)
    g = np.zeros(res ** dim * C * K)
    a = np.zeros_like(g) if want_abs else None
    lib().tgo_query_backward(dim, res, order, C, N, _p(pts, _f32p), _p(_c(dL_df, np.float64), _f64p),
                             _p(_c(dL_dgx, np.float64), _f64p), _p(g, _f64p), _p(a, _f64p))
    return (g, a) if want_abs else g


def query_absscale(dim, res, order, C, coefs, pts):
    pts = _c(pts, np.float32).reshape(-1, dim)
    s = np.zeros((pts.shape[0], C))
    lib().tgo_query_absscale(dim, res, order, C, _p(_c(coefs, np.float64), _f64p), pts.shape[0],
                             _p(pts, _f32p), _p(s, _f64p))
    return s


def query_gradscale(dim, res, order, C, coefs, pts):
    """Per point, channel and axis: the magnitude of the terms of the world-unit spatial gradient,
    sum_i |d w_i / d x_a| sum_k |theta_k phi_k| + w_i sum_k |theta_k d phi_k / d delta_a|  (N, C, dim)."""
    pts = _c(pts, np.float32).reshape(-1, dim)
    s = np.zeros((pts.shape[0], C, dim))
    lib().tgo_query_gradscale(dim, res, order, C, _p(_c(coefs, np.float64), _f64p), pts.shape[0],
                              _p(pts, _f32p), _p(s, _f64p))
    return s


def eval_cell(dim, res, order, C, coefs, cell, t):
    coefs = _c(coefs, np.float64)
    cell = np.ascontiguousarray(cell, np.int32); t = np.ascontiguousarray(t, np.float64)
    f = np.zeros(C); gu = np.zeros(C * dim)
    lib().tgo_eval_cell(dim, res, order, C, _p(coefs, _f64p), _p(cell, _i32p), _p(t, _f64p),
                        _p(f, _f64p), _p(gu, _f64p))
    return f, gu.reshape(C, dim)


def adam(p, g, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-8, step=1, bf16_moments=False):
    """In-place FP64 Adam step on float64 arrays; zeroes g. bf16_moments rounds m and v to BF16 after the update."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().tgo_adam(p.size, _p(p, _f64p), _p(g, _f64p), _p(m, _f64p), _p(v, _f64p), lr, beta1, beta2, eps, step,
                   int(bool(bf16_moments)))


def bf16_round(x):
    """Round every element of x to BF16 (nearest, ties to even), returned as float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = lib().tgo_bf16_round
    return np.array([f(float(e)) for e in x.ravel()]).reshape(x.shape)


def adam_lazy(p, g, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-8, step=1, bf16_moments=False):
    """In-place FP64 lazy (sparse) Adam step: entries with g == 0 keep p, m and v; zeroes g."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().tgo_adam_lazy(p.size, _p(p, _f64p), _p(g, _f64p), _p(m, _f64p), _p(v, _f64p), lr, beta1, beta2, eps,
                        step, int(bool(bf16_moments)))


def sdf_union(spheres, boxes, x):
    sph = _c(spheres, np.float32).reshape(-1); box = _c(boxes, np.float32).reshape(-1)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    return np.array([lib().tgo_sdf_union(len(sph) // 4, _p(sph, _f32p), len(box) // 6, _p(box, _f32p),
                                         _p(x[n], _f64p)) for n in range(x.shape[0])])


def sdf_step(res, order, coefs, pts, spheres, boxes, lambda_eik, k_weight=0.0):
    """One SDF fitting step (Eq. 6 with Eq. 7's weight for k_weight > 0, plus the eikonal term);
    returns (coef_grad, (weighted reconstruction mean, eikonal mean))."""
    pts = _c(pts, np.float32).reshape(-1, 3)
    sph = _c(spheres, np.float32).reshape(-1); box = _c(boxes, np.float32).reshape(-1)
    K = num_coefs(3, order)
    g = np.zeros(res ** 3 * K); loss = np.zeros(3)
    lib().tgo_sdf_step(res, order, _p(_c(coefs, np.float64), _f64p), pts.shape[0], _p(pts, _f32p),
                       len(sph) // 4, _p(sph, _f32p), len(box) // 6, _p(box, _f32p), lambda_eik, k_weight,
                       _p(g, _f64p), _p(loss, _f64p))
    return g, (loss[0], loss[1])


def adaptive_weight1(k, z) -> float:
    """w'(z) of Eq. 7 (1 for k <= 0)."""
    return lib().tgo_adaptive_weight1(k, z)


def tv(res, nv, coefs, lam=1.0, want_grad=True):
    """Total variation term of Sec. 3.2 over a 3-D grid ([vertex][nv] coefficients): (L_TV, lam * dL_TV/dtheta)."""
    c = _c(coefs, np.float64)
    g = np.zeros(res ** 3 * nv) if want_grad else None
    L = lib().tgo_tv(res, nv, _p(c, _f64p), lam, _p(g, _f64p) if want_grad else None)
    return L, g


def uniform(seed, stream, idx) -> float:
    return lib().tgo_uniform(seed, stream, idx)


def lattice_values(res, order, C, coefs, M, channel=0):
    """The field (channel `channel`) at the M^3 lattice x = (i, j, k) / (M - 1), i fastest (FP64)."""
    a = np.arange(M, dtype=np.float64) / (M - 1)
    z, y, x = np.meshgrid(a, a, a, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)
    f, _, _, _ = query(3, res, order, C, coefs, pts, want_grad=False)
    return f.reshape(-1, C)[:, channel].copy()


def marching_tets(M, vals, iso=0.0):
    """Triangles (T, 3, 3) of the iso surface of the M^3 lattice values (i fastest), in cube order."""
    vals = np.ascontiguousarray(vals, np.float64).reshape(-1)
    assert vals.size == M ** 3
    n = lib().tgo_marching_tets(M, _p(vals, _f64p), iso, None, 0)
    tris = np.zeros((max(n, 1), 9))
    lib().tgo_marching_tets(M, _p(vals, _f64p), iso, _p(tris, _f64p), n)
    return tris[:n].reshape(n, 3, 3)


MESH_STREAM = 0x4D455348          # generator stream of the mesh sampler


def sample_mesh(tris, n, seed):
    """n area-weighted points on the triangles (T, 3, 3) given in FP32."""
    t = np.ascontiguousarray(tris, np.float32).reshape(-1)
    out = np.zeros((n, 3))
    lib().tgo_sample_mesh(t.size // 9, _p(t, _f32p), n, seed, MESH_STREAM, _p(out, _f64p))
    return out


def chamfer(A, B):
    """(sum_a min_b |a - b|^2, sum_b min_a |a - b|^2) in FP64; the nearest neighbours come from a k-d tree
    (scipy.spatial.cKDTree, exact)."""
    from scipy.spatial import cKDTree
    A = np.asarray(A, np.float64).reshape(-1, 3); B = np.asarray(B, np.float64).reshape(-1, 3)
    da, _ = cKDTree(B).query(A)
    db, _ = cKDTree(A).query(B)
    return float((da * da).sum()), float((db * db).sum())


def ray_box(o, d):
    o = np.ascontiguousarray(o, np.float64); d = np.ascontiguousarray(d, np.float64)
    n = ctypes.c_double(); f = ctypes.c_double()
    hit = lib().tgo_ray_box(_p(o, _f64p), _p(d, _f64p), ctypes.byref(n), ctypes.byref(f))
    return bool(hit), n.value, f.value


def render(res, od, dcoef, oc, ccoef, rays_o, rays_d, S, seed, ray_base=0, bg=1.0, target=None, want_abs=False):
    """Returns rgb (R,3) and, if target is given, (loss, density grad, colour grad) and, with want_abs, the
    per-coefficient magnitudes of the terms of both gradients (density, colour)."""
    rays_o = _c(rays_o, np.float32).reshape(-1, 3); rays_d = _c(rays_d, np.float32).reshape(-1, 3)
    R = rays_o.shape[0]
    rgb = np.zeros((R, 3))
    train = target is not None
    dg = np.zeros(res ** 3 * num_coefs(3, od)) if train else None
    cg = np.zeros(res ** 3 * 3 * num_coefs(3, oc)) if train else None
    da = np.zeros_like(dg) if train and want_abs else None
    ca = np.zeros_like(cg) if train and want_abs else None
    loss = np.zeros(1)
    lib().tgo_render(res, od, _p(_c(dcoef, np.float64), _f64p), oc, _p(_c(ccoef, np.float64), _f64p), R, S,
                     _p(rays_o, _f32p), _p(rays_d, _f32p), seed, ray_base, bg, _p(rgb, _f64p),
                     _p(_c(target, np.float32), _f32p), _p(dg, _f64p), _p(cg, _f64p), _p(loss, _f64p),
                     _p(da, _f64p), _p(ca, _f64p))
    if not train:
        return rgb
    if want_abs:
        return rgb, float(loss[0]), dg, cg, da, ca
    return rgb, float(loss[0]), dg, cg


def render_blobs(scene, rays_o, rays_d, n_samples=1024, bg=1.0):
    """Ground-truth colours of the blob scene (mu, inv_cov, amp, rgb) along rays, (R, 3) float64."""
    mu, icov, amp, rgb = (np.ascontiguousarray(a, np.float64) for a in scene)
    rays_o = _c(rays_o, np.float32).reshape(-1, 3); rays_d = _c(rays_d, np.float32).reshape(-1, 3)
    out = np.zeros((rays_o.shape[0], 3))
    lib().tgo_render_blobs(mu.shape[0], _p(mu, _f64p), _p(icov, _f64p), _p(amp, _f64p), _p(rgb, _f64p),
                           rays_o.shape[0], _p(rays_o, _f32p), _p(rays_d, _f32p), n_samples, bg, _p(out, _f64p))
    return out


def resample(res_src, order_src, C, coefs, res_dst, order_dst):
    """The src field re-expanded as Taylor data at the vertices of a res_dst grid of order order_dst (3-D)."""
    out = np.zeros(res_dst ** 3 * C * num_coefs(3, order_dst))
    lib().tgo_resample(res_src, order_src, C, _p(_c(coefs, np.float64), _f64p), res_dst, order_dst, _p(out, _f64p))
    return out
