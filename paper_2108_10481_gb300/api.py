"""Python binding of the C ABI: the same names as include/pbbem.h, taking
torch tensors (device memory and streams) and doing argument marshalling only.
Every step of the computation runs in libpbbem's CUDA kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N

# status codes, enumerations (mirror include/pbbem.h)
PB_OK, PB_EINVAL, PB_EMESH, PB_ENOMEM, PB_ENOCONV, PB_ENUMERIC, PB_ECUDA, PB_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
PB_OP_V, PB_OP_K, PB_OP_T, PB_OP_D, PB_OP_M = 0, 1, 2, 3, 4
PB_LAPLACE, PB_YUKAWA = 0, 1
PB_F64, PB_F32, PB_F32_ACCURATE, PB_MIXED = 0, 1, 2, 3
FORMS = {"direct_int": 0, "direct_ext": 1, "direct_int_perm": 2, "direct_ext_perm": 3, "cfie_int": 4,
         "cfie_ext": 5, "pmchwt_int": 6, "pmchwt_ext": 7, "muller_int": 8, "muller_ext": 9, "juffer": 10,
         "lu": 11}
PRECONDS = {"none": 0, "block_diag": 1, "mass": 2, "scaled_mass": 3, "calderon_full": 4, "calderon_int": 5,
            "calderon_ext": 6, "scaled_calderon_int": 7, "scaled_calderon_ext": 8}
# Table 1 of the paper: case -> (formulation, preconditioner)
CASES = {
    1: ("direct_int", "none"), 2: ("direct_int", "block_diag"), 3: ("direct_ext", "none"),
    4: ("direct_ext", "block_diag"), 5: ("direct_int_perm", "none"), 6: ("direct_int_perm", "block_diag"),
    7: ("direct_ext_perm", "none"), 8: ("direct_ext_perm", "block_diag"), 9: ("juffer", "mass"),
    10: ("juffer", "scaled_mass"), 11: ("lu", "none"), 12: ("lu", "mass"), 13: ("muller_int", "mass"),
    14: ("muller_ext", "mass"), 15: ("pmchwt_int", "mass"), 16: ("pmchwt_int", "calderon_full"),
    17: ("pmchwt_int", "calderon_int"), 18: ("pmchwt_int", "calderon_ext"), 19: ("pmchwt_ext", "mass"),
    20: ("pmchwt_ext", "calderon_full"), 21: ("pmchwt_ext", "calderon_ext"), 22: ("pmchwt_ext", "calderon_int"),
    23: ("pmchwt_int", "scaled_calderon_int"), 24: ("pmchwt_int", "scaled_calderon_ext"),
    25: ("pmchwt_ext", "scaled_calderon_ext"), 26: ("pmchwt_ext", "scaled_calderon_int"),
}


class PBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pbbem error {code}: {msg}")
        self.code = code


def _check(rc: int):
    if rc != PB_OK:
        raise PBError(rc, N.load().pb_last_error().decode())
    return rc


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dptr(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _form(form):
    return FORMS[form] if isinstance(form, str) else int(form)


def _prec(pc):
    return PRECONDS[pc] if isinstance(pc, str) else int(pc)


@dataclass
class Params:
    eps_int: float = 4.0
    eps_ext: float = 80.0
    kappa: float = 0.125

    def c(self):
        return N.pb_params(self.eps_int, self.eps_ext, self.kappa)


class _Handle:
    _free = None

    def __init__(self, ptr, owner=None):
        self.ptr = ptr
        self.owner = owner  # keeps the parent alive

    def free(self):
        if self.ptr:
            getattr(N.load(), self._free)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Ctx(_Handle):
    _free = "pb_free_ctx"


class Mesh(_Handle):
    _free = "pb_free_mesh"

    def info(self):
        out = (ctypes.c_int64 * 6)()
        _check(N.load().pb_mesh_info(self.ptr, out))
        return dict(zip(["n_verts", "n_tris", "n_points", "nnz", "n_pairs", "device_bytes"], list(out)))


class Near(_Handle):
    _free = "pb_free_near"


PB_KERNEL_PAIR32, PB_KERNEL_PAIR32_ACCURATE, PB_KERNEL_PAIR64 = 0, 1, 2
PB_KERNEL_NEAR_ADJ, PB_KERNEL_NEAR_COIN, PB_KERNEL_NEAR_BAND = 3, 4, 5
PB_KERNEL_TREE32 = 6
PB_KERNEL_SPMV, PB_KERNEL_CHEB, PB_KERNEL_KRYLOV = 7, 8, 9  # memory-bound: pairs = ops = algorithmic bytes


def pb_profile(ctx: Ctx, enable: bool = True):
    _check(N.load().pb_profile(ctx.ptr, 1 if enable else 0))


def pb_profile_read(ctx: Ctx, kernel: int):
    """dict(launches, ms, pairs, ops) of one pair-kernel family since pb_profile(ctx, True)."""
    n = ctypes.c_int64()
    ms, pairs, ops = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(N.load().pb_profile_read(ctx.ptr, kernel, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(pairs),
                                    ctypes.byref(ops)))
    return {"launches": n.value, "ms": ms.value, "pairs": pairs.value, "ops": ops.value}


def pb_selftest_wait(ctx: Ctx, polls: int = 4096) -> int:
    """Status word left by a bounded wait on a barrier nothing completes."""
    st = ctypes.c_int()
    _check(N.load().pb_selftest_wait(ctx.ptr, int(polls), ctypes.byref(st)))
    return st.value


def pb_measure_peak(ctx: Ctx, kind: int) -> float:
    """FMAs per second of this GPU by microbenchmark: kind 0 FP32, 1 FP64, 2 packed f32x2."""
    out = ctypes.c_double()
    _check(N.load().pb_measure_peak(ctx.ptr, int(kind), ctypes.byref(out)))
    return out.value


def pb_selftest_exp(ctx: Ctx, x: torch.Tensor, stream=None) -> torch.Tensor:
    """e^x (x <= 0) by the near-field kernels' exponential, for x a CUDA float64 tensor."""
    xx = x.contiguous()
    y = torch.empty_like(xx)
    _check(N.load().pb_selftest_exp(ctx.ptr, _dptr(xx, "x"), _dptr(y, "y"), xx.numel(), _stream(stream)))
    return y


def pb_launch_count() -> int:
    return int(N.load().pb_launch_count())


def pb_set_treecode(ctx: Ctx, enable: bool = True, order: int = 6, theta: float = 0.7, min_points: int = 50000):
    """Treecode far field for FP32 applications of meshes with >= min_points far-rule points."""
    _check(N.load().pb_set_treecode(ctx.ptr, 1 if enable else 0, int(order), float(theta), int(min_points)))


def pb_tree_info(mesh: Mesh):
    """Sizes of the mesh's tree (after its first treecode application)."""
    out = (ctypes.c_int64 * 6)()
    _check(N.load().pb_tree_info(mesh.ptr, out))
    return dict(zip(["leaves", "proxied_clusters", "far_entries", "near_entries", "direct_pairs", "proxy_pairs"],
                    list(out)))


def pb_set_graphs(ctx: Ctx, enable: bool = True):
    """Replay GMRES iterations from CUDA graphs (default) or launch them kernel by kernel."""
    _check(N.load().pb_set_graphs(ctx.ptr, 1 if enable else 0))


def pb_version() -> str:
    return N.load().pb_version().decode()


def pb_init(device: int = 0) -> Ctx:
    h = ctypes.c_void_p()
    _check(N.load().pb_init(int(device), ctypes.byref(h)))
    return Ctx(h.value)


def _plan(far_q=6, n_ss=4, band_eta=0.0, band_q=6, n_ss_coin=0, n_ss_edge=0, n_ss_vert=0):
    return N.pb_quad_plan(int(far_q), int(n_ss), float(band_eta), int(band_q), int(n_ss_coin), int(n_ss_edge),
                          int(n_ss_vert))


def plan_dict(p) -> dict:
    """A pb_quad_plan as keyword arguments of pb_mesh_load / pb_submit / pb_solvation_energy."""
    return {k: getattr(p, k) for k, _ in N.pb_quad_plan._fields_}


def pb_mesh_load(ctx: Ctx, verts, tris, far_q: int = 6, n_ss: int = 4, band_eta: float = 0.0,
                 band_q: int = 6, n_ss_coin: int = 0, n_ss_edge: int = 0, n_ss_vert: int = 0) -> Mesh:
    """verts [N_v,3] float64 and tris [N_t,3] int32, numpy (host) or CUDA tensors; the quadrature plan
    (far rule, singular rule and its per-class orders (0: n_ss), optional distance band and its rule)."""
    plan = _plan(far_q, n_ss, band_eta, band_q, n_ss_coin, n_ss_edge, n_ss_vert)
    if isinstance(verts, torch.Tensor) and verts.is_cuda:
        v = verts.contiguous()
        t = tris.to(torch.int32).contiguous()
        mem, vp, tp, nv, nt = 1, v.data_ptr(), t.data_ptr(), v.shape[0], t.shape[0]
        keep = (v, t)
    else:
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        mem, vp, tp, nv, nt = 0, v.ctypes.data, t.ctypes.data, v.shape[0], t.shape[0]
        keep = (v, t)
    h = ctypes.c_void_p()
    _check(N.load().pb_mesh_load(ctx.ptr, ctypes.c_void_p(vp), nv, ctypes.c_void_p(tp), nt, ctypes.byref(plan),
                                 mem, ctypes.byref(h)))
    del keep
    return Mesh(h.value, ctx)


def pb_near_build(ctx: Ctx, mesh: Mesh, kappa: float, stream=None) -> Near:
    h = ctypes.c_void_p()
    _check(N.load().pb_near_build(ctx.ptr, mesh.ptr, float(kappa), ctypes.byref(h), _stream(stream)))
    return Near(h.value, mesh)


def pb_op_apply(ctx: Ctx, mesh: Mesh, near: Near, op: int, kernel: int, prec: int, x: torch.Tensor,
                y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if y is None:
        y = torch.empty_like(x)
    _check(N.load().pb_op_apply(ctx.ptr, mesh.ptr, near.ptr, op, kernel, prec, _dptr(x, "x"), _dptr(y, "y"),
                                _stream(stream)))
    return y


def pb_system_apply(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, x: torch.Tensor, prec: int = PB_F64,
                    alpha: float = 0.0, beta: float = 0.0, y: torch.Tensor | None = None, stream=None):
    if y is None:
        y = torch.empty_like(x)
    p = params.c()
    _check(N.load().pb_system_apply(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), alpha, beta, prec,
                                    _dptr(x, "x"), _dptr(y, "y"), _stream(stream)))
    return y


def pb_system_apply_noalloc(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, x: torch.Tensor,
                            y: torch.Tensor, alpha: float = 0.0, beta: float = 0.0, stream=None):
    """FP32 system application that allocates no device memory: for callers
    that cannot call cudaMalloc (see include/pbbem.h). y must be preallocated
    by the caller; meshes up to the library's 16 MiB scratch limit."""
    p = params.c()
    _check(N.load().pb_system_apply_noalloc(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), alpha, beta,
                                            _dptr(x, "x"), _dptr(y, "y"), _stream(stream)))
    return y


def pb_rhs_charges(ctx: Ctx, mesh: Mesh, xq: torch.Tensor, q: torch.Tensor, params: Params, form,
                   alpha: float = 0.0, beta: float = 0.0, rhs: torch.Tensor | None = None, stream=None,
                   prec: int = PB_F64):
    """prec: PB_F64, or PB_F32_ACCURATE (split-coordinate FP32 pair sums, FP64 tile sums)."""
    nv = mesh.info()["n_verts"]
    if rhs is None:
        rhs = torch.empty(2 * nv, dtype=torch.float64, device=xq.device)
    p = params.c()
    _check(N.load().pb_rhs_charges(ctx.ptr, mesh.ptr, _dptr(xq, "xq"), _dptr(q, "q"), q.numel(), ctypes.byref(p),
                                   _form(form), alpha, beta, _dptr(rhs, "rhs"), int(prec), _stream(stream)))
    return rhs


def solve_opts(tol=1e-6, max_it=500, restart=0, precision=PB_F64, inner_tol=1e-4, max_outer=20, alpha=0.0,
               beta=0.0, pc_a=0.0, pc_b=0.0):
    return N.pb_solve_opts(tol, max_it, restart, precision, inner_tol, max_outer, alpha, beta, pc_a, pc_b)


def pb_solve(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, precond, rhs: torch.Tensor,
             x: torch.Tensor | None = None, opts=None, stream=None, raise_on_noconv: bool = True):
    """Returns (x, info dict)."""
    if x is None:
        x = torch.empty_like(rhs)
    p = params.c()
    o = opts if opts is not None else solve_opts()
    info = N.pb_solve_info()
    rc = N.load().pb_solve(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), _prec(precond),
                           ctypes.byref(o), _dptr(rhs, "rhs"), _dptr(x, "x"), ctypes.byref(info), _stream(stream))
    d = {k: getattr(info, k) for k, _ in N.pb_solve_info._fields_}
    if rc != PB_OK and (raise_on_noconv or rc != PB_ENOCONV):
        _check(rc)
    return x, d


def pb_solve_many(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, precond, rhs: torch.Tensor,
                  x: torch.Tensor | None = None, opts=None, stream=None, raise_on_noconv: bool = True):
    """rhs: [K, 2 N_v] device tensor of K right-hand sides. Returns (x [K, 2 N_v], list of K info dicts)."""
    rhs = rhs.contiguous()
    if x is None:
        x = torch.empty_like(rhs)
    k = rhs.shape[0]
    p = params.c()
    o = opts if opts is not None else solve_opts()
    infos = (N.pb_solve_info * k)()
    rc = N.load().pb_solve_many(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), _prec(precond),
                                ctypes.byref(o), int(k), _dptr(rhs, "rhs"), _dptr(x, "x"), infos, _stream(stream))
    d = [{f: getattr(infos[i], f) for f, _ in N.pb_solve_info._fields_} for i in range(k)]
    if rc != PB_OK and (raise_on_noconv or rc != PB_ENOCONV):
        _check(rc)
    return x, d


def pb_precond_apply(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, precond, x: torch.Tensor,
                     y: torch.Tensor | None = None, opts=None, prec: int = PB_F64, stream=None):
    """y = P^-1 x with the preconditioner pb_solve uses."""
    if y is None:
        y = torch.empty_like(x)
    p = params.c()
    o = opts if opts is not None else solve_opts()
    _check(N.load().pb_precond_apply(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), _prec(precond),
                                     ctypes.byref(o), int(prec), _dptr(x, "x"), _dptr(y, "y"), _stream(stream)))
    return y


def pb_solve_pc(ctx: Ctx, mesh: Mesh, near: Near, pc_mesh: Mesh, pc_near: Near, params: Params, form, precond,
                rhs: torch.Tensor, x: torch.Tensor | None = None, opts=None, stream=None,
                raise_on_noconv: bool = True):
    """Fast Calderon: pb_solve with the preconditioner's operator from pc_mesh/pc_near (the same surface
    loaded with a relaxed plan). Returns (x, info dict)."""
    if x is None:
        x = torch.empty_like(rhs)
    p = params.c()
    o = opts if opts is not None else solve_opts()
    info = N.pb_solve_info()
    rc = N.load().pb_solve_pc(ctx.ptr, mesh.ptr, near.ptr, pc_mesh.ptr, pc_near.ptr, ctypes.byref(p), _form(form),
                              _prec(precond), ctypes.byref(o), _dptr(rhs, "rhs"), _dptr(x, "x"), ctypes.byref(info),
                              _stream(stream))
    d = {k: getattr(info, k) for k, _ in N.pb_solve_info._fields_}
    if rc != PB_OK and (raise_on_noconv or rc != PB_ENOCONV):
        _check(rc)
    return x, d


def pb_energy(ctx: Ctx, mesh: Mesh, x: torch.Tensor, form, xq: torch.Tensor, q: torch.Tensor, params: Params,
              phi: torch.Tensor | None = None, stream=None, prec: int = PB_F64):
    """Returns (dG in paper units, dG in kcal/mol); phi (optional, n_q) receives phi_reac.
    prec: PB_F64, or PB_F32_ACCURATE (split-coordinate FP32 pair sums, FP64 tile sums)."""
    p = params.c()
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(N.load().pb_energy(ctx.ptr, mesh.ptr, _dptr(x, "x"), _form(form), _dptr(xq, "xq"), _dptr(q, "q"),
                              q.numel(), ctypes.byref(p), _dptr(phi, "phi") if phi is not None else None,
                              ctypes.byref(a), ctypes.byref(b), int(prec), _stream(stream)))
    return a.value, b.value


class Server(_Handle):
    """Continuous-batching request server (see pb_server_create in include/pbbem.h)."""
    _free = "pb_server_destroy"


def pb_server_create(ctx: Ctx, hbm_budget_bytes: int, max_active: int = 64) -> Server:
    h = ctypes.c_void_p()
    _check(N.load().pb_server_create(ctx.ptr, int(hbm_budget_bytes), int(max_active), ctypes.byref(h)))
    return Server(h.value, ctx)


def pb_submit(srv: Server, verts, tris, xq, q, params: Params, form, precond, opts=None, tag: int = 0,
              far_q: int = 6, n_ss: int = 4, band_eta: float = 0.0, band_q: int = 6, n_ss_coin: int = 0,
              n_ss_edge: int = 0, n_ss_vert: int = 0):
    """Queue one molecule (host arrays, copied by the library)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    x = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    r = N.pb_request()
    r.verts, r.n_verts = v.ctypes.data, v.shape[0]
    r.tris, r.n_tris = t.ctypes.data, t.shape[0]
    r.xq, r.q, r.n_q = x.ctypes.data, qq.ctypes.data, qq.shape[0]
    r.params = params.c()
    r.form, r.precond = _form(form), _prec(precond)
    r.opts = opts if opts is not None else solve_opts()
    r.plan = _plan(far_q, n_ss, band_eta, band_q, n_ss_coin, n_ss_edge, n_ss_vert)
    r.tag = int(tag)
    _check(N.load().pb_submit(srv.ptr, ctypes.byref(r)))


def pb_server_step(srv: Server):
    """One scheduling step; returns (n_active, n_pending)."""
    a, p = ctypes.c_int(), ctypes.c_int()
    _check(N.load().pb_server_step(srv.ptr, ctypes.byref(a), ctypes.byref(p)))
    return a.value, p.value


def pb_poll(srv: Server, max_results: int = 1024):
    """Finished results as a list of dicts."""
    buf = (N.pb_result * max_results)()
    n = ctypes.c_int()
    _check(N.load().pb_poll(srv.ptr, buf, max_results, ctypes.byref(n)))
    return [{k: getattr(buf[i], k) for k, _ in N.pb_result._fields_} for i in range(n.value)]


def pb_autotune(ctx: Ctx, mesh: Mesh, near: Near, params: Params, form, stream=None):
    """Tune the FP32 far-field launch for this mesh size; returns the choices
    {"fast": {...}, "accurate": {...}} (kernel, shape, tile records, stages,
    targets per thread, split scale, best and default ms)."""
    r = N.pb_tune_result()
    p = params.c()
    _check(N.load().pb_autotune(ctx.ptr, mesh.ptr, near.ptr, ctypes.byref(p), _form(form), ctypes.byref(r),
                                _stream(stream)))
    return {v: {k: getattr(getattr(r, v), k) for k, _ in N.pb_tune_choice._fields_} for v in ("fast", "accurate")}


def pb_autotune_plan(ctx: Ctx, verts, tris, xq, q, params: Params, form, precond, tol_dG: float = 1e-6,
                     reference=(6, 4), opts=None, stream=None):
    """Cheapest quadrature plan whose Delta G stays within tol_dG of the reference plan:
    returns (plan as a dict of pb_mesh_load's keyword arguments, relative change)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    x = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    p = params.c()
    ref = _plan(*reference)
    out = N.pb_quad_plan()
    ch = ctypes.c_double()
    o = opts if opts is not None else solve_opts()
    _check(N.load().pb_autotune_plan(ctx.ptr, ctypes.c_void_p(v.ctypes.data), v.shape[0],
                                     ctypes.c_void_p(t.ctypes.data), t.shape[0], ctypes.c_void_p(x.ctypes.data),
                                     ctypes.c_void_p(qq.ctypes.data), qq.shape[0], ctypes.byref(p), ctypes.byref(ref),
                                     _form(form), _prec(precond), ctypes.byref(o), float(tol_dG), ctypes.byref(out),
                                     ctypes.byref(ch), _stream(stream)))
    return plan_dict(out), ch.value


def pb_solvation_energy(ctx: Ctx, verts: np.ndarray, tris: np.ndarray, xq: np.ndarray, q: np.ndarray,
                        params: Params, form, precond, far_q: int = 6, n_ss: int = 4, opts=None, stream=None,
                        band_eta: float = 0.0, band_q: int = 6, n_ss_coin: int = 0, n_ss_edge: int = 0,
                        n_ss_vert: int = 0):
    """Whole path from host arrays; returns (dG kcal/mol, info dict)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    x = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, 3)
    qq = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    p = params.c()
    plan = _plan(far_q, n_ss, band_eta, band_q, n_ss_coin, n_ss_edge, n_ss_vert)
    o = opts if opts is not None else solve_opts()
    info = N.pb_solve_info()
    out = ctypes.c_double()
    _check(N.load().pb_solvation_energy(ctx.ptr, ctypes.c_void_p(v.ctypes.data), v.shape[0],
                                        ctypes.c_void_p(t.ctypes.data), t.shape[0], ctypes.c_void_p(x.ctypes.data),
                                        ctypes.c_void_p(qq.ctypes.data), qq.shape[0], ctypes.byref(p),
                                        ctypes.byref(plan), _form(form), _prec(precond), ctypes.byref(o),
                                        ctypes.byref(out), ctypes.byref(info), _stream(stream)))
    return out.value, {k: getattr(info, k) for k, _ in N.pb_solve_info._fields_}
