"""Thin ctypes binding of libpp (include/pp.h): argument marshalling only.

Every function keeps the C name and forwards to libpp; device arrays are
torch CUDA float64 tensors (their data_ptr() is passed), host arrays are
numpy float64 arrays.  Nonzero status codes raise PPError with the library's
message.  There is no fallback: if libpp.so is missing or fails to load,
importing this module raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpp.so")

PP_OK, PP_EINVAL, PP_ENOMEM, PP_ENOCONV, PP_ENAN, PP_EBREAKDOWN, PP_ECUDA, PP_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
PP_KIN_HEAVE_PITCH, PP_KIN_FOURIER6, PP_KIN_SPLINE8 = 0, 1, 2
PP_PREC_FP64, PP_PREC_MIXED = 0, 1
STATUS_NAMES = {0: "PP_OK", -1: "PP_EINVAL", -2: "PP_ENOMEM", -3: "PP_ENOCONV", -4: "PP_ENAN",
                -5: "PP_EBREAKDOWN", -6: "PP_ECUDA", -7: "PP_ESTATE"}

EXPORTED = [
    "pp_version", "pp_config_default", "pp_create", "pp_destroy", "pp_last_error", "pp_mesh_create",
    "pp_mesh_destroy", "pp_mesh_info", "pp_residual", "pp_jacobian_blocks", "pp_qoi_rate", "pp_primal_period",
    "pp_tangent_matvec", "pp_adjoint_sweep", "pp_shoot_nk", "pp_periodic_adjoint", "pp_qoi_rate_noalloc",
    "pp_steady_state",
    # include/pp_prof.h
    "pp_prof_select", "pp_prof_read", "pp_prof_counts", "pp_measure_fp64_peak", "pp_sweep_counts",
    "pp_shoot_fixed_point", "pp_periodic_adjoint_fixed_point", "pp_floquet", "pp_hessenberg_eigvals",
    "pp_ogrid_generate", "pp_mesh_ogrid", "pp_shoot_nk_batched", "pp_periodic_adjoint_batched",
    "pp_periodic_adjoint_multi", "pp_motion_eval",
    "pp_stage_apply", "pp_prof_also", "pp_prof_sample", "pp_prof_read_class", "pp_measure_fp64_peak_clock",
    # include/pp_learn.h
    "pp_gemm_f32", "pp_gemm_f64", "pp_bias_act_f32", "pp_gelu_backward_f32", "pp_colsum_f32", "pp_mse_f32",
    "pp_adam_f32", "pp_syevj_f64",
]
PP_K = dict(none=0, jacobian=1, residual=2, stage_matvec=3, block_apply=4, block_inverse=5, krylov=6, other=7,
            stage_matvec32=8, block_apply32=9, krylov32=10, stage_op=11, fold=12, stage_op32=13, arnoldi=14,
            arnoldi32=15)


class pp_config(C.Structure):
    _fields_ = [("p", C.c_int), ("gamma", C.c_double), ("Pr", C.c_double), ("Mach", C.c_double),
                ("Re", C.c_double), ("T", C.c_double), ("kin", C.c_int), ("device", C.c_int),
                ("stream", C.c_void_p), ("newton_tol", C.c_double), ("newton_maxit", C.c_int),
                ("gmres_rtol", C.c_double), ("gmres_restart", C.c_int), ("gmres_maxit", C.c_int),
                ("lin_rtol", C.c_double), ("nk_gmres_rtol", C.c_double), ("nk_restart", C.c_int),
                ("nk_max_newton", C.c_int), ("nk_max_krylov", C.c_int), ("adj_tol", C.c_double),
                ("adj_restart", C.c_int), ("adj_maxit", C.c_int), ("precision", C.c_int),
                ("inner_maxit", C.c_int), ("inner_rtol", C.c_double), ("checkpoint_stride", C.c_int),
                ("nk_fixed_point_pre", C.c_int)]


class pp_shoot_stats(C.Structure):
    _fields_ = [("cold_start", C.c_int), ("newton_iters", C.c_int), ("krylov_iters", C.c_int), ("primal_sweeps", C.c_int),
                ("stage_newton_iters", C.c_int), ("residual", C.c_double * 64), ("seconds", C.c_double)]


class pp_adj_stats(C.Structure):
    _fields_ = [("krylov_iters", C.c_int), ("residual", C.c_double), ("seconds", C.c_double)]


class PPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpp.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_1512_00616_gb300.build")
    lib = C.CDLL(LIB_PATH)
    P, D, I, V = C.c_void_p, C.c_double, C.c_int, None
    dp = C.POINTER(C.c_double)
    sig = {
        "pp_version": (C.c_char_p, []),
        "pp_config_default": (V, [C.POINTER(pp_config)]),
        "pp_create": (I, [C.POINTER(pp_config), C.POINTER(P)]),
        "pp_destroy": (I, [P]),
        "pp_last_error": (C.c_char_p, [P]),
        "pp_mesh_create": (I, [P, dp, I, C.POINTER(C.c_int32), C.POINTER(C.c_int32), I, C.POINTER(P)]),
        "pp_mesh_destroy": (I, [P]),
        "pp_mesh_info": (I, [P, C.POINTER(I), C.POINTER(I), C.POINTER(C.c_int64)]),
        "pp_motion_eval": (I, [I, D, dp, I, D, dp]),
        "pp_residual": (I, [P, P, dp, I, D, P, P]),
        "pp_jacobian_blocks": (I, [P, P, dp, I, D, P, P]),
        "pp_qoi_rate": (I, [P, P, dp, I, D, P, dp]),
        "pp_qoi_rate_noalloc": (I, [P, P, dp, I, D, P, dp]),
        "pp_steady_state": (I, [P, P, dp, I, D, I, P, C.POINTER(I), dp]),
        "pp_primal_period": (I, [P, P, dp, I, P, I, P, P, dp]),
        "pp_tangent_matvec": (I, [P, P, P]),
        "pp_adjoint_sweep": (I, [P, P, dp, P, dp]),
        "pp_shoot_nk": (I, [P, P, dp, I, P, I, D, P, dp, C.POINTER(pp_shoot_stats)]),
        "pp_periodic_adjoint": (I, [P, P, dp, I, P, I, dp, dp, dp, P, C.POINTER(pp_adj_stats)]),
        "pp_shoot_fixed_point": (I, [P, P, dp, I, P, I, D, I, P, dp, C.POINTER(pp_shoot_stats)]),
        "pp_floquet": (I, [P, I, dp, dp, dp]),
        "pp_periodic_adjoint_multi": (I, [P, P, dp, I, P, I, I, dp, dp, dp, P, C.POINTER(pp_adj_stats)]),
        "pp_shoot_nk_batched": (I, [P, P, dp, I, I, P, I, D, P, dp, C.POINTER(pp_shoot_stats), C.POINTER(I)]),
        "pp_periodic_adjoint_batched": (I, [P, P, dp, I, I, P, I, dp, dp, dp, P, C.POINTER(pp_adj_stats)]),
        "pp_ogrid_generate": (I, [I, I, D, C.c_uint64, dp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(I), C.POINTER(I)]),
        "pp_mesh_ogrid": (I, [P, I, I, D, C.c_uint64, C.POINTER(P)]),
        "pp_hessenberg_eigvals": (I, [I, dp, I, dp, dp]),
        "pp_periodic_adjoint_fixed_point": (I, [P, P, dp, I, P, I, dp, D, I, dp, dp, P, C.POINTER(pp_adj_stats)]),
        "pp_prof_select": (I, [I]),
        "pp_prof_read": (I, [C.POINTER(C.c_int64), dp]),
        "pp_prof_counts": (I, [C.POINTER(C.c_int64)]),
        "pp_measure_fp64_peak": (I, [I, dp]),
        "pp_sweep_counts": (I, [P] + [C.POINTER(C.c_int64)] * 4),
        "pp_stage_apply": (I, [P, I, I, I, I, I, P, P]),
        "pp_prof_also": (I, [I]),
        "pp_prof_sample": (I, [I]),
        "pp_prof_read_class": (I, [I, C.POINTER(C.c_int64), dp, dp]),
        "pp_measure_fp64_peak_clock": (I, [I, dp, dp]),
        "pp_gemm_f32": (I, [I, I, I, C.c_float, P, I, I, P, I, I, C.c_float, P, I, P]),
        "pp_gemm_f64": (I, [I, I, I, D, P, I, I, P, I, I, D, P, I, P]),
        "pp_bias_act_f32": (I, [I, I, P, P, P, I, P]),
        "pp_gelu_backward_f32": (I, [I, P, P, P, P]),
        "pp_colsum_f32": (I, [I, I, P, P, P]),
        "pp_mse_f32": (I, [I, P, P, P, P, P]),
        "pp_adam_f32": (I, [I, P, P, P, P, C.c_float, C.c_float, C.c_float, C.c_float, I, P]),
        "pp_syevj_f64": (I, [I, P, P, P, D, I, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


# --------------------------------------------------------------------------- helpers
def _host(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(C.c_double if dtype == np.float64 else C.c_int32))


def _dev(t, name):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    return C.c_void_p(t.data_ptr())


def _check(ctx, code):
    if code != PP_OK:
        msg = _lib.pp_last_error(ctx).decode() if ctx else ""
        raise PPError(code, msg)


# --------------------------------------------------------------------------- entry points
def pp_version():
    return _lib.pp_version().decode()


def pp_config_default(**overrides):
    cfg = pp_config()
    _lib.pp_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def pp_create(cfg=None, **overrides):
    if cfg is None:
        cfg = pp_config_default(**overrides)
    h = C.c_void_p()
    _check(None, _lib.pp_create(C.byref(cfg), C.byref(h)))
    return h


def pp_destroy(ctx):
    _check(None, _lib.pp_destroy(ctx))


def pp_last_error(ctx):
    return _lib.pp_last_error(ctx).decode()


def pp_mesh_create(ctx, verts, tris, ftag):
    v, vp = _host(verts)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    f = np.ascontiguousarray(ftag, dtype=np.int32)
    h = C.c_void_p()
    _check(ctx, _lib.pp_mesh_create(ctx, vp, v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)),
                                    f.ctypes.data_as(C.POINTER(C.c_int32)), t.shape[0], C.byref(h)))
    return h


def pp_ogrid_generate(n_theta, n_r, r_far=10.0, seed=0):
    """(verts [nv, 2], tris [nt, 3], ftag [nt, 3]) of the library's seeded O-grid (host code)."""
    nv, nt = C.c_int(), C.c_int()
    code = _lib.pp_ogrid_generate(int(n_theta), int(n_r), float(r_far), int(seed), None, None, None,
                                  C.byref(nv), C.byref(nt))
    if code != PP_OK:
        raise PPError(code, "pp_ogrid_generate")
    v = np.zeros((nv.value, 2))
    t = np.zeros((nt.value, 3), dtype=np.int32)
    g = np.zeros((nt.value, 3), dtype=np.int32)
    _lib.pp_ogrid_generate(int(n_theta), int(n_r), float(r_far), int(seed), v.ctypes.data_as(C.POINTER(C.c_double)),
                           t.ctypes.data_as(C.POINTER(C.c_int32)), g.ctypes.data_as(C.POINTER(C.c_int32)), None, None)
    return v, t, g


def pp_mesh_ogrid(ctx, n_theta, n_r, r_far=10.0, seed=0):
    out = C.c_void_p()
    _check(ctx, _lib.pp_mesh_ogrid(ctx, int(n_theta), int(n_r), float(r_far), int(seed), C.byref(out)))
    return out


def pp_mesh_destroy(mesh):
    _check(None, _lib.pp_mesh_destroy(mesh))


def pp_motion_eval(kin, T, mu, t):
    """(theta, theta', h') at time t and their derivatives d/dmu_j as a [1 + n_mu, 3] array."""
    m, mp = _host(mu)
    out = np.zeros(3 + 3 * len(m))
    code = _lib.pp_motion_eval(int(kin), float(T), mp, len(m), float(t), out.ctypes.data_as(C.POINTER(C.c_double)))
    if code != PP_OK:
        raise PPError(code, "pp_motion_eval")
    return out.reshape(1 + len(m), 3)


def pp_mesh_info(mesh):
    ne, npn, nu = C.c_int(), C.c_int(), C.c_int64()
    _check(None, _lib.pp_mesh_info(mesh, C.byref(ne), C.byref(npn), C.byref(nu)))
    return ne.value, npn.value, nu.value


def pp_residual(ctx, mesh, mu, t, u, r):
    m, mp = _host(mu)
    _check(ctx, _lib.pp_residual(ctx, mesh, mp, len(m), float(t), _dev(u, "u"), _dev(r, "r")))


def pp_jacobian_blocks(ctx, mesh, mu, t, u, blocks):
    m, mp = _host(mu)
    _check(ctx, _lib.pp_jacobian_blocks(ctx, mesh, mp, len(m), float(t), _dev(u, "u"), _dev(blocks, "blocks")))


def pp_qoi_rate(ctx, mesh, mu, t, u):
    m, mp = _host(mu)
    out = np.zeros(2)
    _check(ctx, _lib.pp_qoi_rate(ctx, mesh, mp, len(m), float(t), _dev(u, "u"), _host(out)[1]))
    return out


def pp_qoi_rate_noalloc(ctx, mesh, mu, t, u):
    m, mp = _host(mu)
    out = np.zeros(2)
    _check(ctx, _lib.pp_qoi_rate_noalloc(ctx, mesh, mp, len(m), float(t), _dev(u, "u"), _host(out)[1]))
    return out


def pp_primal_period(ctx, mesh, mu, u0, Nt, u_traj=None, u_final=None):
    m, mp = _host(mu)
    qoi = np.zeros(4)
    _check(ctx, _lib.pp_primal_period(ctx, mesh, mp, len(m), _dev(u0, "u0"), int(Nt), _dev(u_traj, "u_traj"),
                                      _dev(u_final, "u_final"), qoi.ctypes.data_as(C.POINTER(C.c_double))))
    return qoi


def pp_tangent_matvec(ctx, v, out):
    _check(ctx, _lib.pp_tangent_matvec(ctx, _dev(v, "v"), _dev(out, "out")))


def pp_adjoint_sweep(ctx, lam_Nt, lam0, weights=None, n_mu=0):
    if weights is not None:
        w, wp = _host(weights)
        g = np.zeros(max(n_mu, 1))
        gp = g.ctypes.data_as(C.POINTER(C.c_double)) if n_mu else None
    else:
        wp, g, gp = None, None, None
    _check(ctx, _lib.pp_adjoint_sweep(ctx, _dev(lam_Nt, "lam_Nt"), wp, _dev(lam0, "lam0"), gp))
    return g[:n_mu] if (weights is not None and n_mu) else None


def pp_shoot_nk(ctx, mesh, mu, Nt, tol, u0_out, u0_guess=None, raise_on_noconv=True):
    m, mp = _host(mu)
    qoi = np.zeros(4)
    st = pp_shoot_stats()
    code = _lib.pp_shoot_nk(ctx, mesh, mp, len(m), _dev(u0_guess, "u0_guess"), int(Nt), float(tol),
                            _dev(u0_out, "u0_out"), qoi.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st))
    if code != PP_ENOCONV or raise_on_noconv:
        _check(ctx, code)
    n = min(st.newton_iters + 1, 64)
    stats = dict(cold_start=st.cold_start, newton_iters=st.newton_iters, krylov_iters=st.krylov_iters, primal_sweeps=st.primal_sweeps,
                 stage_newton_iters=st.stage_newton_iters, residual=list(st.residual[:n]), seconds=st.seconds,
                 status=code)
    return qoi, stats


def pp_shoot_nk_batched(ctx, mesh, mu, Nt, tol, u0_out, u0_guess=None, raise_on_noconv=True):
    """mu [B, n_mu] (host); u0_out, u0_guess: CUDA float64 [B * N_u].  Returns (qoi [B, 4], status [B], stats)."""
    m = np.ascontiguousarray(mu, dtype=np.float64)
    B, n_mu = m.shape
    qoi = np.zeros((B, 4))
    st = (pp_shoot_stats * B)()
    status = (C.c_int * B)()
    code = _lib.pp_shoot_nk_batched(ctx, mesh, m.ctypes.data_as(C.POINTER(C.c_double)), n_mu, B,
                                    _dev(u0_guess, "u0_guess"), int(Nt), float(tol), _dev(u0_out, "u0_out"),
                                    qoi.ctypes.data_as(C.POINTER(C.c_double)), st, status)
    if code != PP_ENOCONV or raise_on_noconv:
        _check(ctx, code)
    stats = [dict(newton_iters=s.newton_iters, krylov_iters=s.krylov_iters, cold_start=s.cold_start,
                  residual=list(s.residual[:min(s.newton_iters + 1, 64)]), seconds=s.seconds) for s in st]
    return qoi, np.array(status[:]), stats


def pp_periodic_adjoint_batched(ctx, mesh, mu, Nt, weights, u0, lam_Nt=None):
    """mu [B, n_mu], weights [B, 2] (host); u0, lam_Nt: CUDA float64 [B * N_u].  Returns (F [B], dF/dmu [B, n_mu])."""
    m = np.ascontiguousarray(mu, dtype=np.float64)
    B, n_mu = m.shape
    w = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64), (B, 2)))
    F = np.zeros(B)
    g = np.zeros((B, n_mu))
    st = (pp_adj_stats * B)()
    _check(ctx, _lib.pp_periodic_adjoint_batched(ctx, mesh, m.ctypes.data_as(C.POINTER(C.c_double)), n_mu, B,
                                                 _dev(u0, "u0"), int(Nt), w.ctypes.data_as(C.POINTER(C.c_double)),
                                                 F.ctypes.data_as(C.POINTER(C.c_double)),
                                                 g.ctypes.data_as(C.POINTER(C.c_double)), _dev(lam_Nt, "lam_Nt"), st))
    return F, g


def pp_periodic_adjoint_multi(ctx, mesh, mu, Nt, weights, u0=None, lam_Nt=None):
    """weights [n_qoi, 2]; lam_Nt: CUDA float64 [n_qoi * N_u] or None.  Returns (F [n_qoi],
    dF/dmu [n_qoi, n_mu], stats)."""
    m, mp = _host(mu)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    nq = w.shape[0]
    F = np.zeros(nq)
    g = np.zeros((nq, len(m)))
    st = pp_adj_stats()
    _check(ctx, _lib.pp_periodic_adjoint_multi(ctx, mesh, mp, len(m), _dev(u0, "u0"), int(Nt), nq,
                                               w.ctypes.data_as(C.POINTER(C.c_double)),
                                               F.ctypes.data_as(C.POINTER(C.c_double)),
                                               g.ctypes.data_as(C.POINTER(C.c_double)), _dev(lam_Nt, "lam_Nt"),
                                               C.byref(st)))
    return F, g, dict(sweeps=st.krylov_iters, residual=st.residual, seconds=st.seconds)


def pp_shoot_fixed_point(ctx, mesh, mu, Nt, tol, maxit, u0_guess, u0_out, raise_on_noconv=True):
    m, mp = _host(mu)
    qoi = np.zeros(4)
    st = pp_shoot_stats()
    code = _lib.pp_shoot_fixed_point(ctx, mesh, mp, len(m), _dev(u0_guess, "u0_guess"), int(Nt), float(tol),
                                     int(maxit), _dev(u0_out, "u0_out"), qoi.ctypes.data_as(C.POINTER(C.c_double)),
                                     C.byref(st))
    if code != PP_ENOCONV or raise_on_noconv:
        _check(ctx, code)
    n = min(st.newton_iters + 1, 64)
    return qoi, dict(iterations=st.newton_iters, primal_sweeps=st.primal_sweeps, residual=list(st.residual[:n]),
                     seconds=st.seconds, status=code)


def pp_steady_state(ctx, mesh, mu, u, tol=1e-10, maxit=100):
    m, mp = _host(mu)
    steps, rel = C.c_int(), C.c_double()
    _check(ctx, _lib.pp_steady_state(ctx, mesh, mp, len(m), float(tol), int(maxit), _dev(u, "u"), C.byref(steps),
                                     C.byref(rel)))
    return steps.value, rel.value


def pp_periodic_adjoint(ctx, mesh, mu, Nt, weights, u0=None, lam_Nt=None):
    m, mp = _host(mu)
    w, wp = _host(weights)
    F = np.zeros(1)
    g = np.zeros(len(m))
    st = pp_adj_stats()
    _check(ctx, _lib.pp_periodic_adjoint(ctx, mesh, mp, len(m), _dev(u0, "u0"), int(Nt), wp,
                                         F.ctypes.data_as(C.POINTER(C.c_double)),
                                         g.ctypes.data_as(C.POINTER(C.c_double)), _dev(lam_Nt, "lam_Nt"),
                                         C.byref(st)))
    return float(F[0]), g, dict(krylov_iters=st.krylov_iters, residual=st.residual, seconds=st.seconds)


def pp_periodic_adjoint_fixed_point(ctx, mesh, mu, Nt, weights, tol, maxit, u0=None, lam_Nt=None):
    m, mp = _host(mu)
    w, wp = _host(weights)
    F = np.zeros(1)
    g = np.zeros(len(m))
    st = pp_adj_stats()
    _check(ctx, _lib.pp_periodic_adjoint_fixed_point(ctx, mesh, mp, len(m), _dev(u0, "u0"), int(Nt), wp, float(tol),
                                                     int(maxit), F.ctypes.data_as(C.POINTER(C.c_double)),
                                                     g.ctypes.data_as(C.POINTER(C.c_double)),
                                                     _dev(lam_Nt, "lam_Nt"), C.byref(st)))
    return float(F[0]), g, dict(sweeps=st.krylov_iters, residual=st.residual, seconds=st.seconds)


def pp_floquet(ctx, m):
    """Ritz values (complex, largest modulus first) of Phi from m Arnoldi steps, and h_(m+1,m)."""
    wr, wi, hl = np.zeros(m), np.zeros(m), np.zeros(1)
    _check(ctx, _lib.pp_floquet(ctx, int(m), wr.ctypes.data_as(C.POINTER(C.c_double)),
                                wi.ctypes.data_as(C.POINTER(C.c_double)), hl.ctypes.data_as(C.POINTER(C.c_double))))
    return wr + 1j * wi, float(hl[0])


def pp_hessenberg_eigvals(H):
    """Eigenvalues of an upper Hessenberg matrix (host code of the library)."""
    A = np.array(H, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    wr, wi = np.zeros(n), np.zeros(n)
    code = _lib.pp_hessenberg_eigvals(n, A.ctypes.data_as(C.POINTER(C.c_double)), n,
                                      wr.ctypes.data_as(C.POINTER(C.c_double)), wi.ctypes.data_as(C.POINTER(C.c_double)))
    if code != PP_OK:
        raise PPError(code, "pp_hessenberg_eigvals")
    return wr + 1j * wi


# --------------------------------------------------------------------------- diagnostics (include/pp_prof.h)
def pp_prof_select(kind):
    k = PP_K[kind] if isinstance(kind, str) else int(kind)
    _check(None, _lib.pp_prof_select(k))


def pp_prof_read():
    n, ms = C.c_int64(), C.c_double()
    _check(None, _lib.pp_prof_read(C.byref(n), C.byref(ms)))
    return n.value, ms.value


def pp_prof_sample(stride):
    _check(None, _lib.pp_prof_sample(int(stride)))


def pp_prof_also(kind):
    k = PP_K[kind] if isinstance(kind, str) else int(kind)
    _check(None, _lib.pp_prof_also(k))


def pp_prof_read_class(kind):
    """(timed launches, summed ms, algorithmic bytes) of one timed kernel class."""
    k = PP_K[kind] if isinstance(kind, str) else int(kind)
    n, ms, by = C.c_int64(), C.c_double(), C.c_double()
    _check(None, _lib.pp_prof_read_class(k, C.byref(n), C.byref(ms), C.byref(by)))
    return n.value, ms.value, by.value


def pp_prof_counts():
    a = (C.c_int64 * len(PP_K))()
    _check(None, _lib.pp_prof_counts(a))
    return {k: a[v] for k, v in PP_K.items() if k != "none"}


def pp_measure_fp64_peak(device=0):
    t = C.c_double()
    _check(None, _lib.pp_measure_fp64_peak(int(device), C.byref(t)))
    return t.value


def pp_measure_fp64_peak_clock(device=0):
    """(TFLOP/s, SM MHz inside the probe)."""
    t, mhz = C.c_double(), C.c_double()
    _check(None, _lib.pp_measure_fp64_peak_clock(int(device), C.byref(t), C.byref(mhz)))
    return t.value, mhz.value


def pp_sweep_counts(ctx):
    v = [C.c_int64() for _ in range(4)]
    _check(ctx, _lib.pp_sweep_counts(ctx, *[C.byref(x) for x in v]))
    return dict(newton=v[0].value, gmres_primal=v[1].value, gmres_tangent=v[2].value, gmres_adjoint=v[3].value)


def pp_stage_apply(ctx, step, stage, kind, x, y, trans=False, prec=0):
    """y = one stored stage operator applied to x (kind 0: M - cJ, 1: D^-1, 2: (M - cJ) D^-1)."""
    _check(ctx, _lib.pp_stage_apply(ctx, int(step), int(stage), int(kind), int(bool(trans)), int(prec),
                                    _dev(x, "x"), _dev(y, "y")))


# --------------------------------------------------------------------------- learned warm start (include/pp_learn.h)
def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _lcheck(code, name):
    if code != 0:
        raise PPError(code, name)


def pp_gemm(A, B, C_out, ta=False, tb=False, alpha=1.0, beta=0.0):
    """C_out = alpha op(A) op(B) + beta C_out (row-major torch CUDA tensors, float32 or float64)."""
    import torch
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    f = _lib.pp_gemm_f32 if A.dtype == torch.float32 else _lib.pp_gemm_f64
    _lcheck(f(m, n, k, alpha, _ptr(A), A.shape[1], int(ta), _ptr(B), B.shape[1], int(tb), beta, _ptr(C_out),
              C_out.shape[1], _stream()), "pp_gemm")


def pp_bias_act_f32(Z, b, H, gelu_on):
    _lcheck(_lib.pp_bias_act_f32(Z.shape[0], Z.shape[1], _ptr(Z), _ptr(b), _ptr(H), int(gelu_on), _stream()),
            "pp_bias_act_f32")


def pp_gelu_backward_f32(Z, dH, dZ):
    _lcheck(_lib.pp_gelu_backward_f32(Z.numel(), _ptr(Z), _ptr(dH), _ptr(dZ), _stream()), "pp_gelu_backward_f32")


def pp_colsum_f32(dZ, db):
    _lcheck(_lib.pp_colsum_f32(dZ.shape[0], dZ.shape[1], _ptr(dZ), _ptr(db), _stream()), "pp_colsum_f32")


def pp_mse_f32(Y, T, dY, loss):
    _lcheck(_lib.pp_mse_f32(Y.numel(), _ptr(Y), _ptr(T), _ptr(dY), _ptr(loss), _stream()), "pp_mse_f32")


def pp_adam_f32(w, g, m1, m2, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    _lcheck(_lib.pp_adam_f32(w.numel(), _ptr(w), _ptr(g), _ptr(m1), _ptr(m2), lr, b1, b2, eps, int(step),
                             _stream()), "pp_adam_f32")


def pp_syevj_f64(A, V, w, tol=1e-14, max_sweeps=30):
    _lcheck(_lib.pp_syevj_f64(A.shape[0], _ptr(A), _ptr(V), _ptr(w), tol, max_sweeps, None, _stream()),
            "pp_syevj_f64")
