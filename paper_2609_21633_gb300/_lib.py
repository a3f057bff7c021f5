"""ctypes binding of ``include/terra_wedge.h`` (argument marshalling only).

Every function here has the C name of the entry point it calls.  Device
buffers are torch CUDA tensors (torch provides device memory and streams); the
work itself runs in the library's sm_103a kernels.  The shared library must be
built in-tree (``__graft_entry__.build()``); loading fails loudly otherwise --
there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libterra_wedge.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "terra_wedge.h")

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ENOTCONVERGED, TN_ETIMEOUT, TN_EBUSY, TN_ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
TN_ECANCELED = -8
TN_F64, TN_F32 = 0, 1
TN_BC_FREESLIP, TN_BC_NOSLIP = 0, 1
TN_ETA_F32, TN_ETA_BF16, TN_ETA_F16 = 0, 1, 2
TN_FP64_ELEM_DOUBLE_FLOAT, TN_FP64_ELEM_BINARY64 = 0, 1


class TnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class tn_mesh_opts(ctypes.Structure):
    _fields_ = [("bc_inner", ctypes.c_int), ("bc_outer", ctypes.c_int), ("div_term", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("eta_storage", ctypes.c_int), ("hg_kappa", ctypes.c_double),
                ("radial_quad_points", ctypes.c_int), ("fp64_element", ctypes.c_int)]


class tn_level_info(ctypes.Structure):
    _fields_ = [("lateral_level", ctypes.c_int), ("N", ctypes.c_int), ("n_r", ctypes.c_int), ("pitch", ctypes.c_int),
                ("layer_stride", ctypes.c_int64), ("diamond_stride", ctypes.c_int64), ("n_layout", ctypes.c_int64),
                ("n_unique_nodes", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_wedges", ctypes.c_int64),
                ("depth", ctypes.c_int), ("r_in", ctypes.c_double), ("r_out", ctypes.c_double)]


class tn_visc_law(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("jump_r", ctypes.c_double), ("jump_factor", ctypes.c_double)]


class tn_mg_opts(ctypes.Structure):
    _fields_ = [("pre_smooth", ctypes.c_int), ("post_smooth", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("coarse_max_iters", ctypes.c_int), ("coarse_rtol", ctypes.c_double), ("levels", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


class tn_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("restart", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("mode", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("inner_max_iters", ctypes.c_int),
                ("max_refinements", ctypes.c_int)]


class tn_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("converged", ctypes.c_int)]


TN_SOLVE_F64, TN_SOLVE_MIXED, TN_SOLVE_F64_PREC32 = 0, 1, 2


class tn_server_opts(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("memory_fraction", ctypes.c_double), ("mode", ctypes.c_int),
                ("rtol", ctypes.c_double), ("keep_solutions", ctypes.c_int), ("eta_storage", ctypes.c_int),
                ("hg_kappa", ctypes.c_double), ("radial_quad_points", ctypes.c_int), ("max_batch", ctypes.c_int)]


class tn_convection_opts(ctypes.Structure):
    _fields_ = [("Ra", ctypes.c_double), ("E", ctypes.c_double), ("cfl", ctypes.c_double), ("supg", ctypes.c_int),
                ("mode", ctypes.c_int), ("rtol", ctypes.c_double), ("dt", ctypes.c_double), ("substeps", ctypes.c_int)]


class tn_convection_step_stats(ctypes.Structure):
    _fields_ = [("time", ctypes.c_double), ("dt", ctypes.c_double), ("substeps", ctypes.c_int),
                ("stokes_iterations", ctypes.c_int), ("rel_residual", ctypes.c_double), ("nu_top", ctypes.c_double),
                ("v_rms", ctypes.c_double), ("u_max", ctypes.c_double), ("stokes_seconds", ctypes.c_double),
                ("energy_seconds", ctypes.c_double)]


class tn_request(ctypes.Structure):
    _fields_ = [("lateral_level", ctypes.c_int), ("radial_layers", ctypes.c_int), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double), ("E", ctypes.c_double), ("Ra", ctypes.c_double),
                ("t_degree", ctypes.c_int), ("t_order", ctypes.c_int), ("t_amplitude", ctypes.c_double)]


class tn_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_end", ctypes.c_double), ("batch", ctypes.c_int)]


_lib = None
P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "tn_last_error": ([], ctypes.c_char_p),
    "tn_mesh_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                        ctypes.POINTER(tn_mesh_opts), ctypes.POINTER(P)], ctypes.c_int),
    "tn_mesh_destroy": ([P], ctypes.c_int),
    "tn_mesh_info": ([P, ctypes.c_int, ctypes.POINTER(tn_level_info)], ctypes.c_int),
    "tn_mesh_lateral_points": ([P, ctypes.c_int, P], ctypes.c_int),
    "tn_mesh_canonical_index": ([P, ctypes.c_int, P], ctypes.c_int),
    "tn_set_viscosity": ([P, P, P], ctypes.c_int),
    "tn_set_temperature": ([P, P, ctypes.POINTER(tn_visc_law), P], ctypes.c_int),
    "tn_get_viscosity": ([P, ctypes.c_int, P, P], ctypes.c_int),
    "tn_apply_A": ([P, ctypes.c_int, ctypes.c_int, PP, PP, P], ctypes.c_int),
    "tn_apply_B": ([P, ctypes.c_int, ctypes.c_int, PP, P, P], ctypes.c_int),
    "tn_apply_BT": ([P, ctypes.c_int, ctypes.c_int, P, PP, P], ctypes.c_int),
    "tn_apply_B_static": ([P, ctypes.c_int, ctypes.c_int, PP, P, P], ctypes.c_int),
    "tn_diag_A": ([P, ctypes.c_int, ctypes.c_int, PP, P], ctypes.c_int),
    "tn_diag_pmass": ([P, ctypes.c_int, ctypes.c_int, P, P], ctypes.c_int),
    "tn_operator_steps_host": ([P, ctypes.c_int, ctypes.c_int, PP, PP, PP, P], ctypes.c_int),
    "tn_prolong": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PP, PP, P], ctypes.c_int),
    "tn_restrict": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PP, PP, P], ctypes.c_int),
    "tn_buoyancy": ([P, P, ctypes.c_double, PP, P], ctypes.c_int),
    "tn_set_reference_state": ([P, P, P], ctypes.c_int),
    "tn_energy_residual": ([P, P, PP, ctypes.c_int, P, P], ctypes.c_int),
    "tn_energy_steps": ([P, P, PP, ctypes.c_double, ctypes.c_int, ctypes.c_int, P], ctypes.c_int),
    "tn_energy_diagnostics": ([P, P, PP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), P],
                              ctypes.c_int),
    "tn_energy_stable_dt": ([P, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
    "tn_convection_default_opts": ([ctypes.POINTER(tn_convection_opts)], ctypes.c_int),
    "tn_convection_steps": ([P, P, PP, P, ctypes.c_int, ctypes.POINTER(tn_convection_opts),
                             ctypes.POINTER(tn_convection_step_stats), P], ctypes.c_int),
    "tn_mg_default_opts": ([ctypes.POINTER(tn_mg_opts)], ctypes.c_int),
    "tn_mg_setup": ([P, ctypes.c_int, ctypes.POINTER(tn_mg_opts), PP, P], ctypes.c_int),
    "tn_mg_lambda": ([P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "tn_vcycle": ([P, ctypes.c_int, PP, PP, P], ctypes.c_int),
    "tn_solve_default_opts": ([ctypes.POINTER(tn_solve_opts)], ctypes.c_int),
    "tn_stokes_solve": ([P, ctypes.POINTER(tn_solve_opts), PP, P, PP, P, ctypes.POINTER(tn_solve_stats), P],
                        ctypes.c_int),
    "tn_stokes_solve_batch": ([PP, ctypes.c_int, ctypes.POINTER(tn_solve_opts), PP, PP, PP, PP,
                               ctypes.POINTER(tn_solve_stats), ctypes.POINTER(ctypes.c_int), P], ctypes.c_int),
    "tn_server_default_opts": ([ctypes.POINTER(tn_server_opts)], ctypes.c_int),
    "tn_server_create": ([ctypes.POINTER(tn_server_opts), ctypes.POINTER(P)], ctypes.c_int),
    "tn_server_submit": ([P, ctypes.POINTER(tn_request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "tn_server_poll": ([P, ctypes.c_uint64, ctypes.POINTER(tn_result)], ctypes.c_int),
    "tn_server_wait": ([P, ctypes.c_uint64, ctypes.POINTER(tn_result)], ctypes.c_int),
    "tn_server_solution": ([P, ctypes.c_uint64, P, P], ctypes.c_int),
    "tn_server_stats": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "tn_server_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
    "tn_probe_fma_peak": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), P], ctypes.c_int),
    "tn_server_destroy": ([P], ctypes.c_int),
}


def lib():
    """Load the in-tree shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes, fn.restype = args, res
        _lib = L
    return _lib


def _check(status):
    if status != TN_OK:
        raise TnError(status, lib().tn_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return ctypes.cast(arr, PP), arr


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _prec(dtype):
    import torch
    if dtype == torch.float64:
        return TN_F64
    if dtype == torch.float32:
        return TN_F32
    raise TypeError(f"unsupported dtype {dtype}")


def tn_mesh_create(lateral_level, radial_layers, r_in, r_out, bc_inner=TN_BC_FREESLIP, bc_outer=TN_BC_FREESLIP,
                   div_term=True, max_levels=0, eta_storage=0, hg_kappa=0.0, radial_quad_points=1,
                   fp64_element=TN_FP64_ELEM_DOUBLE_FLOAT):
    opts = tn_mesh_opts(bc_inner, bc_outer, int(bool(div_term)), max_levels, eta_storage, float(hg_kappa),
                        int(radial_quad_points), int(fp64_element))
    out = P()
    _check(lib().tn_mesh_create(lateral_level, radial_layers, r_in, r_out, ctypes.byref(opts), ctypes.byref(out)))
    return out


def tn_mesh_destroy(mesh):
    _check(lib().tn_mesh_destroy(mesh))


def tn_mesh_info(mesh, level=0):
    info = tn_level_info()
    _check(lib().tn_mesh_info(mesh, level, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in tn_level_info._fields_}


def tn_mesh_lateral_points(mesh, level=0):
    import numpy as np
    N = tn_mesh_info(mesh, level)["N"]
    out = np.empty((10, N + 1, N + 1, 3), dtype=np.float64)
    _check(lib().tn_mesh_lateral_points(mesh, level, out.ctypes.data_as(P)))
    return out


def tn_mesh_canonical_index(mesh, level=0):
    import numpy as np
    n = tn_mesh_info(mesh, level)["n_layout"]
    out = np.empty(n, dtype=np.int64)
    _check(lib().tn_mesh_canonical_index(mesh, level, out.ctypes.data_as(P)))
    return out


def tn_set_viscosity(mesh, eta, stream=None):
    _check(lib().tn_set_viscosity(mesh, _ptr(eta), _stream(stream)))


def tn_set_temperature(mesh, T, E, jump_r=0.0, jump_factor=1.0, stream=None):
    law = tn_visc_law(E, jump_r, jump_factor)
    _check(lib().tn_set_temperature(mesh, _ptr(T), ctypes.byref(law), _stream(stream)))


def tn_get_viscosity(mesh, level, eta_out, stream=None):
    _check(lib().tn_get_viscosity(mesh, level, _ptr(eta_out), _stream(stream)))


def tn_apply_A(mesh, level, u, y, stream=None):
    pu, _a = _ptrs(u)
    py, _b = _ptrs(y)
    _check(lib().tn_apply_A(mesh, level, _prec(u[0].dtype), pu, py, _stream(stream)))


def tn_apply_B(mesh, level, u, q, stream=None):
    pu, _a = _ptrs(u)
    _check(lib().tn_apply_B(mesh, level, _prec(u[0].dtype), pu, _ptr(q), _stream(stream)))


def tn_apply_B_static(mesh, level, u, q, stream=None):
    pu, _a = _ptrs(u)
    _check(lib().tn_apply_B_static(mesh, level, _prec(u[0].dtype), pu, _ptr(q), _stream(stream)))


def tn_apply_BT(mesh, level, p, y, stream=None):
    py, _b = _ptrs(y)
    _check(lib().tn_apply_BT(mesh, level, _prec(p.dtype), _ptr(p), py, _stream(stream)))


def tn_diag_A(mesh, level, d, stream=None):
    pd, _a = _ptrs(d)
    _check(lib().tn_diag_A(mesh, level, _prec(d[0].dtype), pd, _stream(stream)))


def tn_diag_pmass(mesh, level, m, stream=None):
    _check(lib().tn_diag_pmass(mesh, level, _prec(m.dtype), _ptr(m), _stream(stream)))


def tn_operator_steps_host(mesh, u_steps, p_steps, out_steps, stream=None):
    """len(u_steps) operator steps from and to host memory (see the header): u_steps[i] is 3 host
    tensors, p_steps[i] one, out_steps[i] 10 (y_A 3, q, y_BT 3, d 3), all of one dtype; pinned
    CPU tensors let the copies overlap the compute.  Stream-ordered on `stream`."""
    n = len(u_steps)
    if len(p_steps) != n or len(out_steps) != n:
        raise ValueError("u_steps, p_steps and out_steps need one entry per step")
    if any(len(s) != 3 for s in u_steps) or any(len(s) != 10 for s in out_steps):
        raise ValueError("3 input and 10 output tensors per step")
    if n == 0:
        _check(lib().tn_operator_steps_host(mesh, TN_F64, 0, None, None, None, _stream(stream)))
        return
    # the C side copies n_layout elements to and from each host pointer on trust: check every
    # tensor's device, contiguity, dtype and size here, before any copy is enqueued
    n0, n1 = tn_mesh_info(mesh, 0)["n_layout"], tn_mesh_info(mesh, 1)["n_layout"]
    dtype = p_steps[0].dtype
    _prec(dtype)
    for i in range(n):
        slots = ([(t, n0, "u") for t in u_steps[i]] + [(p_steps[i], n1, "p")] +
                 [(t, n1 if k == 3 else n0, "out[%d]" % k) for k, t in enumerate(out_steps[i])])
        for t, want, name in slots:
            if t.device.type != "cpu":
                raise ValueError(f"step {i} {name}: host (CPU) tensor expected, got {t.device}")
            if not t.is_contiguous():
                raise ValueError(f"step {i} {name}: tensor must be contiguous")
            if t.dtype != dtype:
                raise ValueError(f"step {i} {name}: dtype {t.dtype}, expected {dtype} like p_steps[0]")
            if t.numel() != want:
                raise ValueError(f"step {i} {name}: {t.numel()} elements, the layout has {want}")
    pu, _a = _ptrs([t for s in u_steps for t in s])
    pp, _b = _ptrs(list(p_steps))
    po, _c = _ptrs([t for s in out_steps for t in s])
    _check(lib().tn_operator_steps_host(mesh, _prec(p_steps[0].dtype), n, pu, pp, po, _stream(stream)))


def tn_prolong(mesh, level, coarse, fine, apply_bc=False, stream=None):
    pc, _a = _ptrs(coarse)
    pf, _b = _ptrs(fine)
    _check(lib().tn_prolong(mesh, level, _prec(coarse[0].dtype), len(coarse), int(apply_bc), pc, pf, _stream(stream)))


def tn_restrict(mesh, level, fine, coarse, apply_bc=False, stream=None):
    pf, _a = _ptrs(fine)
    pc, _b = _ptrs(coarse)
    _check(lib().tn_restrict(mesh, level, _prec(fine[0].dtype), len(fine), int(apply_bc), pf, pc, _stream(stream)))


def tn_buoyancy(mesh, T, Ra, f, stream=None):
    pf, _a = _ptrs(f)
    _check(lib().tn_buoyancy(mesh, _ptr(T), Ra, pf, _stream(stream)))


def tn_set_reference_state(mesh, rho=None, alpha=None):
    """TALA reference profiles at the level-0 node radii (host sequences of N_r values); rho=None
    restores the Boussinesq system."""
    import numpy as np
    if rho is None:
        _check(lib().tn_set_reference_state(mesh, None, None))
        return
    r = np.ascontiguousarray(rho, dtype=np.float64)
    a = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    n = tn_mesh_info(mesh, 0)["n_r"]
    if r.size != n or (a is not None and a.size != n):
        raise ValueError(f"reference profiles need {n} values (one per node layer)")
    _check(lib().tn_set_reference_state(mesh, r.ctypes.data_as(P), None if a is None else a.ctypes.data_as(P)))


def tn_energy_residual(mesh, T, u, R, supg=True, stream=None):
    pu, _a = _ptrs(u) if u is not None else (None, None)
    _check(lib().tn_energy_residual(mesh, _ptr(T), pu, int(bool(supg)), _ptr(R), _stream(stream)))


def tn_energy_steps(mesh, T, u, dt, n_steps, supg=True, stream=None):
    pu, _a = _ptrs(u) if u is not None else (None, None)
    _check(lib().tn_energy_steps(mesh, _ptr(T), pu, float(dt), int(n_steps), int(bool(supg)), _stream(stream)))


def tn_energy_diagnostics(mesh, T, u, stream=None):
    """(nu_top, v_rms)"""
    nu, vr = ctypes.c_double(), ctypes.c_double()
    pu, _a = _ptrs(u)
    _check(lib().tn_energy_diagnostics(mesh, _ptr(T), pu, ctypes.byref(nu), ctypes.byref(vr), _stream(stream)))
    return nu.value, vr.value


def tn_energy_stable_dt(mesh, stream=None):
    out = ctypes.c_double()
    _check(lib().tn_energy_stable_dt(mesh, ctypes.byref(out), _stream(stream)))
    return out.value


def tn_convection_default_opts(**kw):
    o = tn_convection_opts()
    _check(lib().tn_convection_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def tn_convection_steps(mesh, T, u, p, n_steps, opts=None, stream=None, check=True):
    """Returns the per-step stats as a list of dicts."""
    o = opts if opts is not None else tn_convection_default_opts()
    stats = (tn_convection_step_stats * max(1, n_steps))()
    pu, _a = _ptrs(u)
    status = lib().tn_convection_steps(mesh, _ptr(T), pu, _ptr(p), int(n_steps), ctypes.byref(o), stats,
                                       _stream(stream))
    if status != TN_OK and (check or status != TN_ENOTCONVERGED):
        _check(status)
    return [{f: getattr(stats[i], f) for f, _ in tn_convection_step_stats._fields_} for i in range(n_steps)]


def tn_mg_default_opts(**kw):
    o = tn_mg_opts()
    _check(lib().tn_mg_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def tn_mg_setup(mesh, dtype, opts=None, v0=None, stream=None):
    import torch
    prec = _prec(dtype if isinstance(dtype, torch.dtype) else torch.float64)
    o = opts if opts is not None else tn_mg_default_opts()
    if v0 is not None:
        pv, _a = _ptrs(v0)
    else:
        pv, _a = None, None
    _check(lib().tn_mg_setup(mesh, prec, ctypes.byref(o), pv, _stream(stream)))


def tn_mg_lambda(mesh, dtype, level):
    out = ctypes.c_double()
    _check(lib().tn_mg_lambda(mesh, _prec(dtype), level, ctypes.byref(out)))
    return out.value


def tn_vcycle(mesh, r, z, stream=None):
    pr, _a = _ptrs(r)
    pz, _b = _ptrs(z)
    _check(lib().tn_vcycle(mesh, _prec(r[0].dtype), pr, pz, _stream(stream)))


def tn_solve_default_opts(**kw):
    o = tn_solve_opts()
    _check(lib().tn_solve_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def tn_stokes_solve(mesh, f, g, u, p, opts=None, stream=None, check=True):
    """Returns the stats as a dict; raises on failure (TN_ENOTCONVERGED only if check)."""
    o = opts if opts is not None else tn_solve_default_opts()
    st = tn_solve_stats()
    pf, _a = _ptrs(f)
    pu, _b = _ptrs(u)
    status = lib().tn_stokes_solve(mesh, ctypes.byref(o), pf, _ptr(g), pu, _ptr(p), ctypes.byref(st), _stream(stream))
    if status != TN_OK and (check or status != TN_ENOTCONVERGED):
        _check(status)
    return {f: getattr(st, f) for f, _ in tn_solve_stats._fields_}


def tn_stokes_solve_batch(meshes, f, u, p, opts=None, stream=None):
    """Lockstep solve of len(meshes) systems; f[i], u[i]: 3 tensors, p[i]: one.  Returns a list of
    (status, stats dict) per system."""
    n = len(meshes)
    o = opts if opts is not None else tn_solve_default_opts()
    st = (tn_solve_stats * n)()
    status = (ctypes.c_int * n)()
    keep = []
    fa = (ctypes.c_void_p * n)()
    ua = (ctypes.c_void_p * n)()
    for i in range(n):
        pf, a = _ptrs(f[i])
        pu, b = _ptrs(u[i])
        keep += [a, b]
        fa[i] = ctypes.cast(pf, ctypes.c_void_p)
        ua[i] = ctypes.cast(pu, ctypes.c_void_p)
    ma = (ctypes.c_void_p * n)(*[ctypes.cast(m, ctypes.c_void_p) for m in meshes])
    pa = (ctypes.c_void_p * n)(*[t.data_ptr() for t in p])
    s = lib().tn_stokes_solve_batch(ctypes.cast(ma, PP), n, ctypes.byref(o), ctypes.cast(fa, PP), None,
                                    ctypes.cast(ua, PP), ctypes.cast(pa, PP), st, status, _stream(stream))
    if s == TN_EINVAL:
        _check(s)
    return [(status[i], {k: getattr(st[i], k) for k, _ in tn_solve_stats._fields_}) for i in range(n)]


def _result(r):
    return {f: getattr(r, f) for f, _ in tn_result._fields_}


def tn_server_default_opts(**kw):
    o = tn_server_opts()
    _check(lib().tn_server_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def tn_server_create(opts=None):
    o = opts if opts is not None else tn_server_default_opts()
    out = P()
    _check(lib().tn_server_create(ctypes.byref(o), ctypes.byref(out)))
    return out


def tn_server_submit(srv, lateral_level, radial_layers, E, Ra, t_degree, t_order, t_amplitude, r_in=0.55, r_out=1.0):
    req = tn_request(lateral_level, radial_layers, r_in, r_out, E, Ra, t_degree, t_order, t_amplitude)
    t = ctypes.c_uint64()
    _check(lib().tn_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def tn_server_poll(srv, ticket):
    """(done, result dict)"""
    r = tn_result()
    st = lib().tn_server_poll(srv, ticket, ctypes.byref(r))
    if st not in (TN_OK, TN_EBUSY):
        _check(st)
    return st == TN_OK, _result(r)


def tn_server_wait(srv, ticket):
    r = tn_result()
    _check(lib().tn_server_wait(srv, ticket, ctypes.byref(r)))
    return _result(r)


def tn_server_solution(srv, ticket, n_layout0, n_layout1):
    import numpy as np
    u = np.empty(3 * n_layout0)
    p = np.empty(n_layout1)
    _check(lib().tn_server_solution(srv, ticket, u.ctypes.data_as(P), p.ctypes.data_as(P)))
    return u.reshape(3, -1), p


def tn_server_stats(srv):
    q, r, res, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().tn_server_stats(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(res), ctypes.byref(b)))
    return {"queued": q.value, "running": r.value, "resident": res.value, "reserved_bytes": b.value}


def tn_server_cancel(srv, ticket):
    _check(lib().tn_server_cancel(srv, ticket))


def tn_probe_fma_peak(dtype, stream=None):
    """Measured FMA throughput (TFLOP/s) of the current device for torch.float64 / torch.float32."""
    out = ctypes.c_double()
    _check(lib().tn_probe_fma_peak(_prec(dtype), ctypes.byref(out), _stream(stream)))
    return out.value


def tn_server_destroy(srv):
    _check(lib().tn_server_destroy(srv))


def header_entry_points():
    """Names of the functions declared in include/terra_wedge.h."""
    import re
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:tn_status|const char\*)\s+(tn_\w+)\s*\(", src, flags=re.M)))
