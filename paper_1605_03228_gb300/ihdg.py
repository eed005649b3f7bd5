"""Python binding of libihdg (ctypes).  Argument marshalling only: every step of the iHDG
sweep runs in the library's CUDA kernels.  There is no CPU fallback; if the library or a
GPU is missing, the calls raise.

The names follow include/ihdg.h.  Arrays are numpy float64 (host calls) or raw device
pointers (the *_device calls), e.g. from torch tensors via tensor.data_ptr().
"""
import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, NOT_CONVERGED, DIVERGED, ERR_BUSY, ERR_TIMEOUT, ERR_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_NOMEM", 3: "ERR_CUDA", 4: "NOT_CONVERGED", 5: "DIVERGED",
                6: "ERR_BUSY", 7: "ERR_TIMEOUT", 8: "ERR_UNSUPPORTED"}
TRANSPORT, CONVDIFF, SWE = 0, 1, 2
FLUX_UPWIND, FLUX_NPC = 0, 1
KERNEL_AUTO, KERNEL_TENSOR_CORES, KERNEL_CUDA_CORES, KERNEL_GLOBAL = 0, 1, 2, 3
BACKWARD_EULER, CRANK_NICOLSON = 0, 1
# Result.inner_kernel_used: the kernel that ran a mixed solve's inner sweeps
INNER_KERNEL_NAMES = {0: None, 1: "k_inner_tc", 2: "k_inner_blk", 3: "k_inner_reg", 4: "k_inner_tile",
                      5: "k_inner_persist", 6: "k_inner_tcs"}
FP64, MIXED_FP32, MIXED_TF32, MIXED_BF16 = 0, 1, 2, 3


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("p", ctypes.c_int)]


class Coeffs(ctypes.Structure):
    _fields_ = [("pde", ctypes.c_int), ("beta", ctypes.c_double * 3), ("kappa", ctypes.c_double),
                ("nu", ctypes.c_double), ("Phi", ctypes.c_double), ("coriolis_f", ctypes.c_double),
                ("friction", ctypes.c_double), ("dt", ctypes.c_double), ("flux", ctypes.c_int),
                ("tau_gamma", ctypes.c_double), ("time_scheme", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int), ("prec", ctypes.c_int),
                ("diverge_factor", ctypes.c_double), ("inner_max", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("u0", ctypes.c_void_p), ("profile", ctypes.c_int),
                ("inner_kernel", ctypes.c_int), ("sweeps_per_sync", ctypes.c_int), ("tile_shape", ctypes.c_int),
                ("krylov_restart", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("fp64_sweeps", ctypes.c_int), ("lowp_sweeps", ctypes.c_int),
                ("residual", ctypes.c_double), ("status", ctypes.c_int), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("fp64_sweep_ms", ctypes.c_double), ("lowp_sweep_ms", ctypes.c_double),
                ("fp64_launches", ctypes.c_int), ("lowp_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("inner_kernel_used", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Sizes(ctypes.Structure):
    _fields_ = [("n_el", ctypes.c_longlong), ("nvol", ctypes.c_int), ("ncomp", ctypes.c_int), ("nqv", ctypes.c_int),
                ("n_bface", ctypes.c_longlong), ("nqf", ctypes.c_int), ("n_face", ctypes.c_longlong),
                ("nface_nodes", ctypes.c_int), ("n_exp", ctypes.c_int), ("n_in", ctypes.c_int)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("l2_read_gbs", ctypes.c_double), ("sms", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = ["ihdg_create", "ihdg_destroy", "ihdg_last_error", "ihdg_problem_sizes", "ihdg_quadrature_points",
            "ihdg_node_points", "ihdg_solve", "ihdg_workspace_bytes", "ihdg_solve_device", "ihdg_swe_steps",
            "ihdg_swe_steps_device", "ihdg_host_operator", "ihdg_solve_device_static", "ihdg_server_start",
            "ihdg_server_stop", "ihdg_submit", "ihdg_poll", "ihdg_fetch", "ihdg_autotune", "ihdg_measure_peaks",
            "ihdg_face_quadrature_points", "ihdg_var_plan_create", "ihdg_var_plan_destroy", "ihdg_var_plan_info",
            "ihdg_var_solve", "ihdg_var_solve_device", "ihdg_var_host_operator", "ihdg_var_solve_group",
            "ihdg_group_workspace_bytes", "ihdg_solve_group_device", "ihdg_abi_sizes"]
STATIC_SCRATCH_BYTES = 64 * 1024 * 1024

_lib = None


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libihdg.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libihdg.so is not built; run paper_1605_03228_gb300/build.py")
    L = ctypes.CDLL(_build.LIB)
    P, VP, I, D, SZ = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    dp = P(ctypes.c_double)
    L.ihdg_create.argtypes = [P(VP), I]
    L.ihdg_destroy.argtypes = [VP]
    L.ihdg_destroy.restype = None
    L.ihdg_last_error.argtypes = [VP]
    L.ihdg_last_error.restype = ctypes.c_char_p
    L.ihdg_problem_sizes.argtypes = [P(Mesh), P(Coeffs), P(Sizes)]
    L.ihdg_abi_sizes.argtypes = [P(ctypes.c_size_t), I]
    L.ihdg_quadrature_points.argtypes = [P(Mesh), dp, dp]
    L.ihdg_node_points.argtypes = [P(Mesh), dp]
    L.ihdg_solve.argtypes = [VP, P(Mesh), P(Coeffs), dp, dp, P(Options), dp, dp, P(Result)]
    L.ihdg_workspace_bytes.argtypes = [P(Mesh), P(Coeffs), P(Options), P(SZ)]
    L.ihdg_solve_device.argtypes = [VP, P(Mesh), P(Coeffs), VP, VP, P(Options), VP, VP, VP, SZ, VP, P(Result)]
    L.ihdg_swe_steps.argtypes = [VP, P(Mesh), P(Coeffs), dp, I, P(Options), P(I), P(Result)]
    L.ihdg_swe_steps_device.argtypes = [VP, P(Mesh), P(Coeffs), VP, I, P(Options), P(I), VP, SZ, VP, P(Result)]
    L.ihdg_host_operator.argtypes = [P(Mesh), P(Coeffs), I, P(I), P(I), dp]
    L.ihdg_solve_device_static.argtypes = [VP, P(Mesh), P(Coeffs), VP, VP, P(Options), VP, VP, VP, P(Result)]
    L.ihdg_autotune.argtypes = [VP, P(Mesh), P(Coeffs), dp, dp, P(Options), P(Options), dp]
    L.ihdg_server_start.argtypes = [VP, SZ, I]
    L.ihdg_server_stop.argtypes = [VP]
    L.ihdg_submit.argtypes = [VP, P(Mesh), P(Coeffs), dp, dp, P(Options), P(ctypes.c_longlong)]
    L.ihdg_poll.argtypes = [VP, ctypes.c_longlong, P(Result)]
    L.ihdg_fetch.argtypes = [VP, ctypes.c_longlong, dp, dp]
    L.ihdg_measure_peaks.argtypes = [I, P(Peaks)]
    L.ihdg_face_quadrature_points.argtypes = [P(Mesh), dp]
    L.ihdg_var_plan_create.argtypes = [VP, P(Mesh), dp, dp, P(VP)]
    L.ihdg_var_plan_destroy.argtypes = [VP]
    L.ihdg_var_plan_info.argtypes = [VP, P(SZ), dp]
    L.ihdg_var_solve.argtypes = [VP, VP, dp, dp, P(Options), dp, dp, P(Result)]
    L.ihdg_var_solve_device.argtypes = [VP, VP, VP, VP, P(Options), VP, VP, VP, P(Result)]
    L.ihdg_var_host_operator.argtypes = [P(Mesh), dp, dp, ctypes.c_longlong, I, P(I), P(I), dp]
    L.ihdg_var_solve_group.argtypes = [VP, I, P(VP), P(VP), P(VP), P(Options), P(VP), P(VP), VP, P(Result)]
    for name in EXPORTED:
        f = getattr(L, name)
        if name not in ("ihdg_destroy", "ihdg_last_error", "ihdg_var_plan_destroy"):
            f.restype = ctypes.c_int
    L.ihdg_var_plan_destroy.restype = None
    _lib = L
    return L


def make_mesh(dim, n, p, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    m = Mesh()
    m.dim = dim
    for a in range(3):
        m.n[a] = int(n[a]) if a < len(n) else 1
        m.lo[a] = float(lo[a]) if a < len(lo) else 0.0
        m.hi[a] = float(hi[a]) if a < len(hi) else 1.0
    m.p = p
    return m


def make_coeffs(pde, beta=(0.0, 0.0, 0.0), kappa=0.0, nu=0.0, Phi=0.0, coriolis_f=0.0, friction=0.0, dt=0.0,
                flux=0, tau_gamma=0.0, time_scheme=0):
    c = Coeffs()
    c.pde = pde
    c.time_scheme = time_scheme
    c.flux = flux
    c.tau_gamma = tau_gamma
    for a in range(3):
        c.beta[a] = float(beta[a]) if a < len(beta) else 0.0
    c.kappa, c.nu, c.Phi, c.coriolis_f, c.friction, c.dt = kappa, nu, Phi, coriolis_f, friction, dt
    return c


def make_options(tol, max_iters=2000, prec=FP64, diverge_factor=0.0, inner_max=0, inner_rtol=0.0, u0=None,
                 profile=0, inner_kernel=0, sweeps_per_sync=0, tile_shape=0, krylov_restart=0):
    o = Options()
    o.krylov_restart = krylov_restart
    o.tile_shape = tile_shape
    o.inner_kernel = inner_kernel
    o.sweeps_per_sync = sweeps_per_sync
    o.tol, o.max_iters, o.prec, o.diverge_factor = tol, max_iters, prec, diverge_factor
    o.inner_max, o.inner_rtol = inner_max, inner_rtol
    o.u0 = u0
    o.profile = profile
    return o


def measure_peaks(device=0):
    """ihdg_measure_peaks: float64 / float32 FMA rates (TFLOP/s) and L2 read bandwidth (GB/s)."""
    L = load()
    pk = Peaks()
    st = L.ihdg_measure_peaks(int(device), ctypes.byref(pk))
    if st != OK:
        raise IHDGError(st, "ihdg_measure_peaks failed")
    return pk


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


class IHDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def problem_sizes(mesh, coeffs):
    L = load()
    s = Sizes()
    st = L.ihdg_problem_sizes(ctypes.byref(mesh), ctypes.byref(coeffs), ctypes.byref(s))
    if st != OK:
        raise IHDGError(st, "ihdg_problem_sizes")
    return s


def quadrature_points(mesh, coeffs):
    s = problem_sizes(mesh, coeffs)
    L = load()
    q = (mesh.p + 2)
    nqv, nqf = q ** mesh.dim, q ** (mesh.dim - 1)
    vol = np.zeros((s.n_el, nqv, mesh.dim))
    bnd = np.zeros((s.n_bface, nqf, mesh.dim))
    st = L.ihdg_quadrature_points(ctypes.byref(mesh), _dptr(vol), _dptr(bnd))
    if st != OK:
        raise IHDGError(st, "ihdg_quadrature_points")
    return vol, bnd


def face_quadrature_points(mesh):
    """Gauss points of every global face, (n_face, q^(dim-1), dim), global face order."""
    L = load()
    co = make_coeffs(TRANSPORT, beta=(1.0, 0.0, 0.0))
    s = problem_sizes(mesh, co)
    nqf = (mesh.p + 2) ** (mesh.dim - 1)
    xyz = np.zeros((s.n_face, nqf, mesh.dim))
    st = L.ihdg_face_quadrature_points(ctypes.byref(mesh), _dptr(xyz))
    if st != OK:
        raise IHDGError(st, "ihdg_face_quadrature_points")
    return xyz


def var_host_operator(mesh, beta_vol, beta_face, element, which):
    """ihdg_var_host_operator: one element's L_K (which 0) or A_K^{-1} (which 1), host float64."""
    L = load()
    bv = np.ascontiguousarray(beta_vol, dtype=np.float64)
    bf = np.ascontiguousarray(beta_face, dtype=np.float64)
    r, c = ctypes.c_int(0), ctypes.c_int(0)
    st = L.ihdg_var_host_operator(ctypes.byref(mesh), _dptr(bv), _dptr(bf), int(element), int(which), ctypes.byref(r),
                                  ctypes.byref(c), None)
    if st != OK:
        raise IHDGError(st, "ihdg_var_host_operator")
    out = np.zeros((r.value, c.value))
    st = L.ihdg_var_host_operator(ctypes.byref(mesh), _dptr(bv), _dptr(bf), int(element), int(which), ctypes.byref(r),
                                  ctypes.byref(c), _dptr(out))
    if st != OK:
        raise IHDGError(st, "ihdg_var_host_operator")
    return out


def node_points(mesh, coeffs):
    s = problem_sizes(mesh, coeffs)
    L = load()
    nb = (mesh.p + 1) ** mesh.dim
    xyz = np.zeros((s.n_el, nb, mesh.dim))
    st = L.ihdg_node_points(ctypes.byref(mesh), _dptr(xyz))
    if st != OK:
        raise IHDGError(st, "ihdg_node_points")
    return xyz


def host_operator(mesh, coeffs, which):
    """Float64 operator of the library's host precompute: 0 L_E, 1 Q, 2 L_vol, 3 R, 4 PF, 5 PV."""
    L = load()
    r, c = ctypes.c_int(), ctypes.c_int()
    st = L.ihdg_host_operator(ctypes.byref(mesh), ctypes.byref(coeffs), which, ctypes.byref(r), ctypes.byref(c), None)
    if st != OK:
        raise IHDGError(st, "ihdg_host_operator")
    out = np.zeros((r.value, c.value))
    L.ihdg_host_operator(ctypes.byref(mesh), ctypes.byref(coeffs), which, ctypes.byref(r), ctypes.byref(c), _dptr(out))
    return out


def workspace_bytes(mesh, coeffs, opts):
    L = load()
    n = ctypes.c_size_t()
    st = L.ihdg_workspace_bytes(ctypes.byref(mesh), ctypes.byref(coeffs), ctypes.byref(opts), ctypes.byref(n))
    if st != OK:
        raise IHDGError(st, "ihdg_workspace_bytes")
    return n.value


class Context:
    """An ihdg_ctx bound to one CUDA device."""

    def __init__(self, device=0):
        self.L = load()
        self.h = ctypes.c_void_p()
        st = self.L.ihdg_create(ctypes.byref(self.h), device)
        if st != OK:
            raise IHDGError(st, f"ihdg_create(device={device}) failed: no usable sm_103 GPU")

    def close(self):
        if self.h:
            self.L.ihdg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self):
        return self.L.ihdg_last_error(self.h).decode()

    def _check(self, st, name, allow_nonconverged=True):
        if st != OK:
            raise IHDGError(st, f"{name}: {self.last_error()}")

    def solve(self, mesh, coeffs, f_qp, g_qp, opts, want_trace=True, u_out=None, trace_out=None):
        """Host-buffer solve.  Returns (u [n_el, nvol], trace or None, Result).  u_out and
        trace_out, when given, are C-contiguous float64 host arrays of those shapes (e.g.
        views of pinned memory) that receive the results."""
        s = problem_sizes(mesh, coeffs)
        f = np.ascontiguousarray(f_qp, dtype=np.float64)
        g = np.ascontiguousarray(g_qp, dtype=np.float64)
        u = u_out if u_out is not None else np.zeros((s.n_el, s.nvol))
        tr = trace_out if trace_out is not None else (np.zeros((s.n_face, s.nface_nodes)) if want_trace else None)
        assert u.shape == (s.n_el, s.nvol) and u.dtype == np.float64 and u.flags.c_contiguous
        assert tr is None or (tr.shape == (s.n_face, s.nface_nodes) and tr.dtype == np.float64 and tr.flags.c_contiguous)
        res = Result()
        st = self.L.ihdg_solve(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), _dptr(f), _dptr(g),
                               ctypes.byref(opts), _dptr(u), _dptr(tr), ctypes.byref(res))
        self._check(st, "ihdg_solve")
        return u, tr, res

    def autotune(self, mesh, coeffs, f_qp, g_qp, opts):
        """ihdg_autotune: returns (tuned Options, device time of the fastest solve in ms)."""
        f = np.ascontiguousarray(f_qp, dtype=np.float64)
        g = np.ascontiguousarray(g_qp, dtype=np.float64)
        tuned = Options()
        best = ctypes.c_double(0.0)
        st = self.L.ihdg_autotune(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), _dptr(f), _dptr(g),
                                  ctypes.byref(opts), ctypes.byref(tuned), ctypes.byref(best))
        self._check(st, "ihdg_autotune")
        return tuned, best.value

    def solve_device(self, mesh, coeffs, d_f, d_g, opts, d_u, d_tr, d_ws, ws_bytes, stream=0):
        """Device-pointer solve (integer pointers).  Returns Result."""
        res = Result()
        st = self.L.ihdg_solve_device(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), ctypes.c_void_p(d_f),
                                      ctypes.c_void_p(d_g), ctypes.byref(opts), ctypes.c_void_p(d_u),
                                      ctypes.c_void_p(d_tr) if d_tr else None, ctypes.c_void_p(d_ws),
                                      ctypes.c_size_t(ws_bytes), ctypes.c_void_p(stream), ctypes.byref(res))
        self._check(st, "ihdg_solve_device")
        return res

    def solve_device_static(self, mesh, coeffs, d_f, d_g, opts, d_u, d_tr, stream=0):
        """Device-pointer solve that allocates nothing (scratch in the library's static
        device array, see ihdg_solve_device_static).  Returns Result."""
        res = Result()
        st = self.L.ihdg_solve_device_static(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), ctypes.c_void_p(d_f),
                                             ctypes.c_void_p(d_g), ctypes.byref(opts), ctypes.c_void_p(d_u),
                                             ctypes.c_void_p(d_tr) if d_tr else None, ctypes.c_void_p(stream),
                                             ctypes.byref(res))
        self._check(st, "ihdg_solve_device_static")
        return res

    # ---------------------------------------------------------------- variable beta
    def var_plan(self, mesh, beta_vol, beta_face):
        """ihdg_var_plan_create: per-element local solves of transport with a velocity field
        sampled at the volume and face quadrature points.  Returns a VarPlan."""
        bv = np.ascontiguousarray(beta_vol, dtype=np.float64)
        bf = np.ascontiguousarray(beta_face, dtype=np.float64)
        h = ctypes.c_void_p()
        st = self.L.ihdg_var_plan_create(self.h, ctypes.byref(mesh), _dptr(bv), _dptr(bf), ctypes.byref(h))
        self._check(st, "ihdg_var_plan_create")
        return VarPlan(self, mesh, h)

    def var_solve_group(self, plans, d_f, d_g, opts, d_u, d_tr=None, stream=0):
        """ihdg_var_solve_group: device-pointer solves of several plans together (integer
        pointers, one per plan).  Returns a list of Result."""
        n = len(plans)
        arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(int(x) if x else 0) for x in xs])
        res = (Result * n)()
        pl = (ctypes.c_void_p * n)(*[p.h for p in plans])
        st = self.L.ihdg_var_solve_group(self.h, n, pl, arr(d_f), arr(d_g), ctypes.byref(opts), arr(d_u),
                                         arr(d_tr) if d_tr is not None else None, ctypes.c_void_p(stream), res)
        self._check(st, "ihdg_var_solve_group")
        return list(res)

    def group_workspace_bytes(self, meshes, coeffs, opts):
        """ihdg_group_workspace_bytes for the problems (meshes[i], coeffs[i])."""
        n = len(meshes)
        ms = (Mesh * n)(*meshes)
        cs = (Coeffs * n)(*coeffs)
        b = ctypes.c_size_t()
        self._check(self.L.ihdg_group_workspace_bytes(n, ms, cs, ctypes.byref(opts), ctypes.byref(b)),
                    "ihdg_group_workspace_bytes")
        return b.value

    def solve_group_device(self, meshes, coeffs, d_f, d_g, opts, d_u, d_tr, d_ws, ws_bytes, stream=0):
        """ihdg_solve_group_device: float64 solves of several problems together (integer device
        pointers, one per problem; d_tr None or a list with 0 for no trace).  Returns a list of
        Result."""
        n = len(meshes)
        arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(int(x) if x else 0) for x in xs])
        ms = (Mesh * n)(*meshes)
        cs = (Coeffs * n)(*coeffs)
        res = (Result * n)()
        st = self.L.ihdg_solve_group_device(self.h, n, ms, cs, arr(d_f), arr(d_g), ctypes.byref(opts), arr(d_u),
                                            arr(d_tr) if d_tr is not None else None, ctypes.c_void_p(d_ws),
                                            ctypes.c_size_t(ws_bytes), ctypes.c_void_p(stream), res)
        self._check(st, "ihdg_solve_group_device")
        return list(res)

    # ---------------------------------------------------------------- serving
    def server_start(self, hbm_budget_bytes, slots):
        self._check(self.L.ihdg_server_start(self.h, ctypes.c_size_t(hbm_budget_bytes), slots), "ihdg_server_start")

    def server_stop(self):
        self._check(self.L.ihdg_server_stop(self.h), "ihdg_server_stop")

    def submit(self, mesh, coeffs, f_qp, g_qp, opts):
        f = np.ascontiguousarray(f_qp, dtype=np.float64)
        g = np.ascontiguousarray(g_qp, dtype=np.float64)
        t = ctypes.c_longlong()
        st = self.L.ihdg_submit(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), _dptr(f), _dptr(g),
                                ctypes.byref(opts), ctypes.byref(t))
        self._check(st, "ihdg_submit")
        return t.value

    def poll(self, ticket):
        """Result when done, None while busy."""
        res = Result()
        st = self.L.ihdg_poll(self.h, ctypes.c_longlong(ticket), ctypes.byref(res))
        if st == ERR_BUSY:
            return None
        self._check(st, "ihdg_poll")
        return res

    def fetch(self, ticket, mesh, coeffs, want_trace=True):
        s = problem_sizes(mesh, coeffs)
        u = np.zeros((s.n_el, s.nvol))
        tr = np.zeros((s.n_face, s.nface_nodes)) if want_trace else None
        st = self.L.ihdg_fetch(self.h, ctypes.c_longlong(ticket), _dptr(u), _dptr(tr))
        self._check(st, "ihdg_fetch")
        return u, tr

    def swe_steps(self, mesh, coeffs, q, nsteps, opts):
        """Host-buffer shallow-water stepping; q is updated in place.  Returns (iters, Result)."""
        qq = np.ascontiguousarray(q, dtype=np.float64)
        its = (ctypes.c_int * max(nsteps, 1))()
        res = Result()
        st = self.L.ihdg_swe_steps(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), _dptr(qq), nsteps,
                                   ctypes.byref(opts), its, ctypes.byref(res))
        self._check(st, "ihdg_swe_steps")
        q[...] = qq
        return list(its)[:nsteps], res

    def swe_steps_device(self, mesh, coeffs, d_q, nsteps, opts, d_ws, ws_bytes, stream=0):
        its = (ctypes.c_int * max(nsteps, 1))()
        res = Result()
        st = self.L.ihdg_swe_steps_device(self.h, ctypes.byref(mesh), ctypes.byref(coeffs), ctypes.c_void_p(d_q),
                                          nsteps, ctypes.byref(opts), its, ctypes.c_void_p(d_ws),
                                          ctypes.c_size_t(ws_bytes), ctypes.c_void_p(stream), ctypes.byref(res))
        self._check(st, "ihdg_swe_steps_device")
        return list(its)[:nsteps], res


class VarPlan:
    """An ihdg_var_plan: the per-element local solves of one velocity field on one device."""

    def __init__(self, ctx, mesh, h):
        self.ctx, self.mesh, self.h = ctx, mesh, h
        co = make_coeffs(TRANSPORT, beta=(1.0, 0.0, 0.0))
        self.sizes = problem_sizes(mesh, co)

    def close(self):
        if self.h:
            self.ctx.L.ihdg_var_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """(device bytes, host set-up time in ms)."""
        b = ctypes.c_size_t(0)
        ms = ctypes.c_double(0.0)
        self.ctx._check(self.ctx.L.ihdg_var_plan_info(self.h, ctypes.byref(b), ctypes.byref(ms)), "ihdg_var_plan_info")
        return b.value, ms.value

    def solve(self, f_qp, g_qp, opts, want_trace=True):
        """Host-buffer solve: (u [n_el, (p+1)^dim], trace or None, Result)."""
        s = self.sizes
        f = np.ascontiguousarray(f_qp, dtype=np.float64)
        g = np.ascontiguousarray(g_qp, dtype=np.float64)
        u = np.zeros((s.n_el, (self.mesh.p + 1) ** self.mesh.dim))
        tr = np.zeros((s.n_face, s.nface_nodes)) if want_trace else None
        res = Result()
        st = self.ctx.L.ihdg_var_solve(self.ctx.h, self.h, _dptr(f), _dptr(g), ctypes.byref(opts), _dptr(u),
                                       _dptr(tr), ctypes.byref(res))
        self.ctx._check(st, "ihdg_var_solve")
        return u, tr, res

    def solve_device(self, d_f, d_g, opts, d_u, d_tr=0, stream=0):
        """Device-pointer solve (integer pointers).  Returns Result."""
        res = Result()
        st = self.ctx.L.ihdg_var_solve_device(self.ctx.h, self.h, ctypes.c_void_p(d_f), ctypes.c_void_p(d_g),
                                              ctypes.byref(opts), ctypes.c_void_p(d_u),
                                              ctypes.c_void_p(d_tr) if d_tr else None, ctypes.c_void_p(stream),
                                              ctypes.byref(res))
        self.ctx._check(st, "ihdg_var_solve_device")
        return res
