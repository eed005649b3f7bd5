"""CPU tests of libihdg's host side: the library loads and exports every symbol the header
declares; geometry queries agree with the oracle's own point generators; argument checks;
and the library's float64 operators (built independently of the oracle) reproduce one
oracle sweep when applied on the CPU in the export form.  No compute call needs a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import BoxMesh, ConvDiff, Discretisation, ShallowWater, Transport
from paper_1605_03228_gb300 import ihdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ihdg.h")).read()
    return sorted(set(re.findall(r"\b(ihdg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = ihdg.load()
    syms = header_symbols()
    assert len(syms) >= 11
    for s in syms:
        assert hasattr(L, s), s


def test_create_without_gpu_fails_cleanly():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(ihdg.IHDGError) as e:
        ihdg.Context(0)
    assert e.value.status == ihdg.ERR_CUDA


@pytest.mark.parametrize("dim,n,p", [(2, (3, 2), 2), (3, (2, 3, 2), 1)])
def test_points_match_oracle(dim, n, p):
    mesh = ihdg.make_mesh(dim, n, p, lo=(0.1, -0.2, 0.3), hi=(1.3, 0.7, 0.9))
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.5, 0.3))
    vol, bnd = ihdg.quadrature_points(mesh, co)
    nodes = ihdg.node_points(mesh, co)
    om = BoxMesh(dim, n, lo=[0.1, -0.2, 0.3][:dim], hi=[1.3, 0.7, 0.9][:dim])
    disc = Discretisation(om, p)
    assert np.abs(vol - disc.volume_points()).max() < 1e-14
    assert np.abs(bnd - disc.boundary_points()).max() < 1e-14
    assert np.abs(nodes - disc.node_points()).max() < 1e-14


def test_sizes():
    mesh = ihdg.make_mesh(2, (256, 256), 3)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=1e-2)
    s = ihdg.problem_sizes(mesh, co)
    assert (s.n_el, s.nvol, s.ncomp, s.nqv, s.nqf) == (65536, 48, 3, 25, 5)
    assert s.n_face == 2 * 257 * 256 and s.n_bface == 4 * 256
    assert (s.n_exp, s.n_in, s.nface_nodes) == (16, 16, 4)


def test_invalid_arguments_rejected():
    L = ihdg.load()
    s = ihdg.Sizes()
    bad = [
        (ihdg.make_mesh(4, (2, 2), 2), ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1))),
        (ihdg.make_mesh(2, (0, 2), 2), ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1))),
        (ihdg.make_mesh(2, (2, 2), 2, hi=(0.0, 1.0)), ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1))),
        (ihdg.make_mesh(2, (2, 2), 2), ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=0.0)),
        (ihdg.make_mesh(2, (2, 2), 2), ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.0)),
        (ihdg.make_mesh(2, (2, 2), 2), ihdg.make_coeffs(ihdg.TRANSPORT, beta=(0, 0))),
    ]
    for m, c in bad:
        assert L.ihdg_problem_sizes(ctypes.byref(m), ctypes.byref(c), ctypes.byref(s)) == ihdg.ERR_INVALID
    m3 = ihdg.make_mesh(3, (2, 2, 2), 2)
    c3 = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.1)
    assert L.ihdg_problem_sizes(ctypes.byref(m3), ctypes.byref(c3), ctypes.byref(s)) == ihdg.ERR_UNSUPPORTED
    bad_flux = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1), flux=7)
    m2 = ihdg.make_mesh(2, (2, 2), 2)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(bad_flux), ctypes.byref(s)) == ihdg.ERR_INVALID
    bad_tau = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=0.1, tau_gamma=-1.0)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(bad_tau), ctypes.byref(s)) == ihdg.ERR_INVALID
    tau_tr = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1), tau_gamma=1.0)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(tau_tr), ctypes.byref(s)) == ihdg.ERR_UNSUPPORTED
    npc_cd = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=0.1, flux=ihdg.FLUX_NPC)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(npc_cd), ctypes.byref(s)) == ihdg.ERR_UNSUPPORTED
    cn_tr = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1), time_scheme=ihdg.CRANK_NICOLSON)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(cn_tr), ctypes.byref(s)) == ihdg.ERR_UNSUPPORTED
    bad_ts = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.01, time_scheme=7)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(bad_ts), ctypes.byref(s)) == ihdg.ERR_INVALID
    cn_swe = ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.01, time_scheme=ihdg.CRANK_NICOLSON)
    assert L.ihdg_problem_sizes(ctypes.byref(m2), ctypes.byref(cn_swe), ctypes.byref(s)) == ihdg.OK
    m = ihdg.make_mesh(2, (2, 2), 5)
    c = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1))
    assert L.ihdg_problem_sizes(ctypes.byref(m), ctypes.byref(c), ctypes.byref(s)) == ihdg.ERR_UNSUPPORTED
    assert L.ihdg_problem_sizes(None, ctypes.byref(c), ctypes.byref(s)) == ihdg.ERR_INVALID


# ---------------------------------------------------------------- export-form sweep on the CPU
def export_gather(E, om, kinds, own_off, nbr_off, nf, mirror):
    """Trace inputs t (nel, 2d*nf) from exports E (nel, n_exp), as the sweep's step a1."""
    nel, d = om.nel, om.d
    t = np.zeros((nel, 2 * d * nf))
    for K in range(nel):
        for f in range(2 * d):
            nb = om.nbr[K, f]
            for j in range(nf):
                s = f * nf + j
                if kinds[f] == "own":
                    t[K, s] = E[K, own_off[f] + j]
                elif kinds[f] == "nbr":
                    t[K, s] = E[nb, nbr_off[f] + j] if nb >= 0 else 0.0
                elif kinds[f] == "sum":
                    o = E[K, own_off[f] + j]
                    t[K, s] = o + E[nb, nbr_off[f] + j] if nb >= 0 else (2 * o if mirror else 0.0)
    return t


def check_one_sweep(mesh, co, problem, kinds, own_off, nbr_off, mirror, U_prev=None):
    Lvol = ihdg.host_operator(mesh, co, 2)
    R = ihdg.host_operator(mesh, co, 3)
    LE = ihdg.host_operator(mesh, co, 0)
    Q = ihdg.host_operator(mesh, co, 1)
    assert np.abs(LE - R @ Lvol).max() < 1e-12 * max(1, np.abs(LE).max())
    om, disc = problem.mesh, problem.disc
    rng = np.random.default_rng(3)
    U = rng.standard_normal((om.nel, problem.nc, disc.nb))
    E = U.reshape(om.nel, -1) @ R.T
    t = export_gather(E, om, kinds, own_off, nbr_off, disc.ref.nb1 ** (om.d - 1), mirror)
    u_lib = t @ Lvol.T
    if problem.__class__ is ShallowWater:
        zero = np.zeros_like(U)
        u_or = problem.sweep(U, None, None, U_prev=zero)
    else:
        f = np.zeros((om.nel, disc.nq))
        g = np.zeros((om.nbface, disc.nqf))
        u_or = problem.sweep(U, f, g)
    assert np.abs(u_lib - u_or.reshape(om.nel, -1)).max() < 1e-11 * max(1.0, np.abs(u_or).max())
    # the stopping-norm operator: ||L_vol dt||^2 in the problem's norm equals dt^T Q dt
    dt = rng.standard_normal((om.nel, Lvol.shape[1]))
    du = (dt @ Lvol.T).reshape(om.nel, problem.nc, disc.nb)
    assert abs(np.einsum("ki,ij,kj->", dt, Q, dt) - problem.norm2(du)) < 1e-10 * problem.norm2(du)


@pytest.mark.parametrize("p,flux", [(1, "upwind"), (3, "upwind"), (2, "npc"), (3, "npc")])
def test_export_form_matches_oracle_transport(p, flux):
    beta = (1.0, 0.5)
    mesh = ihdg.make_mesh(2, (3, 3), p)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=beta, flux=ihdg.FLUX_NPC if flux == "npc" else ihdg.FLUX_UPWIND)
    om = BoxMesh(2, (3, 3))
    pr = Transport(Discretisation(om, p), np.array(beta), flux=flux)
    nf = p + 1
    kinds = ["nbr", "own", "nbr", "own"]          # beta > 0: -x, -y inflow; +x, +y outflow
    own_off = [(f // 2) * nf for f in range(4)]   # export slot = axis * nf + node
    nbr_off = [(f // 2) * nf for f in range(4)]
    check_one_sweep(mesh, co, pr, kinds, own_off, nbr_off, False)
    # forcing part: u^1 from u^0 = 0 with g = 0 is PV f
    PV = ihdg.host_operator(mesh, co, 5)
    f = np.random.default_rng(1).standard_normal((om.nel, pr.disc.nq))
    u1 = pr.sweep(np.zeros((om.nel, 1, pr.disc.nb)), f, np.zeros((om.nbface, pr.disc.nqf)))
    assert np.abs(f @ PV.T - u1.reshape(om.nel, -1)).max() < 1e-12


@pytest.mark.parametrize("p,gamma", [(1, 0.0), (3, 0.0), (2, 1.0), (3, 0.5)])
def test_export_form_matches_oracle_convdiff(p, gamma):
    beta, kappa, nu = (1.0, -0.7), 0.05, 0.3
    mesh = ihdg.make_mesh(2, (3, 3), p)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa, nu=nu, tau_gamma=gamma)
    om = BoxMesh(2, (3, 3))
    pr = ConvDiff(Discretisation(om, p), np.array(beta), kappa, nu, tau_gamma=gamma or None)
    nf = p + 1
    kinds = ["sum"] * 4
    own_off = [f * nf for f in range(4)]
    nbr_off = [(f ^ 1) * nf for f in range(4)]
    check_one_sweep(mesh, co, pr, kinds, own_off, nbr_off, False)


def test_export_form_matches_oracle_convdiff_3d():
    beta, kappa = (0.6, -0.4, 0.7), 0.1
    mesh = ihdg.make_mesh(3, (2, 2, 2), 1)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=beta, kappa=kappa)
    om = BoxMesh(3, (2, 2, 2))
    pr = ConvDiff(Discretisation(om, 1), np.array(beta), kappa, 0.0)
    nf = 4
    check_one_sweep(mesh, co, pr, ["sum"] * 6, [f * nf for f in range(6)], [(f ^ 1) * nf for f in range(6)], False)


@pytest.mark.parametrize("p", [1, 2])
def test_export_form_matches_oracle_swe(p):
    mesh = ihdg.make_mesh(2, (3, 3), p)
    co = ihdg.make_coeffs(ihdg.SWE, Phi=1.5, dt=0.01, coriolis_f=0.3, friction=0.1)
    om = BoxMesh(2, (3, 3))
    pr = ShallowWater(Discretisation(om, p), 1.5, 0.01, 0.3, 0.1)
    nf = p + 1
    check_one_sweep(mesh, co, pr, ["sum"] * 4, [f * nf for f in range(4)], [(f ^ 1) * nf for f in range(4)], True)


# ------------------------------------------------------------------ variable beta (host)
def _var_case(d, field):
    from oracle.refelem import lagrange_matrix
    if d == 2:
        n, p = (4, 3), 3
        mesh = ihdg.make_mesh(2, n, p, hi=(2.0, 2.0))
        om = BoxMesh(2, n, lo=[0, 0], hi=[2, 2])
    else:
        n, p = (2, 3, 2), 2
        mesh = ihdg.make_mesh(3, n, p)
        om = BoxMesh(3, n)
    return mesh, om, p, field


@pytest.mark.parametrize("d,field", [(2, "e1"), (2, "neg"), (2, "zero_y"), (3, "e2")])
def test_var_operators_match_oracle(d, field):
    """The plan's per-element local solve, built on the host from beta sampled at the library's
    quadrature points, against the oracle's (TransportVar, its own tables): A_K^{-1} and
    L_K = A_K^{-1} G_K, where the oracle's face-point coupling W_Kf times the face nodal basis
    at the face Gauss points is G_K's block of face f (outflow and inflow faces; faces with
    beta.n = 0 couple nothing)."""
    import workloads as W
    from oracle import Discretisation, TransportVar
    from oracle.refelem import lagrange_matrix
    fields = {"e1": W.e1_beta, "e2": W.e2_beta,
              "neg": lambda X: np.stack([-(1.0 + 0.3 * np.sin(X[..., 1])), -0.5 - 0.2 * X[..., 0]], axis=-1),
              "zero_y": lambda X: np.stack([1.0 + 0.5 * X[..., 1], 0.0 * X[..., 0]], axis=-1)}
    mesh, om, p, _ = _var_case(d, field)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, _ = ihdg.quadrature_points(mesh, co)
    fpts = ihdg.face_quadrature_points(mesh)
    disc = Discretisation(om, p)
    assert np.abs(fpts - disc.face_points(np.arange(om.nface))).max() < 1e-13
    assert np.abs(vol - disc.volume_points()).max() < 1e-13
    beta = fields[field]
    pr = TransportVar(disc, beta)
    B1 = lagrange_matrix(disc.ref.nodes1, disc.ref.xq1)
    Bf = B1 if d == 2 else np.kron(B1, B1)
    W_ = pr.trace_coupling()
    for K in (0, om.nel // 2, om.nel - 1):
        Ainv = np.linalg.inv(pr.A[K])
        assert np.allclose(ihdg.var_host_operator(mesh, beta(vol), beta(fpts), K, 1), Ainv, rtol=0, atol=1e-10 * np.abs(Ainv).max())
        G = np.concatenate([W_[f][K] @ Bf for f in range(2 * d)], axis=1)
        Lk = Ainv @ G
        got = ihdg.var_host_operator(mesh, beta(vol), beta(fpts), K, 0)
        assert np.abs(got - Lk).max() < 1e-10 * max(1.0, np.abs(Lk).max())


def test_var_plan_rejects_sign_change_and_needs_device():
    import workloads as W
    mesh = ihdg.make_mesh(2, (3, 3), 2)
    co = ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1.0, 0.0, 0.0))
    vol, _ = ihdg.quadrature_points(mesh, co)
    fpts = ihdg.face_quadrature_points(mesh)
    sign_change = lambda X: np.stack([X[..., 1] - 0.45, np.ones_like(X[..., 0])], axis=-1)
    with pytest.raises(ihdg.IHDGError) as ei:
        ihdg.var_host_operator(mesh, sign_change(vol), sign_change(fpts), 0, 0)
    assert ei.value.status == ihdg.ERR_UNSUPPORTED


def test_group_workspace_bytes_host_only():
    """ihdg_group_workspace_bytes (host only): the per-problem workspaces, each rounded to 256
    bytes, plus the grouped launch's descriptors; shallow water and bad counts are rejected."""
    L = ihdg.load()
    meshes = [ihdg.make_mesh(2, (9, 7), 2), ihdg.make_mesh(2, (12, 12), 4), ihdg.make_mesh(3, (3, 4, 5), 1)]
    coeffs = [ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 0.5)), ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=0.01),
              ihdg.make_coeffs(ihdg.TRANSPORT, beta=(1, 1, 1))]
    opts = ihdg.make_options(1e-8)
    n = len(meshes)
    ms = (ihdg.Mesh * n)(*meshes)
    cs = (ihdg.Coeffs * n)(*coeffs)
    b = ctypes.c_size_t()
    assert L.ihdg_group_workspace_bytes(n, ms, cs, ctypes.byref(opts), ctypes.byref(b)) == ihdg.OK
    per = sum((ihdg.workspace_bytes(m, c, opts) + 255) // 256 * 256 for m, c in zip(meshes, coeffs))
    assert per < b.value <= per + 64 * 1024
    swe = (ihdg.Coeffs * 1)(ihdg.make_coeffs(ihdg.SWE, Phi=1.0, dt=0.01))
    m1 = (ihdg.Mesh * 1)(meshes[0])
    assert L.ihdg_group_workspace_bytes(1, m1, swe, ctypes.byref(opts), ctypes.byref(b)) == ihdg.ERR_INVALID
    assert L.ihdg_group_workspace_bytes(-1, ms, cs, ctypes.byref(opts), ctypes.byref(b)) == ihdg.ERR_INVALID


def test_krylov_workspace_host_only():
    """opts.krylov_restart = m (GMRES around the sweep) adds its basis, m + 1 export vectors of
    n_exp x ld doubles, plus the small Hessenberg and reduction arrays, to the workspace;
    values outside 0..4096 are rejected before any device work."""
    mesh = ihdg.make_mesh(2, (20, 13), 3)
    co = ihdg.make_coeffs(ihdg.CONVDIFF, beta=(1, 1), kappa=0.01)
    s = ihdg.problem_sizes(mesh, co)
    ld = (s.n_el + 31) // 32 * 32
    nvec = s.n_exp * ld
    nblk = (nvec + 1023) // 1024
    w0 = ihdg.workspace_bytes(mesh, co, ihdg.make_options(1e-8))
    for m in (1, 30, 4096):
        wm = ihdg.workspace_bytes(mesh, co, ihdg.make_options(1e-8, krylov_restart=m))
        basis = (m + 1) * nvec * 8
        assert basis <= wm - w0 <= basis + (m + 1) * (m + 8) * 8 + (m + 1) * nblk * 8 + 16 * 256
    for bad in (-1, 4097):
        with pytest.raises(ihdg.IHDGError) as ei:
            ihdg.workspace_bytes(mesh, co, ihdg.make_options(1e-8, krylov_restart=bad))
        assert ei.value.status == ihdg.ERR_INVALID


def test_binding_structs_match_the_c_abi():
    """The ctypes mirrors of the public structs have the C sizes (a field added on one side
    only, or a type mismatch, changes them)."""
    L = ihdg.load()
    out = (ctypes.c_size_t * 6)()
    assert L.ihdg_abi_sizes(out, 6) == ihdg.OK
    mirrors = [ihdg.Mesh, ihdg.Coeffs, ihdg.Options, ihdg.Result, ihdg.Sizes, ihdg.Peaks]
    assert [ctypes.sizeof(m) for m in mirrors] == list(out)
    assert L.ihdg_abi_sizes(None, 6) == ihdg.ERR_INVALID
    part = (ctypes.c_size_t * 2)(0, 0)
    assert L.ihdg_abi_sizes(part, 2) == ihdg.OK and part[1] == out[1]
