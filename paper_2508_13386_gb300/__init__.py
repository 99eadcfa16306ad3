"""GB300 (sm_103a) multilevel elastodynamics timestep library.

Python face of the C ABI in ``include/mls.h`` (libmls.so): argument
marshalling only.  Device arrays are torch CUDA tensors (float64, [n, 3]);
host arrays are numpy arrays.  Every step of the timestep runs in the
library's CUDA kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib

__all__ = ["Solver", "MLP", "MLSError", "lib", "contact_pair_derivatives"]

lib = None


def _get_lib():
    global lib
    if lib is None:
        lib = _lib.load()
    return lib


def tridiag_max_eig(d, e):
    """Largest eigenvalue of the symmetric tridiagonal (d, e) by the library's
    Sturm bisection (mls_tridiag_max_eig)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    P = C.POINTER(C.c_double)
    return float(_get_lib().mls_tridiag_max_eig(d.ctypes.data_as(P), e.ctypes.data_as(P), int(d.size)))


class MLSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_lib.STATUS.get(status, status)}: {message}")
        self.status = status


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _dev(t, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One library context (``mls_ctx``) bound to a CUDA stream."""

    def __init__(self, precision="fp64", preconditioner="jacobi", cycle="additive", omega=1.0,
                 newton_tol=1e-10, pcg_rtol=1e-4, max_newton=50, max_pcg=20000,
                 coarse_refresh=0, pcg_check_every=16, persistent=False, persist_blocks_per_sm=0,
                 direction="pcg", refine_iters=20, paper_tol=1e-3, stream=None, coarse_lag_steps=0,
                 sub_rtol=1e-4, hessian_lag=False):
        self._l = _get_lib()
        self._ctx = C.c_void_p()
        self.opt = _lib.Options()
        self._l.mls_default_options(C.byref(self.opt))
        self._fill(precision, preconditioner, cycle, omega, newton_tol, pcg_rtol, max_newton, max_pcg,
                   coarse_refresh, pcg_check_every, persistent, persist_blocks_per_sm, direction, refine_iters,
                   paper_tol, stream, coarse_lag_steps, sub_rtol, hessian_lag)
        st = self._l.mls_create(C.byref(self._ctx), C.byref(self.opt))
        if st != _lib.MLS_OK:
            raise MLSError(st, "mls_create failed")
        self.n = 0
        self.t = 0
        self.m = 0

    def _fill(self, precision, preconditioner, cycle, omega, newton_tol, pcg_rtol, max_newton, max_pcg,
              coarse_refresh, pcg_check_every, persistent, persist_blocks_per_sm, direction, refine_iters,
              paper_tol, stream, coarse_lag_steps=0, sub_rtol=1e-4, hessian_lag=False):
        o = self.opt
        o.precision = _lib.PRECISION[precision]
        o.preconditioner = _lib.PRECOND[preconditioner]
        o.cycle = _lib.CYCLE[cycle]
        o.omega = float(omega)
        o.newton_tol = float(newton_tol)
        o.pcg_rtol = float(pcg_rtol)
        o.max_newton = int(max_newton)
        o.max_pcg = int(max_pcg)
        o.coarse_refresh = int(coarse_refresh)
        o.coarse_lag_steps = int(coarse_lag_steps)
        o.pcg_check_every = int(pcg_check_every)
        o.persistent = 1 if persistent else 0
        o.persist_blocks_per_sm = int(persist_blocks_per_sm)
        o.direction = ({"pcg": 0, "paper": 1, "paper_literal": 2}[direction] if isinstance(direction, str)
                       else int(direction))
        o.refine_iters = int(refine_iters)
        o.paper_tol = float(paper_tol)
        o.sub_rtol = float(sub_rtol)
        o.hessian_lag = 1 if hessian_lag else 0
        if stream is None:
            o.stream = None
        else:
            o.stream = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)

    def set_options(self, **kw):
        cur = dict(precision={v: k for k, v in _lib.PRECISION.items()}[self.opt.precision],
                   preconditioner=["jacobi", "two_level"][self.opt.preconditioner],
                   cycle=["additive", "multiplicative"][self.opt.cycle], omega=self.opt.omega,
                   newton_tol=self.opt.newton_tol, pcg_rtol=self.opt.pcg_rtol,
                   max_newton=self.opt.max_newton, max_pcg=self.opt.max_pcg,
                   coarse_refresh=self.opt.coarse_refresh, pcg_check_every=self.opt.pcg_check_every,
                   persistent=bool(self.opt.persistent),
                   persist_blocks_per_sm=self.opt.persist_blocks_per_sm, direction=self.opt.direction,
                   refine_iters=self.opt.refine_iters, paper_tol=self.opt.paper_tol, stream=self.opt.stream,
                   coarse_lag_steps=self.opt.coarse_lag_steps, sub_rtol=self.opt.sub_rtol,
                   hessian_lag=bool(self.opt.hessian_lag))
        cur.update(kw)
        self._fill(**cur)
        self._check(self._l.mls_set_options(self._ctx, C.byref(self.opt)))

    def close(self):
        if self._ctx:
            self._l.mls_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != _lib.MLS_OK and st not in allow:
            msg = self._l.mls_last_error(self._ctx)
            raise MLSError(st, msg.decode() if msg else "")
        return st

    # ---- uploads ---------------------------------------------------------------
    def upload_mesh(self, X, tets, E, nu, rho, dirichlet=None):
        X, pX = _host(X, np.float64)
        tets, pT = _host(tets, np.int32)
        E, pE = _host(E, np.float64)
        nu, pN = _host(nu, np.float64)
        rho, pR = _host(rho, np.float64)
        if dirichlet is None:
            pD = None
        else:
            dirichlet, pD = _host(dirichlet, np.uint8)
        self._check(self._l.mls_upload_mesh(self._ctx, X.shape[0], pX, tets.shape[0], pT, pE, pN, pR, pD))
        self.n, self.t = X.shape[0], tets.shape[0]

    def upload_basis(self, origins, vrow, handle, phi):
        origins, pO = _host(origins, np.float64)
        vrow, pV = _host(vrow, np.int32)
        handle, pH = _host(handle, np.int32)
        phi, pP = _host(phi, np.float64)
        self._check(self._l.mls_upload_basis(self._ctx, origins.shape[0], pO, pV, pH, pP))
        self.m = origins.shape[0]

    def upload_cubature(self, scale):
        """Per-element factor w_e / vol_e of an elastic-term cubature for the
        coarse operator (``cubature.build_cubature(...)["scale"]``), or None."""
        if scale is None:
            self._check(self._l.mls_upload_cubature(self._ctx, None))
            return
        scale, ps = _host(scale, np.float64)
        self._check(self._l.mls_upload_cubature(self._ctx, ps))

    def set_forces(self, gravity=(0.0, 0.0, -9.81), contact=False, plane_n=(0.0, 0.0, 1.0), plane_o=0.0,
                   dhat=1e-3, kappa=1e5):
        g, pg = _host(gravity, np.float64)
        pn, ppn = _host(plane_n, np.float64)
        self._check(self._l.mls_set_forces(self._ctx, pg, 1 if contact else 0, ppn, float(plane_o),
                                           float(dhat), float(kappa)))

    def set_friction(self, mu, eps_v=1e-3):
        """Lagged friction (coefficient mu, mollifier velocity eps_v) against the
        contact plane and, with bodies set, between them (mls_set_friction);
        needs contact on (set_forces) or bodies (set_bodies).  mu = 0 turns it off."""
        self._check(self._l.mls_set_friction(self._ctx, float(mu), float(eps_v)))

    def setup_scene(self, scene):
        """Upload a ``synth.Scene``-like object's mesh, materials and loads."""
        self.upload_mesh(scene.X, scene.tets, scene.E, scene.nu, scene.rho, scene.dirichlet)
        self.set_forces(scene.gravity, scene.contact, scene.plane_n, scene.plane_o, scene.dhat, scene.kappa)

    # ---- timestep ----------------------------------------------------------------
    def newton_step(self, x, v, dt, dx=None, allow_notconv=False):
        import torch
        if dx is None:
            dx = torch.empty_like(x)
        st = _lib.Stats()
        allow = (-4,) if allow_notconv else ()
        status = self._check(self._l.mls_newton_step(self._ctx, _dev(x, (self.n, 3)), _dev(v, (self.n, 3)),
                                                     float(dt), _dev(dx, (self.n, 3)), C.byref(st)), allow)
        out = st.as_dict()
        out["status"] = status
        return dx, out

    def newton_step_bdf2(self, x, v, x_prev, v_prev, dt, dx=None, allow_notconv=False):
        """One BDF2 timestep from (x^t, v^t) and (x^{t-1}, v^{t-1}); returns
        dx = x^{t+1} - x^t (device) and the stats."""
        import torch
        if dx is None:
            dx = torch.empty_like(x)
        st = _lib.Stats()
        allow = (-4,) if allow_notconv else ()
        shape = (self.n, 3)
        status = self._check(self._l.mls_newton_step_bdf2(self._ctx, _dev(x, shape), _dev(v, shape),
                                                          _dev(x_prev, shape), _dev(v_prev, shape), float(dt),
                                                          _dev(dx, shape), C.byref(st)), allow)
        out = st.as_dict()
        out["status"] = status
        return dx, out

    def newton_step_host(self, x, v, dt, dx=None):
        x, px = _host(x, np.float64)
        v, pv = _host(v, np.float64)
        if dx is None:
            dx = np.empty_like(x)
        st = _lib.Stats()
        self._check(self._l.mls_newton_step_host(self._ctx, px, pv, float(dt),
                                                 dx.ctypes.data_as(C.c_void_p), C.byref(st)))
        return dx, st.as_dict()

    # ---- stage entry points --------------------------------------------------------
    def eval_elements(self, x):
        import torch
        dev = x.device
        energy = torch.empty(self.t, dtype=torch.float64, device=dev)
        grad = torch.empty(self.t, 12, dtype=torch.float64, device=dev)
        hess = torch.empty(self.t, 12, 12, dtype=torch.float64, device=dev)
        self._check(self._l.mls_eval_elements(self._ctx, _dev(x, (self.n, 3)), _dev(energy), _dev(grad),
                                              _dev(hess)))
        return energy, grad, hess

    def assemble(self, x, x_t, v_t, dt):
        import torch
        g = torch.empty_like(x)
        self._check(self._l.mls_assemble(self._ctx, _dev(x, (self.n, 3)), _dev(x_t, (self.n, 3)),
                                         _dev(v_t, (self.n, 3)), float(dt), _dev(g)))
        return g

    def get_hessian_nnzb(self):
        nnzb = C.c_int64()
        self._check(self._l.mls_get_hessian(self._ctx, None, None, None, C.byref(nnzb)))
        return nnzb.value

    def get_hessian(self):
        nnzb = C.c_int64()
        self._check(self._l.mls_get_hessian(self._ctx, None, None, None, C.byref(nnzb)))
        rp = np.zeros(self.n + 1, dtype=np.int32)
        col = np.zeros(nnzb.value, dtype=np.int32)
        val = np.zeros((nnzb.value, 3, 3), dtype=np.float64)
        self._check(self._l.mls_get_hessian(self._ctx, rp.ctypes.data_as(C.c_void_p),
                                            col.ctypes.data_as(C.c_void_p), val.ctypes.data_as(C.c_void_p),
                                            C.byref(nnzb)))
        return rp, col, val

    def spmv(self, x):
        import torch
        y = torch.empty_like(x)
        self._check(self._l.mls_spmv(self._ctx, _dev(x, (self.n, 3)), _dev(y)))
        return y

    def precond_apply(self, r):
        import torch
        z = torch.empty_like(r)
        self._check(self._l.mls_precond_apply(self._ctx, _dev(r, (self.n, 3)), _dev(z)))
        return z

    def pcg_solve(self, b, rtol, max_iter=20000):
        import torch
        d = torch.empty_like(b)
        it = C.c_int()
        rel = C.c_double()
        st = self._check(self._l.mls_pcg_solve(self._ctx, _dev(b, (self.n, 3)), _dev(d), float(rtol),
                                               int(max_iter), C.byref(it), C.byref(rel)), allow=(-4,))
        return d, it.value, rel.value, st

    def prolong(self, q):
        import torch
        w = torch.empty(self.n, 3, dtype=torch.float64, device=q.device)
        self._check(self._l.mls_prolong(self._ctx, _dev(q, (self.m, 12)), _dev(w)))
        return w

    def restrict(self, r):
        import torch
        z = torch.empty(self.m, 12, dtype=torch.float64, device=r.device)
        self._check(self._l.mls_restrict(self._ctx, _dev(r, (self.n, 3)), _dev(z)))
        return z

    def build_coarse(self):
        self._check(self._l.mls_build_coarse(self._ctx))

    def smoother_omega(self):
        """(omega, lambda_max estimate) of the two-level smoother; see mls_smoother_omega."""
        om, lm = C.c_double(), C.c_double()
        self._check(self._l.mls_smoother_omega(self._ctx, C.byref(om), C.byref(lm)))
        return om.value, lm.value

    def get_coarse_factor(self):
        """Lower Cholesky factor L of the last coarse build (mls_get_coarse_factor)."""
        r = 12 * self.m
        L = np.zeros((r, r))
        self._check(self._l.mls_get_coarse_factor(self._ctx, L.ctypes.data_as(C.c_void_p)))
        return L

    def coarse_shift(self):
        """Relative diagonal shift of the current coarse factor (0: none); see mls_coarse_shift."""
        sig = C.c_double()
        self._check(self._l.mls_coarse_shift(self._ctx, C.byref(sig)))
        return sig.value

    def get_coarse(self):
        r = 12 * self.m
        A = np.zeros((r, r), dtype=np.float64)
        self._check(self._l.mls_get_coarse(self._ctx, A.ctypes.data_as(C.c_void_p)))
        return A

    def energy(self, x, d, alpha):
        E = C.c_double()
        feas = C.c_int()
        self._check(self._l.mls_energy(self._ctx, _dev(x, (self.n, 3)), _dev(d, (self.n, 3)), float(alpha),
                                       C.byref(E), C.byref(feas)))
        return E.value, bool(feas.value)

    # ---- warm start -------------------------------------------------------------
    def warm_start_enable(self, enable=True, record=False):
        self._check(self._l.mls_warm_start_enable(self._ctx, (2 if record else 1) if enable else 0))

    def warm_start_reset(self):
        self._check(self._l.mls_warm_start_reset(self._ctx))

    def warm_start_attach(self, mlp):
        self._check(self._l.mls_warm_start_attach(self._ctx, mlp._h if mlp is not None else None))
        self._attached = mlp  # keep the network alive while attached

    def warm_start_sample(self, features, target):
        self._check(self._l.mls_warm_start_sample(self._ctx, C.c_void_p(features.data_ptr()),
                                                  C.c_void_p(target.data_ptr())))

    def coarse_project(self, x):
        import torch
        q = torch.empty(self.m, 12, dtype=torch.float64, device=x.device)
        self._check(self._l.mls_coarse_project(self._ctx, _dev(x, (self.n, 3)), _dev(q)))
        return q

    def profile_enable(self, classes=()):
        mask = 0
        for c in classes:
            mask |= 1 << _lib.PROF_CLASSES.index(c)
        self._check(self._l.mls_profile_enable(self._ctx, mask))

    def profile_read(self):
        ms = np.zeros(len(_lib.PROF_CLASSES), dtype=np.float64)
        n = np.zeros(len(_lib.PROF_CLASSES), dtype=np.int64)
        self._check(self._l.mls_profile_read(self._ctx, ms.ctypes.data_as(C.c_void_p), n.ctypes.data_as(C.c_void_p)))
        return {c: (float(ms[i]), int(n[i])) for i, c in enumerate(_lib.PROF_CLASSES)}

    def ccd_bound(self, x, d):
        a = C.c_double()
        self._check(self._l.mls_ccd_bound(self._ctx, _dev(x, (self.n, 3)), _dev(d, (self.n, 3)), C.byref(a)))
        return a.value

    # ---- mesh-mesh contact ---------------------------------------------------------
    def set_bodies(self, body, dhat=1e-3, kappa=1e5, spare=0):
        """Mesh-mesh contact between the bodies ``body`` [n] labels (None: off);
        see mls_set_bodies.  Call after upload_mesh, before upload_basis."""
        if body is None:
            self._check(self._l.mls_set_bodies(self._ctx, None, float(dhat), float(kappa), 0))
            return
        b, pb = _host(body, np.int32)
        if b.shape != (self.n,):
            raise ValueError(f"expected {self.n} body labels")
        self._check(self._l.mls_set_bodies(self._ctx, pb, float(dhat), float(kappa), int(spare)))

    def contact_pairs(self, x, d=None):
        """(pt [k, 4], ee [k, 4]) vertex indices of the contact pairs at x
        (d None: distance < dhat) or the candidates over x -> x + d."""
        npt, nee = C.c_int64(), C.c_int64()
        dd = None if d is None else _dev(d, (self.n, 3))
        self._check(self._l.mls_contact_pairs(self._ctx, _dev(x, (self.n, 3)), dd, 0, None, C.byref(npt), None,
                                              C.byref(nee)))
        cap = max(npt.value, nee.value, 1)
        pt = np.zeros((cap, 4), np.int32)
        ee = np.zeros((cap, 4), np.int32)
        self._check(self._l.mls_contact_pairs(self._ctx, _dev(x, (self.n, 3)), dd, int(cap),
                                              pt.ctypes.data_as(C.c_void_p), C.byref(npt),
                                              ee.ctypes.data_as(C.c_void_p), C.byref(nee)))
        return pt[:npt.value], ee[:nee.value]


def contact_pair_derivatives(kind, X, kappa, dhat):
    """Per-pair distance derivatives on the GPU (mls_contact_pair_derivatives):
    kind [P] (0 point-triangle, 1 edge-edge), X [P, 4, 3] -> (d [P],
    grad d [P, 12], Hess d [P, 12, 12], projected barrier Hessian [P, 12, 12])."""
    import torch
    kind = torch.as_tensor(np.asarray(kind, np.int32), device="cuda:0").contiguous()
    X = torch.as_tensor(np.asarray(X, np.float64), device="cuda:0").contiguous()
    P = int(kind.shape[0])
    d = torch.empty(P, dtype=torch.float64, device="cuda:0")
    g = torch.empty((P, 12), dtype=torch.float64, device="cuda:0")
    Hd = torch.empty((P, 12, 12), dtype=torch.float64, device="cuda:0")
    Hb = torch.empty((P, 12, 12), dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    st = _get_lib().mls_contact_pair_derivatives(C.c_void_p(kind.data_ptr()), C.c_void_p(X.data_ptr()), P,
                                                float(kappa), float(dhat), C.c_void_p(d.data_ptr()),
                                                C.c_void_p(g.data_ptr()), C.c_void_p(Hd.data_ptr()),
                                                C.c_void_p(Hb.data_ptr()))
    if st != 0:
        raise MLSError(st, "contact_pair_derivatives")
    return d.cpu().numpy(), g.cpu().numpy(), Hd.cpu().numpy(), Hb.cpu().numpy()


class Batch:
    """Many independent meshes advanced together (``mls_batch``): one graph
    launch per timestep, block-Jacobi PCG, per-mesh Newton decisions."""

    def __init__(self, precision="fp32", preconditioner="jacobi", omega=0.5, newton_tol=1e-5, pcg_rtol=1e-4,
                 max_newton=50, max_pcg=20000, stream=None):
        self._l = _get_lib()
        self._b = C.c_void_p()
        opt = _lib.Options()
        self._l.mls_default_options(C.byref(opt))
        opt.precision = _lib.PRECISION[precision]
        opt.preconditioner = _lib.PRECOND[preconditioner]
        opt.omega = float(omega)
        opt.newton_tol = float(newton_tol)
        opt.pcg_rtol = float(pcg_rtol)
        opt.max_newton = int(max_newton)
        opt.max_pcg = int(max_pcg)
        opt.stream = None if stream is None else C.c_void_p(stream.cuda_stream)
        st = self._l.mls_batch_create(C.byref(self._b), C.byref(opt))
        if st != _lib.MLS_OK:
            raise MLSError(st, "mls_batch_create failed")
        self.n_meshes = 0
        self.vert_offsets = None

    def close(self):
        if self._b:
            self._l.mls_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != _lib.MLS_OK and st not in allow:
            msg = self._l.mls_batch_last_error(self._b)
            raise MLSError(st, msg.decode() if msg else "")
        return st

    def upload_scenes(self, scenes):
        """Concatenate ``synth.Scene``-like meshes (forces from the first)."""
        voff, toff, X, T, E, nu, rho, D = [0], [0], [], [], [], [], [], []
        for sc in scenes:
            nt = len(sc.tets)
            X.append(np.asarray(sc.X, dtype=np.float64))
            T.append(np.asarray(sc.tets, dtype=np.int64) + voff[-1])
            E.append(np.broadcast_to(np.asarray(sc.E, dtype=np.float64), (nt,)))
            nu.append(np.broadcast_to(np.asarray(sc.nu, dtype=np.float64), (nt,)))
            rho.append(np.broadcast_to(np.asarray(sc.rho, dtype=np.float64), (nt,)))
            D.append(np.asarray(sc.dirichlet, dtype=np.uint8) if sc.dirichlet is not None
                     else np.zeros(len(sc.X), dtype=np.uint8))
            voff.append(voff[-1] + len(sc.X))
            toff.append(toff[-1] + nt)
        self.upload(voff, toff, np.concatenate(X), np.concatenate(T), np.concatenate(E), np.concatenate(nu),
                    np.concatenate(rho), np.concatenate(D))
        s0 = scenes[0]
        self.set_forces(s0.gravity, s0.contact, s0.plane_n, s0.plane_o, s0.dhat, s0.kappa)

    def upload(self, vert_offsets, tet_offsets, X, tets, E, nu, rho, dirichlet=None):
        vo, pvo = _host(vert_offsets, np.int32)
        to, pto = _host(tet_offsets, np.int32)
        X, pX = _host(X, np.float64)
        tets, pT = _host(tets, np.int32)
        E, pE = _host(E, np.float64)
        nu, pN = _host(nu, np.float64)
        rho, pR = _host(rho, np.float64)
        pD = None
        if dirichlet is not None:
            dirichlet, pD = _host(dirichlet, np.uint8)
        self._check(self._l.mls_batch_upload(self._b, len(vo) - 1, pvo, pto, pX, pT, pE, pN, pR, pD))
        self.n_meshes = len(vo) - 1
        self.vert_offsets = vo.copy()
        self.n = int(vo[-1])

    def upload_bases(self, bases):
        """Per-mesh bases (dicts with origins, vrow, handle, phi in each mesh's
        own vertex and handle numbering), concatenated in mesh order."""
        hoff, O, VR, H, PH = [0], [], [np.zeros(1, dtype=np.int64)], [], []
        nnz = 0
        for B in bases:
            O.append(np.asarray(B["origins"], dtype=np.float64))
            vr = np.asarray(B["vrow"], dtype=np.int64)
            VR.append(vr[1:] + nnz)
            H.append(np.asarray(B["handle"], dtype=np.int64) + hoff[-1])
            PH.append(np.asarray(B["phi"], dtype=np.float64))
            nnz += int(vr[-1])
            hoff.append(hoff[-1] + len(B["origins"]))
        ho, pho = _host(hoff, np.int32)
        o, po = _host(np.concatenate(O), np.float64)
        vr, pvr = _host(np.concatenate(VR), np.int32)
        h, ph = _host(np.concatenate(H), np.int32)
        f, pf = _host(np.concatenate(PH), np.float64)
        self._check(self._l.mls_batch_upload_basis(self._b, int(hoff[-1]), pho, po, pvr, ph, pf))

    def set_forces(self, gravity=(0.0, 0.0, -9.81), contact=False, plane_n=(0.0, 0.0, 1.0), plane_o=0.0,
                   dhat=1e-3, kappa=1e5):
        g, pg = _host(gravity, np.float64)
        pn, ppn = _host(plane_n, np.float64)
        self._check(self._l.mls_batch_set_forces(self._b, pg, 1 if contact else 0, ppn, float(plane_o),
                                                 float(dhat), float(kappa)))

    def set_friction(self, mu, eps_v=1e-3):
        """Lagged point-plane friction for every mesh (as ``Solver.set_friction``)."""
        self._check(self._l.mls_batch_set_friction(self._b, float(mu), float(eps_v)))

    def retune(self):
        self._check(self._l.mls_batch_retune(self._b))

    def step(self, x, v, dt, dx=None, allow=(-4,)):
        """One timestep of every mesh; returns (dx, per-mesh stats, info).
        Meshes that hit their Newton cap (-4) are reported, not raised."""
        import torch
        if dx is None:
            dx = torch.empty_like(x)
        stats = (_lib.BatchMeshStats * self.n_meshes)()
        info = _lib.BatchInfo()
        status = self._check(self._l.mls_batch_step(self._b, _dev(x, (self.n, 3)), _dev(v, (self.n, 3)), float(dt),
                                                    _dev(dx, (self.n, 3)), stats, C.byref(info)), allow)
        per = [{k: getattr(s, k) for k, _ in _lib.BatchMeshStats._fields_} for s in stats]
        inf = {k: getattr(info, k) for k, _ in _lib.BatchInfo._fields_}
        inf["status"] = status
        return dx, per, inf

    def step_bdf2(self, x, v, x_prev, v_prev, dt, dx=None, allow=(-4,)):
        """One BDF2 timestep of every mesh from (x^t, v^t) and (x^{t-1}, v^{t-1});
        returns (dx, per-mesh stats, info) as ``step``."""
        import torch
        if dx is None:
            dx = torch.empty_like(x)
        stats = (_lib.BatchMeshStats * self.n_meshes)()
        info = _lib.BatchInfo()
        shape = (self.n, 3)
        status = self._check(self._l.mls_batch_step_bdf2(self._b, _dev(x, shape), _dev(v, shape), _dev(x_prev, shape),
                                                         _dev(v_prev, shape), float(dt), _dev(dx, shape), stats,
                                                         C.byref(info)), allow)
        per = [{k: getattr(s, k) for k, _ in _lib.BatchMeshStats._fields_} for s in stats]
        inf = {k: getattr(info, k) for k, _ in _lib.BatchInfo._fields_}
        inf["status"] = status
        return dx, per, inf


class MLP:
    """A network trained and run by the library's kernels (``mls_mlp_*``)."""

    def __init__(self, sizes, init_params, max_batch=256, stream=None):
        self._l = _get_lib()
        self.sizes = list(sizes)
        flat = np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in init_params])
        self._h = C.c_void_p()
        st = self._l.mls_mlp_create(C.byref(self._h), sizes[0], sizes[1], sizes[-1], int(max_batch),
                                    flat.ctypes.data_as(C.c_void_p),
                                    None if stream is None else C.c_void_p(stream.cuda_stream))
        if st != _lib.MLS_OK:
            raise MLSError(st, "mls_mlp_create failed")
        self.n_params = int(self._l.mls_mlp_param_count(self._h))

    def close(self):
        if self._h:
            self._l.mls_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _p(t):
        return C.c_void_p(t.data_ptr())

    def _ok(self, st, what):
        if st != _lib.MLS_OK:
            raise MLSError(st, what)

    def forward(self, X):
        import torch
        Y = torch.empty(X.shape[0], self.sizes[-1], dtype=torch.float32, device=X.device)
        self._ok(self._l.mls_mlp_forward(self._h, self._p(X), X.shape[0], self._p(Y)), "forward")
        return Y

    def set_normalization(self, mean_in, std_in, mean_out, std_out):
        self._ok(self._l.mls_mlp_set_normalization(self._h, self._p(mean_in), self._p(std_in),
                                                   self._p(mean_out), self._p(std_out)), "normalization")

    def train_epoch(self, X, T, order, batch, lr):
        loss = C.c_double()
        self._ok(self._l.mls_mlp_train(self._h, self._p(X), self._p(T), X.shape[0], self._p(order),
                                       order.shape[0], int(batch), C.c_float(lr), C.byref(loss)), "train")
        return loss.value

    def params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        self._ok(self._l.mls_mlp_get_params(self._h, out.ctypes.data_as(C.c_void_p)), "get_params")
        return out


def column_stats(X):
    """Column mean and standard deviation of a float32 CUDA tensor (library kernel)."""
    import torch
    mean = torch.empty(X.shape[1], dtype=torch.float32, device=X.device)
    sd = torch.empty_like(mean)
    st = _get_lib().mls_mlp_column_stats(C.c_void_p(X.data_ptr()), X.shape[0], X.shape[1],
                                         C.c_void_p(mean.data_ptr()), C.c_void_p(sd.data_ptr()), None)
    if st != _lib.MLS_OK:
        raise MLSError(st, "column_stats")
    return mean, sd
