"""Thin Python wrapper over the C ABI: torch tensors in, device pointers out.

PyTorch only provides device memory and streams here; every step of the
simulation runs in libpdgb300's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib

_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


def _check(status: int, where: str):
    if status != _lib.PD_OK:
        L = lib()
        raise _lib.PDError(status, where, f"{L.pd_status_string(status).decode()}: {L.pd_last_error().decode()}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_f32(a, shape=None, device="cuda"):
    if a is None:
        return None
    t = a if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a))
    t = t.to(device=device, dtype=torch.float32).contiguous()
    if shape is not None:
        t = t.reshape(shape)
    return t


PRECISIONS = {"fp32": _lib.PD_PREC_FP32, "bf16": _lib.PD_PREC_BF16, "tf32": _lib.PD_PREC_TF32}


class Mesh:
    """A tet mesh resident on the GPU, stepped by domain-decomposed PD."""

    def __init__(self, rest, tets, pinned=None, tet_domain=None, n_domains=1, density=300.0, vertex_mass=None,
                 stream: torch.cuda.Stream | None = None):
        L = lib()
        self.rest = np.ascontiguousarray(rest, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.n_v = int(self.rest.shape[0])
        self.n_t = int(self.tets.shape[0])
        pin = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
        dom = None if tet_domain is None else np.ascontiguousarray(tet_domain, dtype=np.int32)
        mass = None if vertex_mass is None else np.ascontiguousarray(vertex_mass, dtype=np.float64)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n_pinned = 0 if pin is None else int((pin != 0).sum())
        h = C.c_void_p()
        st = L.pd_create_mesh(self.rest.ctypes.data, self.n_v, self.tets.ctypes.data, self.n_t,
                              None if mass is None else mass.ctypes.data, float(density),
                              None if dom is None else dom.ctypes.data, int(n_domains),
                              None if pin is None else pin.ctypes.data, C.c_void_p(self.stream.cuda_stream),
                              C.byref(h))
        _check(st, "pd_create_mesh")
        self._h = h
        self._keep = {}
        self.dt = None

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pd_destroy_mesh(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up ----------------------------------------------------------------
    def set_materials(self, gamma_s, gamma_v):
        gs = np.ascontiguousarray(np.asarray(gamma_s, dtype=np.float32)) if not isinstance(gamma_s, torch.Tensor) \
            else gamma_s.to(torch.float32).contiguous()
        gv = np.ascontiguousarray(np.asarray(gamma_v, dtype=np.float32)) if not isinstance(gamma_v, torch.Tensor) \
            else gamma_v.to(torch.float32).contiguous()
        p_s = gs.ctypes.data if isinstance(gs, np.ndarray) else gs.data_ptr()
        p_v = gv.ctypes.data if isinstance(gv, np.ndarray) else gv.data_ptr()
        _check(lib().pd_set_materials(self._h, C.c_void_p(p_s), C.c_void_p(p_v)), "pd_set_materials")

    @staticmethod
    def solver_opts(precision="fp32", refine_steps=0, use_graphs=True, correction=False, single_level=False,
                    streaming=False, modal=False, modes=20, jacobi_sweeps=0, jacobi_rho=0.0):
        flags = ((_lib.PD_SOLVE_CORRECTION if correction else 0) | (_lib.PD_SOLVE_SINGLE_LEVEL if single_level else 0)
                 | (_lib.PD_SOLVE_STREAMING if streaming else 0) | (_lib.PD_SOLVE_MODAL if modal else 0))
        return _lib.pd_solver_opts(PRECISIONS[precision], int(refine_steps), 1 if use_graphs else 0, flags,
                                   int(modes), int(jacobi_sweeps), float(jacobi_rho))

    def prefactor(self, dt, **solver):
        o = self.solver_opts(**solver)
        _check(lib().pd_prefactor(self._h, float(dt), C.byref(o)), "pd_prefactor")
        self.dt = float(dt)

    # -- state -----------------------------------------------------------------
    def set_state(self, x=None, v=None):
        xt = _dev_f32(x, (self.n_v, 3))
        vt = _dev_f32(v, (self.n_v, 3))
        _check(lib().pd_set_state(self._h, _ptr(xt), _ptr(vt)), "pd_set_state")
        self._keep["state"] = (xt, vt)   # keep alive until the stream has consumed them

    def get_state(self):
        x = torch.empty((self.n_v, 3), device="cuda", dtype=torch.float32)
        v = torch.empty((self.n_v, 3), device="cuda", dtype=torch.float32)
        _check(lib().pd_get_state(self._h, _ptr(x), _ptr(v)), "pd_get_state")
        return x, v

    def step(self, pin_targets=None, gravity=(0.0, 0.0, -9.81), n_iter=10, x_out=None):
        pt = _dev_f32(pin_targets, (self.n_pinned, 3)) if pin_targets is not None else None
        g = (C.c_float * 3)(*[float(a) for a in gravity])
        _check(lib().pd_step(self._h, _ptr(pt), g, int(n_iter), _ptr(x_out)), "pd_step")
        self._keep["pins"] = pt
        return x_out

    def sync(self):
        _check(lib().pd_sync(self._h), "pd_sync")

    def info(self) -> dict:
        i = _lib.pd_mesh_info()
        _check(lib().pd_get_info(self._h, C.byref(i)), "pd_get_info")
        d = {k: getattr(i, k) for k, _ in _lib.pd_mesh_info._fields_ if k not in ("phase_bytes", "phase_launches")}
        d["phase_bytes"] = {PHASES[k]: int(i.phase_bytes[k]) for k in range(len(PHASES))}
        d["phase_launches"] = {PHASES[k]: int(i.phase_launches[k]) for k in range(len(PHASES))}
        return d

    # -- diagnostics -------------------------------------------------------------
    def local_rhs(self, x, y):
        xt = _dev_f32(x, (self.n_v, 3))
        yt = _dev_f32(y, (self.n_v, 3))
        b = torch.empty((self.n_v, 3), device="cuda", dtype=torch.float32)
        _check(lib().pd_local_rhs(self._h, _ptr(xt), _ptr(yt), _ptr(b)), "pd_local_rhs")
        return b

    def solve(self, r):
        rt = _dev_f32(r, (self.n_v, 3))
        x = torch.empty((self.n_v, 3), device="cuda", dtype=torch.float32)
        _check(lib().pd_solve(self._h, _ptr(rt), _ptr(x)), "pd_solve")
        return x

    def solve_noalloc(self, r, x):
        """pd_solve without any device allocation inside the call: r and x are
        caller-owned device tensors (n_v, 3) float32; the library's temporaries
        come from its fixed 16 MiB static scratch."""
        _check(lib().pd_solve_noalloc(self._h, _ptr(r), _ptr(x)), "pd_solve_noalloc")
        return x

    def enable_timing(self, mask=-1, iteration=-1):
        """Phase events for the kernel classes in `mask` (-1: all); the loop
        phases only in PD iteration `iteration` of each frame (-1: every one)."""
        _check(lib().pd_enable_timing(self._h, int(mask)), "pd_enable_timing")
        _check(lib().pd_set_timing_iteration(self._h, int(iteration)), "pd_set_timing_iteration")

    def phase_times(self) -> dict:
        out = (C.c_float * 24)()
        n = C.c_int32()
        _check(lib().pd_phase_times(self._h, out, 24, C.byref(n)), "pd_phase_times")
        return {lib().pd_phase_name(k).decode(): float(out[k]) for k in range(n.value)}

    def test_offset_phase_counter(self, phase, delta):
        """Testing hook: makes the next streaming solve's wait on `phase` run out."""
        _check(lib().pd_test_offset_phase_counter(self._h, int(phase), int(delta)), "pd_test_offset_phase_counter")

    def test_inflate_copy(self, nbytes):
        """Test hook: make the next tile stream's bounded wait run out (see include/pd.h)."""
        _check(lib().pd_test_inflate_copy(self._h, int(nbytes)), "pd_test_inflate_copy")


class Adjoint:
    """Workspace for equilibrium steps and backward adjoint steps on one mesh."""

    def __init__(self, mesh: Mesh, cg_iters=30):
        self.mesh = mesh
        h = C.c_void_p()
        _check(lib().pd_adjoint_create(mesh._h, int(cg_iters), C.byref(h)), "pd_adjoint_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pd_adjoint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(lib().pd_adjoint_reset(self._h), "pd_adjoint_reset")

    def equilibrium_step(self, pin_targets=None, gravity=(0.0, 0.0, -9.81), n_pd_iter=10, n_newton=3, x_out=None):
        m = self.mesh
        pt = _dev_f32(pin_targets, (m.n_pinned, 3)) if pin_targets is not None else None
        g = (C.c_float * 3)(*[float(a) for a in gravity])
        _check(lib().pd_equilibrium_step(m._h, self._h, _ptr(pt), g, int(n_pd_iter), int(n_newton), _ptr(x_out)),
               "pd_equilibrium_step")
        m._keep["pins"] = pt
        return x_out

    def step(self, x_n, dL_dx, dL_dgs, dL_dgv):
        """One backward step; dL_dgs / dL_dgv (n_t float32 device) are accumulated."""
        m = self.mesh
        xt = _dev_f32(x_n, (m.n_v, 3))
        gt = _dev_f32(dL_dx, (m.n_v, 3))
        _check(lib().pd_adjoint_step(m._h, self._h, _ptr(xt), _ptr(gt), _ptr(dL_dgs), _ptr(dL_dgv)),
               "pd_adjoint_step")
        m._keep["adj"] = (xt, gt)

    def step64(self, x_n, dL_dx, dL_dgs, dL_dgv):
        """pd_adjoint_step64: one backward step at an FP64 state x_n (n_v, 3) float64 on the device."""
        m = self.mesh
        xt = x_n.to(device="cuda", dtype=torch.float64).contiguous()
        gt = _dev_f32(dL_dx, (m.n_v, 3))
        _check(lib().pd_adjoint_step64(m._h, self._h, _ptr(xt), _ptr(gt), _ptr(dL_dgs), _ptr(dL_dgv)),
               "pd_adjoint_step64")
        m._keep["adj"] = (xt, gt)

    def get_state64(self):
        """(x, v) of the FP64 equilibrium state, (n_v, 3) float64 device tensors."""
        m = self.mesh
        x = torch.empty((m.n_v, 3), device="cuda", dtype=torch.float64)
        v = torch.empty((m.n_v, 3), device="cuda", dtype=torch.float64)
        _check(lib().pd_adjoint_get_state64(self._h, _ptr(x), _ptr(v)), "pd_adjoint_get_state64")
        return x, v

    def set_state64(self, x, v):
        m = self.mesh
        xt = x.to(device="cuda", dtype=torch.float64).contiguous()
        vt = v.to(device="cuda", dtype=torch.float64).contiguous()
        _check(lib().pd_adjoint_set_state64(self._h, _ptr(xt), _ptr(vt)), "pd_adjoint_set_state64")
        m._keep["state64"] = (xt, vt)

    def hessian_vec(self, x, v):
        m = self.mesh
        out = torch.empty((m.n_v, 3), device="cuda", dtype=torch.float32)
        xt, vt = _dev_f32(x, (m.n_v, 3)), _dev_f32(v, (m.n_v, 3))   # held until the call returns
        _check(lib().pd_hessian_vec(m._h, _ptr(xt), _ptr(vt), _ptr(out)), "pd_hessian_vec")
        return out

    def residual(self, x, x_prev, v_prev, gravity=(0.0, 0.0, -9.81)):
        m = self.mesh
        out = torch.empty((m.n_v, 3), device="cuda", dtype=torch.float32)
        g = (C.c_float * 3)(*[float(a) for a in gravity])
        xt, xpt, vpt = (_dev_f32(t, (m.n_v, 3)) for t in (x, x_prev, v_prev))   # held until the call returns
        _check(lib().pd_residual(m._h, _ptr(xt), _ptr(xpt), _ptr(vpt), g, _ptr(out)), "pd_residual")
        return out


    # ---- material fitting (Sec. 6.2, 6.3) ----------------------------------------------
    def pose_misfit(self, x, target, with_grad=True):
        """(loss tensor (1,) float64 on the device, dL/dx or None)."""
        m = self.mesh
        xt, tt = _dev_f32(x, (m.n_v, 3)), _dev_f32(target, (m.n_v, 3))
        loss = torch.empty(1, device="cuda", dtype=torch.float64)
        g = torch.empty((m.n_v, 3), device="cuda", dtype=torch.float32) if with_grad else None
        _check(lib().pd_pose_misfit(m._h, _ptr(xt), _ptr(tt), _ptr(g), _ptr(loss)), "pd_pose_misfit")
        return loss, g

    def pose_misfit_accumulate(self, x, target, loss, dl=None):
        """loss (device float64, shape (1,)) += sum_free ||x - target||^2; dl (or None) <- 2 (x - target)."""
        m = self.mesh
        xt, tt = _dev_f32(x, (m.n_v, 3)), _dev_f32(target, (m.n_v, 3))
        _check(lib().pd_pose_misfit_accumulate(m._h, _ptr(xt), _ptr(tt), _ptr(dl), _ptr(loss)),
               "pd_pose_misfit_accumulate")
        return loss

    def tied_gradient(self, gs, gv, ratio, scale=None):
        """dL/dtheta = scale (dL/dgamma_s + ratio dL/dgamma_v) for gamma_s = theta, gamma_v = ratio theta;
        scale is a device float64 tensor of one element or None."""
        m = self.mesh
        out = torch.empty(m.n_t, device="cuda", dtype=torch.float32)
        sc = None if scale is None else scale.to(device="cuda", dtype=torch.float64).reshape(1).contiguous()
        _check(lib().pd_tied_gradient(m._h, _ptr(gs), _ptr(gv), float(ratio), _ptr(sc), _ptr(out)),
               "pd_tied_gradient")
        return out

    def gn_product(self, x, v, active=None, g_scale=2.0):
        m = self.mesh
        xt = _dev_f32(x, (m.n_v, 3))
        vt = _dev_f32(v, (2 * m.n_t,))
        at = None if active is None else torch.as_tensor(active).to(device="cuda", dtype=torch.uint8).contiguous()
        out = torch.empty(2 * m.n_t, device="cuda", dtype=torch.float32)
        _check(lib().pd_gn_product(m._h, self._h, _ptr(xt), _ptr(vt), _ptr(at), float(g_scale), _ptr(out)),
               "pd_gn_product")
        torch.cuda.synchronize()          # inputs converted here are held until the work is done
        return out

    def gn_direction(self, x, grad, active=None, kappa_rel=1e-2, outer_iters=50, g_scale=2.0):
        """(d, kappa) of (P + kappa I) d = -grad."""
        m = self.mesh
        xt = _dev_f32(x, (m.n_v, 3))
        gt = _dev_f32(grad, (2 * m.n_t,))
        at = None if active is None else torch.as_tensor(active).to(device="cuda", dtype=torch.uint8).contiguous()
        d = torch.empty(2 * m.n_t, device="cuda", dtype=torch.float32)
        kap = torch.empty(1, device="cuda", dtype=torch.float64)
        _check(lib().pd_gn_direction(m._h, self._h, _ptr(xt), _ptr(gt), _ptr(at), float(kappa_rel), float(g_scale),
                                     int(outer_iters), _ptr(d), _ptr(kap)), "pd_gn_direction")
        torch.cuda.synchronize()
        return d, kap

    def fit_pose(self, x_prev, v_prev, target, gamma, pin_targets=None, gravity=(0.0, 0.0, -9.81), n_gd=2, n_gn=3,
                 gd_step=0.01, gn_step=1.0, kappa_rel=1e-2, floor=1e-3, max_halvings=12, max_pivots=8,
                 n_pd_iter=30, n_newton=4, outer_iters=50, dt=None, **solver):
        """Two-stage fit of one pose; gamma = [gamma_s | gamma_v] (2 n_t).  Returns
        (gamma tensor, losses array, report dict).  `solver` holds the prefactor
        options used after each material change."""
        m = self.mesh
        if dt is None and m.dt is None:
            raise ValueError("fit_pose needs dt (or a prefactored mesh)")
        xp, vp, tg = (_dev_f32(t, (m.n_v, 3)) for t in (x_prev, v_prev, target))
        pt = _dev_f32(pin_targets, (m.n_pinned, 3)) if pin_targets is not None else None
        gm = _dev_f32(gamma, (2 * m.n_t,)).clone()
        so = m.solver_opts(**solver)
        o = _lib.pd_fit_opts(int(n_gd), int(n_gn), float(gd_step), float(gn_step), float(kappa_rel), float(floor),
                             int(max_halvings), int(max_pivots), int(n_pd_iter), int(n_newton), int(outer_iters),
                             float(dt if dt is not None else m.dt), C.pointer(so))
        losses = np.zeros(int(n_gd) + int(n_gn) + 1, np.float64)
        rep = _lib.pd_fit_report()
        g = (C.c_float * 3)(*[float(a) for a in gravity])
        _check(lib().pd_fit_pose(m._h, self._h, C.byref(o), _ptr(xp), _ptr(vp), _ptr(pt), g, _ptr(tg), _ptr(gm),
                                 losses.ctypes.data_as(C.c_void_p), C.byref(rep)), "pd_fit_pose")
        info = {k: getattr(rep, k) for k, _ in _lib.pd_fit_report._fields_}
        return gm, losses, info


    def harmonic_basis(self, r):
        """(H (r, n_t) float32 on the device: row k = h_{k+1}, lambdas (r,), iterations)."""
        m = self.mesh
        H = torch.empty((int(r), m.n_t), device="cuda", dtype=torch.float32)
        lam = np.zeros(int(r), np.float64)
        it = C.c_int32(0)
        _check(lib().pd_harmonic_basis(m._h, int(r), _ptr(H), lam.ctypes.data_as(C.c_void_p), C.byref(it)),
               "pd_harmonic_basis")
        return H, lam, int(it.value)

    def fit_pose_reduced(self, H, x_prev, v_prev, target, gamma, pin_targets=None, gravity=(0.0, 0.0, -9.81),
                         n_gn=3, gn_step=1.0, kappa_rel=1e-2, floor=1e-3, max_halvings=12, n_pd_iter=30, n_newton=4,
                         dt=None, **solver):
        """Gauss-Newton in gamma = diag(H, H) q; H (r, n_t) as from harmonic_basis.
        Returns (gamma tensor, losses array, report dict)."""
        m = self.mesh
        if dt is None and m.dt is None:
            raise ValueError("fit_pose_reduced needs dt (or a prefactored mesh)")
        Ht = _dev_f32(H).contiguous()
        r = int(Ht.shape[0])
        xp, vp, tg = (_dev_f32(t, (m.n_v, 3)) for t in (x_prev, v_prev, target))
        pt = _dev_f32(pin_targets, (m.n_pinned, 3)) if pin_targets is not None else None
        gm = _dev_f32(gamma, (2 * m.n_t,)).clone()
        so = m.solver_opts(**solver)
        o = _lib.pd_fit_opts(0, int(n_gn), 0.01, float(gn_step), float(kappa_rel), float(floor), int(max_halvings), 0,
                             int(n_pd_iter), int(n_newton), 1, float(dt if dt is not None else m.dt), C.pointer(so))
        losses = np.zeros(int(n_gn) + 1, np.float64)
        rep = _lib.pd_fit_report()
        g = (C.c_float * 3)(*[float(a) for a in gravity])
        _check(lib().pd_fit_pose_reduced(m._h, self._h, C.byref(o), _ptr(Ht), r, _ptr(xp), _ptr(vp), _ptr(pt), g,
                                         _ptr(tg), _ptr(gm), losses.ctypes.data_as(C.c_void_p), C.byref(rep)),
               "pd_fit_pose_reduced")
        info = {k: getattr(rep, k) for k, _ in _lib.pd_fit_report._fields_}
        return gm, losses, info

    def harmonic_initialization(self, x_prev, v_prev, target, gamma, ranks=(1, 10, 30), n_gn=3, **kw):
        """Rank by rank (Sec. 6, Harmonic Initialization): the basis of the largest
        rank once, then Gauss-Newton in its leading r columns for each r.
        Returns (gamma, [(r, losses), ...])."""
        H, _, _ = self.harmonic_basis(max(ranks))
        out = []
        g = gamma
        for r in ranks:
            g, losses, _ = self.fit_pose_reduced(H[:r], x_prev, v_prev, target, g, n_gn=n_gn, **kw)
            out.append((r, losses))
        return g, out


class Server:
    """Serving loop: resident garment simulations advanced in shared batched launches."""

    def __init__(self, hbm_budget_bytes, max_slots=64, n_iter=20, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().pd_server_create(int(hbm_budget_bytes), int(max_slots), int(n_iter),
                                      C.c_void_p(self.stream.cuda_stream), C.byref(h)), "pd_server_create")
        self._h = h
        self._nv = {}
        self._nf = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().pd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, w, n_frames, drive=None):
        """Queue a Workload-like object (rest, tets, tet_domain, n_domains, pinned, gamma_s, gamma_v,
        density, dt, gravity); drive = (amp, freq, axis) of the pinned vertices or None."""
        rest = np.ascontiguousarray(w.rest, np.float64)
        tets = np.ascontiguousarray(w.tets, np.int32)
        dom = np.ascontiguousarray(w.tet_domain, np.int32)
        pin = np.ascontiguousarray(w.pinned, np.uint8)
        gs = np.ascontiguousarray(w.gamma_s, np.float32)
        gv = np.ascontiguousarray(w.gamma_v, np.float32)
        amp, freq, axis = drive if drive is not None else (0.0, 0.0, 0)
        q = _lib.pd_request(rest.ctypes.data, rest.shape[0], tets.ctypes.data, tets.shape[0], dom.ctypes.data,
                            int(w.n_domains), pin.ctypes.data, gs.ctypes.data, gv.ctypes.data, float(w.density),
                            float(w.dt), int(n_frames), (C.c_float * 3)(*w.gravity), float(amp), float(freq),
                            int(axis))
        rid = C.c_int64()
        _check(lib().pd_submit(self._h, C.byref(q), C.byref(rid)), "pd_submit")
        self._nv[rid.value] = rest.shape[0]
        self._nf[rid.value] = int(n_frames)
        return rid.value

    def tick(self):
        n = C.c_int32()
        ms = C.c_float()
        _check(lib().pd_server_tick(self._h, C.byref(n), C.byref(ms)), "pd_server_tick")
        return n.value, ms.value

    def run(self, max_ticks=100000):
        """Tick until no request is queued or resident; returns the ticks run."""
        t = C.c_int32()
        _check(lib().pd_server_run(self._h, int(max_ticks), C.byref(t)), "pd_server_run")
        return t.value

    def poll(self, rid):
        st, fd = C.c_int32(), C.c_int32()
        _check(lib().pd_poll(self._h, int(rid), C.byref(st), C.byref(fd)), "pd_poll")
        return st.value, fd.value

    def fetch(self, rid):
        x = np.empty((self._nv[rid], 3), np.float32)
        ms = np.empty(self._nf[rid], np.float32)
        _check(lib().pd_fetch(self._h, int(rid), x.ctypes.data, ms.ctypes.data), "pd_fetch")
        return x, ms

    def stats(self):
        q, a, u, pk = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().pd_server_stats(self._h, C.byref(q), C.byref(a), C.byref(u), C.byref(pk)), "pd_server_stats")
        return {"queued": q.value, "active": a.value, "used_bytes": u.value, "peak_bytes": pk.value}


def project(F: torch.Tensor, with_sigma=True):
    """Rotation and volume targets of a batch of deformation gradients (n, 3, 3)."""
    F = F.to(device="cuda", dtype=torch.float32).contiguous()
    n = F.shape[0]
    R = torch.empty_like(F)
    V = torch.empty_like(F)
    s = torch.empty((n, 3), device="cuda", dtype=torch.float32) if with_sigma else None
    _check(lib().pd_project(_ptr(F), n, _ptr(R), _ptr(V), _ptr(s), C.c_void_p(torch.cuda.current_stream().cuda_stream)),
           "pd_project")
    return R, V, s


PHASES = ["inertia", "local", "assemble", "dd_condense", "dd_gather", "dd_coarse", "dd_reduce", "dd_backsub",
          "residual", "velocity", "dd_condense2", "dd_gather2", "dd_backsub2", "dd_interior", "dd_interior2",
          "dd_solve", "dd_modal", "dd_jacobi"]


def phase_bit(name: str) -> int:
    return 1 << PHASES.index(name)
