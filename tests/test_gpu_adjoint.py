"""GPU adjoint (Sec. 6.1) against the FP64 adjoint oracle.

Hessian-vector products, the equilibrium residual and equilibrium steps
are compared with the oracle; the gradient of the pose loss with respect to
every per-element parameter is compared with the oracle's adjoint gradient
(itself pinned against central finite differences on the CPU), and the
checkpointed backward pass with one that keeps every step.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import f32, rel  # noqa: E402

from oracle.adjoint import AdjointOracle  # noqa: E402
from oracle.pd_oracle import PDOracle  # noqa: E402
from workloads.meshes import adjoint_slab, slab_workload  # noqa: E402

# measurement records go to $PD_RECORD_DIR when it is set (nothing is written otherwise)
OUT = os.environ.get("PD_RECORD_DIR")


def _record(name, payload):
    if not OUT:
        return
    try:
        os.makedirs(OUT, exist_ok=True)
        with open(os.path.join(OUT, f"adjoint_{name}.json"), "w") as f:
            json.dump(payload, f, indent=1)
    except OSError:
        pass


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _small():
    return slab_workload(6, 6, 2, 0.01, 5, (2, 2), seed=3, n_iter=10, name="adj-small")


GRAVITY32 = tuple(float(np.float32(g)) for g in (0.0, 0.0, -9.81))


def _oracle(w, gs, gv):
    """The FP64 adjoint oracle given the FP32 values the library is given (materials, gravity)."""
    return AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(gs), f32(gv), w.density, w.dt), gravity=GRAVITY32)


def _pins32(w):
    return lambda n: f32(w.pin_targets(n))


def _pair(w, cg_iters=40):
    from paper_2405_12484_gb300.sim import Adjoint, Mesh
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt)
    a = Adjoint(m, cg_iters)
    return m, a, _oracle(w, w.gamma_s, w.gamma_v)


def _deformed(w, rng):
    x = w.rest.copy()
    L = w.rest[:, 1].max()
    x[:, 2] -= 0.03 * (w.rest[:, 1] / L - 1.0) ** 2
    x += 3e-4 * rng.standard_normal(x.shape)
    x[w.pinned.astype(bool)] = w.rest[w.pinned.astype(bool)]
    return x


def test_hessian_vector_product_matches_oracle():
    w = _small()
    m, a, o = _pair(w)
    rng = np.random.default_rng(11)
    x = _deformed(w, rng).astype(np.float32)
    v = rng.standard_normal(x.shape).astype(np.float32)
    v[w.pinned.astype(bool)] = 0.0
    hv = a.hessian_vec(torch.as_tensor(x), torch.as_tensor(v)).cpu().numpy()
    H = o.hessian(x.astype(np.float64))
    ref = np.zeros_like(x, dtype=np.float64)
    ref[o.o.free] = (H @ v.astype(np.float64)[o.o.free].ravel()).reshape(-1, 3)
    e = rel(hv, ref)
    _record("hvp", {"rel_err": e})
    assert e < 1e-4


def test_residual_matches_oracle():
    w = _small()
    m, a, o = _pair(w)
    rng = np.random.default_rng(12)
    xp = _deformed(w, rng)
    vp = 0.05 * rng.standard_normal(xp.shape)
    vp[w.pinned.astype(bool)] = 0
    x = xp + w.dt * vp + 1e-4 * rng.standard_normal(xp.shape)
    x[w.pinned.astype(bool)] = xp[w.pinned.astype(bool)]
    x32, xp32, vp32 = (t.astype(np.float32) for t in (x, xp, vp))
    g = a.residual(torch.as_tensor(x32), torch.as_tensor(xp32), torch.as_tensor(vp32), w.gravity).cpu().numpy()
    y = o.o.inertial_target(xp32.astype(np.float64), vp32.astype(np.float64), w.gravity)
    ref = o.residual(x32.astype(np.float64), y)
    ref[w.pinned.astype(bool)] = 0.0
    e = rel(g, ref)
    _record("residual", {"rel_err": e})
    assert e < 1e-3     # g is a difference of O(M x / dt^2) terms: FP32 cancellation bounds it


def test_equilibrium_steps_match_oracle():
    """Equilibrium steps (PD, then Newton with an FP64 residual at the FP64
    state) against the oracle's equilibria from the same FP32 inputs: the
    FP64 state matches to 1e-9 of the displacement, its FP32 rounding to
    FP32 rounding."""
    w = _small()
    m, a, o = _pair(w)
    x0 = f32(w.rest)
    xs, vs = o.forward(x0, np.zeros_like(x0), _pins32(w), 3)
    x = torch.empty((w.n_v, 3), device="cuda")
    errs, disp64, vel64 = [], [], []
    for n in range(3):
        a.equilibrium_step(torch.as_tensor(w.pin_targets(n), dtype=torch.float32), w.gravity, 10, 4, x_out=x)
        x64, v64 = (t.cpu().numpy() for t in a.get_state64())
        errs.append(rel(x.cpu().numpy(), xs[n + 1]))
        disp64.append(float(np.linalg.norm(x64 - xs[n + 1]) / np.linalg.norm(xs[n + 1] - x0)))
        vel64.append(rel(v64, vs[n + 1]))
    _record("equilibrium", {"e_n": errs, "e_disp64": disp64, "e_vel64": vel64})
    assert max(errs) < 1e-7
    assert max(disp64) < 1e-9
    assert max(vel64) < 1e-9


def _targets(w, n_steps, seed):
    """Target poses: the oracle's trajectory under other seeded materials, rounded to FP32 (both sides get these)."""
    w2 = slab_workload(*w.meta["cubes"], w.meta["h"], w.meta["tets_per_cube"], (2, 2), seed=seed, n_iter=10,
                       name="target")
    At = _oracle(w, w2.gamma_s, w2.gamma_v)
    x0 = f32(w.rest)
    tg, _ = At.forward(x0, np.zeros_like(x0), _pins32(w), n_steps)
    return [f32(t) for t in tg]


def _gpu_gradient(w, n_steps, targets, cg_iters, **kw):
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets, n_steps,
                  n_pd_iter=10, n_newton=4, cg_iters=cg_iters, **kw)
    theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
    L = pose_loss(theta, sim, targets)
    L.backward()
    g = theta.grad.detach().cpu().numpy().astype(np.float64)
    # the forward trajectory (FP64 states), for isolating the backward pass
    sim.adj.set_state64(sim.x0.double(), sim.v0.double())
    xs = [f32(w.rest)]
    x = torch.empty((w.n_v, 3), device="cuda")
    for n in range(n_steps):
        sim.adj.equilibrium_step(sim._pin(n), w.gravity, 10, 4, x_out=x)
        xs.append(sim.adj.get_state64()[0].cpu().numpy())
    sim.adj.close()
    sim.mesh.close()
    return g, xs


def test_adjoint_gradient_matches_oracle_and_checkpointing_is_exact():
    w = _small()
    n_steps = 5
    tg = _targets(w, n_steps, seed=4)
    o = _oracle(w, w.gamma_s, w.gamma_v)
    x0 = f32(w.rest)
    xs, _ = o.forward(x0, np.zeros_like(x0), _pins32(w), n_steps)
    gs_o, gv_o = o.gradient(xs, tg)
    g_or = gs_o + 10.0 * gv_o
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    res = {}
    g2, _ = _gpu_gradient(w, n_steps, targets, 60, checkpoint_every=2)
    g_store, xs_gpu = _gpu_gradient(w, n_steps, targets, 60, store_all=True)
    g_more, _ = _gpu_gradient(w, n_steps, targets, 150, store_all=True)
    # oracle backward pass on the GPU's forward trajectory: separates forward and backward errors
    gs_x, gv_x = o.gradient(xs_gpu, tg)
    g_or_on_gpu_traj = gs_x + 10.0 * gv_x
    res["rel_err_cg60"] = rel(g_store, g_or)
    res["rel_err_cg150"] = rel(g_more, g_or)
    res["rel_err_backward_only_cg60"] = rel(g_store, g_or_on_gpu_traj)
    res["rel_err_forward_only"] = rel(g_or_on_gpu_traj, g_or)
    res["traj_rel_err"] = max(rel(xs_gpu[n], xs[n]) for n in range(1, n_steps + 1))
    _record("gradient_small", res)
    assert np.array_equal(g2, g_store)
    assert res["rel_err_cg60"] < 1e-4, res
    assert res["rel_err_cg150"] < 1e-4, res


def test_adjoint_gradient_mid_slab():
    """An 8,000-tet slab (20x20x4 cubes x 5 tets, 8,000 parameters), 2 equilibrium
    steps, GPU adjoint against the oracle adjoint."""
    w = slab_workload(20, 20, 4, 0.01, 5, (4, 4), seed=1, n_iter=10, name="adj-mid")
    n_steps = 2
    tg = _targets(w, n_steps, seed=5)
    o = _oracle(w, w.gamma_s, w.gamma_v)
    x0 = f32(w.rest)
    xs, _ = o.forward(x0, np.zeros_like(x0), _pins32(w), n_steps, pd_iters=10)
    gs_o, gv_o = o.gradient(xs, tg)
    g_or = gs_o + 10.0 * gv_o
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    g, _ = _gpu_gradient(w, n_steps, targets, 150, checkpoint_every=1)
    idx = np.random.default_rng(7).choice(w.n_t, 20, replace=False)
    e = rel(g, g_or)
    e_inf = float(np.abs(g - g_or).max() / np.abs(g_or).max())
    _record("gradient_mid_slab", {"rel_err_norm": e, "rel_err_inf": e_inf, "n_t": int(w.n_t), "steps": n_steps,
                                  "sampled": {int(i): [float(g[i]), float(g_or[i])] for i in idx}})
    assert e < 1e-4
    assert e_inf < 1e-4


def test_adjoint_full_slab_runs_and_checkpoints_exactly():
    """The 50,000-tet, 50x50x4 slab with 50K parameters over 30 steps with a
    checkpoint every 10 steps: the checkpointed gradient equals the one that keeps
    every step (forward and backward wall times are recorded)."""
    import time
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    w = adjoint_slab()
    n_steps = 30
    out = {}
    grads = {}
    for mode, kw in (("ckpt10", dict(checkpoint_every=10)), ("store", dict(store_all=True))):
        sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets, n_steps,
                      n_pd_iter=10, n_newton=3, cg_iters=60, **kw)
        # targets: the rest shape (the loss measures the sag of the slab)
        targets = [torch.as_tensor(w.rest, dtype=torch.float32, device="cuda")] * (n_steps + 1)
        theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = pose_loss(theta, sim, targets)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        grads[mode] = theta.grad.detach().cpu().numpy()
        out[mode] = {"forward_s": t1 - t0, "backward_s": t2 - t1, "loss": float(L)}
        sim.adj.close()
        sim.mesh.close()
    _record("full_slab", out)
    assert np.all(np.isfinite(grads["store"]))
    assert np.array_equal(grads["ckpt10"], grads["store"])


GOLDEN_50K = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "adjoint_slab50k_30steps.json")


def _loss64(sim, gs, gv, targets64, free, n_steps):
    """L = sum_n sum_free |x_n - xhat_n|^2 from the FP64 equilibrium states (for finite differences)."""
    m, a = sim.mesh, sim.adj
    m.set_materials(gs, gv)
    m.prefactor(sim.dt)
    a.set_state64(sim.x0.double(), sim.v0.double())
    L = torch.zeros((), dtype=torch.float64, device="cuda")
    for n in range(n_steps):
        a.equilibrium_step(sim._pin(n), sim.gravity, sim.n_pd, sim.n_newton)
        d = (a.get_state64()[0] - targets64[n + 1])[free]
        L += (d * d).sum()
    return float(L)


def test_adjoint_config4_against_oracle_and_finite_differences():
    """The 50,000-tet slab (50K stiffness parameters), 30 equilibrium steps,
    a checkpoint every 10 steps: the GPU adjoint gradient against the FP64
    oracle's adjoint gradient (tests/golden, written by a script that calls
    only oracle/) and against central finite differences of the loss of the
    FP64 GPU states, on the 20 parameters drawn with seed 7.  Error measure:
    max over the sample of |g - g_ref| / max over the sample of |g_ref|."""
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    from workloads.meshes import target_trajectory
    with open(GOLDEN_50K) as f:
        gold = json.load(f)
    w = adjoint_slab()
    N = gold["config"]["steps"]
    tg = [f32(t) for t in target_trajectory(w.rest, N, gold["config"]["target_seed"])]
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets, N,
                  n_pd_iter=10, n_newton=4, cg_iters=60, checkpoint_every=10)
    theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
    L = pose_loss(theta, sim, targets)
    L.backward()
    g = theta.grad.detach().cpu().numpy().astype(np.float64)
    idx = np.asarray(gold["indices"])
    g_or = np.asarray(gold["dL_dtheta"])
    e_oracle = float(np.abs(g[idx] - g_or).max() / np.abs(g_or).max())
    e_loss = abs(float(L.detach()) - gold["loss"]) / gold["loss"]
    # the two parameter blocks separately (gamma_v = 10 theta), against the oracle and by central differences
    loss, ckpts, stored = sim.forward(theta.detach(), targets)
    gs_t, gv_t = sim.backward(ckpts, stored, targets)
    gs, gv = (t.cpu().numpy().astype(np.float64) for t in (gs_t, gv_t))
    e_oracle_s = float(np.abs(gs[idx] - gold["dL_dgamma_s"]).max() / np.abs(gold["dL_dgamma_s"]).max())
    e_oracle_v = float(np.abs(gv[idx] - gold["dL_dgamma_v"]).max() / np.abs(gold["dL_dgamma_v"]).max())
    free = torch.as_tensor(~w.pinned.astype(bool), device="cuda")
    targets64 = [torch.as_tensor(t, dtype=torch.float64, device="cuda") for t in tg]
    th32 = np.asarray(w.gamma_s, np.float32)
    gs0, gv0 = th32.copy(), th32 * np.float32(10.0)
    fd_s, fd_v = [], []
    for i in idx:
        for base, other, out in ((gs0, gv0, fd_s), (gv0, gs0, fd_v)):
            h = np.float32(2.0 ** np.round(np.log2(1e-3 * float(base[i]))))   # exact in float32 around base[i]
            lp, lm = base.copy(), base.copy()
            lp[i] += h
            lm[i] -= h
            if base is gs0:
                Lp = _loss64(sim, lp, other, targets64, free, N)
                Lm = _loss64(sim, lm, other, targets64, free, N)
            else:
                Lp = _loss64(sim, other, lp, targets64, free, N)
                Lm = _loss64(sim, other, lm, targets64, free, N)
            out.append((Lp - Lm) / (float(lp[i]) - float(lm[i])))
    fd_s, fd_v = np.asarray(fd_s), np.asarray(fd_v)
    e_fd_s = float(np.abs(gs[idx] - fd_s).max() / np.abs(fd_s).max())
    e_fd_v = float(np.abs(gv[idx] - fd_v).max() / np.abs(fd_v).max())
    fd_theta = fd_s + 10.0 * fd_v
    e_fd = float(np.abs(g[idx] - fd_theta).max() / np.abs(fd_theta).max())
    rec = {"e_oracle_theta": e_oracle, "e_oracle_gamma_s": e_oracle_s, "e_oracle_gamma_v": e_oracle_v,
           "e_fd_theta": e_fd, "e_fd_gamma_s": e_fd_s, "e_fd_gamma_v": e_fd_v, "e_loss": e_loss,
           "per_param": {int(i): {"gpu": float(g[i]), "oracle": float(o), "fd": float(f)}
                         for i, o, f in zip(idx, g_or, fd_theta)}}
    _record("config4_50k", rec)
    sim.adj.close()
    sim.mesh.close()
    assert e_loss < 1e-6, rec
    for k in ("e_oracle_theta", "e_oracle_gamma_s", "e_oracle_gamma_v", "e_fd_theta", "e_fd_gamma_s", "e_fd_gamma_v"):
        assert rec[k] < 1e-4, (k, rec)
