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


def _pair(w, cg_iters=40):
    from paper_2405_12484_gb300.sim import Adjoint, Mesh
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt)
    a = Adjoint(m, cg_iters)
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt))
    return m, a, o


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
    w = _small()
    m, a, o = _pair(w)
    xs, vs = o.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, 3)
    x = torch.empty((w.n_v, 3), device="cuda")
    errs = []
    for n in range(3):
        a.equilibrium_step(torch.as_tensor(w.pin_targets(n), dtype=torch.float32), w.gravity, 10, 4, x_out=x)
        m.sync()
        errs.append(rel(x.cpu().numpy(), xs[n + 1]))
    disp = [float(np.linalg.norm(x.cpu().numpy() - xs[3]) / np.linalg.norm(xs[3] - w.rest))]
    _record("equilibrium", {"e_n": errs, "e_disp_last": disp})
    assert max(errs) < 1e-5


def _targets(w, n_steps, seed):
    w2 = slab_workload(*w.meta["cubes"], w.meta["h"], w.meta["tets_per_cube"], (2, 2), seed=seed, n_iter=10,
                       name="target")
    At = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w2.gamma_s), f32(w2.gamma_v), w.density, w.dt))
    tg, _ = At.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
    return tg


def _gpu_gradient(w, n_steps, targets, cg_iters, **kw):
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets, n_steps,
                  n_pd_iter=10, n_newton=4, cg_iters=cg_iters, **kw)
    theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
    L = pose_loss(theta, sim, targets)
    L.backward()
    g = theta.grad.detach().cpu().numpy().astype(np.float64)
    # the forward trajectory, for isolating the backward pass
    sim.mesh.set_state(sim.x0, sim.v0)
    xs = [w.rest.copy()]
    x = torch.empty((w.n_v, 3), device="cuda")
    for n in range(n_steps):
        sim.adj.equilibrium_step(sim._pin(n), w.gravity, 10, 4, x_out=x)
        xs.append(x.cpu().numpy().astype(np.float64))
    sim.adj.close()
    sim.mesh.close()
    return g, xs


def test_adjoint_gradient_matches_oracle_and_checkpointing_is_exact():
    w = _small()
    n_steps = 5
    tg = _targets(w, n_steps, seed=4)
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt))
    xs, _ = o.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
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
    assert min(res["rel_err_cg60"], res["rel_err_cg150"]) < 1e-4, res


def test_adjoint_gradient_mid_slab():
    """An 8,000-tet slab (20x20x4 cubes x 5 tets, 8,000 parameters), 2 equilibrium
    steps, GPU adjoint against the oracle adjoint."""
    w = slab_workload(20, 20, 4, 0.01, 5, (4, 4), seed=1, n_iter=10, name="adj-mid")
    n_steps = 2
    tg = _targets(w, n_steps, seed=5)
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt))
    xs, _ = o.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps, pd_iters=10)
    gs_o, gv_o = o.gradient(xs, tg)
    g_or = gs_o + 10.0 * gv_o
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    g, _ = _gpu_gradient(w, n_steps, targets, 150, checkpoint_every=1)
    idx = np.random.default_rng(7).choice(w.n_t, 20, replace=False)
    e = rel(g, g_or)
    _record("gradient_mid_slab", {"rel_err_norm": e, "n_t": int(w.n_t), "steps": n_steps,
                                  "sampled": {int(i): [float(g[i]), float(g_or[i])] for i in idx}})
    assert e < 1e-3


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
