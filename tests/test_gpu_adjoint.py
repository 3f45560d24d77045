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

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "gpurun_out")


def _record(name, payload):
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


def test_adjoint_gradient_matches_oracle_and_checkpointing_is_exact():
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    w = _small()
    n_steps = 5
    tg = _targets(w, n_steps, seed=4)
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt))
    xs, _ = o.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps)
    gs_o, gv_o = o.gradient(xs, tg)
    g_or = gs_o + 10.0 * gv_o
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    grads = {}
    for mode, kw in (("ckpt2", dict(checkpoint_every=2)), ("store", dict(store_all=True))):
        sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets,
                      n_steps, n_pd_iter=10, n_newton=4, cg_iters=40, **kw)
        theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
        L = pose_loss(theta, sim, targets)
        L.backward()
        grads[mode] = theta.grad.detach().cpu().numpy().astype(np.float64)
        sim.adj.close()
        sim.mesh.close()
    e = rel(grads["ckpt2"], g_or)
    idx = np.random.default_rng(7).choice(w.n_t, 20, replace=False)
    e_entries = np.abs(grads["ckpt2"][idx] - g_or[idx]) / np.abs(g_or).max()
    _record("gradient_small", {"rel_err_norm": e, "max_entry_err_over_max": float(e_entries.max()),
                               "n_t": int(w.n_t), "steps": n_steps})
    assert np.array_equal(grads["ckpt2"], grads["store"])
    assert e < 1e-4


def test_adjoint_gradient_full_slab_sampled():
    """The 50,000-tet, 50x50x4 slab with 50K parameters: GPU adjoint against the
    oracle adjoint over 2 equilibrium steps (20 sampled parameters reported)."""
    from paper_2405_12484_gb300.diff import DiffSim, pose_loss
    w = adjoint_slab()
    n_steps = 2
    w2 = adjoint_slab(seed=5)
    At = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w2.gamma_s), f32(w2.gamma_v), w.density, w.dt))
    tg, _ = At.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps, pd_iters=5)
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt))
    xs, _ = o.forward(w.rest, np.zeros_like(w.rest), w.pin_targets, n_steps, pd_iters=5)
    gs_o, gv_o = o.gradient(xs, tg)
    g_or = gs_o + 10.0 * gv_o
    targets = [torch.as_tensor(t, dtype=torch.float32, device="cuda") for t in tg]
    sim = DiffSim(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, w.dt, w.pin_targets, n_steps,
                  checkpoint_every=1, n_pd_iter=10, n_newton=4, cg_iters=40)
    theta = torch.as_tensor(w.gamma_s, dtype=torch.float32, device="cuda").requires_grad_(True)
    L = pose_loss(theta, sim, targets)
    L.backward()
    g = theta.grad.detach().cpu().numpy().astype(np.float64)
    idx = np.random.default_rng(7).choice(w.n_t, 20, replace=False)
    e = rel(g, g_or)
    _record("gradient_full_slab", {"rel_err_norm": e, "sampled": {int(i): [float(g[i]), float(g_or[i])] for i in idx},
                                   "n_t": int(w.n_t), "steps": n_steps})
    assert e < 1e-4
