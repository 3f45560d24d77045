"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance (FP32 path): per-step relative position error
e_n = ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-5 when the GPU is fed the
oracle's state at step n-1 (one-step error).  Local step and RHS assembly
are compared entry by entry; the subspace solve against the oracle's full
Cholesky solve.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import f32, make_pair, rel  # noqa: E402

from oracle.pd_oracle import deformation_gradient  # noqa: E402
from oracle.projections import project_both  # noqa: E402
from workloads.meshes import parity_slab, slab_workload, sweater_shell  # noqa: E402

# measurement records go to $PD_RECORD_DIR when it is set (nothing is written otherwise)
OUT = os.environ.get("PD_RECORD_DIR")


def _record(name, payload):
    if not OUT:
        return
    try:
        os.makedirs(OUT, exist_ok=True)
        with open(os.path.join(OUT, f"parity_{name}.json"), "w") as f:
            json.dump(payload, f, indent=1)
    except OSError:
        pass


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _rot(n, rng):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)


def test_projection_matches_oracle():
    from paper_2405_12484_gb300.sim import project
    rng = np.random.default_rng(3)
    n = 4000
    # singular values log-uniform in [0.2, 5], 20% inverted, random rotations on both sides
    s = np.sort(np.exp(rng.uniform(np.log(0.2), np.log(5.0), (n, 3))), axis=1)[:, ::-1].copy()
    s[rng.uniform(size=n) < 0.2, 2] *= -1
    U, W = _rot(n, rng), _rot(n, rng)
    F = (U * s[:, None, :]) @ np.swapaxes(W, 1, 2)
    F = np.concatenate([F, np.eye(3)[None] + 0.05 * rng.standard_normal((1000, 3, 3))])
    F32 = F.astype(np.float32)
    R, V, sg = project(torch.as_tensor(F32))
    R, V, sg = R.cpu().numpy(), V.cpu().numpy(), sg.cpu().numpy()
    Ro, Vo, Uo, so, Wo, do = project_both(F32.astype(np.float64))
    assert np.all(np.isfinite(R)) and np.all(np.isfinite(V))
    assert np.abs(sg - so).max() < 2e-5 * np.abs(so).max()
    # R is unique where sigma_2 + sigma_3 is not tiny
    ok = (so[:, 1] + so[:, 2]) > 0.05
    errR = np.abs(R - Ro)[ok].max()
    # V is unique; compare entries relative to the target scale
    scale = np.maximum(1.0, np.abs(do).max(axis=1))[:, None, None]
    errV = (np.abs(V - Vo) / scale).max()
    cost_g = np.sum((F - V) ** 2, axis=(1, 2))
    cost_o = np.sum((F - Vo) ** 2, axis=(1, 2))
    _record("projection", {"n": int(F.shape[0]), "max_abs_err_R": float(errR), "max_rel_err_V": float(errV),
                           "max_cost_excess": float(np.max(cost_g - cost_o))})
    assert errR < 5e-5
    assert errV < 5e-4
    assert np.all(cost_g <= cost_o * (1 + 1e-4) + 1e-5)
    assert np.abs(np.linalg.det(V.astype(np.float64)) - 1).max() < 1e-4


# the oracle's adversarial singular values (ties, inverted, huge stretch, clamp active)
ADVERSARIAL = [
    (1, 1, 1), (2, 2, 1), (100, 1, 1), (3, 1, 0.2), (1.1, 0.9, -0.3), (0.5, 0.5, 0.5),
    (5, 5, 5), (1.5, 1.5, 1.5), (1.0001, 1.0, 0.9999), (2, 1e-3, 1e-3), (1, 1, 0.0),
    (1, 1, -1), (0.02, 0.02, 0.02), (50, 50, 1e-4), (1.9, 1.8, 1.7), (3, 3, 0.5),
    (10, 0.5, 0.5), (0.3, 0.2, -0.1), (2.5, 0.4, 0.05), (8, 8, 8), (1.2, 1.2, -2.0),
]


def test_projection_adversarial_and_wide_range():
    """The local-step projections on the hard branches of the volume target:
    the oracle's 21 adversarial singular-value triples (each under 50 random
    rotation pairs), 10^4 triples log-uniform in [1e-3, 100] with 20 %
    inverted, and near-ties (relative gaps 1e-6 .. 1e-2).  Compared where the
    answer is unique: the signed singular values, the sorted volume targets
    and the optimal cost ||F - V||^2 (always), R where the polar factor is
    well conditioned; V must satisfy det V = 1 and targets >= 0.01."""
    from paper_2405_12484_gb300.sim import project
    rng = np.random.default_rng(31)
    sig = [np.repeat(np.array(ADVERSARIAL, float), 50, axis=0)]
    wide = np.sort(np.exp(rng.uniform(np.log(1e-3), np.log(100.0), (10000, 3))), axis=1)[:, ::-1].copy()
    wide[rng.uniform(size=10000) < 0.2, 2] *= -1
    sig.append(wide)
    base = np.exp(rng.uniform(np.log(0.05), np.log(20.0), (2000, 1)))
    gaps = 10.0 ** rng.uniform(-6, -2, (2000, 2))
    ties = np.concatenate([base, base * (1 - gaps[:, :1]), base * (1 - gaps[:, :1]) * (1 - gaps[:, 1:])], axis=1)
    ties[rng.uniform(size=2000) < 0.2, 2] *= -1
    sig.append(ties)
    s = np.concatenate(sig)
    n = s.shape[0]
    U, W = _rot(n, rng), _rot(n, rng)
    F32 = ((U * s[:, None, :]) @ np.swapaxes(W, 1, 2)).astype(np.float32)
    F = F32.astype(np.float64)
    R, V, sg = project(torch.as_tensor(F32))
    R, V, sg = (t.cpu().numpy().astype(np.float64) for t in (R, V, sg))
    Ro, Vo, Uo, so, Wo, do = project_both(F)
    assert np.all(np.isfinite(R)) and np.all(np.isfinite(V))
    smax = np.abs(so).max(axis=1)
    e_sig = float((np.abs(sg - so).max(axis=1) / smax).max())
    # targets of the GPU's V (its singular values), sorted, against the oracle's
    dv = np.sort(np.linalg.svd(V, compute_uv=False), axis=1)
    dor = np.sort(np.abs(do), axis=1)
    e_d = float((np.abs(dv - dor) / np.maximum(1.0, dor.max(axis=1, keepdims=True))).max())
    cost_g = np.sum((F - V) ** 2, axis=(1, 2))
    cost_o = np.sum((F - Vo) ** 2, axis=(1, 2))
    excess = (cost_g - cost_o) / np.maximum(cost_o, 1e-6 * smax ** 2)
    # R is unique where sigma_2 + sigma_3 > 0; FP32 error grows with kappa = sigma_1 / (sigma_2 + sigma_3)
    kappa = smax / np.maximum(so[:, 1] + so[:, 2], 1e-30)
    okR = kappa < 1e3
    e_R = float((np.abs(R - Ro).max(axis=(1, 2))[okR] / (2e-5 + 2e-6 * kappa[okR])).max())
    detV = np.linalg.det(V)
    _record("projection_adversarial", {"n": int(n), "max_rel_err_sigma": e_sig, "max_rel_err_targets": e_d,
                                       "max_rel_cost_excess": float(excess.max()),
                                       "max_R_err_over_bound": e_R, "max_det_V_err": float(np.abs(detV - 1).max())})
    assert e_sig < 2e-5
    assert e_d < 5e-4
    assert excess.max() < 3e-4      # FP32 rounding of V's entries, relative to a small optimal cost
    assert e_R < 1.0
    assert np.abs(detV - 1).max() < 1e-3
    assert dv.min() >= 0.01 * (1 - 1e-3)


def _deformed(w, rng, amp=0.02):
    X = w.rest
    x = X.copy()
    L = X[:, 1].max()
    th = 0.6 * X[:, 1] / L                      # bend about the x axis
    x[:, 1] = X[:, 1] * np.cos(th) - X[:, 2] * np.sin(th)
    x[:, 2] = X[:, 1] * np.sin(th) + X[:, 2] * np.cos(th) - amp * (X[:, 1] / L) ** 2
    x += 2e-4 * rng.standard_normal(x.shape)
    return x


def test_local_step_and_rhs_match_oracle():
    w = parity_slab()
    m, o = make_pair(w)
    rng = np.random.default_rng(4)
    x = _deformed(w, rng)
    y = x + 1e-3 * rng.standard_normal(x.shape)
    x32, y32 = x.astype(np.float32), y.astype(np.float32)
    b_gpu = m.local_rhs(torch.as_tensor(x32), torch.as_tensor(y32)).cpu().numpy()
    xd, yd = x32.astype(np.float64), y32.astype(np.float64)
    R, V = o.local(xd)
    b_or = o.rhs(yd, R, V)
    b_or[o.free] -= o.K_fp @ xd[o.pin_ids]
    b_or[o.pin_ids] = 0.0
    inertia = (o.mass / o.dt ** 2)[:, None] * yd
    inertia[o.pin_ids] = 0.0
    e_total = rel(b_gpu, b_or)
    e_elastic = rel(b_gpu[o.free] - inertia[o.free], b_or[o.free] - inertia[o.free])
    _record("local_rhs", {"rel_err_b": e_total, "rel_err_elastic_part": e_elastic})
    assert np.all(b_gpu[o.pin_ids] == 0.0)
    assert e_total < 1e-6
    assert e_elastic < 2e-5


def test_local_step_inverted_and_stretched_tets():
    """Local step and RHS on the parity slab with a 50x stretched band
    (x < 0.03 stretched 50x along x) and an inverted patch (z mirrored and
    halved about the mid-plane for 0.09 < x < 0.13, 0.05 < y < 0.11), so that
    the volume targets take the clamped and inverted branches."""
    w = parity_slab()
    m, o = make_pair(w)
    rng = np.random.default_rng(14)
    X = w.rest
    x = X.copy()
    band = X[:, 0] < 0.03
    x[band, 0] = 50.0 * X[band, 0]
    x[~band, 0] += 49.0 * 0.03
    patch = (X[:, 0] > 0.09) & (X[:, 0] < 0.13) & (X[:, 1] > 0.05) & (X[:, 1] < 0.11)
    zc = 0.5 * X[:, 2].max()
    x[patch, 2] = zc - 0.5 * (X[patch, 2] - zc)
    x += 1e-4 * rng.standard_normal(x.shape)
    x[o.pin_ids] = X[o.pin_ids]
    y = x + 1e-3 * rng.standard_normal(x.shape)
    x32, y32 = x.astype(np.float32), y.astype(np.float32)
    xd, yd = x32.astype(np.float64), y32.astype(np.float64)
    F = deformation_gradient(xd, o.tets, o.g)
    dets = np.linalg.det(F)
    n_inv, n_str = int((dets < 0).sum()), int((np.linalg.svd(F, compute_uv=False)[:, 0] > 20).sum())
    b_gpu = m.local_rhs(torch.as_tensor(x32), torch.as_tensor(y32)).cpu().numpy()
    R, V = o.local(xd)
    b_or = o.rhs(yd, R, V)
    b_or[o.free] -= o.K_fp @ xd[o.pin_ids]
    b_or[o.pin_ids] = 0.0
    inertia = (o.mass / o.dt ** 2)[:, None] * yd
    inertia[o.pin_ids] = 0.0
    e_total = rel(b_gpu, b_or)
    e_elastic = rel(b_gpu[o.free] - inertia[o.free], b_or[o.free] - inertia[o.free])
    _record("local_rhs_inverted_stretched", {"rel_err_b": e_total, "rel_err_elastic_part": e_elastic,
                                             "inverted_tets": n_inv, "stretched_tets": n_str})
    assert n_inv > 100 and n_str > 100
    assert e_total < 1e-6
    assert e_elastic < 2e-5


@pytest.mark.parametrize("prec,refine,tol", [("fp32", 0, 1e-5), ("tf32", 1, 1e-5), ("bf16", 2, 1e-5),
                                              ("bf16", 0, 2e-2)])
def test_subspace_solve_equals_full_cholesky(prec, refine, tol):
    w = parity_slab()
    m, o = make_pair(w, precision=prec, refine=refine)
    rng = np.random.default_rng(5)
    x = _deformed(w, rng)
    R, V = o.local(x)
    b = o.rhs(x + 1e-3 * rng.standard_normal(x.shape), R, V).astype(np.float32)
    xg = m.solve(torch.as_tensor(b)).cpu().numpy()
    xo = o.chol.solve(b.astype(np.float64)[o.free])
    e = rel(xg[o.free], xo)
    _record(f"solve_{prec}_r{refine}", {"rel_err": e})
    assert np.all(xg[o.pin_ids] == 0.0)
    assert e < tol


@pytest.fixture(scope="module")
def slab_traj():
    """Oracle trajectory of the parity slab: 100 steps x 10 PD iterations."""
    w = parity_slab()
    from oracle.pd_oracle import PDOracle
    o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt)
    xs, vs = [w.rest.copy()], [np.zeros_like(w.rest)]
    for n in range(100):
        x, v = o.step(xs[-1], vs[-1], w.pin_targets(n), w.gravity, w.n_iter)
        xs.append(x)
        vs.append(v)
    return w, xs, vs


def test_one_step_error_slab(slab_traj):
    w, xs, vs = slab_traj
    m, _ = make_pair(w, factor_oracle=False)
    out = torch.empty((w.n_v, 3), device="cuda")
    errs = {}
    for n in (1, 2, 10, 25, 50, 75, 100):
        m.set_state(torch.as_tensor(xs[n - 1], dtype=torch.float32), torch.as_tensor(vs[n - 1], dtype=torch.float32))
        m.step(torch.as_tensor(w.pin_targets(n - 1), dtype=torch.float32), w.gravity, w.n_iter, x_out=out)
        m.sync()
        xg = out.cpu().numpy()
        disp = np.linalg.norm(xs[n] - w.rest)
        errs[n] = (rel(xg, xs[n]), float(np.linalg.norm(xg - xs[n]) / disp))
    _record("one_step_slab", {str(k): {"e_n": a, "e_disp": b} for k, (a, b) in errs.items()})
    for n, (e, ed) in errs.items():
        assert e < 1e-5, (n, e)
        # relative to the displacement: FP32 positions carry eps32 |x| of rounding, which is
        # 3e-5 of the 0.4 mm sag after the first step, so the bound is looser while the sag is small
        assert ed < (5e-4 if n < 10 else 1e-5), (n, ed)


def test_trajectory_slab(slab_traj):
    w, xs, vs = slab_traj
    m, _ = make_pair(w, factor_oracle=False)
    out = torch.empty((w.n_v, 3), device="cuda")
    e = []
    for n in range(100):
        m.step(torch.as_tensor(w.pin_targets(n), dtype=torch.float32), w.gravity, w.n_iter, x_out=out)
        if (n + 1) % 10 == 0:
            m.sync()
            e.append(rel(out.cpu().numpy(), xs[n + 1]))
    _record("trajectory_slab", {"e_n_every_10": e})
    assert max(e) < 2e-5


def test_frames_are_bitwise_deterministic():
    w = parity_slab()
    m, _ = make_pair(w, factor_oracle=False)
    outs = []
    for _ in range(2):
        m.set_state(torch.as_tensor(w.rest, dtype=torch.float32), torch.zeros((w.n_v, 3)))
        x = torch.empty((w.n_v, 3), device="cuda")
        for n in range(3):
            m.step(torch.as_tensor(w.pin_targets(n), dtype=torch.float32), w.gravity, w.n_iter, x_out=x)
        m.sync()
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("graphs", [True, False])
def test_graph_and_plain_launches_agree(graphs):
    w = parity_slab()
    m, _ = make_pair(w, use_graphs=graphs, factor_oracle=False)
    x = torch.empty((w.n_v, 3), device="cuda")
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, w.n_iter, x_out=x)
    m.sync()
    assert np.all(np.isfinite(x.cpu().numpy()))
    # compare with the other launch mode
    m2, _ = make_pair(w, use_graphs=not graphs, factor_oracle=False)
    x2 = torch.empty_like(x)
    m2.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, w.n_iter, x_out=x2)
    m2.sync()
    assert torch.equal(x, x2)


def test_edge_cases_single_domain_and_all_interface():
    # one domain: no interface, the coarse phase is skipped
    w = slab_workload(5, 4, 2, 0.01, 6, (1, 1), seed=9, n_iter=6, name="one-domain")
    m, o = make_pair(w)
    x = torch.empty((w.n_v, 3), device="cuda")
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, w.n_iter, x_out=x)
    m.sync()
    xo, _ = o.step(w.rest, np.zeros_like(w.rest), w.pin_targets(0), w.gravity, w.n_iter)
    assert m.info()["n_interface"] == 0
    assert rel(x.cpu().numpy(), xo) < 1e-5
    # every tet its own domain: almost every vertex is on the interface; ragged domains
    w2 = slab_workload(2, 2, 1, 0.01, 6, (1, 1), seed=9, n_iter=4, name="tiny")
    w2.tet_domain = np.arange(w2.n_t, dtype=np.int32)
    w2.n_domains = w2.n_t
    m2, o2 = make_pair(w2)
    x2 = torch.empty((w2.n_v, 3), device="cuda")
    m2.step(torch.as_tensor(w2.pin_targets(0), dtype=torch.float32), w2.gravity, w2.n_iter, x_out=x2)
    m2.sync()
    xo2, _ = o2.step(w2.rest, np.zeros_like(w2.rest), w2.pin_targets(0), w2.gravity, w2.n_iter)
    assert rel(x2.cpu().numpy(), xo2) < 1e-5


def test_ragged_domains_and_momentum_without_pins():
    w = slab_workload(7, 5, 3, 0.01, 5, (3, 2), seed=4, n_iter=8, name="ragged", pin_edge=False)
    m, o = make_pair(w)
    rng = np.random.default_rng(1)
    v0 = 0.3 * rng.standard_normal(w.rest.shape)
    m.set_state(torch.as_tensor(w.rest, dtype=torch.float32), torch.as_tensor(v0, dtype=torch.float32))
    for _ in range(3):
        m.step(None, (0.0, 0.0, 0.0), w.n_iter)
    m.sync()
    x, v = m.get_state()
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    p0 = (o.mass[:, None] * v0).sum(0)
    p = (o.mass[:, None] * v).sum(0)
    assert np.abs(p - p0).max() < 1e-4 * np.abs(o.mass[:, None] * v0).sum()
    xo, vo = w.rest.copy(), v0.copy()
    for _ in range(3):
        xo, vo = o.step(xo, vo, None, (0.0, 0.0, 0.0), w.n_iter)
    assert rel(x, xo) < 1e-5


def test_status_codes_on_device():
    from paper_2405_12484_gb300 import _lib
    from paper_2405_12484_gb300.sim import Mesh
    w = slab_workload(3, 3, 1, 0.01, 6, (1, 1), seed=2, n_iter=3, name="status")
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    with pytest.raises(_lib.PDError) as e:
        m.step(None, w.gravity, 3)
    assert e.value.status == _lib.PD_ERR_NOT_PREFACTORED
    bad = w.gamma_s.copy()
    bad[3] = -1.0
    with pytest.raises(_lib.PDError) as e:
        m.set_materials(bad, w.gamma_v)
    assert e.value.status == _lib.PD_ERR_BAD_MATERIAL
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt)
    xn = torch.as_tensor(w.rest, dtype=torch.float32).clone()
    xn[5, 0] = float("nan")
    m.set_state(xn, torch.zeros_like(xn))
    m.step(None, w.gravity, 3)
    with pytest.raises(_lib.PDError) as e:
        m.sync()
    assert e.value.status == _lib.PD_ERR_NONFINITE
    m.set_state(torch.as_tensor(w.rest, dtype=torch.float32), torch.zeros_like(xn))
    m.step(None, w.gravity, 3)
    m.sync()   # the flag was cleared and the mesh is usable again


@pytest.fixture(scope="module")
def shell_frame():
    """The oracle's first frame of the 390K-tet shell with the benchmark's 20 PD iterations."""
    from oracle.pd_oracle import PDOracle
    w = sweater_shell()
    o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt)
    xo, _ = o.step(w.rest, np.zeros_like(w.rest), w.pin_targets(0), w.gravity, 20)
    return w, xo


def test_shell_full_size_one_frame(shell_frame):
    """The 390K-tet shell in the benchmark's launch configuration (graphs, FP32,
    20 PD iterations) against the oracle's frame."""
    w, xo = shell_frame
    m, _ = make_pair(w, factor_oracle=False)
    info = m.info()
    assert info["n_tets"] == 390000 and info["n_domains"] == 200
    x = torch.empty((w.n_v, 3), device="cuda")
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, 20, x_out=x)
    m.sync()
    e = rel(x.cpu().numpy(), xo)
    disp = float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo - w.rest))
    _record("shell_full_size", {"e_n": e, "e_disp": disp, "pd_iters": 20, "info": info})
    m.close()
    assert e < 1e-5
    assert disp < 1e-3


@pytest.mark.parametrize("prec,refine,correction,tol", [("bf16", 0, True, 1e-5), ("tf32", 0, True, 1e-5),
                                                         ("bf16", 1, False, 1e-3), ("bf16", 2, False, 1e-4),
                                                         ("fp32", 0, True, 1e-5)])
def test_one_step_error_mixed_precision(slab_traj, prec, refine, correction, tol):
    """Mixed precision: BF16/TF32 matrices with FP64-residual refinement or the
    correction form, one-step error against the FP64 oracle."""
    w, xs, vs = slab_traj
    from paper_2405_12484_gb300.sim import Mesh
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt, precision=prec, refine_steps=refine, correction=correction)
    out = torch.empty((w.n_v, 3), device="cuda")
    errs = {}
    for n in (1, 25, 60, 100):
        m.set_state(torch.as_tensor(xs[n - 1], dtype=torch.float32), torch.as_tensor(vs[n - 1], dtype=torch.float32))
        m.step(torch.as_tensor(w.pin_targets(n - 1), dtype=torch.float32), w.gravity, w.n_iter, x_out=out)
        m.sync()
        errs[n] = rel(out.cpu().numpy(), xs[n])
    _record(f"one_step_slab_{prec}_r{refine}_c{int(correction)}", {str(k): v for k, v in errs.items()})
    assert max(errs.values()) < tol, errs


@pytest.mark.parametrize("prec,refine,tol", [("fp32", 0, 1e-5), ("bf16", 2, 1e-5)])
def test_streaming_solve_slab(slab_traj, prec, refine, tol):
    """The fused streaming solve (one cooperative launch per solve): the
    subspace solve against the full Cholesky solve, and one-step errors."""
    w, xs, vs = slab_traj
    from oracle.pd_oracle import PDOracle
    from paper_2405_12484_gb300.sim import Mesh
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt, precision=prec, refine_steps=refine, streaming=True)
    o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt)
    rng = np.random.default_rng(9)
    x = _deformed(w, rng)
    R, V = o.local(x)
    b = o.rhs(x + 1e-3 * rng.standard_normal(x.shape), R, V).astype(np.float32)
    xg = m.solve(torch.as_tensor(b)).cpu().numpy()
    e_solve = rel(xg[o.free], o.chol.solve(b.astype(np.float64)[o.free]))
    out = torch.empty((w.n_v, 3), device="cuda")
    errs = {}
    for n in (1, 50, 100):
        m.set_state(torch.as_tensor(xs[n - 1], dtype=torch.float32), torch.as_tensor(vs[n - 1], dtype=torch.float32))
        m.step(torch.as_tensor(w.pin_targets(n - 1), dtype=torch.float32), w.gravity, w.n_iter, x_out=out)
        m.sync()
        errs[n] = rel(out.cpu().numpy(), xs[n])
    _record(f"streaming_slab_{prec}_r{refine}", {"solve": e_solve, "one_step": {str(k): v for k, v in errs.items()}})
    m.close()
    assert e_solve < tol
    assert max(errs.values()) < tol, errs


def test_shell_full_size_mixed_precision(shell_frame):
    """The 390K-tet shell, BF16 matrices in the correction form, 20 PD
    iterations against the oracle's frame (the FP32 run is the test above)."""
    w, xo = shell_frame
    m, _ = make_pair(w, precision="bf16", factor_oracle=False)
    m.prefactor(w.dt, precision="bf16", correction=True)
    x = torch.empty((w.n_v, 3), device="cuda")
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, 20, x_out=x)
    m.sync()
    e = rel(x.cpu().numpy(), xo)
    disp = float(np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo - w.rest))
    _record("shell_full_size_bf16_correction", {"e_n": e, "e_disp": disp, "pd_iters": 20})
    m.close()
    assert e < 1e-5
    assert disp < 1e-3


def test_streaming_wait_runs_out_and_reports_timeout():
    """Failure detection without a fault: a phase counter that can never reach
    its target makes the streaming solve's bounded wait run out; the launch
    ends, pd_sync reports PD_ERR_TIMEOUT, and the mesh works again afterwards."""
    from paper_2405_12484_gb300 import _lib
    from paper_2405_12484_gb300.sim import Mesh
    w = parity_slab()
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt, streaming=True, use_graphs=False)
    x0 = torch.as_tensor(w.rest, dtype=torch.float32)
    v0 = torch.zeros_like(x0)
    ref = torch.empty((w.n_v, 3), device="cuda")
    m.set_state(x0, v0)
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, 2, x_out=ref)
    m.sync()
    m.test_offset_phase_counter(0, -100000)
    m.set_state(x0, v0)
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, 1)
    with pytest.raises(_lib.PDError) as e:
        m.sync()
    assert e.value.status == _lib.PD_ERR_TIMEOUT
    out = torch.empty_like(ref)
    m.set_state(x0, v0)
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, 2, x_out=out)
    m.sync()
    assert torch.equal(out, ref)
    m.close()


def test_bulk_copy_wait_runs_out_and_reports_timeout():
    """Failure detection without a fault: one tile stage that expects 16 bytes
    more than its bulk copy delivers makes the consumers' bounded wait in
    k_axpy_tma run out; the launch drains its copies and ends, pd_sync reports
    PD_ERR_TIMEOUT, and the mesh works again afterwards (bitwise as before)."""
    from paper_2405_12484_gb300 import _lib
    from paper_2405_12484_gb300.sim import Mesh
    w = parity_slab()
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt)
    x0 = torch.as_tensor(w.rest, dtype=torch.float32)
    v0 = torch.zeros_like(x0)
    pins = torch.as_tensor(w.pin_targets(0), dtype=torch.float32)
    ref = torch.empty((w.n_v, 3), device="cuda")
    m.set_state(x0, v0)
    m.step(pins, w.gravity, 2, x_out=ref)
    m.sync()
    m.test_inflate_copy(16)
    m.set_state(x0, v0)
    m.step(pins, w.gravity, 1)
    with pytest.raises(_lib.PDError) as e:
        m.sync()
    assert e.value.status == _lib.PD_ERR_TIMEOUT
    out = torch.empty_like(ref)
    m.set_state(x0, v0)
    m.step(pins, w.gravity, 2, x_out=out)
    m.sync()
    assert torch.equal(out, ref)
    m.close()


def test_phase_timing_sampled_iteration_leaves_results_unchanged():
    """Phase events (every iteration, or one sampled PD iteration per frame)
    time the kernels without changing a bit of the frame's result; a negative
    iteration other than -1 is rejected."""
    from paper_2405_12484_gb300._lib import PDError
    from paper_2405_12484_gb300.sim import phase_bit
    w = parity_slab()
    m, _ = make_pair(w, factor_oracle=False)
    x0 = torch.as_tensor(w.rest, dtype=torch.float32)
    v0 = torch.zeros((w.n_v, 3))
    outs = {}
    for mode, (mask, it) in {"off": (0, -1), "all": (-1, -1), "sampled": (phase_bit("local"), 3)}.items():
        m.enable_timing(mask, iteration=it)
        m.set_state(x0, v0)
        x = torch.empty((w.n_v, 3), device="cuda")
        for n in range(3):
            m.step(torch.as_tensor(w.pin_targets(n), dtype=torch.float32, device="cuda"), w.gravity, 10, x_out=x)
        m.sync()
        outs[mode] = (x.cpu(), m.phase_times())
    assert torch.equal(outs["off"][0], outs["all"][0])
    assert torch.equal(outs["off"][0], outs["sampled"][0])
    assert outs["all"][1]["local"] > 0 and outs["all"][1]["dd_condense"] > 0
    assert outs["sampled"][1]["local"] > 0 and outs["sampled"][1]["dd_condense"] == 0
    with pytest.raises(PDError):
        m.enable_timing(-1, iteration=-2)
    m.close()
