"""Writes tests/golden/adjoint_slab50k_30steps.json: the FP64 oracle's adjoint
gradient of the pose-matching loss on the 50,000-tet slab over 30 equilibrium
steps, at 20 parameters drawn with seed 7.

Paper passage: Sec. 6.1 (Eq. g, Eq. pxpgamma, Eq. adjoint_state,
Eq. adjoint_state_solve); the oracle (oracle/adjoint.py) follows it.  Calls
only oracle/ and the seeded input generators (workloads/); runs about three
hours on one host core.  The inputs are the FP32-rounded values the GPU
library is given: materials (gamma_s = theta, gamma_v = 10 theta, both
float32), initial state, pinned targets, gravity and the target poses.

    python tests/golden/make_adjoint_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.adjoint import AdjointOracle  # noqa: E402
from oracle.pd_oracle import PDOracle  # noqa: E402
from workloads.meshes import adjoint_slab, target_trajectory  # noqa: E402

N_STEPS = 30
TARGET_SEED = 8
SAMPLE_SEED = 7
PD_ITERS = 10


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def inputs():
    w = adjoint_slab()
    theta = np.asarray(w.gamma_s, np.float32)
    gs = theta.astype(np.float64)
    gv = (theta * np.float32(10.0)).astype(np.float64)     # float32 product, as the library forms it
    targets = [f32(t) for t in target_trajectory(w.rest, N_STEPS, TARGET_SEED)]
    gravity = tuple(float(np.float32(g)) for g in w.gravity)
    return w, gs, gv, targets, gravity


def main():
    w, gs, gv, targets, gravity = inputs()
    o = AdjointOracle(PDOracle(w.rest, w.tets, w.pinned, gs, gv, w.density, w.dt), gravity=gravity)
    x0 = f32(w.rest)
    t0 = time.time()
    xs, vs = [x0], [np.zeros_like(x0)]
    for n in range(N_STEPS):
        x, v = o.equilibrium(xs[-1], vs[-1], f32(w.pin_targets(n)), pd_iters=PD_ITERS)
        xs.append(x)
        vs.append(v)
        print(f"step {n + 1}/{N_STEPS}  {time.time() - t0:.0f} s", flush=True)
    free = o.o.free
    loss = AdjointOracle.loss(xs, targets, free)
    g_s, g_v = o.gradient(xs, targets)
    theta_grad = g_s + 10.0 * g_v
    idx = np.random.default_rng(SAMPLE_SEED).choice(w.n_t, 20, replace=False)
    out = {
        "what": "FP64 oracle adjoint gradient of L = sum_{n=1..30} sum_free |x_n - xhat_n|^2 on the 50x50x4x5 slab",
        "cite": "Sec. 6.1, Eq. g, Eq. pxpgamma, Eq. adjoint_state, Eq. adjoint_state_solve",
        "writer": "tests/golden/make_adjoint_golden.py (oracle/ only)",
        "config": {"mesh": w.name, "n_t": int(w.n_t), "n_v": int(w.n_v), "steps": N_STEPS, "dt": w.dt,
                   "target_seed": TARGET_SEED, "sample_seed": SAMPLE_SEED, "oracle_pd_iters": PD_ITERS,
                   "gamma": "gamma_s = float32(theta), gamma_v = float32(10 theta), theta from adjoint_slab()",
                   "x0": "float32(rest), v0 = 0", "gravity": list(gravity)},
        "loss": loss,
        "indices": [int(i) for i in idx],
        "dL_dgamma_s": [float(g_s[i]) for i in idx],
        "dL_dgamma_v": [float(g_v[i]) for i in idx],
        "dL_dtheta": [float(theta_grad[i]) for i in idx],
        "dL_dtheta_max_abs": float(np.abs(theta_grad).max()),
        "dL_dtheta_norm": float(np.linalg.norm(theta_grad)),
        "final_disp_max": float(np.abs(xs[-1] - x0).max()),
        "seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, "adjoint_slab50k_30steps.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("loss", "dL_dtheta_max_abs", "seconds")}))


if __name__ == "__main__":
    main()
