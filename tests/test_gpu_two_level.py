"""Two-level interface solve (Sec. 7.2's subspace solve with the interface
system itself condensed over groups of domains) on the 390K-tet shell: the
solve through the C ABI against the oracle's sparse Cholesky solve of the
full system, with the two-level and the single-level interface solve."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_helpers import f32, rel  # noqa: E402

from workloads.meshes import sweater_shell  # noqa: E402

# measurement records go to $PD_RECORD_DIR when it is set (nothing is written otherwise)
OUT = os.environ.get("PD_RECORD_DIR")


@pytest.fixture(scope="module")
def shell_pair():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from oracle.pd_oracle import PDOracle
    from paper_2405_12484_gb300.sim import Mesh
    w = sweater_shell()
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt)
    yield w, m, o
    m.close()


def _rhs(w, o, seed):
    """A smooth right-hand side (the inertia term of a sagging state) plus noise."""
    rng = np.random.default_rng(seed)
    x = w.rest + 0.01 * np.sin(w.rest * 7.0) + 1e-4 * rng.standard_normal(w.rest.shape)
    b = (o.mass / o.dt ** 2)[:, None] * x
    b[o.pin_ids] = 0.0
    return b.astype(np.float32)


@pytest.mark.parametrize("prec,refine,single_level,streaming,tol", [
    ("fp32", 0, False, False, 1e-5), ("fp32", 0, True, False, 1e-5), ("bf16", 2, False, False, 1e-5),
    ("tf32", 2, False, False, 1e-5), ("fp32", 0, False, True, 1e-5), ("fp32", 0, True, True, 1e-5),
    ("bf16", 2, False, True, 1e-5)])
def test_shell_interface_solve(shell_pair, prec, refine, single_level, streaming, tol):
    w, m, o = shell_pair
    m.prefactor(w.dt, precision=prec, refine_steps=refine, single_level=single_level, streaming=streaming)
    info = m.info()
    assert info["n_groups"] >= 8
    assert info["two_level"] == (0 if single_level else 1)
    b = _rhs(w, o, 1)
    xg = m.solve(torch.as_tensor(b)).cpu().numpy()
    xo = o.chol.solve(b.astype(np.float64)[o.free])
    e = rel(xg[o.free], xo)
    if OUT:
        try:
            os.makedirs(OUT, exist_ok=True)
            with open(os.path.join(OUT, f"two_level_{prec}_r{refine}_single{int(single_level)}"
                                        f"_stream{int(streaming)}.json"), "w") as f:
                json.dump({"rel_err": e, "n_groups": info["n_groups"], "n_top": info["n_top_interface"],
                           "n_interface": info["n_interface"], "prefactor_s": info["prefactor_seconds"],
                           "device_bytes": info["device_bytes"]}, f, indent=1)
        except OSError:
            pass
    assert np.all(xg[o.pin_ids] == 0.0)
    assert e < tol
