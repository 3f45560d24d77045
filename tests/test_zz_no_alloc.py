"""pd_solve_noalloc: the solve for callers that may not allocate device memory.

Some hosts give each library a fixed memory pool at start-up and forbid
cudaMalloc/cudaFree afterwards (or cannot afford the device-wide
synchronisation an allocation can cause while they run).  For them the
library offers pd_solve_noalloc, which takes every temporary from one fixed
16 MiB static device array.  These tests call it through the C ABI and check
it against pd_solve (which allocates its temporaries) on two calls in a row:
the same kernels run in the same order, so the results must be bitwise
equal, and the device's free memory must not move across either call
(the array itself is loaded by pd_prefactor, while allocation is allowed).
The solver variants cover every branch of the scratch layout: the
single-level interface solve with a refinement step, the two-level
interface solve, the fused streaming solve and the modal solve with
Jacobi sweeps.  The file is collected last; it passes alone or after the
other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _workload(kind):
    from workloads.meshes import parity_slab, sweater_shell
    if kind == "slab":
        return parity_slab()
    # a shell with enough domains and interface vertices for the two-level
    # interface solve, small enough for the fixed scratch
    return sweater_shell(n_theta=200, n_z=60, dom_theta=20, dom_z=6)


CASES = {
    "slab-single-level-refine": ("slab", dict(precision="fp32", refine_steps=1)),
    "slab-streaming": ("slab", dict(precision="fp32", streaming=True)),
    "slab-modal-jacobi": ("slab", dict(precision="fp32", modal=True, modes=20, jacobi_sweeps=4, jacobi_rho=0.99)),
    "shell-two-level": ("shell", dict(precision="fp32")),
    "shell-two-level-bf16-refine": ("shell", dict(precision="bf16", refine_steps=2)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_solve_equals_pd_solve_on_two_calls(case):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12484_gb300.sim import Mesh
    kind, opts = CASES[case]
    w = _workload(kind)
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    try:
        m.set_materials(w.gamma_s, w.gamma_v)
        m.prefactor(w.dt, **opts)
        info = m.info()
        if kind == "shell":
            assert info["two_level"] == 1, "the shell case must exercise the two-level branch"
        g = torch.Generator().manual_seed(7)
        scale = torch.as_tensor(w.rest, dtype=torch.float32).abs().max()
        r1 = (torch.randn((w.n_v, 3), generator=g) * scale).cuda()
        r2 = (torch.randn((w.n_v, 3), generator=g) * scale + 1.0).cuda()
        ref1 = m.solve(r1)
        ref2 = m.solve(r2)
        x1 = torch.full((w.n_v, 3), float("nan"), device="cuda")
        x2 = torch.full((w.n_v, 3), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        m.solve_noalloc(r1, x1)
        free1, _ = torch.cuda.mem_get_info()
        m.solve_noalloc(r2, x2)
        free2, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"the first call took {free0 - free1} bytes of device memory"
        assert free2 == free1, f"the second call took {free1 - free2} bytes of device memory"
        assert torch.equal(x1, ref1)
        assert torch.equal(x2, ref2)
        pins = torch.as_tensor(np.nonzero(w.pinned)[0], device="cuda")
        assert torch.all(x2[pins] == 0)
    finally:
        m.close()


def test_noalloc_requires_prefactor():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12484_gb300 import _lib
    from paper_2405_12484_gb300.sim import Mesh
    from workloads.meshes import slab_workload
    w = slab_workload(3, 3, 1, 0.01, 6, (1, 1), seed=2, n_iter=2, name="np")
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    r = torch.zeros((w.n_v, 3), device="cuda")
    x = torch.empty_like(r)
    with pytest.raises(_lib.PDError) as e:
        m.solve_noalloc(r, x)
    assert e.value.status == _lib.PD_ERR_NOT_PREFACTORED
    m.close()
