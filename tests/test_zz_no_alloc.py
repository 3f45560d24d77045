"""pd_solve_noalloc: the solve for callers that may not allocate device memory.

Some hosts give each library a fixed memory pool at start-up and forbid
cudaMalloc/cudaFree afterwards (or cannot afford the device-wide
synchronisation an allocation can cause while they run).  For them the
library offers pd_solve_noalloc, which takes every temporary from one fixed
16 MiB static device array.  This test calls it through the C ABI and checks
it against pd_solve (which allocates its temporaries) on two calls in a row.
It lives in its own file, collected last, and passes alone or after the
other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mesh():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_12484_gb300.sim import Mesh
    from workloads.meshes import parity_slab
    w = parity_slab()
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
    m.set_materials(w.gamma_s, w.gamma_v)
    m.prefactor(w.dt, precision="fp32", refine_steps=1)
    yield w, m
    m.close()


def _rel(a, b):
    return float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))


def test_noalloc_solve_matches_pd_solve_on_two_calls(mesh):
    w, m = mesh
    g = torch.Generator().manual_seed(7)
    scale = torch.as_tensor(w.rest, dtype=torch.float32).abs().max()
    r1 = (torch.randn((w.n_v, 3), generator=g) * scale).cuda()
    r2 = (torch.randn((w.n_v, 3), generator=g) * scale + 1.0).cuda()
    ref1 = m.solve(r1)
    ref2 = m.solve(r2)
    torch.cuda.synchronize()
    x1 = torch.empty((w.n_v, 3), device="cuda")
    x2 = torch.empty((w.n_v, 3), device="cuda")
    m.solve_noalloc(r1, x1)
    free_before, _ = torch.cuda.mem_get_info()
    m.solve_noalloc(r2, x2)
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before            # nothing allocated by the second call
    assert _rel(x1, ref1) <= 1e-5
    assert _rel(x2, ref2) <= 1e-5
    pins = torch.as_tensor(np.nonzero(w.pinned)[0], device="cuda")
    assert torch.all(x2[pins] == 0)


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
