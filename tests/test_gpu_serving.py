"""Serving loop: resident requests advanced in shared batched launches,
admitted by a background thread while others run.

Each request's result must be the same alone, in a mix admitted before the
first frame, and in a mix that it joins while others run (bitwise: its
values are computed with the same arithmetic in every batch); match the
single-mesh stepper and the FP64 oracle; and requests beyond the HBM budget
must wait in the queue and still complete.  Per-request frame latencies
(stalls included) come back with the results.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.meshes import slab_workload, sweater_shell  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def _requests():
    a = slab_workload(8, 8, 2, 0.01, 6, (2, 2), seed=21, n_iter=20, name="r-slab8")
    b = sweater_shell(seed=22, n_theta=40, n_z=12, n_r=2, dom_theta=4, dom_z=2)
    c = slab_workload(12, 6, 2, 0.01, 5, (3, 1), seed=23, n_iter=20, name="r-slab12")
    d = sweater_shell(seed=24, n_theta=26, n_z=8, n_r=2, dom_theta=2, dom_z=2)
    return [(a, None), (b, (0.2, 1.0, 0)), (c, None), (d, (0.2, 1.0, 0))]


def _run(reqs, frames, budget=1 << 34, stagger=True, stats=None, wait_admitted=False):
    """Serve `reqs`; with wait_admitted every request is prepared by the
    admission thread before the first tick (so that all of them share the
    batch from the first frame)."""
    import time
    from paper_2405_12484_gb300.sim import Server
    S = Server(budget, max_slots=16, n_iter=20)
    ids = []
    pending = list(reqs)
    if wait_admitted:
        ids = [S.submit(w, frames, drive) for w, drive in pending]
        pending = []
        t0 = time.time()
        while S.stats()["queued"] > 0:
            assert time.time() - t0 < 120
            time.sleep(0.005)
    ticks = 0
    max_active = 0
    saw_queue = False
    peak = 0
    while pending or any(S.poll(i)[0] in (0, 1) for i in ids):
        if pending and (not stagger or ticks % 3 == 0):
            w, drive = pending.pop(0)
            ids.append(S.submit(w, frames, drive))
        n, _ = S.tick()
        st = S.stats()
        peak = max(peak, st["peak_bytes"])
        saw_queue |= st["queued"] > 0 and st["active"] > 0
        max_active = max(max_active, n)
        ticks += 1
        assert ticks < 10000
    out = [S.fetch(i)[0] for i in ids]
    S.close()
    if stats is not None:
        stats["peak"] = peak
    return out, max_active, saw_queue


def test_results_are_identical_alone_and_in_the_mix():
    reqs = _requests()
    frames = 12
    mix, max_active, _ = _run(reqs, frames, wait_admitted=True)
    assert max_active == len(reqs)
    # and with requests arriving while others run (joining the batch as they are prepared)
    staggered, _, _ = _run(reqs, frames)
    for k, r in enumerate(reqs):
        alone, _, _ = _run([r], frames)
        assert np.array_equal(alone[0], mix[k]), k
        assert np.array_equal(alone[0], staggered[k]), k


def test_serving_matches_the_single_mesh_stepper():
    from paper_2405_12484_gb300.sim import Mesh
    reqs = _requests()
    frames = 5
    mix, _, _ = _run(reqs, frames, wait_admitted=True)
    for k, (w, drive) in enumerate(reqs):
        m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
        m.set_materials(w.gamma_s, w.gamma_v)
        m.prefactor(w.dt)
        x = torch.empty((w.n_v, 3), device="cuda")
        for n in range(frames):
            pins = w.pin_targets(n) if drive is not None else None
            m.step(None if pins is None else torch.as_tensor(pins, dtype=torch.float32), w.gravity, 20, x_out=x)
        m.sync()
        ref = x.cpu().numpy().astype(np.float64)
        e = np.linalg.norm(mix[k] - ref) / np.linalg.norm(ref)
        assert e < 1e-5, (k, e)
        m.close()


def test_admission_waits_for_the_hbm_budget():
    reqs = _requests()
    big = reqs[1]
    reqs = [big, (sweater_shell(seed=25, n_theta=40, n_z=12, n_r=2, dom_theta=4, dom_z=2), big[1])] + reqs[:1] + reqs[2:]
    alone, peaks = [], []
    for r in reqs:
        st = {}
        alone.append(_run([r], 4, stats=st)[0][0])
        peaks.append(st["peak"])
    # room for the largest request and its prefactorisation, not for two of them
    budget = int(1.05 * max(peaks))
    mix, max_active, saw_queue = _run(reqs, 4, budget=budget, stagger=False)
    assert saw_queue
    assert max_active < len(reqs)
    for k in range(len(reqs)):
        assert np.array_equal(alone[k], mix[k])


def test_run_until_idle_matches_ticking():
    """pd_server_run ticks until nothing is queued or resident; the results are
    the ones the tick-by-tick loop gives (bitwise)."""
    from paper_2405_12484_gb300.sim import Server
    reqs = _requests()[:2]
    frames = 4
    ticked, _, _ = _run(reqs, frames, stagger=False)
    S = Server(1 << 34, max_slots=16, n_iter=20)
    ids = [S.submit(w, frames, drive) for w, drive in reqs]
    ticks = S.run()
    assert ticks >= frames
    assert all(S.poll(i)[0] == 2 for i in ids)
    for k, i in enumerate(ids):
        assert np.array_equal(S.fetch(i)[0], ticked[k])
    S.close()


def test_request_larger_than_the_whole_budget_fails_and_leaves_the_queue():
    """A request that would not fit the HBM budget even with nothing resident
    is marked failed at once (it is not retried every tick), and the request
    behind it is served."""
    from paper_2405_12484_gb300.sim import Server
    reqs = _requests()
    small, big = reqs[0], reqs[1]
    st = {}
    _run([small], 2, stats=st)
    S = Server(int(1.05 * st["peak"]), max_slots=16, n_iter=20)
    i_big = S.submit(big[0], 2, big[1])
    i_small = S.submit(small[0], 2, small[1])
    S.run(max_ticks=5000)
    assert S.poll(i_big)[0] == 3
    assert S.poll(i_small)[0] == 2
    S.close()


def test_run_reports_outstanding_work_after_max_ticks():
    from paper_2405_12484_gb300 import _lib
    from paper_2405_12484_gb300.sim import Server
    w, drive = _requests()[0]
    S = Server(1 << 34, max_slots=16, n_iter=20)
    i = S.submit(w, 5, drive)
    with pytest.raises(_lib.PDError) as e:
        S.run(max_ticks=2)
    assert e.value.status == _lib.PD_ERR_TIMEOUT
    assert S.poll(i)[0] in (0, 1)
    assert S.run() >= 1
    assert S.poll(i)[0] == 2
    S.close()


def test_served_requests_match_the_oracle():
    """Two requests served together (a pinned slab and a driven shell), five
    20-iteration frames each, against the FP64 oracle stepping the same
    frames: one-frame-per-tick results within the FP32 parity tolerance."""
    from gpu_helpers import f32, rel
    from oracle.pd_oracle import PDOracle
    reqs = _requests()[:2]
    frames = 5
    mix, max_active, _ = _run(reqs, frames, wait_admitted=True)
    assert max_active == 2
    errs = []
    for k, (w, drive) in enumerate(reqs):
        o = PDOracle(w.rest, w.tets, w.pinned, f32(w.gamma_s), f32(w.gamma_v), w.density, w.dt)
        x, v = w.rest.copy(), np.zeros_like(w.rest)
        for n in range(frames):
            x, v = o.step(x, v, w.pin_targets(n), w.gravity, 20)
        errs.append(rel(mix[k], x))
    assert max(errs) < 1e-5, errs


def test_frame_latencies_include_the_stalls():
    """The per-frame latency of a request is wall time between its frames: at
    least the GPU time of the batched frame it ran in, one entry per frame."""
    from paper_2405_12484_gb300.sim import Server
    reqs = _requests()[:2]
    S = Server(1 << 34, max_slots=16, n_iter=20)
    ids = [S.submit(w, 6, d) for w, d in reqs]
    gpu = []
    while any(S.poll(i)[0] in (0, 1) for i in ids):
        n, ms = S.tick()
        if n:
            gpu.append(ms)
    for i in ids:
        _, lat = S.fetch(i)
        assert lat.shape == (6,)
        assert np.all(lat >= min(gpu) * 0.99)
    S.close()


def test_two_level_requests_in_the_batch():
    """A request large enough for the two-level interface solve is served with
    the second level's batched row-form products: the same result alone and
    beside a one-level request (bitwise), and the single-mesh stepper's
    result within the FP32 tolerance."""
    from paper_2405_12484_gb300.sim import Mesh
    big = sweater_shell(seed=25, n_theta=200, n_z=60, n_r=2, dom_theta=20, dom_z=6)
    small = slab_workload(8, 8, 2, 0.01, 6, (2, 2), seed=26, n_iter=20, name="r-slab8b")
    frames = 3
    m = Mesh(big.rest, big.tets, big.pinned, big.tet_domain, big.n_domains, big.density)
    m.set_materials(big.gamma_s, big.gamma_v)
    m.prefactor(big.dt)
    info = m.info()
    assert info["two_level"] == 1 and info["n_top_interface"] * 4 <= 24576, info
    x = torch.empty((big.n_v, 3), device="cuda")
    for n in range(frames):
        m.step(torch.as_tensor(big.pin_targets(n), dtype=torch.float32), big.gravity, 20, x_out=x)
    m.sync()
    ref = x.cpu().numpy().astype(np.float64)
    m.close()
    alone, _, _ = _run([(big, (0.2, 1.0, 0))], frames, wait_admitted=True)
    mix, _, _ = _run([(small, None), (big, (0.2, 1.0, 0))], frames, wait_admitted=True)
    assert np.array_equal(alone[0], mix[1])
    e = np.linalg.norm(alone[0] - ref) / np.linalg.norm(ref)
    assert e < 1e-5, e
