"""Seeded synthetic workloads: tet meshes, domain partitions, materials, pins.

This module only builds inputs (geometry, connectivity, labels and seeded
random numbers).  It holds none of the simulation arithmetic: no mass
lumping, no deformation gradients, no projections, no matrices.  Both the
FP64 oracle and the CUDA path consume its arrays.

Workloads (all SI units):

* ``slab6``  -- an nx x ny x nz block of cubes, 6 tets per cube (Kuhn split
  along the main diagonal), lying in the x-y plane; used for the 20x20x2
  parity slab (4,800 tets, 1,323 vertices, 8 domains).
* ``slab5``  -- the same block with 5 tets per cube, alternating cube parity
  so that the face diagonals conform; used for the 50x50x4 differentiable
  slab (50,000 tets, 13,005 vertices).
* ``shell``  -- a thick cylindrical shell periodic in theta, standing along
  z, 6 tets per hex; the sweater-scale stand-in (325 x 100 x 2 hexes:
  390,000 tets, 98,475 vertices, 200 domains).

Material recipes follow the per-element stiffness of the paper's energy
(Eq. energy, Sec. 6): gamma_s per element, gamma_v = 10 gamma_s.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

# Six tets of a unit cube: one per axis permutation, each a monotone lattice
# path from corner (0,0,0) to corner (1,1,1) (Kuhn / Freudenthal split).
_KUHN_PATHS = []
for _perm in itertools.permutations(range(3)):
    _c = [0, 0, 0]
    _path = [tuple(_c)]
    for _ax in _perm:
        _c[_ax] += 1
        _path.append(tuple(_c))
    _KUHN_PATHS.append(_path)

# Five-tet split: a central tet on the four corners of one parity class plus
# four corner tets, one at each corner of the other class.
_EVEN = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
_ODD = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]


def _corner_tets_5(center_class, apex_class):
    tets = [list(center_class)]
    for a in apex_class:
        nbrs = [c for c in center_class if sum(abs(a[i] - c[i]) for i in range(3)) == 1]
        tets.append([a] + nbrs)
    return tets


_FIVE_EVEN = _corner_tets_5(_EVEN, _ODD)
_FIVE_ODD = _corner_tets_5(_ODD, _EVEN)


@dataclass
class Workload:
    """A complete synthetic input for the simulator."""

    name: str
    rest: np.ndarray            # (n_v, 3) float64 rest positions
    tets: np.ndarray            # (n_t, 4) int32 vertex indices, positive orientation
    tet_domain: np.ndarray      # (n_t,)  int32 domain label in [0, n_domains)
    n_domains: int
    pinned: np.ndarray          # (n_v,)  uint8, 1 = Dirichlet vertex
    gamma_s: np.ndarray         # (n_t,)  float64 strain stiffness (Pa)
    gamma_v: np.ndarray         # (n_t,)  float64 volume stiffness (Pa)
    density: float = 300.0      # kg / m^3
    dt: float = 1.0 / 150.0
    gravity: tuple = (0.0, 0.0, -9.81)
    n_iter: int = 10
    meta: dict = field(default_factory=dict)

    @property
    def n_v(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_t(self) -> int:
        return int(self.tets.shape[0])

    @property
    def pinned_ids(self) -> np.ndarray:
        return np.nonzero(self.pinned)[0].astype(np.int32)

    def pin_targets(self, frame: int) -> np.ndarray:
        """Prescribed positions of the pinned vertices at the END of `frame`
        (frame 0 advances t from 0 to dt), in increasing vertex-id order."""
        base = self.rest[self.pinned_ids]
        drive = self.meta.get("drive")
        if drive is None:
            return base.copy()
        amp, freq, axis = drive
        t = (frame + 1) * self.dt
        out = base.copy()
        out[:, axis] += amp * np.sin(2.0 * np.pi * freq * t)
        return out


def _orient(pos: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap the last two corners of tets with negative signed volume."""
    a = pos[tets[:, 1]] - pos[tets[:, 0]]
    b = pos[tets[:, 2]] - pos[tets[:, 0]]
    c = pos[tets[:, 3]] - pos[tets[:, 0]]
    s = np.einsum("ij,ij->i", a, np.cross(b, c))
    t = tets.copy()
    neg = s < 0
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def _grid_index(nx, ny, nz):
    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i
    return vid


def slab(nx: int, ny: int, nz: int, h: float, tets_per_cube: int = 6):
    """Block of nx*ny*nz cubes of edge h; returns (rest, tets, cube_ijk)."""
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    vid = _grid_index(nx, ny, nz)
    n_v = (nx + 1) * (ny + 1) * (nz + 1)
    rest = np.zeros((n_v, 3))
    ids = vid(ii, jj, kk).ravel()
    rest[ids, 0] = ii.ravel() * h
    rest[ids, 1] = jj.ravel() * h
    rest[ids, 2] = kk.ravel() * h
    tets, cubes = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if tets_per_cube == 6:
                    pattern = _KUHN_PATHS
                else:
                    pattern = _FIVE_EVEN if (i + j + k) % 2 == 0 else _FIVE_ODD
                for p in pattern:
                    tets.append([vid(i + a, j + b, k + c) for (a, b, c) in p])
                    cubes.append((i, j, k))
    tets = np.asarray(tets, dtype=np.int64)
    tets = _orient(rest, tets).astype(np.int32)
    return rest, tets, np.asarray(cubes, dtype=np.int32)


def shell_mesh(n_theta: int, n_z: int, n_r: int, radius: float, height: float, thickness: float):
    """Thick cylinder periodic in theta; (n_theta, n_z, n_r) hexes, 6 tets each.

    Returns (rest, tets, hex_ijk) with vertex id = (k_z * n_theta + i_theta) * (n_r+1) + j_r.
    """
    nr1 = n_r + 1

    def vid(i, k, j):
        return (k * n_theta + (i % n_theta)) * nr1 + j

    n_v = n_theta * (n_z + 1) * nr1
    rest = np.zeros((n_v, 3))
    th = 2.0 * np.pi * np.arange(n_theta) / n_theta
    rr = radius - 0.5 * thickness + thickness * np.arange(nr1) / n_r
    zz = height * np.arange(n_z + 1) / n_z
    K, I, J = np.meshgrid(np.arange(n_z + 1), np.arange(n_theta), np.arange(nr1), indexing="ij")
    ids = vid(I, K, J).ravel()
    rest[ids, 0] = (rr[J] * np.cos(th[I])).ravel()
    rest[ids, 1] = (rr[J] * np.sin(th[I])).ravel()
    rest[ids, 2] = zz[K].ravel()
    tets, hexes = [], []
    for k in range(n_z):
        for i in range(n_theta):
            for j in range(n_r):
                for p in _KUHN_PATHS:
                    # lattice axes: 0 -> theta, 1 -> z, 2 -> r
                    tets.append([vid(i + a, k + b, j + c) for (a, b, c) in p])
                    hexes.append((i, k, j))
    tets = np.asarray(tets, dtype=np.int64)
    tets = _orient(rest, tets).astype(np.int32)
    return rest, tets, np.asarray(hexes, dtype=np.int32)


def loguniform_stiffness(n: int, seed: int, lo: float = 1e3, hi: float = 1e5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def parity_slab(seed: int = 1, n_iter: int = 10) -> Workload:
    """20x20x2 cubes of 1 cm, 6 tets each: 4,800 tets, 1,323 vertices.

    Edge y = 0.2 pinned (63 vertices); 8 domains = 4 (x) x 2 (y) patches of
    5x10x2 cubes; theta_e log-uniform in [1e3, 1e5] Pa from `seed`.
    """
    return slab_workload(20, 20, 2, 0.01, 6, (4, 2), seed, n_iter, name="slab20x20x2")


def slab_workload(nx, ny, nz, h, tpc, dom_xy, seed, n_iter, name=None, pin_edge=True) -> Workload:
    rest, tets, cubes = slab(nx, ny, nz, h, tpc)
    dx, dy = dom_xy
    bx = np.minimum(cubes[:, 0] * dx // nx, dx - 1)
    by = np.minimum(cubes[:, 1] * dy // ny, dy - 1)
    tet_domain = (by * dx + bx).astype(np.int32)
    pinned = np.zeros(rest.shape[0], np.uint8)
    if pin_edge:
        pinned[np.isclose(rest[:, 1], ny * h)] = 1
    theta = loguniform_stiffness(tets.shape[0], seed)
    return Workload(
        name=name or f"slab{nx}x{ny}x{nz}",
        rest=rest, tets=tets, tet_domain=tet_domain, n_domains=dx * dy, pinned=pinned,
        gamma_s=theta, gamma_v=10.0 * theta, n_iter=n_iter,
        meta={"drive": None, "cubes": (nx, ny, nz), "h": h, "tets_per_cube": tpc},
    )


def adjoint_slab(seed: int = 1, n_iter: int = 10) -> Workload:
    """50x50x4 cubes x 5 tets: 50,000 tets, 13,005 vertices; 25 domains."""
    return slab_workload(50, 50, 4, 0.01, 5, (5, 5), seed, n_iter, name="slab50x50x4x5")


def sweater_shell(seed: int = 2, n_theta: int = 325, n_z: int = 100, n_r: int = 2,
                  dom_theta: int = 25, dom_z: int = 8, n_iter: int = 20) -> Workload:
    """Thick cylindrical shell standing in for the paper's sweater mesh.

    Radius 0.3 m, height 0.6 m, thickness 1 cm as 2 hex layers.  At the
    default sizes: 390,000 tets, 98,475 vertices, 200 domains.  Materials:
    vertical cable bands 2 cm wide alternating 1e5 / 1e4 Pa, times
    (1 + 0.2 U[-1, 1]) seeded noise, gamma_v = 10 gamma_s.  The top ring is
    pinned and driven by x(t) = x0 + 0.2 sin(2 pi t) e_x.
    """
    radius, height, thick = 0.3, 0.6, 0.01
    rest, tets, hexes = shell_mesh(n_theta, n_z, n_r, radius, height, thick)
    dt_ = np.minimum(hexes[:, 0] * dom_theta // n_theta, dom_theta - 1)
    dz_ = np.minimum(hexes[:, 1] * dom_z // n_z, dom_z - 1)
    tet_domain = (dz_ * dom_theta + dt_).astype(np.int32)
    # band index from the arc length of the hex's theta-cell centre
    arc = radius * 2.0 * np.pi * (hexes[:, 0] + 0.5) / n_theta
    stiff = (np.floor(arc / 0.02).astype(np.int64) % 2) == 0
    base = np.where(stiff, 1e5, 1e4)
    rng = np.random.default_rng(seed)
    theta = base * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=tets.shape[0]))
    pinned = np.zeros(rest.shape[0], np.uint8)
    pinned[np.isclose(rest[:, 2], height)] = 1
    return Workload(
        name=f"shell{n_theta}x{n_z}x{n_r}",
        rest=rest, tets=tets, tet_domain=tet_domain, n_domains=dom_theta * dom_z, pinned=pinned,
        gamma_s=theta, gamma_v=10.0 * theta, n_iter=n_iter,
        meta={"drive": (0.2, 1.0, 0), "shape": (n_theta, n_z, n_r)},
    )


def serving_requests(n_req: int = 64, rate: float = 20.0, seed_arrival: int = 11, seed_size: int = 12,
                     t_lo: float = 5e3, t_hi: float = 2e5):
    """Poisson request stream: (arrival_s, generator, n_tets_target, seed) tuples."""
    rng_a = np.random.default_rng(seed_arrival)
    arrivals = np.cumsum(rng_a.exponential(1.0 / rate, size=n_req))
    rng_s = np.random.default_rng(seed_size)
    sizes = np.exp(rng_s.uniform(np.log(t_lo), np.log(t_hi), size=n_req))
    gens = np.where(rng_s.uniform(size=n_req) < 0.5, "slab", "shell")
    return [(float(a), str(g), int(s), 1000 + i) for i, (a, g, s) in enumerate(zip(arrivals, gens, sizes))]


def request_workload(gen: str, n_tets: float, seed: int, n_iter: int = 20) -> Workload:
    """Mesh of roughly n_tets tets for a serving request (domains ~ T / 2000)."""
    n_dom_target = max(1, int(round(n_tets / 2000.0)))
    if gen == "slab":
        n = max(2, int(round(np.sqrt(n_tets / 12.0))))
        side = int(max(1, round(np.sqrt(n_dom_target))))
        side = min(side, n)
        w = slab_workload(n, n, 2, 0.01, 6, (side, side), seed, n_iter, name=f"req-slab{n}")
        return w
    n_z = max(2, int(round(np.sqrt(n_tets / (12.0 * 3.25)))))
    n_theta = max(3, int(round(3.25 * n_z)))
    dz = max(1, int(round(np.sqrt(n_dom_target / 3.125))))
    dth = max(1, int(round(n_dom_target / dz)))
    dz = min(dz, n_z)
    dth = min(dth, n_theta)
    return sweater_shell(seed=seed, n_theta=n_theta, n_z=n_z, n_r=2, dom_theta=dth, dom_z=dz, n_iter=n_iter)


def target_trajectory(rest: np.ndarray, n_steps: int, seed: int) -> list:
    """Seeded target poses xhat_0 .. xhat_{n_steps} for a pose-matching loss.

    The rest shape plus a smooth seeded displacement that grows linearly
    with the step index: a sag along the length (y), a bulge across the
    width (x) and a sideways sway, with amplitudes drawn from `seed`
    (centimetre scale on a 0.5 m slab).  Plain geometry: no mechanics.
    """
    rng = np.random.default_rng(seed)
    a, b, c = rng.uniform(0.5, 1.5, size=3)
    lo, hi = rest.min(axis=0), rest.max(axis=0)
    span = np.where(hi - lo > 0, hi - lo, 1.0)
    u = (rest - lo) / span
    disp = np.zeros_like(rest)
    disp[:, 2] = -0.02 * a * (1.0 - u[:, 1]) ** 2 + 0.004 * b * np.sin(np.pi * u[:, 0])
    disp[:, 0] = 0.005 * c * (1.0 - u[:, 1]) ** 2
    return [rest + (n / max(n_steps, 1)) * disp for n in range(n_steps + 1)]
