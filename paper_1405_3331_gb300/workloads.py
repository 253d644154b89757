"""Seeded synthetic inputs for the cue-field / growth-cone simulation.

This module only draws inputs (grid sizes, physical constants, source cells
and emissions, initial cone positions and directions, targets); it contains
none of the model's arithmetic, so both the CUDA path and the FP64 oracle can
be fed from it.  All draws use numpy's PCG64 with an explicit seed.

The workloads follow the paper's setting (Sec. 4.3: cue sources placed
pseudo-randomly with various diffusion rates; Sec. 3.4: each axon starts on a
randomly attributed direction) at the sizes of the five benchmark
configurations:

  c1  2D 128^2,   4 sources (e = 1),         64 cones,     500 steps
  c2  2D 2048^2,  64 sources (e ~ U[0.5,2]), 16,384 cones, 5,000 steps,
      cones stop within radius 2 of a source
  c3  3D 256^3,   128 sources,               65,536 cones, 2,000 steps
  c4  512 independent 2D instances of uneven size and physics, 1,000 steps
  c5  2D 1024^2,  32 sources, 4,096 cones, 2,000 steps, wall clamp, targets

Initial directions: 2D angle ~ U[0, 2pi); 3D by the trigonometric sphere
method of Sec. 3.2 (z ~ U[-1,1], t ~ U[0,2pi), r = sqrt(1-z^2)).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

PHILOX_SEED_BASE = 0x5EED0000


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    h: float
    D: float
    lam: float
    dt: float
    src_cell: np.ndarray            # int32 [n_src], linear node index i + nx (j + ny k)
    src_emit: np.ndarray            # float32 [n_src], emission per step
    src_map: Optional[np.ndarray]   # float32 field-shaped rate map, or None
    pos: np.ndarray                 # float32 [dim, n]
    dir: np.ndarray                 # float32 [dim, n]
    active: np.ndarray              # uint8 [n]
    w_prev: float = 0.5
    w_grad: float = 0.4
    w_noise: float = 0.1
    step_len: float = 0.5
    stop_radius: float = 0.0
    grad_eps: float = 1e-15
    wall_mode: int = 0
    seed: int = PHILOX_SEED_BASE
    nsteps: int = 1
    C0: Optional[np.ndarray] = None  # float32 field-shaped initial field (None = zeros)
    targets: Optional[np.ndarray] = None  # float32 [dim, n] (adjoint workload)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.dim == 3 else (self.ny, self.nx)

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.shape))

    @property
    def n_axons(self) -> int:
        return int(self.active.shape[0])

    @property
    def n_src(self) -> int:
        return int(self.src_cell.shape[0])

    def field0(self) -> np.ndarray:
        if self.C0 is not None:
            return self.C0.astype(np.float32, copy=True)
        return np.zeros(self.shape, np.float32)


def _distinct_cells(rng, n_cells, n_src):
    if n_src == 0:
        return np.zeros(0, np.int32)
    return np.sort(rng.choice(n_cells, size=n_src, replace=False)).astype(np.int32)


def _cell_coords(cells, nx, ny, dim, h):
    cells = cells.astype(np.int64)
    x = (cells % nx) * h
    y = ((cells // nx) % ny) * h
    if dim == 3:
        z = (cells // (nx * ny)) * h
        return np.stack([x, y, z])
    return np.stack([x, y])


def _directions(rng, dim, n):
    if dim == 2:
        t = rng.uniform(0.0, 2.0 * np.pi, n)
        return np.stack([np.cos(t), np.sin(t)])
    z = rng.uniform(-1.0, 1.0, n)
    t = rng.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(t), r * np.sin(t), z])


def _positions(rng, extents, h, n, avoid=None, radius=0.0):
    """Uniform positions in [0,(N-1)h]^dim, redrawn while within ``radius`` of ``avoid``."""
    dim = len(extents)
    hi = np.array([(e - 1) * h for e in extents], dtype=np.float64)[:, None]
    pos = rng.uniform(0.0, 1.0, (dim, n)) * hi
    if avoid is not None and radius > 0 and n > 0 and avoid.shape[1] > 0:
        for _ in range(1000):
            bad = np.zeros(n, bool)
            for s in range(avoid.shape[1]):
                d2 = ((pos - avoid[:, s:s + 1]) ** 2).sum(0)
                bad |= d2 <= radius * radius
            if not bad.any():
                break
            pos[:, bad] = rng.uniform(0.0, 1.0, (dim, int(bad.sum()))) * hi
    return pos


def make(name, dim, nx, ny, nz=1, *, h=1.0, D=1.0, lam=0.01, dt=0.2, n_src=4, emit=(1.0, 1.0),
         n_axons=64, stop_radius=0.0, wall_mode=0, nsteps=1, seed=0, philox_seed=None,
         src_map=False, targets=False, C0=None, w=(0.5, 0.4, 0.1), step_len=0.5,
         grad_eps=1e-15) -> Workload:
    """Draw one workload.  ``C0`` may be None (zeros), 'random' (U[0,1]), 'smooth' or 'ramp';
    ``src_map`` may be False (none), True / 'random' (U[0,1] per node) or 'zeros'."""
    rng = np.random.default_rng(seed)
    nz = nz if dim == 3 else 1
    extents = (nx, ny, nz)[:dim]
    n_cells = nx * ny * nz
    cells = _distinct_cells(rng, n_cells, n_src)
    if emit[0] == emit[1]:
        e = np.full(n_src, emit[0], np.float32)
    else:
        e = rng.uniform(emit[0], emit[1], n_src).astype(np.float32)
    src_xy = _cell_coords(cells, nx, ny, dim, h)
    pos = _positions(rng, extents, h, n_axons, avoid=src_xy, radius=stop_radius)
    dirs = _directions(rng, dim, n_axons)
    shape = (nz, ny, nx) if dim == 3 else (ny, nx)
    if src_map == "zeros":
        smap = np.zeros(shape, np.float32)
    elif src_map:                                   # True or "random": U[0, 1] per node
        smap = rng.uniform(0.0, 1.0, shape).astype(np.float32)
    else:
        smap = None
    tg = _positions(rng, extents, h, n_axons).astype(np.float32) if targets else None
    if isinstance(C0, str):
        if C0 == "random":
            C0 = rng.uniform(0.0, 1.0, shape).astype(np.float32)
        elif C0 == "smooth":
            C0 = _smooth_field(rng, shape)
        elif C0 == "ramp":
            C0 = _ramp_field(rng, shape)
        else:
            raise ValueError(C0)
    return Workload(
        name=name, dim=dim, nx=nx, ny=ny, nz=nz, h=h, D=D, lam=lam, dt=dt,
        src_cell=cells, src_emit=e, src_map=smap,
        pos=pos.astype(np.float32), dir=dirs.astype(np.float32),
        active=np.ones(n_axons, np.uint8),
        w_prev=w[0], w_grad=w[1], w_noise=w[2], step_len=step_len, stop_radius=stop_radius,
        grad_eps=grad_eps, wall_mode=wall_mode,
        seed=PHILOX_SEED_BASE + (seed if philox_seed is None else philox_seed),
        nsteps=nsteps, C0=C0, targets=tg)


def _smooth_field(rng, shape):
    """A positive field made of a few random Gaussian bumps plus a small random floor."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    out = np.full(shape, 0.01)
    for _ in range(6):
        centre = [rng.uniform(0, s) for s in shape]
        width = rng.uniform(0.1, 0.4) * max(shape)
        amp = rng.uniform(0.5, 5.0)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        out += amp * np.exp(-r2 / (2.0 * width * width))
    out += rng.uniform(0.0, 1e-3, shape)
    return out.astype(np.float32)


def _ramp_field(rng, shape):
    """A tilted plane of slope 0.05 per node along a random direction, plus bumps too shallow
    (slope below 0.005) to create a local maximum: a cue field with no interior critical point."""
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    axis = rng.standard_normal(len(shape))
    axis /= np.linalg.norm(axis)
    out = 1.0 + 0.05 * sum(a * (g - 0.5 * (s - 1)) for a, g, s in zip(axis, grids, shape))
    out -= out.min() - 0.5
    for _ in range(4):
        centre = [rng.uniform(0, s) for s in shape]
        width = 0.25 * max(shape)
        r2 = sum((g - c) ** 2 for g, c in zip(grids, centre))
        out += 0.005 * width * np.sqrt(np.e) * rng.uniform(0.2, 1.0) * np.exp(-r2 / (2.0 * width * width))
    return out.astype(np.float32)


# ---------------------------------------------------------------- configs
def config_c1(seed=0) -> Workload:
    return make("c1-2d-128", 2, 128, 128, h=1.0, D=1.0, lam=0.01, dt=0.2, n_src=4,
                emit=(1.0, 1.0), n_axons=64, nsteps=500, seed=seed, philox_seed=1)


def config_c2(seed=1) -> Workload:
    return make("c2-2d-2048", 2, 2048, 2048, h=1.0, D=1.0, lam=0.005, dt=0.2, n_src=64,
                emit=(0.5, 2.0), n_axons=16384, stop_radius=2.0, nsteps=5000, seed=seed,
                philox_seed=2)


def config_c2_clustered(seed=8) -> Workload:
    """The 2048^2 workload with its 16,384 cones starting clustered: four 48 x 48 node squares
    (4,096 cones each, uniform inside) centred on four points of the grid, wall clamp and no
    source stop, so no cone leaves the run and the cones stay crowded into a few field tiles."""
    w = make("c2-2d-2048-clustered", 2, 2048, 2048, h=1.0, D=1.0, lam=0.005, dt=0.2, n_src=64,
             emit=(0.5, 2.0), n_axons=16384, wall_mode=1, nsteps=5000, seed=seed, philox_seed=8)
    rng = np.random.default_rng(seed + 1000)
    centres = np.array([[512.0, 512.0], [1536.0, 512.0], [512.0, 1536.0], [1536.0, 1536.0]])
    pos = np.empty((2, 16384))
    for q in range(4):
        pos[:, q * 4096:(q + 1) * 4096] = centres[q][:, None] + rng.uniform(-24.0, 24.0, (2, 4096))
    w.pos = pos.astype(np.float32)
    return w


def config_c3(seed=2) -> Workload:
    return make("c3-3d-256", 3, 256, 256, 256, h=1.0, D=1.0, lam=0.01, dt=0.15, n_src=128,
                emit=(0.5, 2.0), n_axons=65536, nsteps=2000, seed=seed, philox_seed=3)


def config_c5(seed=4, n=1024, n_src=32, n_axons=4096, nsteps=2000) -> Workload:
    """Adjoint workload.  The dense rate map is the learnable per-node source term and its
    gradient is taken at M = 0 (a white-noise map makes the field rough and the cone paths
    chaotic, so the endpoint loss has no useful derivative)."""
    return make(f"c5-adjoint-2d-{n}", 2, n, n, h=1.0, D=1.0, lam=0.01, dt=0.2, n_src=n_src,
                emit=(0.5, 2.0), n_axons=n_axons, wall_mode=1, nsteps=nsteps, seed=seed,
                philox_seed=5, src_map="zeros", targets=True)


def config_c4(seed=3, n_instances=512, nsteps=1000) -> List[Workload]:
    """Batched: independent 2D instances, sides ~U{64..1024}, D ~ U[0.5,2],
    lambda ~ 10^U[-3,-1], dt = 0.2/D, 4-64 sources, 256-4096 cones."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_instances):
        nx = int(rng.integers(64, 1025))
        ny = int(rng.integers(64, 1025))
        D = float(rng.uniform(0.5, 2.0))
        lam = float(10.0 ** rng.uniform(-3.0, -1.0))
        n_src = int(rng.integers(4, 65))
        n_ax = int(rng.integers(256, 4097))
        sub = int(rng.integers(0, 2**31 - 1))
        out.append(make(f"c4-inst{b}", 2, nx, ny, h=1.0, D=D, lam=lam, dt=0.2 / D, n_src=n_src,
                        emit=(0.5, 2.0), n_axons=n_ax, nsteps=nsteps, seed=sub, philox_seed=4 + 16 * b))
    return out


def hbm_probe_2d(seed=5) -> Workload:
    """2D 8192^2 (256 MiB per buffer), C2 physics: the field cannot stay in L2."""
    return make("probe-2d-8192", 2, 8192, 8192, D=1.0, lam=0.005, dt=0.2, n_src=64,
                emit=(0.5, 2.0), n_axons=16384, stop_radius=2.0, nsteps=200, seed=seed,
                philox_seed=6)


def hbm_probe_3d(seed=6) -> Workload:
    """3D 512^3 (512 MiB per buffer), C3 physics."""
    return make("probe-3d-512", 3, 512, 512, 512, D=1.0, lam=0.01, dt=0.15, n_src=128,
                emit=(0.5, 2.0), n_axons=65536, nsteps=200, seed=seed, philox_seed=7)


@dataclasses.dataclass
class GraphWorkload:
    """Inputs of the connectivity stage: neurons, the growth cones grown from them, and the
    uniform grid that bins the neurons."""
    name: str
    npos: np.ndarray        # float32 [2, n_neurons]
    pos: np.ndarray         # float32 [2, n_cones]
    owner: np.ndarray       # int32 [n_cones]: the neuron each cone grows from
    active: np.ndarray      # uint8 [n_cones]
    radius: float           # connection distance (the sum of the two radii)
    cell: float             # grid cell side (>= radius)
    grid: tuple             # cells per axis
    source: int = 0         # BFS source vertex

    @property
    def n_neurons(self) -> int:
        return int(self.npos.shape[1])

    @property
    def n_cones(self) -> int:
        return int(self.pos.shape[1])


def config_graph(seed=7, extent=2048.0, n_neurons=262144, cones_per_neuron=4, reach=48.0,
                 radius=2.0) -> GraphWorkload:
    """Connectivity on the 2048^2 domain: neurons uniform in it, each with `cones_per_neuron`
    cones that have grown up to `reach` from it (uniform direction, uniform distance, clamped
    into the domain); 95% of the cones still growing; cells of side `radius`."""
    rng = np.random.default_rng(seed)
    hi = extent - 1.0
    npos = rng.uniform(0.0, hi, (2, n_neurons))
    owner = np.repeat(np.arange(n_neurons, dtype=np.int32), cones_per_neuron)
    n = owner.size
    ang = rng.uniform(0.0, 2.0 * np.pi, n)
    dist = rng.uniform(0.0, reach, n)
    pos = npos[:, owner] + np.stack([np.cos(ang), np.sin(ang)]) * dist
    pos = np.clip(pos, 0.0, hi)
    active = (rng.uniform(0.0, 1.0, n) < 0.95).astype(np.uint8)
    side = int(np.ceil(extent / radius))
    return GraphWorkload(name=f"graph-2d-{int(extent)}", npos=npos.astype(np.float32), pos=pos.astype(np.float32),
                         owner=owner, active=active, radius=radius, cell=radius, grid=(side, side))
