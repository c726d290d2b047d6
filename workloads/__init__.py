"""Seeded, synthetic input generators shared by the oracle and the CUDA path.

This module holds scene, source and grid *descriptions* only: plain Python
data, none of the transport arithmetic.  Both sides marshal these
descriptions into their own structures (the oracle through its private C
structs, the product through the C-ABI in ``include/smcrt.h``).

Geometry follows the paper's model (Sec. 2.2-2.3): a scene is a list of SDF
primitives, each optical region owns a postfix CSG program over them and
its own (mu_a, mu_s, g, n); a bounding box closes the volume of interest.
Units are cm and cm^-1 throughout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Primitive kinds (Sec. 2.2, Eq. 2-3; box and capsule used in Sec. 4; torus
# and capped cylinder among the basic shapes of the Fig. 1 gallery).
SPHERE, BOX, CAPSULE, TORUS, CYLINDER = "sphere", "box", "capsule", "torus", "cylinder"
# Domain operations of a primitive's frame (Sec. 2.2, Fig. 1 i, o, p, q).
XF_NONE, ELONGATE, TWIST, BEND, REPEAT = "none", "elongate", "twist", "bend", "repeat"
# CSG node kinds (Sec. 2.2, Fig. 1 e-h).  'prim' pushes a primitive.
PRIM, UNION, SMOOTH_UNION, INTERSECT, SUBTRACT = (
    "prim", "union", "smooth_union", "intersect", "subtract")
# Source kinds (photon release, Sec. 2.1 and the experiments of Sec. 3-4).
PENCIL, DISC, SQUARE, ISO_POINT = "pencil", "disc", "square", "iso"
# Step rules: plain sphere tracing (Sec. 2.3), or segment stepping (longer
# steps bounded along the ray; Sec. 5 names segment tracing).
SPHERE_TRACING, SEGMENT = "sphere_tracing", "segment"


@dataclass(frozen=True)
class Xform:
    """Frame of a primitive: a point with local coordinates l sits at
    s R l + t (R row-major, orthonormal).  op acts on the local point:
    elongate (a[0..2] half lengths), twist about local z / bend in the local
    x-y plane (a[0] turns per unit length, a[1] the radius the shape reaches
    from the axis), repeat (a[0..2] periods, 0 = none; a[3] copies each
    way)."""
    rot: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    t: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    s: float = 1.0
    op: str = XF_NONE
    a: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)


def rotation(axis: Sequence[float], degrees: float) -> Tuple[float, ...]:
    """Row-major rotation matrix about a unit axis (Rodrigues' formula)."""
    x, y, z = (float(v) for v in axis)
    n = math.sqrt(x * x + y * y + z * z)
    x, y, z = x / n, y / n, z / n
    th = math.radians(degrees)
    c, s, C1 = math.cos(th), math.sin(th), 1.0 - math.cos(th)
    return (c + x * x * C1, x * y * C1 - z * s, x * z * C1 + y * s,
            y * x * C1 + z * s, c + y * y * C1, y * z * C1 - x * s,
            z * x * C1 - y * s, z * y * C1 + x * s, c + z * z * C1)


@dataclass(frozen=True)
class Prim:
    """sphere: (cx, cy, cz, r); box: (cx, cy, cz, hx, hy, hz);
    capsule: (ax, ay, az, bx, by, bz, r); torus: (cx, cy, cz, R, r) about
    the z axis; cylinder: (cx, cy, cz, r, half height) along z.  With a
    frame the parameters are local coordinates."""
    kind: str
    params: Tuple[float, ...]
    xform: Optional[Xform] = None


@dataclass(frozen=True)
class Node:
    """One postfix CSG node: op, primitive index (for 'prim'), k (smooth)."""
    op: str
    prim: int = -1
    k: float = 0.0


@dataclass(frozen=True)
class Region:
    program: Tuple[Node, ...]
    mu_a: float
    mu_s: float
    g: float
    n: float


@dataclass(frozen=True)
class Scene:
    prims: Tuple[Prim, ...]
    regions: Tuple[Region, ...]
    ambient_n: float
    bbox_lo: Tuple[float, float, float]
    bbox_hi: Tuple[float, float, float]
    delta: float = 1e-6
    max_steps: int = 100_000
    stepping: str = SPHERE_TRACING


@dataclass(frozen=True)
class Source:
    kind: str
    pos: Tuple[float, float, float]
    dir: Tuple[float, float, float]
    radius: float = 0.0  # disc radius, or half side of the square


@dataclass(frozen=True)
class Grid:
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    n: Tuple[int, int, int]

    @property
    def size(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def voxel_volume(self) -> float:
        return float(np.prod([(h - l) / k for l, h, k in zip(self.lo, self.hi, self.n)]))


@dataclass(frozen=True)
class Workload:
    name: str
    scene: Scene
    source: Source
    grid: Grid
    npackets: int
    seed: int
    precision: str = "mixed"  # 'fp64' or 'mixed'

    def with_packets(self, n: int) -> "Workload":
        return replace(self, npackets=int(n))

    def with_stepping(self, stepping: str) -> "Workload":
        if stepping not in (SPHERE_TRACING, SEGMENT):
            raise ValueError(stepping)
        return replace(self, scene=replace(self.scene, stepping=stepping))


def prim_program(indices: Sequence[int], op: str = UNION, k: float = 0.0) -> Tuple[Node, ...]:
    """Left fold of ``op`` over the listed primitives, as a postfix program."""
    nodes: List[Node] = [Node(PRIM, int(indices[0]))]
    for i in indices[1:]:
        nodes.append(Node(PRIM, int(i)))
        nodes.append(Node(op, -1, k))
    return tuple(nodes)


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014), used only to derive
    per-job seeds for the served mix."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


# ---------------------------------------------------------------------------
# The five workloads.  Their concrete numbers are synthetic stand-ins
# for the scenes the paper describes (vessel network Sec. 4, glass bottle
# Sec. 4 / Fig. 7, layered tissue as in the Jacques slab of Sec. 3.1).
# ---------------------------------------------------------------------------

def sphere_pencil(npackets: int = 100_000, seed: int = 1, precision: str = "fp64") -> Workload:
    """Pencil beam at the pole of a turbid sphere r=1 cm (mu_a=1, mu_s=10,
    g=0.9, n=1.38) in air; 50^3 grid over the 2 cm cube."""
    scene = Scene(
        prims=(Prim(SPHERE, (0.0, 0.0, 0.0, 1.0)),),
        regions=(Region(prim_program([0]), 1.0, 10.0, 0.9, 1.38),),
        ambient_n=1.0,
        bbox_lo=(-1.25, -1.25, -1.25), bbox_hi=(1.25, 1.25, 1.25))
    return Workload("sphere_pencil_1e5_50c", scene,
                    Source(PENCIL, (0.0, 0.0, 1.2), (0.0, 0.0, -1.0)),
                    Grid((-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (50, 50, 50)),
                    npackets, seed, precision)


def three_layer_slab(npackets: int = 10_000_000, seed: int = 2, precision: str = "mixed",
                     grid_n: int = 100) -> Workload:
    """Three stacked box layers (0.1 / 0.2 / 1.0 cm), pencil beam at normal
    incidence; 100^3 grid over [-1,1]^2 x [-1.3,0]."""
    L = 5.0
    prims = (
        Prim(BOX, (0.0, 0.0, -0.05, L, L, 0.05)),   # z in [-0.1, 0]
        Prim(BOX, (0.0, 0.0, -0.20, L, L, 0.10)),   # z in [-0.3, -0.1]
        Prim(BOX, (0.0, 0.0, -0.80, L, L, 0.50)),   # z in [-1.3, -0.3]
    )
    regions = (
        Region(prim_program([0]), 0.1, 100.0, 0.90, 1.5),
        Region(prim_program([1]), 2.0, 50.0, 0.80, 1.3),
        Region(prim_program([2]), 0.5, 10.0, 0.95, 1.4),
    )
    scene = Scene(prims, regions, 1.0, (-5.1, -5.1, -1.4), (5.1, 5.1, 0.1))
    return Workload(f"three_layer_slab_{npackets:.0e}_{grid_n}c".replace("+0", ""), scene,
                    Source(PENCIL, (0.0, 0.0, 0.05), (0.0, 0.0, -1.0)),
                    Grid((-1.0, -1.0, -1.3), (1.0, 1.0, 0.0), (grid_n, grid_n, grid_n)),
                    npackets, seed, precision)


def vessel_tree_capsules(seed: int = 3, n: int = 64, cube: float = 0.5):
    """Seeded random branching tree of capsules inside a cube [0, cube]^3.

    Root at the top centre heading -z with radius 200 um; every further
    capsule starts at a uniformly chosen existing endpoint, heads within a
    45 degree cone about its parent's direction, has length U(0.02, 0.08) cm
    and radius parent * U(0.7, 0.95) clamped to [20, 200] um.  Endpoints are
    clamped inside the cube.  (Stand-in for the DeepVesselNet network of
    Sec. 4, which is not available.)"""
    rng = np.random.Generator(np.random.PCG64(seed))
    caps = []  # (a, b, r, dir)
    ends = []  # (point, dir, r)
    a = np.array([cube / 2, cube / 2, cube])
    d = np.array([0.0, 0.0, -1.0])
    r = 0.02
    for i in range(n):
        if i > 0:
            a, pd, pr = ends[int(rng.integers(len(ends)))]
            # direction inside a 45 degree cone about pd
            ct = 1.0 - rng.random() * (1.0 - math.cos(math.pi / 4))
            st = math.sqrt(max(0.0, 1.0 - ct * ct))
            ph = 2 * math.pi * rng.random()
            t1 = np.cross(pd, [1.0, 0.0, 0.0] if abs(pd[0]) < 0.9 else [0.0, 1.0, 0.0])
            t1 /= np.linalg.norm(t1)
            t2 = np.cross(pd, t1)
            d = ct * pd + st * (math.cos(ph) * t1 + math.sin(ph) * t2)
            d /= np.linalg.norm(d)
            r = min(0.02, max(0.002, pr * rng.uniform(0.7, 0.95)))
        length = rng.uniform(0.02, 0.08)
        b = np.clip(a + length * d, 0.0, cube)
        if np.linalg.norm(b - a) < 1e-4:  # clamped flat against a face: nudge inward
            b = np.clip(a - length * d, 0.0, cube)
        caps.append((tuple(map(float, a)), tuple(map(float, b)), float(r)))
        ends.append((b.copy(), d.copy(), r))
    return caps


def vessel_network(npackets: int = 100_000_000, seed: int = 3, precision: str = "mixed",
                   grid_n: int = 200, ncap: int = 64, smooth: bool = True) -> Workload:
    """5 mm tissue cube (mu_a=0.5, mu_s=100, g=0.9, n=1.4) with a 64-capsule
    smooth-union (k = 10 um) vessel tree (blood mu_a=20, mu_s=200, g=0.98,
    n=1.4); uniform square illumination of the top face; 200^3 grid.
    smooth=False joins the capsules by a plain union instead."""
    caps = vessel_tree_capsules(seed, ncap)
    prims = [Prim(BOX, (0.25, 0.25, 0.25, 0.25, 0.25, 0.25))]
    for a, b, r in caps:
        prims.append(Prim(CAPSULE, a + b + (r,)))
    regions = (
        Region(prim_program([0]), 0.5, 100.0, 0.90, 1.4),
        Region(prim_program(list(range(1, ncap + 1)), SMOOTH_UNION, 1e-3) if smooth
               else prim_program(list(range(1, ncap + 1))), 20.0, 200.0, 0.98, 1.4),
    )
    scene = Scene(tuple(prims), regions, 1.0, (-0.03, -0.03, -0.03), (0.53, 0.53, 0.53))
    return Workload(f"vessel_network_{ncap}cap_{grid_n}c" + ("" if smooth else "_hard"), scene,
                    Source(SQUARE, (0.25, 0.25, 0.525), (0.0, 0.0, -1.0), 0.25),
                    Grid((0.0, 0.0, 0.0), (0.5, 0.5, 0.5), (grid_n, grid_n, grid_n)),
                    npackets, seed, precision)


def vessel_network_hard(npackets: int = 2_000_000, seed: int = 3, precision: str = "mixed",
                        grid_n: int = 100) -> Workload:
    """The vessel tree with a plain union of its 64 capsules (sharp joints):
    a hard region of capsules, so segment stepping bounds moves by ray-capsule
    distances (and, in mixed mode, by the culled region's distance)."""
    return vessel_network(npackets, seed, precision, grid_n, 64, smooth=False)


def glass_container(npackets: int = 100_000_000, seed: int = 5, precision: str = "mixed",
                    mu_s: float = 20.0, grid_n: int = 128) -> Workload:
    """Glass shell sphere(3) minus sphere(2.8) (n=1.5, clear) holding a
    turbid liquid (mu_s=20, mu_a=0.01, g=0.7, n=1.33); 1 cm wide disc beam;
    128^3 grid over [-3.2, 3.2]^3."""
    prims = (Prim(SPHERE, (0.0, 0.0, 0.0, 3.0)), Prim(SPHERE, (0.0, 0.0, 0.0, 2.8)))
    regions = (
        Region((Node(PRIM, 0), Node(PRIM, 1), Node(SUBTRACT)), 0.0, 0.0, 0.0, 1.5),
        Region(prim_program([1]), 0.01, mu_s, 0.7, 1.33),
    )
    scene = Scene(prims, regions, 1.0, (-3.3, -3.3, -3.3), (3.3, 3.3, 3.3))
    return Workload(f"glass_container_mus{mu_s:g}_{grid_n}c", scene,
                    Source(DISC, (0.0, 0.0, 3.2), (0.0, 0.0, -1.0), 0.5),
                    Grid((-3.2, -3.2, -3.2), (3.2, 3.2, 3.2), (grid_n, grid_n, grid_n)),
                    npackets, seed, precision)


def glass_sphere_beam(npackets: int = 27_000_000, seed: int = 9, precision: str = "mixed",
                      beam_radius: float = 0.3, grid_n: int = 200, grid=None) -> Workload:
    """The smooth-surface test of Sec. 3.2 (Fig. 5): a clear glass sphere
    (n = 1.46, radius 1 cm) centred at (0.5, 0, -1) cm in air, lit from above
    by a uniform disc beam of radius 0.3 cm along the sphere's axis; about
    2.7e7 photons.  The paper leaves the medium's extent, the grid and the
    beam profile open: the bounding box holds the sphere and its focal region
    below, and the grid covers the bounding box at grid_n^3 unless given."""
    prims = (Prim(SPHERE, (0.5, 0.0, -1.0, 1.0)),)
    regions = (Region(prim_program([0]), 0.0, 0.0, 0.0, 1.46),)
    lo, hi = (-1.5, -2.0, -4.0), (2.5, 2.0, 0.5)
    scene = Scene(prims, regions, 1.0, lo, hi)
    g = grid if grid is not None else Grid((-1.5, -2.0, -4.0), (2.5, 2.0, 0.0), (grid_n, grid_n, grid_n))
    return Workload(f"glass_sphere_beam_{npackets:.0e}".replace("+0", ""), scene,
                    Source(DISC, (0.5, 0.0, 0.25), (0.0, 0.0, -1.0), beam_radius), g, npackets, seed, precision)


def served_mix(njobs: int = 200, seed: int = 4, budget_lo: float = 1e4, budget_hi: float = 1e7,
               stepping: str = SPHERE_TRACING):
    """Served mix: jobs drawn from the four scene families with optics redrawn
    uniformly within each family's ranges, log-uniform packet budgets, grid
    sides from {50, 64, 100, 128, 200}, per-job seed splitmix64(seed, j).
    Returns a list of Workloads; arrival times are drawn by the caller at a
    rate matched to measured capacity."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = (50, 64, 100, 128, 200)
    jobs = []
    for j in range(njobs):
        fam = int(rng.integers(4))
        budget = int(round(math.exp(rng.uniform(math.log(budget_lo), math.log(budget_hi)))))
        side = int(sides[int(rng.integers(len(sides)))])
        jseed = splitmix64((seed << 32) + j)
        if fam == 0:
            w = sphere_pencil(budget, jseed, "mixed")
            r = w.scene.regions[0]
            reg = replace(r, mu_a=float(rng.uniform(0.5, 2.0)), mu_s=float(rng.uniform(5, 20)),
                          g=float(rng.uniform(0.8, 0.95)), n=float(rng.uniform(1.33, 1.45)))
            w = replace(w, scene=replace(w.scene, regions=(reg,)))
        elif fam == 1:
            w = three_layer_slab(budget, jseed, "mixed")
            regs = tuple(replace(r, mu_a=float(rng.uniform(0.1, 2.0)), mu_s=float(rng.uniform(10, 100)),
                                 g=float(rng.uniform(0.8, 0.95)), n=float(rng.uniform(1.3, 1.5)))
                         for r in w.scene.regions)
            w = replace(w, scene=replace(w.scene, regions=regs))
        elif fam == 2:
            w = vessel_network(budget, 3, "mixed", ncap=64)
            t, v = w.scene.regions
            t = replace(t, mu_a=float(rng.uniform(0.3, 1.0)), mu_s=float(rng.uniform(50, 150)))
            v = replace(v, mu_a=float(rng.uniform(10, 30)), mu_s=float(rng.uniform(100, 300)))
            w = replace(w, seed=jseed, scene=replace(w.scene, regions=(t, v)))
        else:
            w = glass_container(budget, jseed, "mixed", mu_s=float(rng.uniform(5, 50)))
        g = w.grid
        w = replace(w, grid=Grid(g.lo, g.hi, (side, side, side)),
                    name=f"mix{j:03d}_{w.name.split('_')[0]}")
        jobs.append(w.with_stepping(stepping))
    return jobs


# ---------------------------------------------------------------------------
# Closed-form test scenes (pins for the oracle).
# ---------------------------------------------------------------------------

def slab_scene(mu_a: float, mu_s: float, g: float, n: float, thickness: float,
               ambient_n: float = 1.0, half: float = 20.0) -> Scene:
    """Laterally wide slab z in [-thickness, 0] in an ambient medium."""
    prims = (Prim(BOX, (0.0, 0.0, -thickness / 2, half, half, thickness / 2)),)
    return Scene(prims, (Region(prim_program([0]), mu_a, mu_s, g, n),), ambient_n,
                 (-half + 0.5, -half + 0.5, -thickness - 0.5), (half - 0.5, half - 0.5, 0.5))


def halfspace_scene(n_upper: float, n_lower: float, mu_a_lower: float = 0.0) -> Scene:
    """A clear upper region (box z in [0, 2], wider than the bounding box) over
    an ambient lower half-space; escapes happen only through the bounding box,
    so exactly one refractive interface (z = 0) exists in the volume."""
    prims = (Prim(BOX, (0.0, 0.0, 1.0, 10.0, 10.0, 1.0)),)
    return Scene(prims, (Region(prim_program([0]), 0.0, 0.0, 0.0, n_upper),), n_lower,
                 (-5.0, -5.0, -1.0), (5.0, 5.0, 1.0))


def clear_halfspace_lower(n_upper: float, n_lower: float) -> Scene:
    """Mirror of ``halfspace_scene``: the region is the lower box, ambient above."""
    prims = (Prim(BOX, (0.0, 0.0, -1.0, 10.0, 10.0, 1.0)),)
    return Scene(prims, (Region(prim_program([0]), 0.0, 0.0, 0.0, n_lower),), n_upper,
                 (-5.0, -5.0, -1.0), (5.0, 5.0, 1.0))


def isotropic_sphere(tau: float, radius: float = 0.5) -> Scene:
    """Pure isotropic scatterer (g = 0, mu_a = 0) of radial optical depth tau,
    index-matched to its surroundings (Sec. 3.1, Eq. 4)."""
    prims = (Prim(SPHERE, (0.0, 0.0, 0.0, radius)),)
    b = radius + 0.1
    return Scene(prims, (Region(prim_program([0]), 0.0, tau / radius, 0.0, 1.0),), 1.0,
                 (-b, -b, -b), (b, b, b))


# Table 1 (Sec. 3.1): absorption and reduced scattering per wavelength, for
# a slab with g = 0.9 and n = 1.38 under air.
JACQUES_OPTICS = {420: (1.8, 82.0), 630: (0.23, 21.0)}


def penetration_depth(mu_a: float, mus_reduced: float) -> float:
    """delta = 1 / sqrt(3 mu_a (mu_a + mu_s (1 - g))) (Sec. 3.1, with Eq. 5)."""
    return 1.0 / math.sqrt(3.0 * mu_a * (mu_a + mus_reduced))


def jacques_slab(wavelength_nm: int = 630, npackets: int = 10_000_000, seed: int = 6,
                 precision: str = "mixed", grid_n: Tuple[int, int, int] = (200, 200, 400)) -> Workload:
    """The semi-infinite slab of the validation against Jacques et al. (Sec.
    3.1, Table 1) at the size of its timing case (Table 2: 1e7 photons, a
    200 x 200 x 400 grid): g = 0.9, n = 1.38 under air, light uniformly
    incident on the surface.  The slab is z in [-40 delta, 0], 100 cm wide;
    the source is a uniform 4 x 4 cm square just above the surface, going -z;
    the grid covers x, y in [-1, 1] cm and z in [-16 delta, 0]."""
    mua, musp = JACQUES_OPTICS[wavelength_nm]
    g = 0.9
    d = penetration_depth(mua, musp)
    scene = slab_scene(mua, musp / (1.0 - g), g, 1.38, 40.0 * d, half=50.0)
    return Workload(f"jacques_slab_{wavelength_nm}nm", scene,
                    Source(SQUARE, (0.0, 0.0, 0.05), (0.0, 0.0, -1.0), 2.0),
                    Grid((-1.0, -1.0, -16.0 * d), (1.0, 1.0, 0.0), grid_n), npackets, seed, precision)


def iso_sphere(tau: float = 100.0, npackets: int = 1_000_000, seed: int = 7, precision: str = "mixed",
               grid_n: int = 200) -> Workload:
    """Photons released isotropically from the centre of a pure isotropic
    scatterer of radius 0.5 cm and radial optical depth tau (Sec. 3.1, Eq. 4;
    at tau = 100 with 1e6 photons and a 200^3 grid, the timing case of
    Table 2)."""
    return Workload(f"iso_sphere_tau{tau:g}", isotropic_sphere(tau, 0.5),
                    Source(ISO_POINT, (0.0, 0.0, 0.0), (0.0, 0.0, -1.0)),
                    Grid((-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), (grid_n, grid_n, grid_n)),
                    npackets, seed, precision)


def sdf_gallery(npackets: int = 1_000_000, seed: int = 8, precision: str = "mixed",
                grid_n: int = 100) -> Workload:
    """The shapes and operations of the Fig. 1 gallery in one transport scene
    (Sec. 2.2): a tissue block z in [-2, 0] holding a tilted torus, a box
    rotated about an oblique axis, a twisted bar, a bent bar, an elongated
    sphere, a 5 x 5 array of repeated spheres (index-matched) and a capped
    cylinder scaled by 1.5, each its own region with its own optics and
    refractive index; disc beam r = 1.5 cm from above."""
    prims = (
        Prim(BOX, (0.0, 0.0, -1.0, 2.0, 2.0, 1.0)),
        Prim(TORUS, (0.0, 0.0, 0.0, 0.5, 0.15), Xform(rot=rotation((1, 0, 0), 45.0), t=(-1.0, -1.0, -1.0))),
        Prim(BOX, (0.0, 0.0, 0.0, 0.4, 0.2, 0.2), Xform(rot=rotation((1, 1, 1), 30.0), t=(1.0, -1.0, -1.0))),
        Prim(BOX, (0.0, 0.0, 0.0, 0.15, 0.15, 0.5),
             Xform(t=(-1.0, 1.0, -1.0), op=TWIST, a=(0.25, 0.2122, 0.0, 0.0))),
        Prim(BOX, (0.0, 0.0, 0.0, 0.6, 0.1, 0.1), Xform(t=(1.0, 1.0, -1.0), op=BEND, a=(0.15, 0.61, 0.0, 0.0))),
        Prim(SPHERE, (0.0, 0.0, 0.0, 0.1), Xform(t=(0.0, 0.0, -0.5), op=ELONGATE, a=(0.3, 0.0, 0.0, 0.0))),
        Prim(SPHERE, (0.0, 0.0, 0.0, 0.08), Xform(t=(0.0, 0.0, -1.6), op=REPEAT, a=(0.3, 0.3, 0.0, 2.0))),
        Prim(CYLINDER, (0.0, 0.0, 0.0, 0.2, 0.25), Xform(t=(0.0, 0.0, -1.0), s=1.5)),
    )
    regions = (
        Region(prim_program([0]), 0.2, 20.0, 0.8, 1.37),
        Region(prim_program([1]), 1.0, 50.0, 0.9, 1.45),
        Region(prim_program([2]), 0.5, 10.0, 0.8, 1.5),
        Region(prim_program([3]), 2.0, 30.0, 0.9, 1.4),
        Region(prim_program([4]), 0.3, 5.0, 0.7, 1.33),
        Region(prim_program([5]), 5.0, 100.0, 0.95, 1.4),
        Region(prim_program([6]), 3.0, 60.0, 0.9, 1.37),
        Region(prim_program([7]), 0.1, 2.0, 0.5, 1.55),
    )
    scene = Scene(prims, regions, 1.0, (-2.1, -2.1, -2.1), (2.1, 2.1, 0.2))
    return Workload(f"sdf_gallery_{grid_n}c", scene, Source(DISC, (0.0, 0.0, 0.1), (0.0, 0.0, -1.0), 1.5),
                    Grid((-2.0, -2.0, -2.0), (2.0, 2.0, 0.0), (grid_n, grid_n, grid_n)), npackets, seed, precision)


def all_configs():
    """The four single-job workloads at their stated sizes."""
    return [sphere_pencil(), three_layer_slab(), vessel_network(), glass_container()]
