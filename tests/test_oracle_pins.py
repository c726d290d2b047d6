"""Pins for the FP64 CPU oracle: each test ties one part of the oracle to
something other than itself -- published known answers, closed forms of
the physics, exact invariants, or brute force on small inputs.

Paper references: Eq. 1 (free path), Eq. 2-3 (sphere SDF), Sec. 2.2 (CSG),
Sec. 2.3 / Fig. 2-3 (sphere tracing, Fresnel at index changes), Sec. 3.1
(Eq. 4 scattering count, HG phase function, Table 1 penetration depth),
Sec. 3.1-3.2 (rectangular fluence bins).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from conftest import read_golden

FX = O.FX


# --------------------------------------------------------------------------
# Random numbers: Philox4x32-10 known answers and the uniform mapping.
# --------------------------------------------------------------------------

def test_philox_known_answers():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniforms_in_half_open_unit_interval():
    # xi = (w + 1) 2^-32 lies in (0, 1] so that -ln(xi) (Eq. 1) is finite;
    # the stream is keyed by (seed, packet id) and counted by event.
    u = O.uniforms(seed=123, pid=7, event0=0, ncalls=5000)
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    w = O.philox([0, 0, 7, 0], [123, 0])
    assert np.array_equal(u[:4], (np.array(w, dtype=np.float64) + 1.0) / 2.0 ** 32)
    # different packet ids and seeds give different streams
    assert not np.array_equal(u[:4], O.uniforms(123, 8)[:4])
    assert not np.array_equal(u[:4], O.uniforms(124, 7)[:4])


# --------------------------------------------------------------------------
# Project-written ln and sin/cos: accuracy against libm.
# --------------------------------------------------------------------------

def _ulp_err(a, b):
    return abs(a - b) / math.ulp(b) if b != 0 else abs(a)


def test_log_accuracy():
    rng = np.random.default_rng(0)
    xs = np.concatenate([
        (rng.integers(0, 2 ** 32, 20000).astype(np.float64) + 1.0) / 2.0 ** 32,
        rng.uniform(1e-300, 1.0, 2000), rng.uniform(1.0, 1e6, 2000),
        [1.0, 0.5, 2.0, math.sqrt(2.0), 1 / math.sqrt(2.0), 2.0 ** -32, 0.999999]])
    worst = max(_ulp_err(O.log(x), math.log(x)) for x in xs if x != 1.0)
    assert worst <= 2.0, worst
    assert O.log(1.0) == 0.0


def test_sincos2pi_accuracy():
    rng = np.random.default_rng(1)
    ts = np.concatenate([(rng.integers(0, 2 ** 32, 20000) + 1.0) / 2.0 ** 32,
                         [0.125, 0.25, 0.375, 0.5, 0.75, 1.0, 2.0 ** -32]])
    for t in ts:
        s, c = O.sincos2pi(t)
        # absolute error against libm of 2 pi t (2 pi t itself rounds at 4e-16)
        assert abs(s - math.sin(2 * math.pi * t)) < 2e-15
        assert abs(c - math.cos(2 * math.pi * t)) < 2e-15
        assert abs(s * s + c * c - 1.0) < 4e-16
    s, c = O.sincos2pi(0.25)
    assert s == 1.0 and c == 0.0 or abs(c) < 1e-300


# --------------------------------------------------------------------------
# SDFs (Sec. 2.2): exact distances by brute force, and CSG semantics.
# --------------------------------------------------------------------------

def _one_region_scene(prims, program):
    return W.Scene(tuple(prims), (W.Region(tuple(program), 0.0, 0.0, 0.0, 1.0),), 1.0,
                   (-10.0, -10.0, -10.0), (10.0, 10.0, 10.0))


def test_sphere_sdf_eq2():
    sc = _one_region_scene([W.Prim(W.SPHERE, (0.3, -0.2, 0.1, 0.7))], W.prim_program([0]))
    rng = np.random.default_rng(2)
    for p in rng.uniform(-2, 2, (200, 3)):
        want = np.linalg.norm(p - [0.3, -0.2, 0.1]) - 0.7
        assert abs(O.region_sdf(sc, 0, p) - want) < 1e-14


def _fib_sphere(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


def test_box_sdf_brute_force():
    c, h = np.array([0.1, 0.2, -0.3]), np.array([0.5, 0.25, 0.4])
    sc = _one_region_scene([W.Prim(W.BOX, tuple(c) + tuple(h))], W.prim_program([0]))
    # dense sample of the box surface: 6 faces on a 161x161 lattice
    m = 161
    a = np.linspace(-1, 1, m)
    A, B = np.meshgrid(a, a)
    pts = []
    for ax in range(3):
        o = [k for k in range(3) if k != ax]
        for s in (-1, 1):
            f = np.zeros((m * m, 3))
            f[:, ax] = s * h[ax]
            f[:, o[0]] = A.ravel() * h[o[0]]
            f[:, o[1]] = B.ravel() * h[o[1]]
            pts.append(f)
    surf = np.concatenate(pts) + c
    spacing = 2 * h.max() / (m - 1)
    rng = np.random.default_rng(3)
    for p in rng.uniform(-1.5, 1.5, (150, 3)) + c:
        dmin = np.sqrt(((surf - p) ** 2).sum(1)).min()
        inside = np.all(np.abs(p - c) < h)
        d = O.region_sdf(sc, 0, p)
        assert (d < 0) == inside
        assert abs(abs(d) - dmin) <= spacing, (p, d, dmin)


def test_capsule_sdf_brute_force():
    a, b, r = np.array([0.0, 0.1, 0.2]), np.array([0.6, -0.3, 0.5]), 0.15
    sc = _one_region_scene([W.Prim(W.CAPSULE, tuple(a) + tuple(b) + (r,))], W.prim_program([0]))
    t = np.linspace(0, 1, 20001)[:, None]
    seg = a + t * (b - a)
    rng = np.random.default_rng(4)
    for p in rng.uniform(-1, 1, (200, 3)):
        want = np.sqrt(((seg - p) ** 2).sum(1)).min() - r
        assert abs(O.region_sdf(sc, 0, p) - want) < 1e-4 * np.linalg.norm(b - a)


def test_csg_semantics():
    s1 = W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 1.0))
    s2 = W.Prim(W.SPHERE, (0.8, 0.0, 0.0, 0.6))
    rng = np.random.default_rng(5)
    pts = rng.uniform(-2, 2, (100, 3))
    d1 = np.linalg.norm(pts, axis=1) - 1.0
    d2 = np.linalg.norm(pts - [0.8, 0, 0], axis=1) - 0.6
    for op, want in [(W.UNION, np.minimum(d1, d2)), (W.INTERSECT, np.maximum(d1, d2)),
                     (W.SUBTRACT, np.maximum(d1, -d2))]:
        sc = _one_region_scene([s1, s2], [W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(op)])
        got = np.array([O.region_sdf(sc, 0, p) for p in pts])
        assert np.allclose(got, want, atol=1e-14), op
    # smooth union: equals the hard union where the operands differ by >= k,
    # lies below it (never above) and by at most k/4 where they are close.
    k = 0.3
    sc = _one_region_scene([s1, s2], [W.Node(W.PRIM, 0), W.Node(W.PRIM, 1),
                                      W.Node(W.SMOOTH_UNION, -1, k)])
    got = np.array([O.region_sdf(sc, 0, p) for p in pts])
    hard = np.minimum(d1, d2)
    far = np.abs(d1 - d2) >= k
    assert np.allclose(got[far], hard[far], atol=1e-14)
    assert np.all(got <= hard + 1e-14) and np.all(hard - got <= k / 4 + 1e-14)
    # at equal operands the rounding is exactly k/4
    mid = np.array([0.4, 0.0, 0.0])
    e1 = np.linalg.norm(mid) - 1.0
    sc2 = _one_region_scene([W.Prim(W.SPHERE, (0, 0, 0, 1.0)), W.Prim(W.SPHERE, (0.8, 0, 0, 0.4 - e1))],
                            [W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(W.SMOOTH_UNION, -1, k)])
    assert abs(O.region_sdf(sc2, 0, mid) - (e1 - k / 4)) < 1e-14

# --------------------------------------------------------------------------
# More primitives, frames and domain operations (Sec. 2.2, Fig. 1 gallery).
# --------------------------------------------------------------------------

def _sdf(prim, p):
    return O.region_sdf(_one_region_scene([prim], W.prim_program([0])), 0, p)


def test_torus_sdf_brute_force():
    c, R, r = np.array([0.2, -0.1, 0.3]), 0.6, 0.2
    prim = W.Prim(W.TORUS, tuple(c) + (R, r))
    # dense parametric sample of the surface
    u, v = np.meshgrid(np.linspace(0, 2 * np.pi, 721), np.linspace(0, 2 * np.pi, 241))
    surf = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], -1)
    surf = surf.reshape(-1, 3) + c
    spacing = 2 * np.pi * (R + r) / 720
    rng = np.random.default_rng(11)
    for p in rng.uniform(-1.2, 1.2, (120, 3)) + c:
        q = p - c
        inside = (math.hypot(q[0], q[1]) - R) ** 2 + q[2] ** 2 < r * r
        d = _sdf(prim, p)
        assert (d < 0) == inside
        assert abs(abs(d) - np.sqrt(((surf - p) ** 2).sum(1)).min()) <= spacing, p


def test_cylinder_sdf_brute_force():
    c, r, h = np.array([-0.1, 0.2, 0.0]), 0.4, 0.3
    prim = W.Prim(W.CYLINDER, tuple(c) + (r, h))
    u, z = np.meshgrid(np.linspace(0, 2 * np.pi, 481), np.linspace(-h, h, 121))
    side = np.stack([r * np.cos(u), r * np.sin(u), z], -1).reshape(-1, 3)
    uu, rr = np.meshgrid(np.linspace(0, 2 * np.pi, 481), np.linspace(0, r, 81))
    caps = [np.stack([rr * np.cos(uu), rr * np.sin(uu), np.full_like(rr, s * h)], -1).reshape(-1, 3)
            for s in (-1, 1)]
    surf = np.concatenate([side] + caps) + c
    spacing = 2 * np.pi * r / 480 + 2 * h / 120
    rng = np.random.default_rng(12)
    for p in rng.uniform(-1.0, 1.0, (120, 3)) + c:
        q = p - c
        inside = math.hypot(q[0], q[1]) < r and abs(q[2]) < h
        d = _sdf(prim, p)
        assert (d < 0) == inside
        assert abs(abs(d) - np.sqrt(((surf - p) ** 2).sum(1)).min()) <= spacing, p


def test_rigid_frame_box_brute_force():
    # a box placed by a rotation about an oblique axis, a translation and a
    # uniform scale: its distance is the distance to the placed surface
    h = np.array([0.5, 0.2, 0.3])
    X = W.Xform(rot=W.rotation((1.0, 2.0, -0.5), 37.0), t=(0.3, -0.4, 0.2), s=1.3)
    prim = W.Prim(W.BOX, (0.0, 0.0, 0.0) + tuple(h), X)
    Rm = np.array(X.rot).reshape(3, 3)
    m = 121
    a = np.linspace(-1, 1, m)
    A, B = np.meshgrid(a, a)
    faces = []
    for ax in range(3):
        o = [k for k in range(3) if k != ax]
        for sgn in (-1, 1):
            f = np.zeros((m * m, 3))
            f[:, ax] = sgn * h[ax]
            f[:, o[0]] = A.ravel() * h[o[0]]
            f[:, o[1]] = B.ravel() * h[o[1]]
            faces.append(f)
    surf = X.s * np.concatenate(faces) @ Rm.T + np.array(X.t)     # world = s R l + t
    spacing = X.s * 2 * h.max() / (m - 1)
    rng = np.random.default_rng(13)
    for p in rng.uniform(-1.5, 1.5, (120, 3)):
        loc = Rm.T @ (p - np.array(X.t)) / X.s
        inside = np.all(np.abs(loc) < h)
        d = _sdf(prim, p)
        assert (d < 0) == inside
        assert abs(abs(d) - np.sqrt(((surf - p) ** 2).sum(1)).min()) <= spacing, p


def test_quarter_turn_and_scale_identities():
    # a quarter turn about z swaps the box's x and y half extents; a scaled
    # sphere is the sphere of scaled radius
    rng = np.random.default_rng(14)
    qt = W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.5, 0.2, 0.3), W.Xform(rot=W.rotation((0, 0, 1), 90.0), t=(0.1, 0.2, 0.3)))
    swapped = W.Prim(W.BOX, (0.1, 0.2, 0.3, 0.2, 0.5, 0.3))
    sc = W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 0.4), W.Xform(t=(0.2, 0.0, -0.1), s=2.5))
    big = W.Prim(W.SPHERE, (0.2, 0.0, -0.1, 1.0))
    for p in rng.uniform(-2, 2, (100, 3)):
        assert abs(_sdf(qt, p) - _sdf(swapped, p)) < 1e-12
        assert abs(_sdf(sc, p) - _sdf(big, p)) < 1e-12


def test_elongated_sphere_is_capsule():
    # elongating a sphere of radius r by h along x gives the capsule on the
    # segment [-h, h] x {0} x {0} of radius r (Fig. 1 o)
    h, r = 0.35, 0.2
    el = W.Prim(W.SPHERE, (0.0, 0.0, 0.0, r), W.Xform(t=(0.1, -0.2, 0.3), op=W.ELONGATE, a=(h, 0.0, 0.0, 0.0)))
    cap = W.Prim(W.CAPSULE, (0.1 - h, -0.2, 0.3, 0.1 + h, -0.2, 0.3, r))
    rng = np.random.default_rng(15)
    for p in rng.uniform(-1.5, 1.5, (200, 3)):
        assert abs(_sdf(el, p) - _sdf(cap, p)) < 1e-12


def test_repetition_is_union_of_copies():
    # repeating a centred sphere with periods (0.5, 0.7) and 2 copies each way
    # equals the union of the 25 explicit spheres, everywhere (Fig. 1 i)
    r, c = 0.15, (0.5, 0.7, 0.0)
    rep = W.Prim(W.SPHERE, (0.0, 0.0, 0.0, r), W.Xform(t=(0.1, 0.0, 0.0), op=W.REPEAT, a=c + (2.0,)))
    copies = [W.Prim(W.SPHERE, (0.1 + i * c[0], j * c[1], 0.0, r)) for i in range(-2, 3) for j in range(-2, 3)]
    union = _one_region_scene(copies, W.prim_program(list(range(len(copies)))))
    rng = np.random.default_rng(16)
    for p in rng.uniform(-2.5, 2.5, (300, 3)):
        assert abs(_sdf(rep, p) - O.region_sdf(union, 0, p)) < 1e-12


def _membership_twist(p, h, k, bend=False):
    # inside test written from the definition: rotate (x, y) by 2 pi k z
    # (twist) or 2 pi k x (bend), then test the box
    th = 2 * math.pi * k * (p[0] if bend else p[2])
    x = math.cos(th) * p[0] - math.sin(th) * p[1]
    y = math.sin(th) * p[0] + math.cos(th) * p[1]
    return abs(x) < h[0] and abs(y) < h[1] and abs(p[2]) < h[2]


@pytest.mark.parametrize("op", [W.TWIST, W.BEND])
def test_twist_bend_sign_and_safe_bound(op):
    # the twisted / bent box: negative exactly inside the deformed shape, and
    # a safe sphere-tracing distance: no point of the ball of radius |d(p)|
    # about p changes membership (the deformation stretches space, so the
    # distance is divided by the map's stretch bound; Sec. 5 on non-bounded
    # SDFs).  Membership is written from the definition, independently.
    h = (0.5, 0.12, 0.4) if op == W.BEND else (0.15, 0.1, 0.6)
    k = 0.3
    rho = math.hypot(h[0], h[1])
    prim = W.Prim(W.BOX, (0.0, 0.0, 0.0) + h, W.Xform(op=op, a=(k, rho, 0.0, 0.0)))
    bend = op == W.BEND
    rng = np.random.default_rng(17 if op == W.TWIST else 18)
    pts = rng.uniform(-0.8, 0.8, (300, 3))
    d = np.array([_sdf(prim, p) for p in pts])
    for p, dv in zip(pts, d):
        assert (dv < 0) == _membership_twist(p, h, k, bend), p
    dirs = _fib_sphere(200)
    tight = 0
    for p, dv in zip(pts[:150], d[:150]):
        inside = dv < 0
        for f in (0.5, 0.999999):
            for q in p + f * abs(dv) * dirs:
                assert _membership_twist(q, h, k, bend) == inside, (p, dv, q)
        # not vacuous: a ball a few times larger reaches the other side
        tight += any(_membership_twist(q, h, k, bend) != inside for q in p + 3.0 * abs(dv) * dirs)
    assert tight > 100


def test_rotated_scaled_slab_beer_lambert():
    # transport through a placed primitive: a non-scattering, index-matched
    # slab of local thickness 0.5, scaled by 1.4 and tilted 30 degrees, with
    # the beam along its normal: T = exp(-mu * 0.7)
    mu, n = 1.1, 40000
    Rm = W.rotation((1.0, 0.0, 0.0), 30.0)
    slab = W.Prim(W.BOX, (0.0, 0.0, 0.0, 3.0, 3.0, 0.25), W.Xform(rot=Rm, t=(0.0, 0.0, -1.0), s=1.4))
    sc = W.Scene((slab,), (W.Region(W.prim_program([0]), mu, 0.0, 0.0, 1.0),), 1.0, (-4, -4, -4), (4, 4, 4))
    nrm = np.array(Rm).reshape(3, 3) @ np.array([0.0, 0.0, 1.0])
    start = np.array([0.0, 0.0, -1.0]) + 1.5 * nrm
    _, tot, _ = _run(sc, W.Source(W.PENCIL, tuple(start), tuple(-nrm)), n, 23, fluence=False)
    assert _within(_frac(tot, "T"), math.exp(-mu * 0.7), n)
    assert tot["fresnel"] == 0


def test_gallery_energy_and_segment_safety():
    wl = W.sdf_gallery(400, grid_n=20)
    _, tot, rec = O.run(wl, records=True)
    pb = rec["R"] + rec["T"] + rec["A"] + rec["killed"] - rec["gain"]
    assert np.all(np.abs(pb - FX) <= 0.5 * (rec["scatters"] + 3) + 1)
    assert tot["fresnel"] > 0 and tot["max_steps_hit"] == 0
    # the same transport with segment stepping: identical physics, R/T/A agree
    _, ts, _ = O.run(wl.with_stepping(W.SEGMENT).with_packets(4000), 10_000, 14_000)
    _, tp, _ = O.run(wl.with_packets(4000), 20_000, 24_000)
    for key in ("R", "T", "A"):
        assert abs(_frac(ts, key) - _frac(tp, key)) < 5 * math.sqrt(0.25 / 4000) * 1.5



def test_scene_eval_region_priority_and_dmin():
    # two nested regions: later index wins where both contain p
    sc = W.Scene((W.Prim(W.SPHERE, (0, 0, 0, 1.0)), W.Prim(W.SPHERE, (0, 0, 0, 0.5))),
                 (W.Region(W.prim_program([0]), 0, 0, 0, 1.3), W.Region(W.prim_program([1]), 0, 0, 0, 1.5)),
                 1.0, (-2, -2, -2), (2, 2, 2))
    e = O.scene_eval(sc, [0.0, 0.0, 0.2])
    assert e["region"] == 1 and abs(e["dmin"] - 0.3) < 1e-15 and e["istar"] == 1
    e = O.scene_eval(sc, [0.0, 0.0, 0.8])
    assert e["region"] == 0 and abs(e["dmin"] - 0.2) < 1e-15 and e["istar"] == 0
    e = O.scene_eval(sc, [0.0, 0.0, 1.9])
    assert e["region"] == -1 and abs(e["dmin"] - 0.1) < 1e-15 and e["istar"] == -1
    assert abs(e["dbox"] + 0.1) < 1e-15


def test_normal_unit_gradient():
    # |grad d| = 1 for exact SDFs away from the medial axis; the normal
    # points out of the region.
    sc = _one_region_scene([W.Prim(W.SPHERE, (0.1, 0.0, 0.0, 1.0))], W.prim_program([0]))
    rng = np.random.default_rng(6)
    for v in _fib_sphere(50):
        p = np.array([0.1, 0, 0]) + v * (1.0 + rng.uniform(-5e-7, 5e-7))
        n = O.surface_normal(sc, 0, p)
        assert np.allclose(n, v, atol=1e-8)
    sc = _one_region_scene([W.Prim(W.BOX, (0, 0, 0, 1.0, 2.0, 3.0))], W.prim_program([0]))
    assert np.allclose(O.surface_normal(sc, 0, [0.2, 2.0, 0.1]), [0, 1, 0], atol=1e-9)
    assert np.allclose(O.surface_normal(sc, 0, [0.2, 0.5, -3.0]), [0, 0, -1], atol=1e-9)


# --------------------------------------------------------------------------
# Henyey-Greenstein sampling and the scattering rotation.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("g", [0.0, 0.3, 0.7, 0.9, 0.98, -0.5])
def test_hg_moments(g):
    # HG Legendre moments: <cos> = g, <P2(cos)> = g^2 -> <cos^2> = (1 + 2 g^2)/3.
    n = 200000
    xi = (np.arange(n) + 0.5) / n
    c = np.array([O.hg_cos(g, x) for x in xi[::20]])  # every 20th of the stratified grid
    assert abs(c.mean() - g) < 2e-3
    assert abs((c * c).mean() - (1 + 2 * g * g) / 3) < 2e-3
    assert np.all(np.abs(c) <= 1.0)


def test_hg_endpoints():
    for g in (0.3, 0.9):
        # xi -> 1 gives forward scattering, xi -> 0 backward (inverse CDF)
        assert abs(O.hg_cos(g, 1.0) - 1.0) < 1e-12
        assert abs(O.hg_cos(g, 0.0) + 1.0) < 1e-12


def test_scatter_rotation():
    rng = np.random.default_rng(7)
    for _ in range(300):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        if rng.random() < 0.1:
            u = np.array([0.0, 0.0, rng.choice([-1.0, 1.0])])
        ct = rng.uniform(-1, 1)
        v = O.scatter_dir(u, ct, rng.uniform(0, 1))
        assert abs(np.linalg.norm(v) - 1) < 1e-15
        assert abs(v @ u - ct) < 1e-12
    # azimuth: for u = +z, phi = 2 pi xi is measured from the first basis
    # vector; quarter turns map to orthogonal directions
    u = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])
    vs = [O.scatter_dir(u, 0.0, t) for t in (0.25, 0.5, 0.75, 1.0)]
    for i in range(4):
        assert abs(vs[i] @ vs[(i + 1) % 4]) < 1e-12
        assert abs(vs[i] @ vs[(i + 2) % 4] + 1) < 1e-12


# --------------------------------------------------------------------------
# Fresnel coefficients and the interface geometry (Sec. 2.3).
# --------------------------------------------------------------------------

def _fresnel_closed(n1, n2, ti):
    st = n1 / n2 * math.sin(ti)
    if st >= 1:
        return 1.0
    tt = math.asin(st)
    if ti == 0:
        return ((n1 - n2) / (n1 + n2)) ** 2
    rs = (math.sin(ti - tt) / math.sin(ti + tt)) ** 2
    rp = (math.tan(ti - tt) / math.tan(ti + tt)) ** 2
    return 0.5 * (rs + rp)


def test_fresnel_closed_forms():
    assert abs(O.fresnel(1.0, 1.38, 1.0)[0] - 0.025493) < 1e-6     # (0.38/2.38)^2
    for n1, n2 in [(1.0, 1.5), (1.5, 1.0), (1.33, 1.5), (1.5, 1.33)]:
        for ti in np.linspace(0.01, 1.55, 40):
            R, ct = O.fresnel(n1, n2, math.cos(ti))
            assert abs(R - _fresnel_closed(n1, n2, ti)) < 1e-12
    # Brewster angle: p-polarised reflection vanishes, R = Rs / 2
    tb = math.atan(1.5)
    R, _ = O.fresnel(1.0, 1.5, math.cos(tb))
    tt = math.asin(math.sin(tb) / 1.5)
    assert abs(R - 0.5 * (math.sin(tb - tt) / math.sin(tb + tt)) ** 2) < 1e-14
    # total internal reflection beyond the critical angle
    tc = math.asin(1.0 / 1.5)
    assert O.fresnel(1.5, 1.0, math.cos(tc + 1e-6))[0] == 1.0
    assert O.fresnel(1.5, 1.0, math.cos(tc - 1e-3))[0] < 1.0


def test_interface_snell_geometry_flat():
    sc = W.halfspace_scene(1.0, 1.5)  # air region above z = 0, glass below
    for ti in np.linspace(0.05, 1.4, 12):
        u0 = np.array([math.sin(ti), 0.0, -math.cos(ti)])
        outcomes = set()
        for pid in range(64):
            rc, p, u = O.interface_once(sc, [0.1, 0.2, 3e-7], u0, seed=9, pid=pid)
            assert rc == 1
            assert abs(np.linalg.norm(u) - 1) < 1e-14
            if u[2] > 0:   # reflected: mirror image, stays above
                assert np.allclose(u, [u0[0], 0, -u0[2]], atol=1e-12) and p[2] > 0
                outcomes.add("R")
            else:          # refracted: Snell's law, coplanar, below the surface
                tt = math.asin(math.sin(ti) / 1.5)
                assert np.allclose(u, [math.sin(tt), 0, -math.cos(tt)], atol=1e-9)
                assert p[2] < 0
                outcomes.add("T")
            assert abs(abs(p[2]) - 2e-6) < 1e-9   # pushed 2 delta off the surface
        assert "T" in outcomes


def test_interface_snell_geometry_sphere():
    # refraction into a sphere at impact parameter b: sin(ti) = b / r
    r, n = 1.0, 1.46
    sc = W.Scene((W.Prim(W.SPHERE, (0, 0, 0, r)),), (W.Region(W.prim_program([0]), 0, 0, 0, n),),
                 1.0, (-2, -2, -2), (2, 2, 2))
    for b in (0.1, 0.5, 0.9, 0.99):
        hit = np.array([b, 0.0, math.sqrt(r * r - b * b)])
        p = hit * (1 + 4e-7)
        for pid in range(16):
            rc, q, u = O.interface_once(sc, p, [0, 0, -1.0], seed=1, pid=pid)
            assert rc == 1
            nrm = hit / r
            if u @ nrm < 0:
                ti = math.asin(b / r)
                tt = math.asin(math.sin(ti) / n)
                # transmitted direction: angle tt to -normal, in the plane
                assert abs(-(u @ nrm) - math.cos(tt)) < 1e-8
                assert abs(u[1]) < 1e-12
                assert abs(np.linalg.norm(q) - (r - 2e-6)) < 1e-9


# --------------------------------------------------------------------------
# Track-length tally (Sec. 3.1-3.2): DDA against brute force.
# --------------------------------------------------------------------------

def test_dda_total_and_brute_force():
    grid = W.Grid((-1.0, -0.5, 0.0), (1.0, 0.5, 2.0), (8, 5, 7))
    rng = np.random.default_rng(8)
    lo, hi, n = np.array(grid.lo), np.array(grid.hi), np.array(grid.n)
    for k in range(60):
        p = rng.uniform(-1.5, 2.5, 3)
        u = rng.normal(size=3)
        if k % 10 == 0:
            u[rng.integers(3)] = 0.0
        u /= np.linalg.norm(u)
        L = rng.uniform(0, 4)
        flu, pieces = O.tally_segment(grid, p, u, L, w=0.75)
        # brute force: midpoint sampling of the segment, binned by voxel
        m = 40000
        t = (np.arange(m) + 0.5) / m * L
        x = p + t[:, None] * u
        ins = np.all((x >= lo) & (x < hi), 1)
        idx = np.floor((x[ins] - lo) / ((hi - lo) / n)).astype(int)
        want = np.zeros(grid.n[::-1])
        np.add.at(want, (idx[:, 2], idx[:, 1], idx[:, 0]), 0.75 * L / m)
        got = flu / FX
        assert abs(got.sum() - want.sum()) < 1e-6 + 2 * 0.75 * L / m
        assert np.abs(got - want).max() < 4 * 0.75 * L / m + 1e-9
        assert pieces == np.count_nonzero(flu) or pieces >= np.count_nonzero(flu)


def test_dda_axis_aligned_exact():
    grid = W.Grid((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (4, 4, 4))
    flu, pieces = O.tally_segment(grid, [0.3, 0.6, -0.5], [0, 0, 1.0], 2.0, w=1.0)
    col = flu[:, 2, 1] / FX
    assert np.allclose(col, 0.25, atol=1e-9) and pieces == 4
    assert flu.sum() == flu[:, 2, 1].sum()


# --------------------------------------------------------------------------
# Whole-transport closed forms (Eq. 1, Fresnel at the boundaries).
# --------------------------------------------------------------------------

def _run(scene, source, n, seed, grid=None, **kw):
    grid = grid or W.Grid((-1, -1, -1), (1, 1, 1), (1, 1, 1))
    wl = W.Workload("pin", scene, source, grid, n, seed, "fp64")
    return O.run(wl, **kw)


def _frac(tot, key):
    return tot[key] / FX / tot["packets"]


def _within(p_hat, p, n, k=4.0):
    sig = math.sqrt(max(p * (1 - p), 1e-12) / n)
    return abs(p_hat - p) <= k * sig


def test_beer_lambert_matched_slab():
    mu, L, n = 1.3, 1.0, 40000
    sc = W.slab_scene(mu, 0.0, 0.0, 1.0, L)
    _, tot, _ = _run(sc, W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)), n, 21, fluence=False)
    assert _within(_frac(tot, "T"), math.exp(-mu * L), n)
    assert tot["R"] == 0
    assert tot["fresnel"] == 0


def test_beer_lambert_fluence_profile():
    # straight, non-scattering, index-matched: the track length in a voxel
    # slab [z0, z1] below the surface is (exp(-mu z0) - exp(-mu z1)) / mu.
    mu, L, n, nz = 2.0, 1.0, 40000, 10
    sc = W.slab_scene(mu, 0.0, 0.0, 1.0, L)
    g = W.Grid((-1, -1, -L), (1, 1, 0), (1, 1, nz))
    flu, tot, _ = _run(sc, W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)), n, 22, grid=g)
    got = flu[::-1, 0, 0] / FX / n
    z = np.linspace(0, L, nz + 1)
    want = (np.exp(-mu * z[:-1]) - np.exp(-mu * z[1:])) / mu
    # per-packet track length in bin i is in [0, dz]; bound the std by dz/2
    sig = (L / nz) / 2 / math.sqrt(n)
    assert np.all(np.abs(got - want) < 5 * sig)


def test_slab_multiple_reflections():
    # absorbing, non-scattering slab of index n in air at normal incidence:
    # R_tot = R + (1-R)^2 R e^{-2mL} / (1 - R^2 e^{-2mL}),
    # T_tot = (1-R)^2 e^{-mL} / (1 - R^2 e^{-2mL}),  R = ((n-1)/(n+1))^2.
    mu, L, nidx, n = 0.4, 1.0, 1.5, 60000
    sc = W.slab_scene(mu, 0.0, 0.0, nidx, L)
    _, tot, _ = _run(sc, W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)), n, 23, fluence=False)
    R = ((nidx - 1) / (nidx + 1)) ** 2
    e1, e2 = math.exp(-mu * L), math.exp(-2 * mu * L)
    Rt = R + (1 - R) ** 2 * R * e2 / (1 - R * R * e2)
    Tt = (1 - R) ** 2 * e1 / (1 - R * R * e2)
    assert _within(_frac(tot, "R"), Rt, n)
    assert _within(_frac(tot, "T"), Tt, n)


def _reflected_fraction(scene, th, z_src, n, seed):
    """Fraction reflected at z = 0, measured with a thin tally slab used as a
    detector on the source side: incident and reflected rays cross it at
    different x, and each crossing leaves a track of length dz / cos(th)."""
    up = z_src > 0
    x_hit = abs(z_src) * math.tan(th)
    z0 = 0.2 if up else -0.21
    dz = 0.01
    grid = W.Grid((x_hit - 2.0, -1.0, z0), (x_hit + 2.0, 1.0, z0 + dz), (2, 1, 1))
    d = (math.sin(th), 0.0, -math.cos(th)) if up else (math.sin(th), 0.0, math.cos(th))
    flu, tot, _ = _run(scene, W.Source(W.PENCIL, (0, 0, z_src), d), n, seed, grid=grid)
    return flu[0, 0, 1] / FX / n / (dz / math.cos(th))


@pytest.mark.parametrize("theta_deg", [0.0, 30.0, 40.0])
def test_flat_fresnel_near_normal(theta_deg):
    # below 45 degrees the reflected packet leaves against the source
    # direction, so the R tally itself is the Fresnel reflectance
    th = math.radians(theta_deg)
    n = 30000
    src = W.Source(W.PENCIL, (0, 0, 0.5), (math.sin(th), 0.0, -math.cos(th)))
    _, tot, _ = _run(W.halfspace_scene(1.0, 1.5), src, n, 24, fluence=False)
    assert _within(_frac(tot, "R"), _fresnel_closed(1.0, 1.5, th), n)


@pytest.mark.parametrize("theta_deg", [20.0, 60.0, 80.0])
def test_flat_fresnel_oblique(theta_deg):
    th = math.radians(theta_deg)
    n = 30000
    got = _reflected_fraction(W.halfspace_scene(1.0, 1.5), th, 0.5, n, 24)
    assert _within(got, _fresnel_closed(1.0, 1.5, th), n)


@pytest.mark.parametrize("theta_deg", [20.0, 40.0, 45.0, 70.0])
def test_flat_fresnel_from_inside_and_tir(theta_deg):
    th = math.radians(theta_deg)
    n = 30000
    got = _reflected_fraction(W.clear_halfspace_lower(1.0, 1.5), th, -0.5, n, 25)
    want = _fresnel_closed(1.5, 1.0, th)
    if want == 1.0:
        assert abs(got - 1.0) < 1e-8       # total internal reflection (2^-32 rounding)
    else:
        assert _within(got, want, n)


@pytest.mark.parametrize("b", [0.2, 0.6, 0.9])
def test_spherical_fresnel(b):
    # pencil at impact parameter b on a strongly absorbing sphere: whatever
    # refracts in is absorbed, so the escaping fraction is R(asin(b / r)).
    r, nidx, n = 1.0, 1.46, 30000
    sc = W.Scene((W.Prim(W.SPHERE, (0, 0, 0, r)),),
                 (W.Region(W.prim_program([0]), 500.0, 0.0, 0.0, nidx),), 1.0, (-2, -2, -2), (2, 2, 2))
    _, tot, _ = _run(sc, W.Source(W.PENCIL, (b, 0, 1.5), (0, 0, -1)), n, 26, fluence=False)
    esc = (tot["R"] + tot["T"]) / FX / n
    assert _within(esc, _fresnel_closed(1.0, nidx, math.asin(b / r)), n)


def test_clear_sphere_snell_path():
    # one deterministic ray through a clear sphere at impact parameter b,
    # forced to refract (matching indices inside and out excluded): with an
    # absorbing thin shell below we check where the refracted ray lands.
    r, nidx, b = 1.0, 1.5, 0.5
    sc = W.Scene((W.Prim(W.SPHERE, (0, 0, 0, r)),), (W.Region(W.prim_program([0]), 0.0, 0.0, 0.0, nidx),),
                 1.0, (-3, -3, -3), (3, 3, 3))
    ti = math.asin(b / r)
    tt = math.asin(math.sin(ti) / nidx)
    # fluence grid: thin voxels across x at z = 0 (the ray's x there is known)
    g = W.Grid((-1.0, -0.1, -1e-3), (1.0, 0.1, 1e-3), (400, 1, 1))
    flu, tot, rec = _run(sc, W.Source(W.PENCIL, (b, 0, 2.0), (0, 0, -1)), 400, 27, grid=g,
                         records=True)
    # first refracted segment: from the entry point along the Snell direction
    hit = np.array([b, 0, math.sqrt(r * r - b * b)])
    nrm = hit / r
    d_in = np.array([0, 0, -1.0])
    eta = 1 / nidx
    ci = -(d_in @ nrm)
    ct = math.cos(tt)
    t_dir = eta * d_in + (eta * ci - ct) * nrm
    s = -hit[2] / t_dir[2]
    x0 = hit[0] + s * t_dir[0]
    hot = np.argmax(flu[0, 0, :])
    xc = -1.0 + (hot + 0.5) * 2.0 / 400
    assert abs(xc - x0) <= 2.0 / 400
    # 1 - R(ti) of the packets entered and crossed z = 0 at x0
    frac = flu[0, 0, hot] / FX / (2e-3 / abs(t_dir[2])) / 400
    R = _fresnel_closed(1.0, nidx, ti)
    assert abs(frac - (1 - R)) < 4 * math.sqrt(R * (1 - R) / 400) + 1e-9


# --------------------------------------------------------------------------
# Conservation, reproducibility, and the paper's own validation numbers.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("factory", [W.sphere_pencil, W.three_layer_slab, W.vessel_network, W.glass_container])
def test_energy_conservation(factory):
    wl = factory().with_packets(400)
    _, tot, rec = O.run(wl, records=True)
    bal = tot["R"] + tot["T"] + tot["A"] + tot["killed"] - tot["gain"]
    # every fx() rounding is at most half a unit; bound by deposits per packet
    assert abs(bal - 400 * FX) <= 0.5 * (tot["scatters"] + 3 * 400) + 1
    # per packet as well
    pb = rec["R"] + rec["T"] + rec["A"] + rec["killed"] - rec["gain"]
    assert np.all(np.abs(pb - FX) <= 0.5 * (rec["scatters"] + 3) + 1)


def test_roulette_is_unbiased():
    # Russian roulette below the weight threshold (Sec. 2.1 reuses the
    # earlier codes' absorption routine; threshold 1e-4, survival 1/m with
    # weight x m) must not change the expected energy: a survivor gains
    # w (m - 1) with probability 1/m, a loser is killed with w with
    # probability 1 - 1/m, both w (m - 1) / m in expectation -- equal only
    # when the survival chance and the multiplier match.  In a medium that
    # no packet leaves (albedo 0.9, mean free path 1e-3 cm, 1 cm from the
    # surface), every packet meets roulette and all of its weight is
    # absorbed in expectation: E[A] = 1, i.e. E[killed - gain] = 0 per
    # packet.  The energy identity R + T + A + killed - gain = 1 holds for
    # any survival threshold, so only this expectation pins it.
    mu_a, mu_s = 100.0, 900.0
    sc = W.Scene((W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 1.0)),),
                 (W.Region(W.prim_program([0]), mu_a, mu_s, 0.0, 1.0),), 1.0,
                 (-1.1, -1.1, -1.1), (1.1, 1.1, 1.1))
    n = 20000
    _, tot, rec = _run(sc, W.Source(W.ISO_POINT, (0, 0, 0), (0, 0, -1)), n, 41, fluence=False, records=True)
    assert tot["R"] == 0 and tot["T"] == 0 and tot["max_steps_hit"] == 0
    killed = rec["killed"].astype(np.float64) / FX
    gain = rec["gain"].astype(np.float64) / FX
    # every packet ends in a roulette kill of a weight below the threshold
    assert np.all(rec["killed"] > 0) and np.all(killed < 1e-4)
    # survivors: each gain is (m - 1) w with w below the threshold; about one
    # survival in nine roulette events, so the 2e4 kills come with ~2.2e3
    # survivals -- over 2.2e4 roulette events in all
    events = n + np.count_nonzero(gain)
    assert events > 2.1e4 and np.all(gain < 9e-3)
    d = killed - gain
    z = d.mean() / (d.std() / math.sqrt(n))
    assert abs(z) < 3.0, (d.mean(), d.std(), z)
    # the expected kill per packet is the closed form of the first roulette
    # event: with no survivors the packet dies with w = 0.9^k < 1e-4
    k = math.ceil(math.log(1e-4) / math.log(mu_s / (mu_a + mu_s)))
    w_first = (mu_s / (mu_a + mu_s)) ** k
    assert abs(np.median(killed[gain == 0]) - w_first) < 1e-9


def test_thread_count_independence():
    wl = W.sphere_pencil(600)
    f1, t1, _ = O.run(wl, threads=1)
    f8, t8, _ = O.run(wl, threads=8, chunk=7)
    assert np.array_equal(f1, f8) and t1 == t8


def test_packet_id_additivity():
    # a job is the sum of its packet-id blocks (resume from any prefix)
    wl = W.three_layer_slab(300, grid_n=20)
    fa, ta, _ = O.run(wl, 0, 300)
    fb, tb, _ = O.run(wl, 0, 120)
    fc, tc, _ = O.run(wl, 120, 300)
    assert np.array_equal(fa, fb + fc)
    for k in ("R", "T", "A", "killed", "gain", "scatters", "steps"):
        assert ta[k] == tb[k] + tc[k]


@pytest.mark.parametrize("row", read_golden("eq4_scatterings.txt"))
def test_eq4_mean_scatterings(row):
    tau, radius, tol = float(row[0]), float(row[1]), float(row[2])
    sc = W.isotropic_sphere(tau, radius)
    _, tot, _ = _run(sc, W.Source(W.ISO_POINT, (0, 0, 0), (0, 0, -1)), 20000, 31, fluence=False)
    mean = tot["scatters"] / tot["packets"]
    want = tau * tau / 2 + tau
    assert abs(mean - want) / want < tol, (tau, mean, want)
    assert tot["A"] == 0   # pure scatterer


@pytest.mark.slow
@pytest.mark.parametrize("row", read_golden("table1_penetration.txt"))
def test_table1_penetration_depth(row):
    # deep in a semi-infinite slab the fluence decays as exp(-z k1 / delta)
    # with Table 1's k1 = 1.00 (Eq. 5).  Diffusion is approximate, so the
    # fitted k1 must lie within 8% -- using mu_s instead of mu_s (1 - g)
    # would change it by a factor of three.
    mua, musp, k1, dpaper = float(row[1]), float(row[2]), float(row[4]), float(row[7])
    g = 0.9
    assert abs(1 / math.sqrt(3 * mua * (mua + musp)) - dpaper) < 6e-4
    thick = 30 * dpaper
    sc = W.slab_scene(mua, musp / (1 - g), g, 1.38, thick, half=50.0)
    nz = 120
    grid = W.Grid((-49, -49, -thick), (49, 49, 0), (1, 1, nz))
    flu, tot, _ = _run(sc, W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)), 20000, 11, grid=grid)
    phi = flu[::-1, 0, 0].astype(float)
    z = (np.arange(nz) + 0.5) * thick / nz
    sel = (z > 4 * dpaper) & (z < 12 * dpaper)
    slope = np.polyfit(z[sel], np.log(phi[sel]), 1)[0]
    assert abs(-slope * dpaper - k1) < 0.08
    # absolute level: the laterally integrated fluence of a pencil beam per
    # incident photon equals the fluence rate under uniform illumination per
    # unit irradiance, Psi / Psi0 of Eq. 5 with Table 1's C1, k1, C2, k2.
    # The paper notes that bin shapes keep codes from matching exactly; 6 %.
    C1, C2, k2 = float(row[3]), float(row[5]), float(row[6])
    dz = thick / nz
    psi = phi / FX / dz / tot["packets"]
    for m in (1, 2, 4):
        want = C1 * math.exp(-k1 * m) - C2 * math.exp(-k2 * m)
        got = float(np.interp(m * dpaper, z, psi))
        assert abs(got - want) / want < 0.06, (m, got, want)


# --------------------------------------------------------------------------
# Photon release (Sec. 2.1): source distributions.
# --------------------------------------------------------------------------

def _clear_scene():
    # one tiny region far away: the packets cross only ambient medium
    return W.Scene((W.Prim(W.SPHERE, (5.0, 5.0, 5.0, 0.1)),),
                   (W.Region(W.prim_program([0]), 0.0, 0.0, 0.0, 1.0),), 1.0, (-6, -6, -6), (6, 6, 6))


def _launch_histogram(src, n, R, m=48):
    # a clear medium and a thin tally slab just below the source plane: each
    # packet leaves track length dz in the voxel under its launch point, so
    # the slab is a histogram of launch positions
    dz = 0.01
    grid = W.Grid((-R, -R, -0.2 - dz), (R, R, -0.2), (m, m, 1))
    flu, tot, _ = _run(_clear_scene(), src, n, 41, grid=grid)
    h = flu[0] / FX / dz
    assert abs(h.sum() - n) < 1e-6 * n
    c = (np.arange(m) + 0.5) / m * 2 * R - R
    X, Y = np.meshgrid(c, c)
    return h / n, X, Y


def test_disc_source_uniform_over_disc():
    R, n = 0.5, 40000
    p, X, Y = _launch_histogram(W.Source(W.DISC, (0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R), n, R)
    r2 = float((p * (X * X + Y * Y)).sum())
    # uniform disc: <rho^2> = R^2 / 2 (a radius drawn uniformly would give R^2 / 3)
    assert abs(r2 - R * R / 2) < 0.02 * R * R
    inner = float(p[X * X + Y * Y < (R / 2) ** 2].sum())
    assert abs(inner - 0.25) < 0.02


def test_square_source_uniform_over_square():
    R, n = 0.4, 40000
    p, X, Y = _launch_histogram(W.Source(W.SQUARE, (0.0, 0.0, 0.0), (0.0, 0.0, -1.0), R), n, R, m=8)
    # 64 equal cells: each holds 1/64 of the packets (binomial 4 sigma)
    sig = math.sqrt((1 / 64) * (63 / 64) / n)
    assert np.all(np.abs(p - 1 / 64) < 4 * sig)


def test_isotropic_source_directions():
    n = 40000
    src = W.Source(W.ISO_POINT, (0.0, 0.0, 0.0), (0.0, 0.0, -1.0))
    # half the directions point against dir (counted as R), exactly in expectation
    _, tot, _ = _run(_clear_scene(), src, n, 43, fluence=False)
    assert _within(_frac(tot, "R"), 0.5, n)
    # track-length density of a unit isotropic point source in a clear medium
    # is 1 / (4 pi |x|^2): the expected track length in a box is its volume
    # integral (3D midpoint quadrature of the closed form)
    grid = W.Grid((-2.0, -2.0, 0.5), (2.0, 2.0, 0.6), (1, 1, 1))
    flu, _, _ = _run(_clear_scene(), src, n, 44, grid=grid)
    got = flu[0, 0, 0] / FX / n
    mx, mz = 200, 20
    xs = (np.arange(mx) + 0.5) / mx * 4 - 2
    zs = 0.5 + (np.arange(mz) + 0.5) / mz * 0.1
    X, Y, Z = np.meshgrid(xs, xs, zs, indexing="ij")
    want = float((1.0 / (4 * math.pi * (X * X + Y * Y + Z * Z))).sum() * (4 / mx) ** 2 * (0.1 / mz))
    assert abs(got - want) < 0.03 * want


# --------------------------------------------------------------------------
# Segment stepping (scene option; Sec. 5 names segment tracing as the cure
# for many small steps near parallel surfaces): the move along u is bounded
# by the distance to each primitive's delta/2-offset surface.
# --------------------------------------------------------------------------

def _csg_scene():
    """Hard CSG of boxes and spheres (intersection, subtraction, union) in
    two regions, plus a smooth-union region of capsules."""
    prims = (W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.6, 0.4, 0.5)),
             W.Prim(W.SPHERE, (0.3, 0.0, 0.1, 0.45)),
             W.Prim(W.SPHERE, (-0.5, 0.2, -0.2, 0.3)),
             W.Prim(W.BOX, (-0.2, -0.3, 0.4, 0.2, 0.3, 0.15)),
             W.Prim(W.CAPSULE, (0.5, 0.5, -0.6, 0.9, 0.6, 0.2, 0.08)),
             W.Prim(W.CAPSULE, (0.9, 0.6, 0.2, 0.7, -0.2, 0.5, 0.06)))
    r0 = (W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(W.SUBTRACT), W.Node(W.PRIM, 2), W.Node(W.UNION))
    r1 = (W.Node(W.PRIM, 3), W.Node(W.PRIM, 0), W.Node(W.INTERSECT))
    r2 = (W.Node(W.PRIM, 4), W.Node(W.PRIM, 5), W.Node(W.SMOOTH_UNION, -1, 0.05))
    regs = (W.Region(r0, 1.0, 5.0, 0.5, 1.4), W.Region(r1, 0.5, 2.0, 0.0, 1.2),
            W.Region(r2, 2.0, 10.0, 0.9, 1.4))
    return W.Scene(prims, regs, 1.0, (-1.2, -1.2, -1.2), (1.2, 1.2, 1.2), delta=1e-3,
                   stepping=W.SEGMENT)


def _capsule_scene():
    """A hard union of capsules in several orientations, and a capsule minus
    a sphere: every capsule bounds moves by its ray bound."""
    prims = (W.Prim(W.CAPSULE, (-0.6, 0.0, 0.0, 0.6, 0.0, 0.0, 0.15)),
             W.Prim(W.CAPSULE, (0.0, -0.7, 0.3, 0.1, 0.7, 0.2, 0.1)),
             W.Prim(W.CAPSULE, (-0.5, -0.5, -0.6, 0.5, 0.4, 0.6, 0.08)),
             W.Prim(W.CAPSULE, (0.7, 0.7, -0.8, 0.7, 0.72, 0.8, 0.12)),
             W.Prim(W.CAPSULE, (-0.8, 0.6, 0.6, -0.2, 0.6, 0.6, 0.2)),
             W.Prim(W.SPHERE, (-0.5, 0.6, 0.6, 0.18)))
    r0 = W.prim_program([0, 1, 2, 3])
    r1 = (W.Node(W.PRIM, 4), W.Node(W.PRIM, 5), W.Node(W.SUBTRACT))
    regs = (W.Region(r0, 1.0, 5.0, 0.5, 1.4), W.Region(r1, 0.5, 2.0, 0.0, 1.2))
    return W.Scene(prims, regs, 1.0, (-1.2, -1.2, -1.2), (1.2, 1.2, 1.2), delta=1e-3,
                   stepping=W.SEGMENT)


SEGMENT_SCENES = {
    "csg": _csg_scene,
    "capsules": _capsule_scene,
    "sphere": lambda: W.sphere_pencil().scene,
    "slab": lambda: W.three_layer_slab().scene,
    "glass": lambda: W.glass_container().scene,
    "vessel": lambda: W.vessel_network().scene,
    "vessel_hard": lambda: W.vessel_network_hard().scene,
    "gallery": lambda: W.sdf_gallery().scene,
}


@pytest.mark.parametrize("name", list(SEGMENT_SCENES))
def test_segment_step_never_reaches_a_surface(name):
    # brute force along the move: every region's SDF keeps its sign and the
    # scene distance stays >= delta/2 (sampled densely), and the move is never
    # shorter than the sphere-tracing step d_min - delta/2
    from dataclasses import replace
    sc = replace(SEGMENT_SCENES[name](), stepping=W.SEGMENT)
    dh = 0.5 * sc.delta
    rng = np.random.default_rng(hash(name) % 2**32)
    lo, hi = np.array(sc.bbox_lo), np.array(sc.bbox_hi)
    checked = longer = 0
    for _ in range(90):
        p = lo + (hi - lo) * rng.random(3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        e = O.scene_eval(sc, p)
        if e["dmin"] < sc.delta or e["dbox"] > 0:
            continue
        t = O.segment_step(sc, p, u)
        assert t >= e["dmin"] - dh
        longer += t > e["dmin"] - dh + 1e-12
        signs = [np.sign(O.region_sdf(sc, r, p)) for r in range(len(sc.regions))]
        for s in np.linspace(0.0, t, 160):
            q = p + s * u
            eq = O.scene_eval(sc, q)
            assert eq["dmin"] >= dh - 1e-12, (name, p, u, t, s, eq)   # rounding of |p - c| - r
            assert eq["dbox"] < 0
            assert [np.sign(O.region_sdf(sc, r, q)) for r in range(len(sc.regions))] == signs
        checked += 1
    assert checked > 20 and longer > checked // 4


def test_segment_step_exact_for_planes_and_spheres():
    # the bound is exact where it can be: the move ends on the delta/2-offset
    # surface of a box face or a sphere (straight-line geometry)
    d = 1e-3
    box = W.Scene((W.Prim(W.BOX, (0.0, 0.0, -1.0, 10.0, 10.0, 1.0)),),
                  (W.Region(W.prim_program([0]), 0.0, 1.0, 0.0, 1.5),), 1.0,
                  (-5, -5, -3), (5, 5, 3), delta=d, stepping=W.SEGMENT)
    for c in (1.0, 0.5, 0.05, 1e-3):
        u = np.array([math.sqrt(1 - c * c), 0.0, -c])
        t = O.segment_step(box, (0.0, 0.0, 0.7), u)
        assert math.isclose(t, (0.7 - d / 2) / c, rel_tol=1e-12) or t == pytest.approx((5 - d / 2) / math.sqrt(1 - c * c), rel=1e-12)
        # from inside, towards the bottom face z = -2
        t = O.segment_step(box, (0.0, 0.0, -0.5), np.array([math.sqrt(1 - c * c), 0.0, -c]))
        want = min((1.5 - d / 2) / c, (5 - d / 2) / math.sqrt(1 - c * c) if c < 1 else math.inf)
        assert math.isclose(t, want, rel_tol=1e-12)
    # moving away from the only face: the move reaches the bounding box
    t = O.segment_step(box, (0.0, 0.0, 0.5), np.array([0.0, 0.0, 1.0]))
    assert math.isclose(t, 3.0 - 0.5 - d / 2, rel_tol=1e-12)
    r = 1.0
    sph = W.Scene((W.Prim(W.SPHERE, (0.0, 0.0, 0.0, r)),),
                  (W.Region(W.prim_program([0]), 0.0, 1.0, 0.0, 1.4),), 1.0,
                  (-3, -3, -3), (3, 3, 3), delta=d, stepping=W.SEGMENT)
    for b in (0.0, 0.5, 0.99):
        # outside, aimed at impact parameter b: entry of the grown sphere
        p = np.array([b, 0.0, 2.0])
        t = O.segment_step(sph, p, np.array([0.0, 0.0, -1.0]))
        rr = r + d / 2
        assert math.isclose(t, 2.0 - math.sqrt(rr * rr - b * b), rel_tol=1e-12)
        # inside from the centre line: exit of the shrunk sphere
        p = np.array([b * 0.5, 0.0, 0.0])
        t = O.segment_step(sph, p, np.array([0.0, 0.0, 1.0]))
        rr = r - d / 2
        assert math.isclose(t, math.sqrt(rr * rr - (b * 0.5) ** 2), rel_tol=1e-12)
    # a ray that misses the grown sphere is bounded by the bounding box only
    t = O.segment_step(sph, (1.2, 0.0, 2.0), np.array([0.0, 0.0, -1.0]))
    assert math.isclose(t, 5.0 - d / 2, rel_tol=1e-12)


def test_segment_step_exact_for_capsules():
    # capsule from (-h, 0, 0) to (h, 0, 0), radius r: the move ends on the
    # delta/2-offset surface of the cylinder or of an end ball
    d, h, r = 1e-3, 0.5, 0.2
    cap = W.Scene((W.Prim(W.CAPSULE, (-h, 0.0, 0.0, h, 0.0, 0.0, r)),),
                  (W.Region(W.prim_program([0]), 0.0, 1.0, 0.0, 1.5),), 1.0,
                  (-3, -3, -3), (3, 3, 3), delta=d, stepping=W.SEGMENT)
    rg, rs = r + d / 2, r - d / 2
    down, along = np.array([0.0, 0.0, -1.0]), np.array([-1.0, 0.0, 0.0])
    for x0 in (-0.4, 0.0, 0.3):
        # outside, across the axis: entry of the grown cylinder
        assert math.isclose(O.segment_step(cap, (x0, 0.0, 2.0), down), 2.0 - rg, rel_tol=1e-12)
        # inside, across the axis at offset y0: exit of the shrunk cylinder
        for y0 in (0.0, 0.1, 0.19):
            t = O.segment_step(cap, (x0, y0, 0.0), np.array([0.0, 0.0, 1.0]))
            assert math.isclose(t, math.sqrt(rs * rs - y0 * y0), rel_tol=1e-12)
    for y0 in (0.0, 0.1, 0.2):
        # outside, parallel to the axis: entry of the grown end ball
        t = O.segment_step(cap, (2.0, y0, 0.0), along)
        assert math.isclose(t, 2.0 - h - math.sqrt(rg * rg - y0 * y0), rel_tol=1e-12)
        # inside, along the axis: exit through the far end ball
        t = O.segment_step(cap, (0.1, y0 * 0.5, 0.0), np.array([1.0, 0.0, 0.0]))
        assert math.isclose(t, h - 0.1 + math.sqrt(rs * rs - (y0 * 0.5) ** 2), rel_tol=1e-12)
    # a ray that misses the grown capsule is bounded by the bounding box only
    t = O.segment_step(cap, (0.0, 0.3, 2.0), down)
    assert math.isclose(t, 5.0 - d / 2, rel_tol=1e-12)
    # oblique rays from outside, aimed near the capsule: no sampled point of
    # the move comes closer than delta/2, and a ray that meets the capsule
    # stops where the SDF is delta/2
    rng = np.random.default_rng(3)
    hit = 0
    for _ in range(60):
        p = rng.uniform(-1.5, 1.5, 3)
        if O.region_sdf(cap, 0, p) <= d:
            continue
        aim = np.array([rng.uniform(-h - r, h + r), rng.normal(0.0, 0.12), rng.normal(0.0, 0.12)])
        u = aim - p
        u /= np.linalg.norm(u)
        t = O.segment_step(cap, p, u)
        ts = np.linspace(0.0, t, 400)
        dist = np.array([O.region_sdf(cap, 0, p + s * u) for s in ts])
        assert dist.min() >= d / 2 - 1e-12
        if t < 4.0 and abs(O.region_sdf(cap, 0, p + t * u) - d / 2) < 1e-9:
            hit += 1
    assert hit > 10


def test_segment_step_exact_for_placed_primitives():
    # a frame without a domain operation maps rays to rays: the move ends on
    # the world surface offset by delta/2 for any rotation and scale
    d = 1e-3
    down = np.array([0.0, 0.0, -1.0])

    def one(prim):
        return W.Scene((prim,), (W.Region(W.prim_program([0]), 0.0, 1.0, 0.0, 1.5),), 1.0,
                       (-5, -5, -5), (5, 5, 5), delta=d, stepping=W.SEGMENT)
    for s in (0.5, 1.0, 1.5):
        rz = W.rotation((0, 0, 1), 90.0)
        box = one(W.Prim(W.BOX, (0.0, 0.0, 0.0, 0.4, 0.3, 0.2), W.Xform(rot=rz, t=(0.2, 0.1, -1.0), s=s)))
        assert math.isclose(O.segment_step(box, (0.2, 0.1, 1.0), down), 2.0 - (0.2 * s + d / 2), rel_tol=1e-12)
        # along x the box shows its local y half extent (quarter turn about z)
        t = O.segment_step(box, (3.0, 0.1, -1.0), np.array([-1.0, 0.0, 0.0]))
        assert math.isclose(t, 3.0 - 0.2 - (0.3 * s + d / 2), rel_tol=1e-12)
        # from inside along +y: the exit of the shrunk box at local x half extent
        t = O.segment_step(box, (0.2, 0.1, -1.0), np.array([0.0, 1.0, 0.0]))
        assert math.isclose(t, 0.4 * s - d / 2, rel_tol=1e-12)
        sph = one(W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 0.3), W.Xform(t=(0.0, 0.0, -1.0), s=s)))
        for b in (0.0, 0.1):
            rr = 0.3 * s + d / 2
            t = O.segment_step(sph, (b, 0.0, 1.0), down)
            assert math.isclose(t, 2.0 - math.sqrt(rr * rr - b * b), rel_tol=1e-12)
        # a capsule along local x turned to lie along world y
        cap = one(W.Prim(W.CAPSULE, (-0.5, 0.0, 0.0, 0.5, 0.0, 0.0, 0.1), W.Xform(rot=rz, t=(0.0, 0.0, -1.0), s=s)))
        t = O.segment_step(cap, (0.0, 0.4 * s, 1.0), down)
        assert math.isclose(t, 2.0 - (0.1 * s + d / 2), rel_tol=1e-12)
        t = O.segment_step(cap, (0.0, 3.0, -1.0), np.array([0.0, -1.0, 0.0]))
        assert math.isclose(t, 3.0 - 0.5 * s - (0.1 * s + d / 2), rel_tol=1e-12)
    # a domain operation keeps the isotropic bound: the move is the
    # sphere-tracing step d_min - delta/2
    el = one(W.Prim(W.SPHERE, (0.0, 0.0, 0.0, 0.1), W.Xform(t=(0.0, 0.0, -1.0), op=W.ELONGATE, a=(0.3, 0.0, 0.0, 0.0))))
    p = (0.0, 0.0, 1.0)
    e = O.scene_eval(el, p)
    assert math.isclose(O.segment_step(el, p, down), e["dmin"] - d / 2, rel_tol=1e-12)


def _brute_force_move(sc, p, u, t, n=400):
    """Every region keeps its sign along the move and the scene distance
    stays >= delta/2 (sampled densely)."""
    p = np.asarray(p, dtype=float)
    signs = [np.sign(O.region_sdf(sc, r, p)) for r in range(len(sc.regions))]
    for s in np.linspace(0.0, t, n):
        q = p + s * u
        e = O.scene_eval(sc, q)
        assert e["dmin"] >= 0.5 * sc.delta - 1e-12, (p, u, t, s, e)
        assert [np.sign(O.region_sdf(sc, r, q)) for r in range(len(sc.regions))] == signs, (p, u, t, s)


def _one_region(prims, program, lo=(-5, -5, -5), hi=(5, 5, 5), d=1e-3):
    return W.Scene(tuple(prims), (W.Region(program, 0.0, 1.0, 0.0, 1.5),), 1.0, lo, hi, delta=d,
                   stepping=W.SEGMENT)


def test_segment_step_smooth_fold_margin():
    # three smooth unions of one sphere with itself: the blend adds up to
    # k/4 + k h (1 - h) + ... below min; for equal operands the fold gives
    # a - k/4, then a - k (5/32 + 15/64) = a - 0.390625 k, so the surface is
    # at radius r + 0.390625 k, beyond the r + k/4 a single margin would take
    r, k, d = 0.3, 0.2, 1e-3
    sph = W.Prim(W.SPHERE, (0.0, 0.0, 0.0, r))
    prog = (W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(W.SMOOTH_UNION, -1, k),
            W.Node(W.PRIM, 2), W.Node(W.SMOOTH_UNION, -1, k))
    sc = _one_region([sph, sph, sph], prog, d=d)
    rs = r + 0.390625 * k
    assert abs(O.region_sdf(sc, 0, (0.0, 0.0, rs))) < 1e-12
    down = np.array([0.0, 0.0, -1.0])
    # the margin is the sum over both folds, k/2: a ray passing the centre
    # at a distance below r + k/2 + delta/2 stops on that grown sphere
    # (longer than the isotropic step), also where it would miss the
    # surface itself, and where a k/4 margin would let it cross the surface
    for x0 in (0.36, 0.39):
        t = O.segment_step(sc, (x0, 0.0, 2.0), down)
        rg = r + 0.5 * k + d / 2
        assert math.isclose(t, 2.0 - math.sqrt(rg * rg - x0 * x0), rel_tol=1e-12)
        _brute_force_move(sc, (x0, 0.0, 2.0), down, t)
    # past the grown sphere: only the bounding box bounds the move
    assert math.isclose(O.segment_step(sc, (0.45, 0.0, 2.0), down), 7.0 - d / 2, rel_tol=1e-12)
    # oblique rays that graze the blended surface
    rng = np.random.default_rng(11)
    for _ in range(40):
        p = rng.normal(size=3)
        p *= 1.5 / np.linalg.norm(p)
        aim = rng.normal(0.0, 0.3, 3)
        u = (aim - p) / np.linalg.norm(aim - p)
        t = O.segment_step(sc, p, u)
        _brute_force_move(sc, p, u, t, n=200)
    # two spheres side by side, a ray down their bisecting plane: the blend
    # reaches k/4 below both (equal operands) and the surface lies on the
    # spheres grown by k/4
    a, b = W.Prim(W.SPHERE, (-0.05, 0.0, 0.0, 0.2)), W.Prim(W.SPHERE, (0.05, 0.0, 0.0, 0.2))
    two = _one_region([a, b], (W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(W.SMOOTH_UNION, -1, k)), d=d)
    zs = math.sqrt(0.25 ** 2 - 0.05 ** 2)
    assert abs(O.region_sdf(two, 0, (0.0, 0.0, zs))) < 1e-12
    t = O.segment_step(two, (0.0, 0.0, 1.0), down)
    ze = math.sqrt((0.25 + d / 2) ** 2 - 0.05 ** 2)
    assert math.isclose(t, 1.0 - ze, rel_tol=1e-12)
    # a bounding box whose exit lies past the blended surface but short of the
    # spheres' own distance: the spheres are not passed over as unable to bind
    cut = W.Scene((a, b), (W.Region(two.regions[0].program, 0.0, 1.0, 0.0, 1.5),), 1.0, (-2, -2, 0.22),
                  (2, 2, 2), delta=d, stepping=W.SEGMENT)
    t = O.segment_step(cut, (0.0, 0.0, 1.0), down)
    assert math.isclose(t, 1.0 - ze, rel_tol=1e-12)
    _brute_force_move(cut, (0.0, 0.0, 1.0), down, t)
    # more than eight smooth unions: the region keeps its isotropic bound
    many = [W.Prim(W.SPHERE, (0.1 * i, 0.0, 0.0, 0.2)) for i in range(10)]
    prog = [W.Node(W.PRIM, 0)]
    for i in range(1, 10):
        prog += [W.Node(W.PRIM, i), W.Node(W.SMOOTH_UNION, -1, 0.05)]
    soft = _one_region(many, tuple(prog), d=d)
    p = (0.45, 0.0, 2.0)
    e = O.scene_eval(soft, p)
    assert math.isclose(O.segment_step(soft, p, down), e["dmin"] - d / 2, rel_tol=1e-12)


def test_segment_step_exact_for_cylinders_and_tori():
    d = 1e-3
    down = np.array([0.0, 0.0, -1.0])
    cyl = _one_region([W.Prim(W.CYLINDER, (0.0, 0.0, 0.0, 0.3, 0.5))], W.prim_program([0]), d=d)
    # outside: the cylinder grown by delta/2 in radius and half height
    assert math.isclose(O.segment_step(cyl, (0.1, 0.0, 2.0), down), 2.0 - (0.5 + d / 2), rel_tol=1e-12)
    assert math.isclose(O.segment_step(cyl, (2.0, 0.0, 0.2), np.array([-1.0, 0.0, 0.0])), 2.0 - (0.3 + d / 2),
                        rel_tol=1e-12)
    # a ray past the rim (cap plane reached outside the grown radius) goes on
    # to the side wall
    u = np.array([-1.0, 0.0, -1.0]) / math.sqrt(2.0)
    t = O.segment_step(cyl, (1.5, 0.0, 1.0), u)
    assert math.isclose(t, (1.5 - (0.3 + d / 2)) * math.sqrt(2.0), rel_tol=1e-12)
    # inside: the exit of the cylinder shrunk by delta/2
    assert math.isclose(O.segment_step(cyl, (0.0, 0.0, 0.0), np.array([0.0, 0.0, 1.0])), 0.5 - d / 2,
                        rel_tol=1e-12)
    assert math.isclose(O.segment_step(cyl, (0.0, 0.0, 0.0), np.array([1.0, 0.0, 0.0])), 0.3 - d / 2,
                        rel_tol=1e-12)
    tor = _one_region([W.Prim(W.TORUS, (0.0, 0.0, 0.0, 0.5, 0.15))], W.prim_program([0]), d=d)
    # outside, in the ring's plane and from above the core circle: d - delta/2
    assert math.isclose(O.segment_step(tor, (2.0, 0.0, 0.0), np.array([-1.0, 0.0, 0.0])), 2.0 - 0.65 - d / 2,
                        rel_tol=1e-12)
    assert math.isclose(O.segment_step(tor, (0.5, 0.0, 1.0), down), 1.0 - 0.15 - d / 2, rel_tol=1e-12)
    # down the axis through the hole: only the bounding box bounds the move
    assert math.isclose(O.segment_step(tor, (0.0, 0.0, 1.0), down), 6.0 - d / 2, rel_tol=1e-12)
    # inside the tube: the exit of the ball of radius r - delta/2 about the
    # nearest point of the core circle, longer than the isotropic 0.1 - delta/2
    # when the ray runs across the tube
    rb = 0.15 - d / 2
    for u in (np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])):
        t = O.segment_step(tor, (0.5, 0.0, 0.05), u)
        assert math.isclose(t, math.sqrt(rb * rb - 0.05 * 0.05), rel_tol=1e-12)
        _brute_force_move(tor, (0.5, 0.0, 0.05), u, t)
    # straight down through the core circle: the ball's far side
    assert math.isclose(O.segment_step(tor, (0.5, 0.0, 0.05), np.array([0.0, 0.0, -1.0])), rb + 0.05,
                        rel_tol=1e-12)
    # placed by a frame (quarter turn about x, scale 2): the ring's axis is
    # world y, so a ray down world y through the hole meets nothing
    rx = W.rotation((1, 0, 0), 90.0)
    ptor = _one_region([W.Prim(W.TORUS, (0.0, 0.0, 0.0, 0.5, 0.15), W.Xform(rot=rx, t=(0.0, 0.0, -1.0), s=2.0))],
                       W.prim_program([0]), d=d)
    assert math.isclose(O.segment_step(ptor, (0.0, 3.0, -1.0), np.array([0.0, -1.0, 0.0])), 8.0 - d / 2,
                        rel_tol=1e-12)
    assert math.isclose(O.segment_step(ptor, (0.0, 0.0, 2.0), down), 3.0 - 2.0 * 0.65 - d / 2, rel_tol=1e-12)
    pcyl = _one_region([W.Prim(W.CYLINDER, (0.0, 0.0, 0.0, 0.3, 0.5), W.Xform(rot=rx, t=(0.0, 0.0, -1.0), s=1.5))],
                       W.prim_program([0]), d=d)
    # the cylinder's axis is world y: from above, its side at 1.5 * 0.3
    assert math.isclose(O.segment_step(pcyl, (0.0, 0.2, 2.0), down), 3.0 - (1.5 * 0.3 + d / 2), rel_tol=1e-12)
    # brute force from random points and directions, hard CSG of both
    both = W.Scene((W.Prim(W.TORUS, (0.0, 0.0, 0.0, 0.5, 0.15)), W.Prim(W.CYLINDER, (0.4, 0.0, 0.1, 0.2, 0.3)),
                    W.Prim(W.TORUS, (0.0, 0.0, 0.0, 0.4, 0.1), W.Xform(rot=W.rotation((1, 1, 0), 60.0),
                                                                      t=(-0.3, 0.2, 0.0)))),
                   (W.Region((W.Node(W.PRIM, 0), W.Node(W.PRIM, 1), W.Node(W.SUBTRACT)), 0.0, 1.0, 0.0, 1.5),
                    W.Region(W.prim_program([2]), 0.0, 1.0, 0.0, 1.3)),
                   1.0, (-1.2, -1.2, -1.2), (1.2, 1.2, 1.2), delta=d, stepping=W.SEGMENT)
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(150):
        p = rng.uniform(-1.1, 1.1, 3)
        if O.scene_eval(both, p)["dmin"] < d:
            continue
        aim = rng.normal(0.0, 0.4, 3)
        u = (aim - p) / np.linalg.norm(aim - p)
        _brute_force_move(both, p, u, O.segment_step(both, p, u), n=200)
        checked += 1
    assert checked > 100


def _seg(sc):
    from dataclasses import replace
    return replace(sc, stepping=W.SEGMENT)


def test_segment_stepping_closed_forms():
    # Beer-Lambert and the slab's multiple reflections hold under segment
    # stepping, and a packet crosses the matched slab in one move
    mu, L, n = 1.3, 1.0, 40000
    _, tot, _ = _run(_seg(W.slab_scene(mu, 0.0, 0.0, 1.0, L)), W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)),
                     n, 21, fluence=False)
    assert _within(_frac(tot, "T"), math.exp(-mu * L), n)
    assert tot["steps"] <= 6 * n
    mu, L, nidx, n = 0.4, 1.0, 1.5, 60000
    _, tot, _ = _run(_seg(W.slab_scene(mu, 0.0, 0.0, nidx, L)), W.Source(W.PENCIL, (0, 0, 0.2), (0, 0, -1)),
                     n, 23, fluence=False)
    R = ((nidx - 1) / (nidx + 1)) ** 2
    e1, e2 = math.exp(-mu * L), math.exp(-2 * mu * L)
    assert _within(_frac(tot, "R"), R + (1 - R) ** 2 * R * e2 / (1 - R * R * e2), n)
    assert _within(_frac(tot, "T"), (1 - R) ** 2 * e1 / (1 - R * R * e2), n)


@pytest.mark.parametrize("theta_deg", [20.0, 70.0, 80.0])
def test_segment_stepping_flat_fresnel(theta_deg):
    th = math.radians(theta_deg)
    n = 30000
    got = _reflected_fraction(_seg(W.halfspace_scene(1.0, 1.5)), th, 0.5, n, 24)
    assert _within(got, _fresnel_closed(1.0, 1.5, th), n)


@pytest.mark.parametrize("b", [0.6, 0.97])
def test_segment_stepping_spherical_fresnel(b):
    r, nidx, n = 1.0, 1.46, 30000
    sc = W.Scene((W.Prim(W.SPHERE, (0, 0, 0, r)),),
                 (W.Region(W.prim_program([0]), 500.0, 0.0, 0.0, nidx),), 1.0, (-2, -2, -2), (2, 2, 2),
                 stepping=W.SEGMENT)
    _, tot, _ = _run(sc, W.Source(W.PENCIL, (b, 0, 1.5), (0, 0, -1)), n, 26, fluence=False)
    esc = (tot["R"] + tot["T"]) / FX / n
    assert _within(esc, _fresnel_closed(1.0, nidx, math.asin(b / r)), n)


@pytest.mark.parametrize("factory", [W.sphere_pencil, W.three_layer_slab, W.vessel_network, W.glass_container])
def test_segment_stepping_same_transport_fewer_steps(factory):
    # same physics: R, T, A agree with sphere tracing within Monte Carlo
    # error (per-packet variances), energy closes per packet, and fewer steps
    wl = factory().with_packets(3000)
    _, t0, r0 = O.run(wl, records=True)
    _, t1, r1 = O.run(wl.with_stepping(W.SEGMENT), records=True)
    for k in ("R", "T", "A"):
        a, b = r0[k] / FX, r1[k] / FX
        se = math.sqrt((a.var() + b.var()) / len(a)) + 1e-12
        assert abs(a.mean() - b.mean()) < 4 * se, k
    pb = r1["R"] + r1["T"] + r1["A"] + r1["killed"] - r1["gain"]
    assert np.all(np.abs(pb - FX) <= 0.5 * (r1["scatters"] + 3) + 1)
    assert t1["steps"] < 0.7 * t0["steps"]


def test_glass_sphere_focuses_at_the_ball_lens_focal_length():
    # The clear glass sphere of Sec. 3.2 (n = 1.46, radius 1 cm) is a ball
    # lens: a narrow beam along its axis focuses at nR / (2 (n - 1)) from the
    # centre (paraxial optics, two refractions at the spherical surface).  The
    # fluence in a thin column on the axis is largest where the beam is
    # narrowest; the midpoint of its half-maximum span is the focus.
    n, R = 1.46, 1.0
    z_focus = -1.0 - n * R / (2.0 * (n - 1.0))
    grid = W.Grid((0.498, -0.002, -3.0), (0.502, 0.002, -2.2), (1, 1, 160))
    wl = W.glass_sphere_beam(1_000_000, beam_radius=0.1, grid=grid, precision="fp64")
    flu, tot, _ = O.run(wl)
    col = flu[:, 0, 0].astype(np.float64)
    z = -3.0 + (np.arange(160) + 0.5) * 0.005
    half = z[col > 0.5 * col.max()]
    mid = 0.5 * (half.min() + half.max())
    assert abs(mid - z_focus) < 0.015, (mid, z_focus)
    # nothing absorbs in clear glass and air: every packet is reflected or
    # transmitted
    assert tot["A"] == 0 and tot["R"] + tot["T"] == wl.npackets * 2 ** 32


def test_capsule_bound_safe_for_rays_nearly_parallel_to_the_axis():
    # the cylinder part's quadratic is worst conditioned when the ray runs
    # almost along the axis, close to the wall: brute force along the move,
    # from inside and from outside, at angles down to 1e-9 rad
    d = 1e-6
    r = 0.05
    cap = W.Scene((W.Prim(W.CAPSULE, (0.0, 0.0, -1.0, 0.0, 0.0, 1.0, r)),),
                  (W.Region(W.prim_program([0]), 0.0, 1.0, 0.0, 1.5),), 1.0,
                  (-2, -2, -3), (2, 2, 3), delta=d, stepping=W.SEGMENT)
    checked = 0
    for off in (r - 4 * d, r - 1e-3, r + 4 * d, r + 1e-3):      # inside and outside the wall
        for ang in (0.0, 1e-9, 1e-6, 1e-4, 1e-2):
            for sgn in (1.0, -1.0):                              # towards and away from the wall
                p = np.array([off, 0.0, -0.5])
                u = np.array([sgn * math.sin(ang), 0.0, math.cos(ang)])
                if abs(O.region_sdf(cap, 0, p)) <= d:
                    continue
                t = O.segment_step(cap, p, u)
                s0 = np.sign(O.region_sdf(cap, 0, p))
                for s in np.linspace(0.0, t, 400):
                    q = p + s * u
                    v = O.region_sdf(cap, 0, q)
                    assert np.sign(v) == s0 and abs(v) >= d / 2 - 1e-12, (off, ang, sgn, t, s, v)
                checked += 1
    assert checked == 40
