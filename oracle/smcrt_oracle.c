/*
 * smcrt_oracle.c -- plain, slow, FP64 CPU oracle for SDF-based Monte Carlo
 * radiation transfer (signedMCRT, McMillan, Bruce & Dholakia).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA path: every structure below is private.
 *
 * What it computes, step by step in the paper's order (Sec. 2.1, 2.3,
 * Fig. 2 right panel, Fig. 3):
 *   - launch a packet (Sec. 2.1 "releasing photons"),
 *   - sample an optical depth tau = -ln(xi)                    (Eq. 1),
 *   - sphere-trace: d_sdf = min over all SDFs of |d|, step while the
 *     remaining optical depth is not reached               (Sec. 2.3),
 *   - at d_sdf < delta check the refractive index on both sides; if it
 *     changes compute the SDF-gradient normal by numerical differentiation
 *     and apply Fresnel reflection / Snell refraction  (Sec. 1, Sec. 2.3),
 *   - positive bounding-box SDF or an outward boundary hit terminates the
 *     packet                                                  (Sec. 2.3),
 *   - interaction: absorption weight, Henyey-Greenstein scattering
 *     (Sec. 3.1) with Russian roulette,
 *   - track-length fluence in rectangular voxel bins      (Sec. 3.1-3.2).
 *
 * Points the paper leaves open (xi in (0,1], delta, normal step, push-off,
 * Fresnel form, roulette constants, RNG) take one reading each, stated at
 * its use below.
 *
 * Bit-reproducibility conventions: IEEE +,-,*,/,sqrt only, compiled with
 * -ffp-contract=off, fixed expression order; ln and sin/cos are written
 * here from textbook series (atanh series for ln; Taylor series after
 * reduction to a quarter turn), not taken from libm.  Tallies are int64
 * fixed point (2^-32 units), so the result is independent of the order in
 * which packets are processed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_STACK 16
#define OR_FX 4294967296.0 /* 2^32: fixed-point scale of every tally */

/* ------------------------------------------------------------------------
 * Private structures (not shared with the CUDA side).
 * ---------------------------------------------------------------------- */
/* kind: 0 sphere, 1 box, 2 capsule, 3 torus, 4 capped cylinder; xform: 0 none,
 * k > 0 the primitive sits in frame xforms[k - 1] */
typedef struct { int32_t kind; int32_t xform; double p[7]; } or_prim;
/* Placement and domain operation of a primitive (Sec. 2.2: SDFs can be
 * translated, rotated, scaled, twisted, bent, elongated, repeated).  A point
 * with local coordinates l sits at s R l + t (R row-major, orthonormal).
 * op on the local point: 0 none, 1 elongate (a[0..2] half lengths),
 * 2 twist about local z (a[0] turns per unit length, a[1] radius reached by
 * the shape), 3 bend in the local x-y plane (same parameters, angle from x),
 * 4 repeat (a[0..2] periods, 0 = not repeated; a[3] copies each way). */
typedef struct { double rot[9], t[3], s; int32_t op, pad; double a[4]; } or_xform;
typedef struct { int32_t op; int32_t prim; double k; } or_node;         /* 0 prim,1 union,2 smooth,3 inter,4 sub */
typedef struct { int32_t begin, count; double mu_a, mu_s, g, n; } or_region;
typedef struct {
    const or_prim *prims; int32_t nprims;
    const or_node *nodes; int32_t nnodes;
    const or_region *regions; int32_t nregions;
    double ambient_n;
    double bbox_lo[3], bbox_hi[3];
    double delta;
    int64_t max_steps;
    int32_t stepping;          /* 0 sphere tracing (Sec. 2.3), 1 segment stepping (below) */
    int32_t pad;
    const or_xform *xforms; int32_t nxforms;
    int32_t pad2;
} or_scene;
typedef struct { int32_t kind; int32_t pad; double pos[3], dir[3], radius; } or_source; /* 0 pencil,1 disc,2 square,3 iso */
typedef struct { double lo[3], hi[3]; int32_t n[3]; int32_t pad; } or_grid;
typedef struct {
    int64_t R, T, A, killed, gain;       /* fixed point, 2^-32 weight units */
    int64_t packets, scatters, steps, scene_evals, prog_evals, prim_evals;
    int64_t interfaces, fresnel, pieces, max_steps_hit;
    /* work counters (no effect on the transport): primitive SDF evaluations
     * by kind (sphere, box, capsule, torus, cylinder), smooth-union
     * operations, segment-stepping bound calls and the primitive ray bounds
     * taken in them by kind */
    int64_t prim_kind[5], smooth_ops, seg_calls, seg_kind[5];
    int64_t seg_moves;    /* segment-stepping moves that did not end in an interaction */
    int64_t seg_dist[5];  /* primitive distances taken by the bounds, by kind */
} or_totals;
typedef struct { int64_t R, T, A, killed, gain, scatters, steps, pad; } or_packet;

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"): 10 rounds of two 32x32->64 multiplies
 * with the published multipliers and Weyl key increments.
 * ---------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Packet random stream: key = (seed lo, seed hi), counter = (event, 0, id
 * lo, id hi).  One call gives four uniforms xi_j = (w_j + 1) * 2^-32, which
 * lie in (0, 1] so that -ln(xi) of Eq. 1 is finite. */
typedef struct { uint32_t key[2]; uint32_t id_lo, id_hi; uint32_t event; } or_rng;

static void or_draw4(or_rng *r, double xi[4])
{
    uint32_t ctr[4] = { r->event, 0u, r->id_lo, r->id_hi };
    uint32_t w[4];
    or_philox4x32_10(ctr, r->key, w);
    r->event += 1u;
    for (int j = 0; j < 4; ++j) xi[j] = ((double)w[j] + 1.0) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------
 * ln(x) for positive normal x: x = m 2^e with m in (sqrt(1/2), sqrt(2)],
 * ln m = 2 atanh(s), s = (m-1)/(m+1), atanh series to s^21 (|s| <= 0.1716,
 * so the first omitted term is below 3e-17 relative).
 * ---------------------------------------------------------------------- */
double or_log(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    uint64_t mb = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > 1.4142135623730951) { m = m * 0.5; e = e + 1; }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double poly = 1.0 / 21.0;
    poly = poly * z + 1.0 / 19.0;
    poly = poly * z + 1.0 / 17.0;
    poly = poly * z + 1.0 / 15.0;
    poly = poly * z + 1.0 / 13.0;
    poly = poly * z + 1.0 / 11.0;
    poly = poly * z + 1.0 / 9.0;
    poly = poly * z + 1.0 / 7.0;
    poly = poly * z + 1.0 / 5.0;
    poly = poly * z + 1.0 / 3.0;
    poly = poly * z + 1.0;
    double lnm = 2.0 * s * poly;
    return (double)e * 0.6931471805599453 + lnm;
}

/* sin(2 pi t) and cos(2 pi t): t = f + q/4 with q the nearest quarter turn
 * (exact for t a multiple of 2^-32), angle a = 2 pi f in [-pi/4, pi/4],
 * Taylor series of sin to a^17 and cos to a^16 (omitted terms < 1e-17),
 * then a quarter-turn rotation by q. */
void or_sincos2pi(double t, double *sn, double *cs)
{
    double q = floor(t * 4.0 + 0.5);
    double f = t - q * 0.25;
    double a = f * 6.283185307179586;
    double z = a * a;
    double sp = 1.0 / 355687428096000.0;          /* 1/17! */
    sp = sp * z - 1.0 / 1307674368000.0;          /* 1/15! */
    sp = sp * z + 1.0 / 6227020800.0;             /* 1/13! */
    sp = sp * z - 1.0 / 39916800.0;               /* 1/11! */
    sp = sp * z + 1.0 / 362880.0;                 /* 1/9!  */
    sp = sp * z - 1.0 / 5040.0;                   /* 1/7!  */
    sp = sp * z + 1.0 / 120.0;                    /* 1/5!  */
    sp = sp * z - 1.0 / 6.0;                      /* 1/3!  */
    double s = a + a * (z * sp);
    double cp = 1.0 / 20922789888000.0;           /* 1/16! */
    cp = cp * z - 1.0 / 87178291200.0;            /* 1/14! */
    cp = cp * z + 1.0 / 479001600.0;              /* 1/12! */
    cp = cp * z - 1.0 / 3628800.0;                /* 1/10! */
    cp = cp * z + 1.0 / 40320.0;                  /* 1/8!  */
    cp = cp * z - 1.0 / 720.0;                    /* 1/6!  */
    cp = cp * z + 1.0 / 24.0;                     /* 1/4!  */
    cp = cp * z - 0.5;                            /* 1/2!  */
    double c = 1.0 + z * cp;
    int qi = ((int)q) & 3;
    if (qi == 0)      { *sn = s;  *cs = c;  }
    else if (qi == 1) { *sn = c;  *cs = -s; }
    else if (qi == 2) { *sn = -s; *cs = -c; }
    else              { *sn = -c; *cs = s;  }
}

/* ------------------------------------------------------------------------
 * Signed distance functions (Sec. 2.2): negative inside, positive outside.
 * ---------------------------------------------------------------------- */
static double sdf_sphere(const double p[3], const double *q)
{   /* Eq. 2: |p - c| - r */
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - q[3];
}

static double sdf_box(const double p[3], const double c[3], const double h[3])
{   /* exact box distance: length(max(|p-c|-h, 0)) + min(max component, 0) */
    double qx = fabs(p[0] - c[0]) - h[0];
    double qy = fabs(p[1] - c[1]) - h[1];
    double qz = fabs(p[2] - c[2]) - h[2];
    double mx = fmax(qx, 0.0), my = fmax(qy, 0.0), mz = fmax(qz, 0.0);
    double outside = sqrt(mx * mx + my * my + mz * mz);
    double inside = fmin(fmax(qx, fmax(qy, qz)), 0.0);
    return outside + inside;
}

static double sdf_capsule(const double p[3], const double *q)
{   /* distance to segment [a, b] minus r */
    double pax = p[0] - q[0], pay = p[1] - q[1], paz = p[2] - q[2];
    double bax = q[3] - q[0], bay = q[4] - q[1], baz = q[5] - q[2];
    double t = (pax * bax + pay * bay + paz * baz) / (bax * bax + bay * bay + baz * baz);
    t = fmin(fmax(t, 0.0), 1.0);
    double dx = pax - bax * t, dy = pay - bay * t, dz = paz - baz * t;
    return sqrt(dx * dx + dy * dy + dz * dz) - q[6];
}

static double sdf_torus(const double p[3], const double *q)
{   /* ring of major radius R = q[3] about the z axis through c, tube radius
     * r = q[4]: distance to the core circle minus r */
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    double ring = sqrt(dx * dx + dy * dy) - q[3];
    return sqrt(ring * ring + dz * dz) - q[4];
}

static double sdf_cylinder(const double p[3], const double *q)
{   /* capped cylinder along z through c, radius q[3], half height q[4]:
     * the exact distance of a 2D box in (radial, axial) coordinates */
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    double a = sqrt(dx * dx + dy * dy) - q[3];
    double b = fabs(dz) - q[4];
    double ma = fmax(a, 0.0), mb = fmax(b, 0.0);
    return fmin(fmax(a, b), 0.0) + sqrt(ma * ma + mb * mb);
}

static double sdf_base(int kind, const double *q, const double p[3])
{
    if (kind == 0) return sdf_sphere(p, q);
    if (kind == 1) return sdf_box(p, q, q + 3);
    if (kind == 2) return sdf_capsule(p, q);
    if (kind == 3) return sdf_torus(p, q);
    return sdf_cylinder(p, q);
}

/* A primitive in its frame: map p to local coordinates (inverse placement),
 * apply the domain operation, evaluate, scale back by s and divide by the
 * operation's Lipschitz bound L, so the value never exceeds the true
 * distance and sphere tracing stays safe (the paper's caution about
 * non-bounded SDFs, Sec. 5). */
static double sdf_xprim(const or_prim *pr, const or_xform *X, const double p[3])
{
    double vx = p[0] - X->t[0], vy = p[1] - X->t[1], vz = p[2] - X->t[2];
    double q[3];
    q[0] = (X->rot[0] * vx + X->rot[3] * vy + X->rot[6] * vz) / X->s;
    q[1] = (X->rot[1] * vx + X->rot[4] * vy + X->rot[7] * vz) / X->s;
    q[2] = (X->rot[2] * vx + X->rot[5] * vy + X->rot[8] * vz) / X->s;
    double L = 1.0;
    if (X->op == 1) {                        /* elongate: stretch the centre */
        for (int a = 0; a < 3; ++a) q[a] = q[a] - fmin(fmax(q[a], -X->a[a]), X->a[a]);
    } else if (X->op == 2 || X->op == 3) {   /* twist about z / bend about the x-y plane */
        double rho = sqrt(q[0] * q[0] + q[1] * q[1]);
        double sn, cs;
        or_sincos2pi(X->a[0] * (X->op == 2 ? q[2] : q[0]), &sn, &cs);
        double x = cs * q[0] - sn * q[1];
        double y = sn * q[0] + cs * q[1];
        q[0] = x; q[1] = y;
        /* largest stretch of the map within radius rho of the axis, with
         * m = 2 pi a0 rho: its Jacobian is a rotation times I + m N, N of
         * norm one; for the twist the largest singular value of
         * [[I, m e], [0, 1]] is (m + sqrt(m^2 + 4)) / 2, for the bend that
         * of I + m N is 1 + m.  rho: the larger of the point's and the
         * shape's radius, so the bound holds on the whole segment from the
         * point to the surface (rho is convex along it). */
        double m = 6.283185307179586 * X->a[0] * fmax(rho, X->a[1]);
        L = X->op == 2 ? 0.5 * (m + sqrt(m * m + 4.0)) : 1.0 + m;
    } else if (X->op == 4) {                 /* repetition: nearest copy, at most a[3] each way */
        for (int a = 0; a < 3; ++a) {
            double c = X->a[a];
            if (c > 0.0) {
                double k = floor(q[a] / c + 0.5);
                k = fmin(fmax(k, -X->a[3]), X->a[3]);
                q[a] = q[a] - c * k;
            }
        }
    }
    return X->s * sdf_base(pr->kind, pr->p, q) / L;
}

static double sdf_prim(const or_scene *S, const or_prim *pr, const double p[3])
{
    if (pr->xform > 0) return sdf_xprim(pr, &S->xforms[pr->xform - 1], p);
    return sdf_base(pr->kind, pr->p, p);
}

/* CSG on two distances: a is the left (earlier) operand, b the right. */
static double csg_apply(int op, double a, double b, double k)
{
    if (op == 1) return fmin(a, b);                    /* union        */
    if (op == 3) return fmax(a, b);                    /* intersection */
    if (op == 4) return fmax(a, -b);                   /* a minus b    */
    /* smooth union: polynomial smooth minimum of the SDF literature cited
     * with the gallery (Fig. 1 e); h blends, k*h*(1-h) rounds the join. */
    double h = 0.5 + 0.5 * (b - a) / k;
    h = fmin(fmax(h, 0.0), 1.0);
    double m = b * (1.0 - h) + a * h;
    return m - k * h * (1.0 - h);
}

/* Evaluate region r's postfix program at p. */
static double region_sdf(const or_scene *S, int r, const double p[3], or_totals *T)
{
    double st[OR_MAX_STACK];
    int sp = 0;
    const or_region *R = &S->regions[r];
    for (int i = 0; i < R->count; ++i) {
        const or_node *nd = &S->nodes[R->begin + i];
        if (nd->op == 0) {
            st[sp++] = sdf_prim(S, &S->prims[nd->prim], p);
            if (T) { T->prim_evals += 1; T->prim_kind[S->prims[nd->prim].kind] += 1; }
        } else {
            double b = st[--sp];
            double a = st[--sp];
            st[sp++] = csg_apply(nd->op, a, b, nd->k);
            if (T && nd->op == 2) T->smooth_ops += 1;
        }
    }
    return st[0];
}

static void bbox_center_half(const or_scene *S, double c[3], double h[3])
{
    for (int a = 0; a < 3; ++a) {
        c[a] = (S->bbox_lo[a] + S->bbox_hi[a]) * 0.5;
        h[a] = (S->bbox_hi[a] - S->bbox_lo[a]) * 0.5;
    }
}

static double bbox_sdf(const or_scene *S, const double p[3])
{
    double c[3], h[3];
    bbox_center_half(S, c, h);
    return sdf_box(p, c, h);
}

/* Full scene evaluation (Sec. 2.3): every region's SDF and the bounding
 * box.  region = highest-index region whose SDF is negative (-1 ambient);
 * d_min = min |d| over regions, then the bounding box; istar is the
 * surface attaining it (lowest region index on ties, box = -1 last). */
typedef struct { double dmin; double dstar; int istar; int region; double dbox; double dsoft; } or_eval;

/* Segment stepping bounds a region by rays to its primitives, widened by a
 * margin of k/4 per smooth union (below).  A region with more smooth unions
 * than this ("soft") keeps the isotropic bound |d| - delta/2: its margin
 * would grow past what the ray bound gains. */
#define OR_SEG_MAX_SMOOTH 8

static int region_soft(const or_scene *S, int r)
{
    const or_region *R = &S->regions[r];
    int n = 0;
    for (int i = 0; i < R->count; ++i)
        if (S->nodes[R->begin + i].op == 2) n += 1;
    return n > OR_SEG_MAX_SMOOTH;
}

static or_eval scene_eval(const or_scene *S, const double p[3], or_totals *T)
{
    or_eval E;
    E.dmin = INFINITY; E.dstar = 0.0; E.istar = -1; E.region = -1;
    E.dsoft = INFINITY;      /* min |d| over soft regions */
    for (int r = 0; r < S->nregions; ++r) {
        double d = region_sdf(S, r, p, T);
        if (d < 0.0) E.region = r;
        double ad = fabs(d);
        if (ad < E.dmin) { E.dmin = ad; E.istar = r; E.dstar = d; }
        if (region_soft(S, r) && ad < E.dsoft) E.dsoft = ad;
    }
    E.dbox = bbox_sdf(S, p);
    if (fabs(E.dbox) < E.dmin) { E.dmin = fabs(E.dbox); E.istar = -1; E.dstar = E.dbox; }
    if (T) T->scene_evals += 1;
    return E;
}

static int scene_region(const or_scene *S, const double p[3], or_totals *T)
{
    return scene_eval(S, p, T).region;
}

/* The SDF of one surface: region program, or the bounding box for -1. */
static double surface_sdf(const or_scene *S, int istar, const double p[3], or_totals *T)
{
    if (T) T->prog_evals += 1;
    if (istar < 0) return bbox_sdf(S, p);
    return region_sdf(S, istar, p, T);
}

/* Normal by numerical differentiation of the surface SDF (Sec. 1 "numerical
 * differentiation to provide the surface normals"): central differences
 * with step h, then normalised.  Returns 0 for a vanishing gradient. */
static int surface_normal(const or_scene *S, int istar, const double p[3], double h,
                          double n[3], or_totals *T)
{
    double g[3];
    for (int a = 0; a < 3; ++a) {
        double pp[3] = { p[0], p[1], p[2] };
        double pm[3] = { p[0], p[1], p[2] };
        pp[a] = p[a] + h;
        pm[a] = p[a] - h;
        g[a] = surface_sdf(S, istar, pp, T) - surface_sdf(S, istar, pm, T);
    }
    double l2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (!(l2 > 0.0)) return 0;
    double l = sqrt(l2);
    n[0] = g[0] / l; n[1] = g[1] / l; n[2] = g[2] / l;
    return 1;
}

static double region_n(const or_scene *S, int r) { return r < 0 ? S->ambient_n : S->regions[r].n; }

static void normalise(double u[3])
{
    double l = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    u[0] = u[0] / l; u[1] = u[1] / l; u[2] = u[2] / l;
}

/* Orthonormal basis (b1, b2) perpendicular to the unit vector n, branchless
 * construction of Duff, Burgess, Christensen, Hery, Kensler, Liani and
 * Villemin, "Building an Orthonormal Basis, Revisited" (JCGT 6(1), 2017). */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double sg = copysign(1.0, n[2]);
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sg * n[0] * n[0] * a; b1[1] = sg * b; b1[2] = -sg * n[0];
    b2[0] = b; b2[1] = sg + n[1] * n[1] * a; b2[2] = -n[1];
}

/* ------------------------------------------------------------------------
 * Track-length fluence tally (Sec. 3.1-3.2: fluence grid, rectangular bins).
 * The segment p + t u, t in [0, len], is clipped to the grid box and split
 * by a 3D DDA (Amanatides & Woo, Eurographics 1987).  The parametric
 * distance to each axis' next plane is recomputed from the segment start
 * (not accumulated).  Each piece adds llrint(w * piece * 2^32) to its
 * voxel; ties between axes advance x before y before z.
 * ---------------------------------------------------------------------- */
void or_tally(const or_grid *G, const double p[3], const double u[3], double len, double w,
              int64_t *flu, int64_t *pieces)
{
    if (!flu || !(len > 0.0) || !(w > 0.0)) return;
    double tin = 0.0, tout = len;
    double dl[3];
    for (int a = 0; a < 3; ++a) {
        dl[a] = (G->hi[a] - G->lo[a]) / (double)G->n[a];
        if (u[a] != 0.0) {
            double t0 = (G->lo[a] - p[a]) / u[a];
            double t1 = (G->hi[a] - p[a]) / u[a];
            double tmin = fmin(t0, t1), tmax = fmax(t0, t1);
            tin = fmax(tin, tmin);
            tout = fmin(tout, tmax);
        } else if (p[a] < G->lo[a] || p[a] > G->hi[a]) {
            return;
        }
    }
    if (!(tin < tout)) return;
    int idx[3], step[3];
    double tnext[3];
    for (int a = 0; a < 3; ++a) {
        double x = p[a] + tin * u[a];
        double f = floor((x - G->lo[a]) / dl[a]);
        int i = (int)fmin(fmax(f, 0.0), (double)(G->n[a] - 1));
        idx[a] = i;
        if (u[a] > 0.0) {
            step[a] = 1;
            tnext[a] = ((G->lo[a] + (double)(i + 1) * dl[a]) - p[a]) / u[a];
        } else if (u[a] < 0.0) {
            step[a] = -1;
            tnext[a] = ((G->lo[a] + (double)i * dl[a]) - p[a]) / u[a];
        } else {
            step[a] = 0;
            tnext[a] = INFINITY;
        }
    }
    double t = tin;
    int guard = G->n[0] + G->n[1] + G->n[2] + 3;
    while (guard-- > 0) {
        int ax;
        if (tnext[0] <= tnext[1] && tnext[0] <= tnext[2]) ax = 0;
        else if (tnext[1] <= tnext[2]) ax = 1;
        else ax = 2;
        double tend = fmin(tnext[ax], tout);
        double piece = tend - t;
        if (piece > 0.0) {
            int64_t v = llrint(w * piece * OR_FX);
            size_t off = ((size_t)idx[2] * (size_t)G->n[1] + (size_t)idx[1]) * (size_t)G->n[0] + (size_t)idx[0];
            flu[off] += v;
            if (pieces) *pieces += 1;
            t = tend;
        }
        if (tnext[ax] >= tout) break;
        idx[ax] += step[ax];
        if (idx[ax] < 0 || idx[ax] >= G->n[ax]) break;
        if (step[ax] > 0)
            tnext[ax] = ((G->lo[ax] + (double)(idx[ax] + 1) * dl[ax]) - p[ax]) / u[ax];
        else
            tnext[ax] = ((G->lo[ax] + (double)idx[ax] * dl[ax]) - p[ax]) / u[ax];
    }
}

static int64_t fx(double x) { return llrint(x * OR_FX); }

/* Henyey-Greenstein sample of cos(theta) (Sec. 3.1 "Henyey-Greenstein phase
 * function"), inverse-CDF form; isotropic for |g| < 1e-6. */
double or_hg_cos(double g, double xi)
{
    double c;
    if (fabs(g) < 1e-6) {
        c = 2.0 * xi - 1.0;
    } else {
        double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
        c = (1.0 + g * g - t * t) / (2.0 * g);
    }
    return fmin(fmax(c, -1.0), 1.0);
}

/* New direction after scattering by polar cosine ct and azimuth 2 pi xi. */
void or_scatter_dir(double u[3], double ct, double xi_phi)
{
    double st = sqrt((1.0 - ct) * (1.0 + ct));
    double sp, cp;
    or_sincos2pi(xi_phi, &sp, &cp);
    double b1[3], b2[3];
    onb(u, b1, b2);
    double a1 = st * cp, a2 = st * sp;
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = a1 * b1[k] + a2 * b2[k] + ct * u[k];
    normalise(v);
    u[0] = v[0]; u[1] = v[1]; u[2] = v[2];
}

/* Fresnel reflectance for unpolarised light (average of s and p), 1 for
 * total internal reflection.  Also returns cos of the transmitted angle. */
double or_fresnel(double n1, double n2, double ci, double *ct_out)
{
    double eta = n1 / n2;
    double st2 = eta * eta * ((1.0 - ci) * (1.0 + ci));
    if (st2 >= 1.0) { if (ct_out) *ct_out = 0.0; return 1.0; }
    double ct = sqrt(1.0 - st2);
    double rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
    double rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
    if (ct_out) *ct_out = ct;
    return 0.5 * (rs * rs + rp * rp);
}

/* Interface step (Sec. 2.3: d_sdf < delta).  Returns 0 if the packet is not
 * approaching surface istar (caller then takes a forced step of delta), 1 if
 * it was handled (moved across or reflected), 2 if it escaped through the
 * bounding box. */
static int interface_step(const or_scene *S, or_eval *E, double p[3], double u[3],
                          or_rng *rng, or_totals *T)
{
    double nrm[3];
    if (!surface_normal(S, E->istar, p, S->delta, nrm, T)) return 0;
    double c = u[0] * nrm[0] + u[1] * nrm[1] + u[2] * nrm[2];
    int approaching = (c > 0.0 && E->dstar < 0.0) || (c < 0.0 && E->dstar >= 0.0);
    if (!approaching) return 0;
    if (E->istar < 0) return 2;               /* outward through the box */
    T->interfaces += 1;
    /* localise: project onto the surface along the normal (no tally) */
    double q[3] = { p[0], p[1], p[2] };
    double tol = S->delta * 1e-3;
    for (int it = 0; it < 3; ++it) {
        double dq = surface_sdf(S, E->istar, q, T);
        if (fabs(dq) <= tol) break;
        q[0] = q[0] - dq * nrm[0]; q[1] = q[1] - dq * nrm[1]; q[2] = q[2] - dq * nrm[2];
    }
    double sg = c > 0.0 ? 1.0 : -1.0;
    double e = 2.0 * S->delta * sg;
    double pf[3] = { q[0] + e * nrm[0], q[1] + e * nrm[1], q[2] + e * nrm[2] };
    double pn[3] = { q[0] - e * nrm[0], q[1] - e * nrm[1], q[2] - e * nrm[2] };
    int rf = scene_region(S, pf, T);
    int rn = scene_region(S, pn, T);
    double n1 = region_n(S, rn), n2 = region_n(S, rf);
    if (n1 == n2) {                            /* no index change: cross */
        p[0] = pf[0]; p[1] = pf[1]; p[2] = pf[2];
        return 1;
    }
    T->fresnel += 1;
    double ci = fabs(c);
    double ct;
    double R = or_fresnel(n1, n2, ci, &ct);
    int reflect = 1;
    if (R < 1.0) {
        double xi[4];
        or_draw4(rng, xi);
        reflect = xi[0] <= R;
    }
    if (reflect) {
        double c2 = 2.0 * c;
        u[0] = u[0] - c2 * nrm[0]; u[1] = u[1] - c2 * nrm[1]; u[2] = u[2] - c2 * nrm[2];
        normalise(u);
        p[0] = pn[0]; p[1] = pn[1]; p[2] = pn[2];
    } else {
        double eta = n1 / n2;
        double k = sg * (eta * ci - ct);
        u[0] = eta * u[0] - k * nrm[0]; u[1] = eta * u[1] - k * nrm[1]; u[2] = eta * u[2] - k * nrm[2];
        normalise(u);
        p[0] = pf[0]; p[1] = pf[1]; p[2] = pf[2];
    }
    return 1;
}

/* Launch (photon release) for packet id: one Philox call; xi0, xi1 place or
 * orient the packet, xi3 gives the first optical depth. */
static void launch(const or_source *src, double p[3], double u[3], double *tau, or_rng *rng)
{
    double xi[4];
    or_draw4(rng, xi);
    p[0] = src->pos[0]; p[1] = src->pos[1]; p[2] = src->pos[2];
    u[0] = src->dir[0]; u[1] = src->dir[1]; u[2] = src->dir[2];
    if (src->kind == 1 || src->kind == 2) {
        double b1[3], b2[3];
        onb(src->dir, b1, b2);
        double c1, c2;
        if (src->kind == 1) {                  /* uniform disc of radius R */
            double rho = src->radius * sqrt(xi[0]);
            double sn, cs;
            or_sincos2pi(xi[1], &sn, &cs);
            c1 = rho * cs; c2 = rho * sn;
        } else {                               /* uniform square, half side R */
            c1 = src->radius * (2.0 * xi[0] - 1.0);
            c2 = src->radius * (2.0 * xi[1] - 1.0);
        }
        for (int k = 0; k < 3; ++k) p[k] = src->pos[k] + c1 * b1[k] + c2 * b2[k];
    } else if (src->kind == 3) {               /* isotropic point */
        double ct = 2.0 * xi[0] - 1.0;
        double st = sqrt((1.0 - ct) * (1.0 + ct));
        double sn, cs;
        or_sincos2pi(xi[1], &sn, &cs);
        u[0] = st * cs; u[1] = st * sn; u[2] = ct;
    }
    *tau = -or_log(xi[3]);
}

/* ------------------------------------------------------------------------
 * Segment stepping (scene option; Sec. 5 names segment tracing, which
 * lengthens sphere-tracing steps with bounds taken along the ray, as the
 * remedy for the many small steps of packets travelling nearly parallel to
 * a surface).  Sphere tracing moves by d_min, a bound valid in every
 * direction.  Along the packet's own direction u a longer move is safe.
 *
 * Margin of a region: M = sum of k/4 over its smooth unions (0 for hard
 * CSG).  A smooth union lies between min(a, b) - k/4 and min(a, b) (the
 * blend term k h (1 - h) peaks at h = 1/2), and min, max and max(a, -b)
 * move by at most the largest change of their operands, so the region's
 * SDF F stays within M of its hard version H (every smooth union replaced
 * by min).  H takes, at each point, the value or the negated value of one
 * of its primitives; hence F = 0 only where some primitive has |d_i| <= M.
 * A three-fold smooth union of one sphere reaches 0.39 k below min, so the
 * sum over the folds, not a single k/4, is needed.  Soft regions (more than
 * OR_SEG_MAX_SMOOTH smooth unions) take their isotropic |d| - delta/2.
 *
 * Primitive bound with margin e = M + delta/2 (M the largest margin of the
 * regions that use the primitive): the distance along the ray until |d_i|
 * can fall to e:
 *   - sphere, box, capsule, capped cylinder: outside, the entry of the shape
 *     grown by e (for boxes and cylinders the grown box, which holds the
 *     rounded one); inside, the exit of the shape shrunk by e (exactly the
 *     set d_i < -e of these convex shapes);
 *   - torus from outside: the entry of the annular slab that holds the tube
 *     grown by e, and at least d_i - e; from inside, the exit of the ball of
 *     radius r - e about the nearest point of the core circle;
 *   - the same shapes placed by a frame without a domain operation, in the
 *     frame's coordinates; domain operations: |d_i| - e.
 * On [0, t) every primitive keeps |d_i| > e, so no region's sign changes and
 * every region's |F| stays above delta/2.  The bounding box adds its exit
 * distance, shrunk by delta/2.  The step is max(d_min - delta/2, minimum of
 * the bounds): never shorter than plain sphere tracing.  It ends delta/2
 * short of the first surface, where the next evaluation finds d_min < delta
 * and the interface routine of Sec. 2.3 runs unchanged.
 *
 * The primitives of the regions that are not soft are visited once each,
 * in the order of first use by those regions, after the bounding box and
 * the soft regions' bound.  A primitive whose |d_i| - e is not
 * below the bound so far cannot lower it (its ray bound is at least that,
 * the SDF being 1-Lipschitz) and is passed over; one with |d_i| <= e ends
 * the search with 0.
 * ---------------------------------------------------------------------- */
static double segment_sphere(const double *q, double d, const double p[3], const double u[3], double dh)
{
    double rr = d > 0.0 ? q[3] + dh : q[3] - dh;
    double ox = p[0] - q[0], oy = p[1] - q[1], oz = p[2] - q[2];
    double b = ox * u[0] + oy * u[1] + oz * u[2];
    double cc = ox * ox + oy * oy + oz * oz - rr * rr;
    double disc = b * b - cc;
    double t;
    if (d > 0.0) {                       /* outside: entry of the grown sphere */
        if (b >= 0.0 || disc < 0.0) return INFINITY;
        t = cc / (sqrt(disc) - b);       /* near root, free of cancellation */
    } else {                             /* inside: exit of the shrunk sphere */
        if (disc < 0.0) return 0.0;
        if (b > 0.0) t = -cc / (b + sqrt(disc));
        else t = sqrt(disc) - b;
    }
    return t > 0.0 ? t : 0.0;
}

static double segment_box(const double c[3], const double h[3], double d, const double p[3],
                          const double u[3], double dh)
{
    double e = d > 0.0 ? dh : -dh;
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = c[a] - (h[a] + e), hi = c[a] + (h[a] + e);
        if (u[a] != 0.0) {
            double t0 = (lo - p[a]) / u[a], t1 = (hi - p[a]) / u[a];
            tn = fmax(tn, fmin(t0, t1));
            tf = fmin(tf, fmax(t0, t1));
        } else if (p[a] < lo || p[a] > hi) {
            return d > 0.0 ? INFINITY : 0.0;
        }
    }
    if (d > 0.0) {                       /* outside: entry of the grown box */
        if (tn > tf || tf < 0.0) return INFINITY;
        return tn > 0.0 ? tn : 0.0;
    }
    return tf > 0.0 ? tf : 0.0;          /* inside: exit of the shrunk box */
}

/* Interval [t0, t1] of the ray p + t u inside the ball of radius rr whose
 * centre is at p - o (t0 > t1: missed).  The far root of a quadratic comes
 * from the near one through the product of the roots (no cancellation). */
static void ray_ball(double ox, double oy, double oz, double rr, const double u[3], double *t0, double *t1)
{
    double b = ox * u[0] + oy * u[1] + oz * u[2];
    double cc = ox * ox + oy * oy + oz * oz - rr * rr;
    double disc = b * b - cc;
    *t0 = INFINITY; *t1 = -INFINITY;
    if (disc < 0.0) return;
    double sq = sqrt(disc);
    if (b > 0.0) {
        double q = -(b + sq);
        *t0 = q; *t1 = cc / q;
    } else {
        double q = sq - b;
        if (q > 0.0) { *t1 = q; *t0 = cc / q; }
        else { *t0 = 0.0; *t1 = 0.0; }
    }
}

/* Interval of the ray inside the cylinder of radius rr about the axis a + s ba,
 * between the planes s = 0 and s = 1 (o = p - a, L2 = |ba|^2).  The parts of
 * o and u across the axis are formed first, so a ray nearly parallel to the
 * axis keeps its small cross-axis motion accurate. */
static void ray_cylinder(double ox, double oy, double oz, double bax, double bay, double baz, double L2,
                         double rr, const double u[3], double *t0, double *t1)
{
    double uw = u[0] * bax + u[1] * bay + u[2] * baz;
    double ow = ox * bax + oy * bay + oz * baz;
    double lo = -INFINITY, hi = INFINITY;
    *t0 = INFINITY; *t1 = -INFINITY;
    if (uw != 0.0) {                     /* between the end planes */
        double s0 = -ow / uw, s1 = (L2 - ow) / uw;
        lo = fmin(s0, s1); hi = fmax(s0, s1);
    } else if (ow < 0.0 || ow > L2) {
        return;
    }
    double k = uw / L2, m = ow / L2;
    double vx = u[0] - k * bax, vy = u[1] - k * bay, vz = u[2] - k * baz;
    double wx = ox - m * bax, wy = oy - m * bay, wz = oz - m * baz;
    double A = vx * vx + vy * vy + vz * vz;
    double B = wx * vx + wy * vy + wz * vz;
    double C = wx * wx + wy * wy + wz * wz - rr * rr;
    if (A > 0.0) {                       /* A t^2 + 2 B t + C <= 0 */
        double disc = B * B - A * C;
        if (disc < 0.0) return;
        double sq = sqrt(disc), c0, c1;
        if (B > 0.0) {
            double q = -(B + sq);
            c0 = q / A; c1 = C / q;
        } else {
            double q = sq - B;
            if (q > 0.0) { c1 = q / A; c0 = C / q; }
            else { c0 = 0.0; c1 = 0.0; }
        }
        lo = fmax(lo, c0); hi = fmin(hi, c1);
    } else if (C > 0.0) {
        return;
    }
    *t0 = lo; *t1 = hi;
}

/* Capsule (convex: the cylinder between its end planes and the two end
 * balls): from outside, the earliest entry of a part of the capsule grown by
 * dh; from inside, the latest exit from a part of the capsule shrunk by dh. */
static double segment_capsule(const double *q, double d, const double p[3], const double u[3], double dh)
{
    double rr = d > 0.0 ? q[6] + dh : q[6] - dh;
    double ox = p[0] - q[0], oy = p[1] - q[1], oz = p[2] - q[2];
    double bax = q[3] - q[0], bay = q[4] - q[1], baz = q[5] - q[2];
    double L2 = bax * bax + bay * bay + baz * baz;
    double t0[3], t1[3];
    ray_ball(ox, oy, oz, rr, u, &t0[0], &t1[0]);
    ray_ball(ox - bax, oy - bay, oz - baz, rr, u, &t0[1], &t1[1]);
    ray_cylinder(ox, oy, oz, bax, bay, baz, L2, rr, u, &t0[2], &t1[2]);
    double t;
    if (d > 0.0) {
        t = INFINITY;
        for (int k = 0; k < 3; ++k)
            if (t0[k] <= t1[k] && t1[k] >= 0.0) t = fmin(t, t0[k]);
    } else {
        t = 0.0;
        for (int k = 0; k < 3; ++k)
            if (t0[k] <= t1[k]) t = fmax(t, t1[k]);
    }
    return t > 0.0 ? t : 0.0;
}

/* Capped cylinder along z (radius q[3], half height q[4]): convex, the
 * slab |z - c_z| <= h cut by the infinite cylinder; grown by e from outside,
 * shrunk by e from inside (the margin's sign follows d). */
static double segment_cylinder(const double *q, double d, const double p[3], const double u[3], double e)
{
    double g = d > 0.0 ? e : -e;
    double rr = q[3] + g, hh = q[4] + g;
    double t0, t1;
    ray_cylinder(p[0] - q[0], p[1] - q[1], p[2] - q[2] + hh, 0.0, 0.0, 2.0 * hh, 4.0 * hh * hh, rr, u, &t0, &t1);
    if (d > 0.0) {
        if (!(t0 <= t1) || t1 < 0.0) return INFINITY;
        return t0 > 0.0 ? t0 : 0.0;
    }
    if (!(t0 <= t1)) return 0.0;
    return t1 > 0.0 ? t1 : 0.0;
}

/* Torus about z (major radius q[3], tube q[4]) from outside: the tube grown
 * by e lies in the annular slab R - r' <= rho <= R + r', |z - c_z| <= r'
 * (r' = r + e); the ray's first point in that slab, and never less than
 * d - e.  From inside: the tube shrunk by e holds the ball of radius r - e
 * about the point of the core circle nearest p (which that ball contains,
 * at depth |d| - e), so the ray's exit from the ball bounds the move
 * (p on the axis: |d| - e). */
static double segment_torus(const double *q, double d, const double p[3], const double u[3], double e)
{
    if (d < 0.0) {
        double dx = p[0] - q[0], dy = p[1] - q[1];
        double rho = sqrt(dx * dx + dy * dy);
        if (!(rho > 0.0)) return -d - e;
        double ball[4] = {q[0] + q[3] * dx / rho, q[1] + q[3] * dy / rho, q[2], q[4]};
        return segment_sphere(ball, d, p, u, e);
    }
    double R = q[3], rt = q[4] + e;
    double ox = p[0] - q[0], oy = p[1] - q[1], oz = p[2] - q[2] + rt;
    double a0, a1;
    ray_cylinder(ox, oy, oz, 0.0, 0.0, 2.0 * rt, 4.0 * rt * rt, R + rt, u, &a0, &a1);
    double lo = fmax(a0, 0.0), hi = a1;
    if (!(lo <= hi)) return INFINITY;
    if (R - rt > 0.0) {                  /* the hole rho < R - r' is not in the slab */
        double b0, b1;
        ray_cylinder(ox, oy, oz, 0.0, 0.0, 2.0 * rt, 4.0 * rt * rt, R - rt, u, &b0, &b1);
        if (b0 <= lo && lo < b1) lo = b1;
        if (!(lo < hi)) return INFINITY;   /* left the slab inside the hole */
    }
    return fmax(lo, d - e);
}

/* The shape kinds with a ray bound, in the primitive's own coordinates. */
static double segment_base(int kind, const double *q, double d, const double p[3], const double u[3], double e)
{
    if (kind == 0) return segment_sphere(q, d, p, u, e);
    if (kind == 1) return segment_box(q, q + 3, d, p, u, e);
    if (kind == 2) return segment_capsule(q, d, p, u, e);
    if (kind == 3) return segment_torus(q, d, p, u, e);
    return segment_cylinder(q, d, p, u, e);
}

/* A primitive placed by a frame without a domain operation: the frame
 * (rotation R, translation t, uniform scale s) maps the ray p + t' u to the
 * local ray q + (t' / s) w with q = R^T (p - t) / s and the unit direction
 * w = R^T u, and local distances are world distances over s.  So the world
 * bound is s times the local bound with margin e / s; only the sign of d and
 * (for the torus) its value over s are used. */
static double segment_xprim(const or_prim *pr, const or_xform *X, double d, const double p[3], const double u[3],
                            double e)
{
    double vx = p[0] - X->t[0], vy = p[1] - X->t[1], vz = p[2] - X->t[2];
    double q[3], w[3];
    q[0] = (X->rot[0] * vx + X->rot[3] * vy + X->rot[6] * vz) / X->s;
    q[1] = (X->rot[1] * vx + X->rot[4] * vy + X->rot[7] * vz) / X->s;
    q[2] = (X->rot[2] * vx + X->rot[5] * vy + X->rot[8] * vz) / X->s;
    w[0] = X->rot[0] * u[0] + X->rot[3] * u[1] + X->rot[6] * u[2];
    w[1] = X->rot[1] * u[0] + X->rot[4] * u[1] + X->rot[7] * u[2];
    w[2] = X->rot[2] * u[0] + X->rot[5] * u[1] + X->rot[8] * u[2];
    return X->s * segment_base(pr->kind, pr->p, d / X->s, q, w, e / X->s);
}

/* Bound of one primitive whose distance d satisfies |d| > e. */
static double segment_prim(const or_scene *S, const or_prim *pr, double d, const double p[3], const double u[3],
                           double e)
{
    if (pr->xform == 0) return segment_base(pr->kind, pr->p, d, p, u, e);
    if (S->xforms[pr->xform - 1].op == 0) return segment_xprim(pr, &S->xforms[pr->xform - 1], d, p, u, e);
    return fabs(d) - e;                  /* domain operations: isotropic bound */
}

/* Sum of k/4 over the smooth unions of region r (0: hard CSG). */
static double region_margin(const or_scene *S, int r)
{
    const or_region *R = &S->regions[r];
    double m = 0.0;
    for (int i = 0; i < R->count; ++i)
        if (S->nodes[R->begin + i].op == 2) m = m + 0.25 * S->nodes[R->begin + i].k;
    return m;
}

/* 1 if node i of region r is the first use of its primitive by a region
 * that is not soft (regions in order, nodes in program order). */
static int first_use(const or_scene *S, int r, int i)
{
    int prim = S->nodes[S->regions[r].begin + i].prim;
    for (int r2 = 0; r2 <= r; ++r2) {
        if (region_soft(S, r2)) continue;
        const or_region *R = &S->regions[r2];
        int end = r2 == r ? i : R->count;
        for (int j = 0; j < end; ++j)
            if (S->nodes[R->begin + j].op == 0 && S->nodes[R->begin + j].prim == prim) return 0;
    }
    return 1;
}

/* Largest margin of the regions, not soft, that use primitive prim. */
static double prim_margin(const or_scene *S, int prim)
{
    double m = 0.0;
    for (int r = 0; r < S->nregions; ++r) {
        if (region_soft(S, r)) continue;
        const or_region *R = &S->regions[r];
        for (int j = 0; j < R->count; ++j)
            if (S->nodes[R->begin + j].op == 0 && S->nodes[R->begin + j].prim == prim) {
                m = fmax(m, region_margin(S, r));
                break;
            }
    }
    return m;
}

/* Largest safe move from p along u (scene evaluated at p in E). */
static double segment_bound(const or_scene *S, const or_eval *E, const double p[3], const double u[3],
                            or_totals *T)
{
    double dh = 0.5 * S->delta;
    double c[3], h[3];
    bbox_center_half(S, c, h);
    double t = fmin(segment_box(c, h, E->dbox, p, u, dh), E->dsoft - dh);
    if (T) T->seg_calls += 1;
    for (int r = 0; r < S->nregions; ++r) {
        if (region_soft(S, r)) continue;
        const or_region *R = &S->regions[r];
        for (int i = 0; i < R->count; ++i) {
            const or_node *nd = &S->nodes[R->begin + i];
            if (nd->op != 0 || !first_use(S, r, i)) continue;
            const or_prim *pr = &S->prims[nd->prim];
            double e = prim_margin(S, nd->prim) + dh;
            double d = sdf_prim(S, pr, p);
            if (T) T->seg_dist[pr->kind] += 1;
            if (!(fabs(d) > e)) return 0.0;
            if (fabs(d) - e >= t) continue;
            t = fmin(t, segment_prim(S, pr, d, p, u, e));
            if (T) T->seg_kind[pr->kind] += 1;
        }
    }
    return t;
}

#define OR_W_ROULETTE 1e-4
#define OR_ROULETTE_M 10.0

/* Propagate one packet to termination. */
static void run_packet(const or_scene *S, const or_source *src, const or_grid *G, uint64_t id,
                       uint64_t seed, int64_t *flu, or_totals *T, or_packet *rec)
{
    or_rng rng;
    rng.key[0] = (uint32_t)seed; rng.key[1] = (uint32_t)(seed >> 32);
    rng.id_lo = (uint32_t)id; rng.id_hi = (uint32_t)(id >> 32);
    rng.event = 0u;
    double p[3], u[3], tau, w = 1.0;
    launch(src, p, u, &tau, &rng);
    or_packet P;
    memset(&P, 0, sizeof P);
    int64_t nsteps = 0;
    for (;;) {
        or_eval E = scene_eval(S, p, T);
        if (E.dbox > 0.0) goto escape;         /* outside the volume of interest */
        double L;
        int traced = 0;                        /* counting only: a tracing move */
        if (E.dmin < S->delta) {
            int r = interface_step(S, &E, p, u, &rng, T);
            if (r == 2) goto escape;
            if (r == 1) goto next_step;
            L = S->delta;                      /* not approaching: forced step */
        } else {
            L = E.dmin - 0.5 * S->delta;       /* stop short: never cross by rounding */
            traced = 1;
            if (S->stepping == 1) L = fmax(L, segment_bound(S, &E, p, u, T));
        }
        {
            double mu_a = 0.0, mu_s = 0.0, g = 0.0;
            if (E.region >= 0) {
                mu_a = S->regions[E.region].mu_a;
                mu_s = S->regions[E.region].mu_s;
                g = S->regions[E.region].g;
            }
            double mu_t = mu_a + mu_s;
            if (mu_t > 0.0 && tau < mu_t * L) {
                double s = tau / mu_t;
                or_tally(G, p, u, s, w, flu, &T->pieces);
                p[0] = p[0] + s * u[0]; p[1] = p[1] + s * u[1]; p[2] = p[2] + s * u[2];
                /* interaction: absorption weight, HG scattering, roulette */
                double xi[4];
                or_draw4(&rng, xi);
                double wn = w * (mu_s / mu_t);
                P.A += fx(w - wn);
                w = wn;
                double ct = or_hg_cos(g, xi[0]);
                or_scatter_dir(u, ct, xi[1]);
                P.scatters += 1;
                if (w < OR_W_ROULETTE) {
                    if (xi[2] <= 1.0 / OR_ROULETTE_M) {
                        P.gain += fx(w * (OR_ROULETTE_M - 1.0));
                        w = w * OR_ROULETTE_M;
                    } else {
                        P.killed += fx(w);
                        goto done;
                    }
                }
                tau = -or_log(xi[3]);
            } else {
                or_tally(G, p, u, L, w, flu, &T->pieces);
                if (traced && S->stepping == 1) T->seg_moves += 1;
                tau = tau - mu_t * L;
                p[0] = p[0] + L * u[0]; p[1] = p[1] + L * u[1]; p[2] = p[2] + L * u[2];
            }
        }
    next_step:
        nsteps += 1;
        if (nsteps >= S->max_steps) { P.killed += fx(w); T->max_steps_hit += 1; goto done; }
        continue;
    escape:
        if (u[0] * src->dir[0] + u[1] * src->dir[1] + u[2] * src->dir[2] < 0.0) P.R += fx(w);
        else P.T += fx(w);
        goto done;
    }
done:
    P.steps = nsteps;
    T->R += P.R; T->T += P.T; T->A += P.A; T->killed += P.killed; T->gain += P.gain;
    T->scatters += P.scatters; T->steps += nsteps; T->packets += 1;
    if (rec) *rec = P;
}

/* ------------------------------------------------------------------------
 * Entry points (ctypes).
 * ---------------------------------------------------------------------- */

/* Propagate packets [id_begin, id_end).  flu (may be NULL) is accumulated
 * into, [nz][ny][nx] with x fastest; totals are accumulated into *tot;
 * rec (may be NULL) receives one record per packet.  Returns 0, or a
 * negative code for an invalid scene. */
int or_run(const or_scene *S, const or_source *src, const or_grid *G, uint64_t id_begin,
           uint64_t id_end, uint64_t seed, int64_t *flu, or_totals *tot, or_packet *rec)
{
    if (!S || !src || !G || !tot) return -1;
    if (!(S->delta > 0.0) || S->nregions < 0 || S->stepping < 0 || S->stepping > 1) return -2;
    for (int i = 0; i < S->nprims; ++i) {
        if (S->prims[i].kind < 0 || S->prims[i].kind > 4) return -8;
        if (S->prims[i].xform < 0 || S->prims[i].xform > S->nxforms) return -9;
    }
    for (int i = 0; i < S->nxforms; ++i)
        if (!(S->xforms[i].s > 0.0) || S->xforms[i].op < 0 || S->xforms[i].op > 4) return -10;
    for (int r = 0; r < S->nregions; ++r) {     /* postfix stack check */
        int sp = 0;
        const or_region *R = &S->regions[r];
        if (R->count <= 0 || R->begin < 0 || R->begin + R->count > S->nnodes) return -3;
        for (int i = 0; i < R->count; ++i) {
            const or_node *nd = &S->nodes[R->begin + i];
            if (nd->op == 0) {
                if (nd->prim < 0 || nd->prim >= S->nprims) return -4;
                if (++sp > OR_MAX_STACK) return -5;
            } else {
                if (sp < 2) return -6;
                --sp;
            }
        }
        if (sp != 1) return -7;
    }
    for (uint64_t id = id_begin; id < id_end; ++id)
        run_packet(S, src, G, id, seed, flu, tot, rec ? &rec[id - id_begin] : NULL);
    return 0;
}

/* Scene evaluation at one point, for tests. */
void or_scene_eval(const or_scene *S, const double p[3], double *dmin, int *istar, int *region,
                   double *dbox, double *dstar)
{
    or_totals T;
    memset(&T, 0, sizeof T);
    or_eval E = scene_eval(S, p, &T);
    *dmin = E.dmin; *istar = E.istar; *region = E.region; *dbox = E.dbox; *dstar = E.dstar;
}

/* The segment-stepping move from p along u (for tests); 0 if p is within
 * delta of a surface (no tracing step is taken there). */
double or_segment_step(const or_scene *S, const double p[3], const double u[3])
{
    or_eval E = scene_eval(S, p, NULL);
    if (!(E.dmin >= S->delta)) return 0.0;
    return fmax(E.dmin - 0.5 * S->delta, segment_bound(S, &E, p, u, NULL));
}

double or_region_sdf(const or_scene *S, int r, const double p[3])
{
    return region_sdf(S, r, p, NULL);
}

int or_surface_normal(const or_scene *S, int istar, const double p[3], double n[3])
{
    or_totals T;
    memset(&T, 0, sizeof T);
    return surface_normal(S, istar, p, S->delta, n, &T);
}

/* One interface event at p (within delta of a surface) with a given uniform
 * for the Fresnel choice; for tests of the reflect/refract geometry. */
int or_interface_once(const or_scene *S, double p[3], double u[3], uint64_t seed, uint64_t id)
{
    or_totals T;
    memset(&T, 0, sizeof T);
    or_rng rng;
    rng.key[0] = (uint32_t)seed; rng.key[1] = (uint32_t)(seed >> 32);
    rng.id_lo = (uint32_t)id; rng.id_hi = (uint32_t)(id >> 32);
    rng.event = 0u;
    or_eval E = scene_eval(S, p, &T);
    if (!(E.dmin < S->delta)) return -1;
    return interface_step(S, &E, p, u, &rng, &T);
}

void or_draw_uniforms(uint64_t seed, uint64_t id, uint32_t event0, int ncalls, double *out)
{
    or_rng rng;
    rng.key[0] = (uint32_t)seed; rng.key[1] = (uint32_t)(seed >> 32);
    rng.id_lo = (uint32_t)id; rng.id_hi = (uint32_t)(id >> 32);
    rng.event = event0;
    for (int i = 0; i < ncalls; ++i) or_draw4(&rng, out + 4 * i);
}

int or_sizeof(int which)
{
    switch (which) {
    case 0: return (int)sizeof(or_prim);
    case 1: return (int)sizeof(or_node);
    case 2: return (int)sizeof(or_region);
    case 3: return (int)sizeof(or_scene);
    case 4: return (int)sizeof(or_source);
    case 5: return (int)sizeof(or_grid);
    case 6: return (int)sizeof(or_totals);
    case 7: return (int)sizeof(or_packet);
    case 8: return (int)sizeof(or_xform);
    default: return -1;
    }
}
