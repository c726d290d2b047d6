// smcrt_k32.cu -- mixed-precision packet kernel.
//
// Sphere tracing, HG scattering, roulette and the DDA tally run in FP32
// (compiled with approximate FP32 division/sqrt).  The surface threshold
// delta32 is at least 64 FP32 ulps of the scene extent, the normal is a
// central difference with step h32 = 32 delta32.  FP64 is used only where
// the Fresnel/Snell cosines are ill-conditioned: near grazing (cos_i < 0.05)
// and within 0.01 of the critical angle's sin^2 = 1, where the point is re-localised and
// the normal and cosines recomputed in FP64 (Sec. 2.3 interface handling).
// Tallies are the same exact int64 fixed point as the FP64 path.
#include "smcrt_kernel.cuh"

namespace smcrt {

namespace {

constexpr float kGrazeCos = 0.05f;    // FP64 refinement below this |cos_i|
constexpr float kCritBand = 0.01f;    // ... and within this band of sin^2_t = 1
constexpr float kLandCos = 0.25f;     // line-preserving landing down to this |cos| of the new direction

// Where a packet lands after a Fresnel decision at the surface point q.  The
// decision is taken on the ray through q, so the packet continues on that
// ray: it moves along its new direction v until it is a (= 2 delta32) from
// the tangent plane, on the chosen side sd = +-1 along n.  A push along n
// instead would shift the ray sideways by a sin(theta) at every event; at
// concentric spheres that shift accumulates in r sin(theta) (the quantity
// Snell's law conserves between them), and a packet near the critical angle
// of a glass shell drifts into total internal reflection at both walls and
// stays there.  Directions within kLandCos of the plane move a / kLandCos
// along v and the rest of the distance along n, so no landing moves more than
// 4 a.  The path of the landing is charged afterwards (cross32).
__device__ __forceinline__ void land32(float qx, float qy, float qz, float vx, float vy, float vz, float nx,
                                       float ny, float nz, float a, float sd, float &px, float &py, float &pz)
{
    const float c = fabsf(vx * nx + vy * ny + vz * nz);
    const float s = __fdividef(a, fmaxf(c, kLandCos));
    const float rest = sd * fmaxf(a - s * c, 0.f);
    px = qx + s * vx + rest * nx;
    py = qy + s * vy + rest * ny;
    pz = qz + s * vz + rest * nz;
}

// The interface shortcut in FP32.  A packet reaches a surface when it is
// within delta32 of it, is placed on the surface point q and lands about
// 2 delta32 beyond it; the FP64 reference makes the same moves at its delta
// (30 times smaller for the layered slab), where the path skipped is
// negligible.  At delta32 it is not: the approach from the arrival point p to
// the surface (|d| / |cos| along the ray, |cos| floored like the landing's)
// and the landing q -> P would pass through medium without attenuation or
// fluence, which measurably raised the slab's transmission (by 0.15 % of T
// at 1e7 packets, paired against the FP64 kernel; the bias grows linearly
// with the threshold in the oracle).  So the mixed kernel treats that path
// as travelled: when the optical depth left runs out on the approach, the
// packet interacts on the near side (at its arrival point) instead of
// crossing; otherwise the crossing (cross32) charges the optical depth of
// both pieces, each with its own region's mu_t (the packet interacts at once
// if the landing exhausts it), and their length is tallied with the next
// move: its segment is extended back from the landing point by that length
// (the pieces are a few delta32 long, far below a voxel, and reach at most
// one voxel boundary beyond the surface).  Depositing them separately added
// atomics to the voxel where a pencil beam enters, which every packet's
// first tally piece already hits, and serialised there (10 % of the slab's
// time).

// Length of the approach from a point |dstar| from the surface along a ray
// with |u.n| = |cdot| (floored at kLandCos, as the landing is).  Explicitly
// rounded operations here and in cross32's charge: no multiply-add is
// contracted, so every register-budget instantiation computes the same bits.
__device__ __forceinline__ float approach_len32(float dstar, float cdot)
{
    return __fdividef(fabsf(dstar), fmaxf(fabsf(cdot), kLandCos));
}

__device__ __forceinline__ float hg_cos32(float g, float xi)
{
    float c;
    if (fabsf(g) < 1e-6f) {
        c = 2.f * xi - 1.f;
    } else {
        const float t = __fdividef(__fmaf_rn(-g, g, 1.f), __fmaf_rn(2.f * g, xi, 1.f - g));
        c = __fdividef(__fmaf_rn(-t, t, __fmaf_rn(g, g, 1.f)), 2.f * g);
    }
    return fminf(fmaxf(c, -1.f), 1.f);
}

__device__ __forceinline__ void normalise32(float &x, float &y, float &z)
{
    const float il = rsqrtf(__fmaf_rn(x, x, __fmaf_rn(y, y, z * z)));
    x *= il; y *= il; z *= il;
}

__device__ __forceinline__ void scatter32(float &ux, float &uy, float &uz, float ct, float xi_phi)
{
    const float st = sqrtf(fmaxf((1.f - ct) * (1.f + ct), 0.f));
    float sp, cp;
    __sincosf(6.2831853f * xi_phi, &sp, &cp);
    float b1[3], b2[3];
    onb32(ux, uy, uz, b1, b2);
    const float a1 = st * cp, a2 = st * sp;
    float vx = __fmaf_rn(a1, b1[0], __fmaf_rn(a2, b2[0], ct * ux));
    float vy = __fmaf_rn(a1, b1[1], __fmaf_rn(a2, b2[1], ct * uy));
    float vz = __fmaf_rn(a1, b1[2], __fmaf_rn(a2, b2[2], ct * uz));
    normalise32(vx, vy, vz);
    ux = vx; uy = vy; uz = vz;
}

__device__ __forceinline__ float region_n32(const DevScene &S, int r)
{
    return r < 0 ? S.ambient_n32 : (*(S.reg32 + 2 * r + 1)).x;
}

__device__ __forceinline__ double region_n64(const DevScene &S, int r)
{
    return r < 0 ? S.ambient_n : __ldg(S.reg64 + 8 * r + 3);
}

// FP64 interface localisation for a crossing whose normal must be accurate:
// four FP64 evaluations of the surface's own SDF program -- d(p), then
// forward differences d(p + delta e_a) for the normal (truncation error
// delta * curvature) -- a Newton step onto the surface along that normal,
// and the Fresnel decision (uniform xi), reflected or refracted direction
// and landing (land32), all in FP64.  A ray tangent in FP64 does not cross:
// it stays on the near side with its direction unchanged.
template <bool G>
__device__ __noinline__ void refine64(const DevScene &S, int istar, int rnear, int rfar, float sg32, uint32_t xiw,
                                      float &px, float &py, float &pz, float &ux, float &uy, float &uz,
                                      float nx32, float ny32, float nz32)
{
    const double x = px, y = py, z = pz;
    const double h = S.delta;
    const double d0 = surface64<G>(S, istar, x, y, z);
    const double gx = surface64<G>(S, istar, x + h, y, z) - d0;
    const double gy = surface64<G>(S, istar, x, y + h, z) - d0;
    const double gz = surface64<G>(S, istar, x, y, z + h) - d0;
    double nx = nx32, ny = ny32, nz = nz32;
    const double l2 = gx * gx + gy * gy + gz * gz;
    if (l2 > 0.0) {
        const double il = 1.0 / sqrt(l2);
        nx = gx * il; ny = gy * il; nz = gz * il;
    }
    const double qx = x - d0 * nx, qy = y - d0 * ny, qz = z - d0 * nz;
    double vx = ux, vy = uy, vz = uz;
    const double c = vx * nx + vy * ny + vz * nz;
    const double sg = c > 0.0 ? 1.0 : -1.0;
    const double e = 2.0 * (double)S.delta32 * sg;
    if (sg != (double)sg32) {   // tangent in FP64: no crossing, stay on the near side
        const double en = -2.0 * (double)S.delta32 * (double)sg32;
        px = (float)(qx + en * nx);
        py = (float)(qy + en * ny);
        pz = (float)(qz + en * nz);
        return;
    }
    const double n1 = region_n64(S, rnear), n2 = region_n64(S, rfar);
    const double ci = fabs(c);
    const double eta = n1 / n2;
    const double st2 = eta * eta * ((1.0 - ci) * (1.0 + ci));
    double R = 1.0, ct = 0.0;
    if (st2 < 1.0) {
        ct = sqrt(1.0 - st2);
        const double rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
        const double rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
        R = 0.5 * (rs * rs + rp * rp);
    }
    double sx;
    if (u01_64(xiw) <= R) {
        const double c2 = 2.0 * c;
        vx -= c2 * nx; vy -= c2 * ny; vz -= c2 * nz;
        sx = -e;
    } else {
        const double k = sg * (eta * ci - ct);
        vx = eta * vx - k * nx; vy = eta * vy - k * ny; vz = eta * vz - k * nz;
        sx = e;
    }
    const double il = 1.0 / sqrt(vx * vx + vy * vy + vz * vz);
    vx *= il; vy *= il; vz *= il;
    ux = (float)vx; uy = (float)vy; uz = (float)vz;
    // line-preserving landing (land32), in FP64
    const double a = fabs(e), cv = fabs(vx * nx + vy * ny + vz * nz);
    const double s = a / fmax(cv, (double)kLandCos);
    const double rest = (sx > 0.0 ? 1.0 : -1.0) * fmax(a - s * cv, 0.0);
    px = (float)(qx + s * vx + rest * nx);
    py = (float)(qy + s * vy + rest * ny);
    pz = (float)(qz + s * vz + rest * nz);
}

// A crossing of a surface (Sec. 2.3), out of line: Fresnel reflection or
// Snell refraction when the refractive index changes (FP32 on planar faces,
// refine64 where the cosines are ill-conditioned or the normal is noisy),
// or a straight crossing when it does not (matched); the line-preserving
// landing; and the charge of the interface shortcut: the optical depth of
// the approach (arrival point a to the surface) and of the landing (surface
// point q to the landing point P), each with its own region's mu_t; their
// length is returned for the next move's tally.  The new state is returned
// by value, so the loop's own variables stay in registers.
struct Crossed {
    float px, py, pz, ux, uy, uz, tau;
    float pend;      // the shortcut's length, tallied with the next move
    int refined;
};

template <bool G>
static __device__ __noinline__ Crossed cross32(const DevScene &S, float ux, float uy, float uz, float qx, float qy,
                                               float qz, float nx, float ny, float nz, float tau, float dstar,
                                               float cdot, int istar, int rnear, int rfar, uint32_t xiw, bool matched)
{
    const float sg = cdot > 0.f ? 1.f : -1.f;
    const float a = 2.f * S.delta32;
    Crossed o;
    o.refined = 0;
    o.ux = ux; o.uy = uy; o.uz = uz;
    if (matched) {                                  // same index: cross on the ray
        land32(qx, qy, qz, ux, uy, uz, nx, ny, nz, a, sg, o.px, o.py, o.pz);
    } else {
        const float n1 = region_n32(S, rnear), n2 = region_n32(S, rfar);
        const float ci = fabsf(cdot);
        const float eta = n1 / n2;
        const float st2 = eta * eta * ((1.f - ci) * (1.f + ci));
        const int zeros = (nx == 0.f) + (ny == 0.f) + (nz == 0.f);
        const bool curved_noisy = !S.analytic_nrm && zeros != 2;   // probe normals on curved faces
        if (ci < kGrazeCos || fabsf(st2 - 1.f) < kCritBand || curved_noisy) {
            o.refined = 1;
            o.px = qx; o.py = qy; o.pz = qz;
            refine64<G>(S, istar, rnear, rfar, sg, xiw, o.px, o.py, o.pz, o.ux, o.uy, o.uz, nx, ny, nz);
        } else {                                    // planar face: the FP32 normal is exact
            float R = 1.f, ct = 0.f;
            if (st2 < 1.f) {
                ct = sqrtf(1.f - st2);
                const float rs = __fdividef(n1 * ci - n2 * ct, n1 * ci + n2 * ct);
                const float rp = __fdividef(n1 * ct - n2 * ci, n1 * ct + n2 * ci);
                R = 0.5f * (rs * rs + rp * rp);
            }
            float sd;
            if (u01_32(xiw) <= R) {
                const float c2 = 2.f * cdot;
                o.ux -= c2 * nx; o.uy -= c2 * ny; o.uz -= c2 * nz;
                sd = -sg;
            } else {
                const float k = sg * (eta * ci - ct);
                o.ux = eta * o.ux - k * nx; o.uy = eta * o.uy - k * ny; o.uz = eta * o.uz - k * nz;
                sd = sg;
            }
            normalise32(o.ux, o.uy, o.uz);
            land32(qx, qy, qz, o.ux, o.uy, o.uz, nx, ny, nz, a, sd, o.px, o.py, o.pz);
        }
    }
    // the side the packet landed on: beyond the surface (refracted, matched)
    // or back on the near side (reflected, or tangent in FP64)
    const bool far = __fmul_rn(__fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(o.px, qx), nx),
                                                   __fmul_rn(__fsub_rn(o.py, qy), ny)),
                                         __fmul_rn(__fsub_rn(o.pz, qz), nz)),
                               sg) > 0.f;
    const int rside = far ? rfar : rnear;
    // the shortcut's charge (explicitly rounded: no contraction)
    const float lnear = approach_len32(dstar, cdot);
    const float dx = __fsub_rn(o.px, qx), dy = __fsub_rn(o.py, qy), dz = __fsub_rn(o.pz, qz);
    const float lfar = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
    const float mn = rnear >= 0 ? (*(S.reg32 + 2 * rnear)).x : 0.f;
    const float mf = rside >= 0 ? (*(S.reg32 + 2 * rside)).x : 0.f;
    o.tau = fmaxf(__fsub_rn(__fsub_rn(tau, __fmul_rn(mn, lnear)), __fmul_rn(mf, lfar)), 0.f);
    o.pend = __fadd_rn(lnear, lfar);
    return o;
}

// Photon release (Sec. 2.1), out of line: position and direction from the
// source (pencil, disc, square, isotropic point) and the first optical depth
// (Eq. 1), from one Philox call's words.
struct Launched {
    float px, py, pz, ux, uy, uz, tau;
};

static __device__ __noinline__ Launched launch32(const DevScene &S, uint4 r)
{
    Launched o;
    const float x0 = u01_32(r.x), x1 = u01_32(r.y);
    o.px = S.src_pos32[0]; o.py = S.src_pos32[1]; o.pz = S.src_pos32[2];
    o.ux = S.src_dir32[0]; o.uy = S.src_dir32[1]; o.uz = S.src_dir32[2];
    if (S.src_kind == 1 || S.src_kind == 2) {
        float c1, c2;
        if (S.src_kind == 1) {
            const float rho = S.src_radius32 * sqrtf(x0);
            float sn, cs;
            __sincosf(6.2831853f * x1, &sn, &cs);
            c1 = rho * cs;
            c2 = rho * sn;
        } else {
            c1 = S.src_radius32 * (2.f * x0 - 1.f);
            c2 = S.src_radius32 * (2.f * x1 - 1.f);
        }
        o.px += c1 * S.src_b132[0] + c2 * S.src_b232[0];
        o.py += c1 * S.src_b132[1] + c2 * S.src_b232[1];
        o.pz += c1 * S.src_b132[2] + c2 * S.src_b232[2];
    } else if (S.src_kind == 3) {
        const float ct = 2.f * x0 - 1.f;
        const float st = sqrtf(fmaxf((1.f - ct) * (1.f + ct), 0.f));
        float sn, cs;
        __sincosf(6.2831853f * x1, &sn, &cs);
        o.ux = st * cs; o.uy = st * sn; o.uz = ct;
    }
    o.tau = -__logf(u01_32(r.w));
    return o;
}

// Per-warp shared state: the staged scene and the warp's tally slots.
// Scene-table staging (a launch option the autotuner tries): the warp copies
// the instruction stream, primitive kinds, FP32 primitive and region tables
// and region ranges of its job into shared memory when they fit here.
constexpr int kStageBytes = 4096;
// One job as a warp holds it: its scene, its tally accumulator, its constants.
struct JobSlot {
    DevScene S;
    WarpAcc acc;
    JobConst jc;
    int rdone;               // served rounds: this job's parked list is used up for the round
    int idone;               // ... and its ids are all claimed
};
struct WarpShared {          // plan launches: one job at a time, tables optionally staged
    JobSlot slot;
    __align__(16) unsigned char tab[kStageBytes];
};
// Served rounds: two jobs at a time.  A warp's lanes carry packets of either
// job; the warp feeds new packets from one slot and, when that job runs out
// of ids, stages the next job with work into the other slot as soon as no
// lane holds a packet there -- lanes refill from the next job instead of
// the warp draining each job it visits.  Tables are read from global memory.
constexpr int kMultiSlots = 2;
struct WarpSharedMulti {
    JobSlot slot[kMultiSlots];
};

__device__ __forceinline__ void stage_tables(WarpShared *ws, int lane)
{
    DevScene &SS = ws->slot.S;
    const int ni = SS.ninstr, np = SS.nprims, nr = SS.nregions;
    const int w_ins = 4 * ni, w_kind = np, w_p32 = 8 * np, w_r32 = 8 * nr, w_rr = 2 * nr;   // 4-byte words
    const int o1 = 0, o2 = o1 + ((w_ins + 3) & ~3), o3 = o2 + ((w_kind + 3) & ~3), o4 = o3 + ((w_p32 + 3) & ~3),
              o5 = o4 + ((w_r32 + 3) & ~3), end = o5 + w_rr;
    if (end * 4 > kStageBytes) return;
    uint32_t *T = reinterpret_cast<uint32_t *>(ws->tab);
    const uint32_t *a = reinterpret_cast<const uint32_t *>(SS.instr);
    for (int k = lane; k < w_ins; k += 32) T[o1 + k] = a[k];
    a = reinterpret_cast<const uint32_t *>(SS.pkind);
    for (int k = lane; k < w_kind; k += 32) T[o2 + k] = a[k];
    a = reinterpret_cast<const uint32_t *>(SS.p32);
    for (int k = lane; k < w_p32; k += 32) T[o3 + k] = a[k];
    a = reinterpret_cast<const uint32_t *>(SS.reg32);
    for (int k = lane; k < w_r32; k += 32) T[o4 + k] = a[k];
    a = reinterpret_cast<const uint32_t *>(SS.rrange);
    for (int k = lane; k < w_rr; k += 32) T[o5 + k] = a[k];
    __syncwarp();
    if (lane == 0) {
        SS.instr = reinterpret_cast<const Instr *>(T + o1);
        SS.pkind = reinterpret_cast<const int32_t *>(T + o2);
        SS.p32 = reinterpret_cast<const float4 *>(T + o3);
        SS.reg32 = reinterpret_cast<const float4 *>(T + o4);
        SS.rrange = reinterpret_cast<const int2 *>(T + o5);
    }
    __syncwarp();
}

// Served rounds: the first job of jobs[start, ...) (cyclically) with work
// for a warp -- new ids or parked packets -- other than `exclude`; -1 if
// none.  The lanes look at 32 entries at a time.  A descriptor without
// scene or totals, or a scene that needs the general-shape kernel in the
// plain one, is flagged in the launch's and the job's status words and
// skipped from then on.  Warp-collective; the result is warp-uniform.
template <bool G>
__device__ int multi_find(JobWork *jobs, int njobs, int start, int exclude, unsigned long long &skip, int *status,
                          int lane)
{
    for (int b = 0; b < njobs; b += 32) {
        const int k = b + lane;
        int j = start + k;
        if (j >= njobs) j -= njobs;
        bool work = false, bad = false;
        if (k < njobs && j != exclude && !((skip >> j) & 1ull)) {
            JobWork *J = jobs + j;
            const unsigned long long nxt = *(volatile unsigned long long *)&J->next;
            bool parked = false;
            if (J->defer != nullptr) {
                const int in = J->defer_in & 1;
                parked = min(*(volatile unsigned *)&J->defer->count[in], J->defer->cap) >
                         *(volatile unsigned *)&J->defer->cursor[in];
            }
            // a cancelled job's ids are no work (its parked packets still are)
            const bool fresh = nxt < J->end && *(volatile int32_t *)&J->cancelled == 0;
            if (fresh || parked) {
                if (J->scene == nullptr || J->totals == nullptr || (!G && J->scene->general)) {
                    bad = true;
                    atomicOr(status, kStatusBadJob);
                    if (J->jstat != nullptr) atomicOr(J->jstat, kStatusBadJob);
                } else {
                    work = true;
                }
            }
        }
        // bad jobs are skipped by this warp from now on (warp-uniform mask)
        for (unsigned m = __ballot_sync(SMCRT_FULL, bad); m != 0u; m &= m - 1u) {
            int jb = start + b + (__ffs(m) - 1);
            if (jb >= njobs) jb -= njobs;
            skip |= 1ull << jb;
        }
        const unsigned hit = __ballot_sync(SMCRT_FULL, work);
        if (hit != 0u) {
            const int j0 = start + b + (__ffs(hit) - 1);
            return j0 >= njobs ? j0 - njobs : j0;
        }
    }
    return -1;
}

// Served rounds: stage job J into a slot (scene header copied from global
// memory, constants, zeroed accumulator).  Warp-collective.
__device__ __forceinline__ void multi_stage(JobSlot *sl, JobWork *J, int lane)
{
    const long long *s8 = reinterpret_cast<const long long *>(J->scene);
    long long *d8 = reinterpret_cast<long long *>(&sl->S);
    for (int i = lane; i < (int)(sizeof(DevScene) / 8); i += 32) d8[i] = s8[i];
    if (lane == 0) {
        jobconst_fill(&sl->jc, J);
        sl->rdone = 0;
        sl->idone = 0;
    }
    wacc_clear(&sl->acc, lane);
    __syncwarp();
}

// One warp works through packet ids of job J until the job's cursor passes
// its end.  Iteration structure (all lanes execute every stage; a lane's
// phase only selects operands or predicates a short update):
//   1 refill dead lanes (one atomicAdd per warp),
//   2 one FP32 scene evaluation at the lane's phase point,
//   3 classify: escape / start interface / move / normal bookkeeping /
//     far-near regions / Fresnel,
//   4 the track-length tally of this iteration's move (one call site),
//   5 one Philox call serving launch, interaction and Fresnel draws,
//   6 the consumers: release a packet, scatter (HG + roulette), Fresnel.
//
// MULTI = false (plan launches): one job, jobs[0], in slots[0].  MULTI =
// true (served rounds): the warp works through the table jobs[0, njobs)
// starting at `first`, holding up to two jobs in slots[0..1] (see
// WarpSharedMulti); each lane's packet belongs to the job of its slot js.
template <bool G, bool MULTI>
__device__ bool run_job_mixed(JobSlot *slots, JobWork *jobs, int njobs, int first, int *status, int lane)
{
    const DevScene &S0 = slots[0].S;
    const float delta0 = S0.delta32, hstep0 = S0.h32;
    const volatile JobConst *const jc0 = &slots[0].jc;
    JobWork *const J = jobs;
    int js = 0;                          // the lane's job slot
    // served rounds (warp-uniform): the slot fed with new packets, the job of
    // each slot (-1: none), the next table entry to look at, and the jobs
    // this warp found unusable (a descriptor without scene or totals)
    int feed = 0, sj0 = -1, sj1 = -1, scan = first;
    unsigned long long skip = 0ull;
    // served rounds: no job had work left when this warp last looked.  Its
    // packets then park sooner (after the round's drain budget instead of the
    // full one), so a round is not held open by a few long-lived packets
    // while the rest of the GPU idles; they resume next round among new work.
    bool drained = false;
    // served rounds: a search found no job with work; within a round none
    // appears later (ids only get claimed, parked lists only get resumed),
    // so idle lanes retire without asking again
    bool nomore = false;
    if (MULTI) {
        const int nj = multi_find<G>(jobs, njobs, scan, -1, skip, status, lane);
        if (nj < 0) return false;
        multi_stage(slots, jobs + nj, lane);
        sj0 = nj;
        scan = nj + 1 < njobs ? nj + 1 : 0;
    }

    bool alive = false, retired = false;
    float px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0, w = 0, tau = 0;
    float qx = 0, qy = 0, qz = 0;        // FAR / NEAR: surface point; TRACE: crawl anchor
    // Crawl: a packet within delta32 of a surface that it is leaving takes
    // forced steps of delta32 along u.  Adding the same small step to an
    // FP32 position again and again rounds the same way every time, and over
    // a few hundred steps (a near-tangent departure from a concave wall) the
    // bias carries the packet across the wall unnoticed.  So the crawl keeps
    // an anchor q and its length cs along u, and places the packet at
    // q + cs u (one rounding, whatever the step count).  cs < 0: no crawl.
    float cs = -1.f;
    float pend = 0.f;                    // track length of a crossing's shortcut, tallied with the next move
    float nx = 0, ny = 0, nz = 0, cdot = 0, fplus = 0, dstar = 0;
    int phase = kTrace, sub = 0, istar = -1, reg = -1, rfar = -1;
    int nsteps = 0;
    unsigned pscat = 0, npieces = 0;
    long long pA = 0, pG = 0;
    uint32_t id_lo = 0, id_hi = 0, event = 0;
    uint32_t t_acq = 0;
    bool timed_out = false;              // the launch's time limit stopped the refills

    for (;;) {
        // ---- 1. refill: this job's parked packets first, then new ids
        if (MULTI) {
            unsigned need = __ballot_sync(SMCRT_FULL, !alive && !retired);
            if (nomore) {
                if (!alive) retired = true;
                need = 0u;
            }
            for (int pass = 0; need != 0u && pass < 4; ++pass) {
                JobSlot *const sf = slots + feed;
                JobWork *const Jf = jobs + (feed ? sj1 : sj0);
                JobDefer *const dfr = (JobDefer *)sf->jc.dfr;
                if (dfr != nullptr && !*(volatile int *)&sf->rdone) {   // the feed job's parked packets
                    const int din = sf->jc.din;
                    const int leader = __ffs(need) - 1;
                    unsigned base = 0u, avail = 0u;
                    if (lane == leader) {
                        avail = min(*(volatile unsigned *)&dfr->count[din], dfr->cap);
                        base = atomicAdd(&dfr->cursor[din], (unsigned)__popc(need));
                    }
                    base = __shfl_sync(SMCRT_FULL, base, leader);
                    avail = __shfl_sync(SMCRT_FULL, avail, leader);
                    // the list only shrinks during a round (new parks go to the
                    // other one): once the cursor passes its count, stop asking
                    if (base + (unsigned)__popc(need) >= avail) {
                        if (lane == 0) *(volatile int *)&sf->rdone = 1;
                        __syncwarp();
                    }
                    if (!alive && !retired) {
                        const unsigned k = base + (unsigned)__popc(need & ((1u << lane) - 1u));
                        if (k < avail) {
                            const DeferState &d = dfr->buf[din][k];
                            px = (float)d.p[0]; py = (float)d.p[1]; pz = (float)d.p[2];
                            ux = (float)d.u[0]; uy = (float)d.u[1]; uz = (float)d.u[2];
                            w = (float)d.w; tau = (float)d.tau;
                            pA = d.pA; pG = d.pG;
                            id_lo = d.id_lo; id_hi = d.id_hi; event = d.event;
                            nsteps = (int)d.nsteps; pscat = d.pscat;
                            phase = kTrace;
                            cs = __uint_as_float(d.pad[0]);
                            pend = __uint_as_float(d.pad[1]);
                            if (cs >= 0.f) {
                                qx = px; qy = py; qz = pz;
                                px = __fmaf_rn(cs, ux, qx); py = __fmaf_rn(cs, uy, qy); pz = __fmaf_rn(cs, uz, qz);
                            }
                            t_acq = (uint32_t)clock();
                            alive = true;
                            js = feed;
                        }
                    }
                    need = __ballot_sync(SMCRT_FULL, !alive && !retired);
                }
                if (need != 0u && !*(volatile int *)&sf->idone) {   // the feed job's new ids
                    const int leader = __ffs(need) - 1;
                    unsigned long long base = 0;
                    if (lane == leader)
                        base = *(volatile int32_t *)&Jf->cancelled
                                   ? ~0ull
                                   : atomicAdd(&Jf->next, (unsigned long long)__popc(need));
                    base = __shfl_sync(SMCRT_FULL, base, leader);
                    if (base == ~0ull || base + (unsigned long long)__popc(need) >= sf->jc.end) {
                        if (lane == 0) *(volatile int *)&sf->idone = 1;
                        __syncwarp();
                    }
                    if (!alive && !retired) {
                        const unsigned long long id =
                            base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                        if (base != ~0ull && id < sf->jc.end) {
                            id_lo = (uint32_t)id;
                            id_hi = (uint32_t)(id >> 32);
                            event = 0u;
                            phase = kLaunch;
                            t_acq = (uint32_t)clock();
                            alive = true;
                            js = feed;
                        }
                    }
                    need = __ballot_sync(SMCRT_FULL, !alive && !retired);
                }
                if (need == 0u) break;
                // the feed job has no work left for these lanes: feed the
                // other slot with the next job that has some, once no lane
                // holds a packet there
                const int o = 1 - feed;
                if (__ballot_sync(SMCRT_FULL, alive && js == o) != 0u) break;
                const int oj = o ? sj1 : sj0;
                if (oj >= 0) wacc_flush(&slots[o].acc, jobs[oj].totals, lane);
                const int nj = multi_find<G>(jobs, njobs, scan, feed ? sj1 : sj0, skip, status, lane);
                if (o) sj1 = -1; else sj0 = -1;
                if (nj < 0) {                  // no job has work left: idle lanes retire
                    if (!alive) retired = true;
                    drained = true;
                    nomore = true;
                    break;
                }
                multi_stage(slots + o, jobs + nj, lane);
                if (o) sj1 = nj; else sj0 = nj;
                scan = nj + 1 < njobs ? nj + 1 : 0;
                feed = o;
            }
            if (__all_sync(SMCRT_FULL, retired)) break;
        } else {
            // plan launches: new ids only (parking belongs to served rounds,
            // which run the multi-job kernel; leaving it out of this one
            // keeps its loop smaller)
            const unsigned need = __ballot_sync(SMCRT_FULL, !alive && !retired);
            const volatile JobConst *const jc = jc0;
            const bool want = !alive && !retired;
            if (need) {
                const int leader = __ffs(need) - 1;
                unsigned long long base = 0;
                if (lane == leader) {
                    if (*(volatile int32_t *)&J->cancelled) base = ~0ull;
                    else if (SMCRT_RARE(past_deadline(jc))) base = ~0ull - 1u;   // device time limit
                    else base = atomicAdd(&J->next, (unsigned long long)__popc(need));
                }
                base = __shfl_sync(SMCRT_FULL, base, leader);
                timed_out = timed_out || base == ~0ull - 1u;
                if (want) {
                    const unsigned long long id = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                    if (base >= ~0ull - 1u || id >= jc->end) {
                        retired = true;
                    } else {
                        id_lo = (uint32_t)id;
                        id_hi = (uint32_t)(id >> 32);
                        event = 0u;
                        phase = kLaunch;
                        t_acq = (uint32_t)clock();
                        alive = true;
                    }
                }
            }
            if (__all_sync(SMCRT_FULL, retired)) break;
        }

        // the lane's job: its scene, constants and accumulator (one job in a
        // plan launch; compile-time slot 0 there)
        const DevScene &S = MULTI ? slots[js].S : S0;
        const float delta = MULTI ? S.delta32 : delta0, hstep = MULTI ? S.h32 : hstep0;
        const volatile JobConst *const jc = MULTI ? &slots[js].jc : jc0;
        WarpAcc *const wa = MULTI ? &slots[js].acc : &slots[0].acc;

        // ---- 2. the scene evaluation of this iteration
        const float sg = cdot > 0.f ? 1.f : -1.f;
        float ex = px, ey = py, ez = pz;
        int sel = -2;
        if (G && SMCRT_RARE(phase == kNrm)) {   // probe normals: general instantiation only
            const float hh = (sub & 1) ? -hstep : hstep;
            const int a = sub >> 1;
            if (a == 0) ex = px + hh; else if (a == 1) ey = py + hh; else ez = pz + hh;
            sel = istar;
        } else if (SMCRT_RARE(phase == kFar || phase == kNear)) {
            const float e = (phase == kFar ? 2.f : -2.f) * delta * sg;
            ex = qx + e * nx; ey = qy + e * ny; ez = qz + e * nz;
        }
        const Eval32 E = scene_eval32<G>(S, ex, ey, ez, sel);
        if (MULTI) {                           // evaluations counted per job slot
            for (int k = 0; k < kMultiSlots; ++k) {
                const unsigned ev = __ballot_sync(SMCRT_FULL, alive && phase != kLaunch && js == k);
                if (lane == 0 && ev != 0u) wadd(&slots[k].acc, kEvals, __popc(ev));
            }
        } else {
            const unsigned ev = __ballot_sync(SMCRT_FULL, alive && phase != kLaunch);
            if (lane == 0) wadd(wa, kEvals, __popc(ev));
        }

        // ---- 3. classify
        bool move = false, fresnel = false, iter_done = false, nrm_ready = false;
        bool seg_step = false;                 // a tracing move that segment stepping may lengthen
        bool crawl = false;                    // a forced step away from a surface
        bool fin = false;                      // the packet ends this iteration
        bool near_hit = false;                 // interacts before reaching the surface
        bool matched = false;                  // a crossing without an index change
        long long fin_R = 0, fin_T = 0, fin_K = 0;
        float L = 0.f;
        int rnear = -1;
        if (alive) {
            if (phase == kTrace) {
                if (SMCRT_RARE(E.dbox > 0.f)) {
                    {                                          // leaves the volume: R or T
                        const long long v = fx32(w);
                        if (ux * S.src_dir32[0] + uy * S.src_dir32[1] + uz * S.src_dir32[2] < 0.f) fin_R = v; else fin_T = v;
                        fin = true;
                        alive = false;
                    }
                } else {
                    reg = E.region;
                    if (SMCRT_RARE(E.dmin < delta)) {
                        istar = E.istar;
                        dstar = E.dstar;
                        if (!G || S.analytic_nrm) {        // gradient of a short program, now
                            grad_surface32(S, istar, px, py, pz, nx, ny, nz);
                            nrm_ready = true;
                        } else {                           // six probes in the next iterations
                            phase = kNrm;
                            sub = 0;
                        }
                    } else {
                        L = E.dmin - 0.5f * delta;
                        move = true;
                        seg_step = S.stepping == SMCRT_STEP_SEGMENT;
                    }
                }
            } else if (G && SMCRT_RARE(phase == kNrm)) {
                const float f = E.dsel;
                if ((sub & 1) == 0) {
                    fplus = f;
                } else {
                    const float gg = fplus - f;
                    const int a = sub >> 1;
                    if (a == 0) nx = gg; else if (a == 1) ny = gg; else nz = gg;
                }
                if (++sub >= 6) nrm_ready = true;
            } else if (phase == kFar) {
                rfar = E.region;
                phase = kNear;
            } else if (phase == kNear) {
                rnear = E.region;
                // matched indices cross on the ray, as a Fresnel landing does
                // (cross32).  A push along n alone never advances along u, and
                // where the normal turns between the two sides (a smooth
                // union's crease) a packet moving along the wall was pushed
                // back and forth across it until the step cap.
                matched = region_n32(S, rnear) == region_n32(S, rfar);
                fresnel = true;
            }
        }

        // ---- 3b. a normal is ready (analytic, or after the sixth probe)
        if (SMCRT_RARE(nrm_ready)) {
            const float l2 = nx * nx + ny * ny + nz * nz;
            bool approaching = false;
            if (l2 > 0.f) {
                const float il = rsqrtf(l2);
                nx *= il; ny *= il; nz *= il;
                cdot = ux * nx + uy * ny + uz * nz;
                approaching = (cdot > 0.f && dstar < 0.f) || (cdot < 0.f && dstar >= 0.f);
            }
            if (!approaching) {
                L = delta;                          // forced step along u
                move = true;
                crawl = true;
            } else if (istar < 0) {                 // leaves the volume: R or T
                const long long v = fx32(w);
                if (ux * S.src_dir32[0] + uy * S.src_dir32[1] + uz * S.src_dir32[2] < 0.f) fin_R = v; else fin_T = v;
                fin = true;
                alive = false;
            } else if (tau < __fmul_rn(reg >= 0 ? (*(S.reg32 + 2 * reg)).x : 0.f, approach_len32(dstar, cdot))) {
                // the optical depth runs out before the surface: interact here,
                // at the arrival point (inside this region by evaluation).  Moving
                // on by tau / mu_t could round the point across the surface, and
                // a packet scattered just inside a clear glass wall can take a
                // direction that total internal reflection traps at both walls.
                near_hit = true;
            } else {
                wadd(wa, kIntf, 1);
                qx = px - dstar * nx; qy = py - dstar * ny; qz = pz - dstar * nz;
                cs = -1.f;
                phase = kFar;
            }
        }

        // ---- 4. move: interaction point or sphere-trace step, one tally site
        bool interact = near_hit;
        if (SMCRT_RARE(near_hit)) {
            cs = -1.f;
            phase = kTrace;                        // also after the sixth probe
            iter_done = true;
        }
        if (move) {
            float mu_t = 0.f, imu_t = 0.f;
            if (reg >= 0) {
                const float4 RG = (*(S.reg32 + 2 * reg));
                mu_t = RG.x; imu_t = RG.y;
            }
            interact = mu_t > 0.f && tau < mu_t * L;
            if (SMCRT_RARE(seg_step && !interact)) {           // segment stepping: a longer move along u
                L = fmaxf(L, segment_bound32<G>(S, E.dsoft, E.dbox, px, py, pz, ux, uy, uz));
                interact = mu_t > 0.f && tau < mu_t * L;
            }
            const float seg = interact ? tau * imu_t : L;
            long long *const flu = (long long *)jc->flu;
            // the segment starts back at the surface after a crossing (pend)
            if (flu) tally32(S, flu, __fmaf_rn(-pend, ux, px), __fmaf_rn(-pend, uy, py), __fmaf_rn(-pend, uz, pz), ux,
                             uy, uz, seg + pend, w, &npieces);
            pend = 0.f;
            if (SMCRT_RARE(crawl)) {
                if (cs < 0.f) { qx = px; qy = py; qz = pz; cs = 0.f; }
                cs += seg;
                px = __fmaf_rn(cs, ux, qx); py = __fmaf_rn(cs, uy, qy); pz = __fmaf_rn(cs, uz, qz);
            } else {
                px = __fmaf_rn(seg, ux, px); py = __fmaf_rn(seg, uy, py); pz = __fmaf_rn(seg, uz, pz);
                cs = -1.f;
            }
            tau = __fmaf_rn(-mu_t, seg, tau);
            phase = kTrace;
            iter_done = true;
        }

        // ---- 5. one Philox call for every lane that draws this iteration
        const bool draws = alive && (phase == kLaunch || interact || (fresnel && !matched));
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (__any_sync(SMCRT_FULL, draws)) {
            r = philox4x32_10(make_uint4(event, 0u, id_lo, id_hi), jc->k0, jc->k1);
            if (draws) event += 1u;
        }

        // ---- 6. consumers
        if (SMCRT_RARE(alive && phase == kLaunch)) {           // photon release (Sec. 2.1)
            const Launched L0 = launch32(S, r);
            px = L0.px; py = L0.py; pz = L0.pz;
            ux = L0.ux; uy = L0.uy; uz = L0.uz;
            tau = L0.tau;
            w = 1.f;
            nsteps = 0; pA = 0; pG = 0; pscat = 0;
            cs = -1.f;
            pend = 0.f;
            phase = kTrace;
        }
        if (interact) {                            // implicit capture, HG, roulette
            const float4 RG = (*(S.reg32 + 2 * reg));
            const float wn = w * RG.z;
            pA += fx32(w - wn);
            w = wn;
            scatter32(ux, uy, uz, hg_cos32(RG.w, u01_32(r.x)), u01_32(r.y));
            pscat += 1u;
            cs = -1.f;
            tau = -__logf(u01_32(r.w));
            if (SMCRT_RARE(w < (float)kWRoulette)) {
                if (u01_32(r.z) <= (float)(1.0 / kRouletteM)) {
                    pG += fx32(w * (float)(kRouletteM - 1.0));
                    w = w * (float)kRouletteM;
                } else {
                    fin_K = fx32(w);
                    fin = true;
                    alive = false;
                }
            }
        }
        if (SMCRT_RARE(fresnel)) {                             // reflect, refract or cross (Sec. 2.3)
            const Crossed c = cross32<G>(S, ux, uy, uz, qx, qy, qz, nx, ny, nz, tau, dstar, cdot, istar, rnear, rfar,
                                         r.x, matched);
            if (!matched) wadd(wa, kFres, 1);
            if (c.refined) wadd(wa, kRefined, 1);
            px = c.px; py = c.py; pz = c.pz;
            ux = c.ux; uy = c.uy; uz = c.uz;
            tau = c.tau;
            pend = c.pend;
            phase = kTrace;
            iter_done = true;
        }
        if (iter_done && alive) {
            nsteps += 1;
            if (SMCRT_RARE(nsteps >= S.max_steps)) {
                wadd(wa, kCap, 1);
                fin_K = fx32(w);
                fin = true;
                alive = false;
            }
        }
        // ---- a terminated packet: one bookkeeping site per iteration
        if (SMCRT_RARE(fin)) {
            wadd(wa, kR, fin_R); wadd(wa, kT, fin_T); wadd(wa, kKilled, fin_K);
            wadd(wa, kA, pA); wadd(wa, kGain, pG); wadd(wa, kScat, pscat); wadd(wa, kSteps, nsteps);
            wadd(wa, kPackets, 1);
            if (MULTI) {                       // a lane's pieces and time go to its packet's job
                wadd(wa, kPieces, npieces);
                npieces = 0u;
                wadd(wa, kBusy, (long long)(((uint32_t)clock() - t_acq) >> 5));
            }
            // per-packet records belong to plan launches (served jobs have none)
            smcrt_packet_record *const recs = (smcrt_packet_record *)jc->recs;
            if (!MULTI && recs) {
                smcrt_packet_record r;
                r.R = fin_R; r.T = fin_T; r.A = pA; r.killed = fin_K; r.gain = pG;
                r.scatters = pscat; r.steps = nsteps; r.reserved = 0;
                const unsigned long long id = ((unsigned long long)id_hi << 32) | id_lo;
                recs[id - jc->begin] = r;
            }
        }
        // ---- park a straggler at a trace boundary (served rounds).  A
        // packet in a crawl is parked as its anchor and crawl length, from
        // which the resume recomputes the same position.
        if (MULTI && SMCRT_RARE(alive && phase == kTrace && jc->budget > 0u &&
                                (uint32_t)clock() - t_acq > (drained ? jc->drain : jc->budget))) {
            JobDefer *const dfr = (JobDefer *)jc->dfr;
            const int din = jc->din;
            const unsigned k = atomicAdd(&dfr->count[1 - din], 1u);
            if (k < dfr->cap) {
                DeferState &d = dfr->buf[1 - din][k];
                const bool in_crawl = cs >= 0.f;
                d.p[0] = in_crawl ? qx : px; d.p[1] = in_crawl ? qy : py; d.p[2] = in_crawl ? qz : pz;
                d.pad[0] = __float_as_uint(cs);
                d.pad[1] = __float_as_uint(pend);
                d.u[0] = ux; d.u[1] = uy; d.u[2] = uz;
                d.w = w; d.tau = tau;
                d.pA = pA; d.pG = pG;
                d.id_lo = id_lo; d.id_hi = id_hi; d.event = event;
                d.nsteps = (uint32_t)nsteps; d.pscat = pscat;
                wadd(wa, kParked, 1);
                if (MULTI) {
                    wadd(wa, kPieces, npieces);
                    npieces = 0u;
                    wadd(wa, kBusy, (long long)(((uint32_t)clock() - t_acq) >> 5));
                }
                alive = false;
            } else {
                // list full: run on and try again after another budget (the
                // time so far is the job's busy time, as a parked segment's is)
                atomicAdd(&dfr->overflow, 1u);
                if (MULTI) wadd(wa, kBusy, (long long)(((uint32_t)clock() - t_acq) >> 5));
                t_acq = (uint32_t)clock();
            }
        }
    }
    if (MULTI) {                               // the jobs still in the slots
        __syncwarp();
        if (sj0 >= 0) wacc_flush(&slots[0].acc, jobs[sj0].totals, lane);
        if (sj1 >= 0) wacc_flush(&slots[1].acc, jobs[sj1].totals, lane);
        return false;
    }
    const long long pc = warp_sum((long long)npieces);
    if (lane == 0) wadd(&slots[0].acc, kPieces, pc);
    return timed_out;
}

template <int kMinBlocks, bool G>
__global__ void __launch_bounds__(128, kMinBlocks) packets_mixed(JobWork *jobs, int njobs, int *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    WarpShared *ws = reinterpret_cast<WarpShared *>(smem) + warp;
    for (int jj = 0; jj < njobs; ++jj) {
        JobWork *J = jobs + (gw + jj) % njobs;
        unsigned long long nxt = 0, e = 0;
        const DevScene *src = nullptr;
        if (lane == 0) {
            nxt = *(volatile unsigned long long *)&J->next;
            e = J->end;
            src = J->scene;
        }
        int parked = 0;
        if (lane == 0 && J->defer != nullptr) {
            const int in = J->defer_in & 1;
            parked = min(*(volatile unsigned *)&J->defer->count[in], J->defer->cap) >
                     *(volatile unsigned *)&J->defer->cursor[in];
        }
        nxt = __shfl_sync(SMCRT_FULL, nxt, 0);
        e = __shfl_sync(SMCRT_FULL, e, 0);
        parked = __shfl_sync(SMCRT_FULL, parked, 0);
        src = (const DevScene *)__shfl_sync(SMCRT_FULL, (unsigned long long)src, 0);
        if (nxt >= e && !parked) continue;
        if (src == nullptr || J->totals == nullptr) {
            if (lane == 0) {
                atomicOr(status, kStatusBadJob);
                if (J->jstat != nullptr) atomicOr(J->jstat, kStatusBadJob);
            }
            continue;
        }
        const long long *s8 = reinterpret_cast<const long long *>(src);
        long long *d8 = reinterpret_cast<long long *>(&ws->slot.S);
        for (int i = lane; i < (int)(sizeof(DevScene) / 8); i += 32) d8[i] = s8[i];
        __syncwarp();
        if (J->stage) stage_tables(ws, lane);
        if (!G && ws->slot.S.general) {      // a scene with general shapes needs the G instantiation
            if (lane == 0) {
                atomicOr(status, kStatusBadJob);
                if (J->jstat != nullptr) atomicOr(J->jstat, kStatusBadJob);
            }
            continue;
        }
        if (lane == 0) jobconst_fill(&ws->slot.jc, J);
        wacc_clear(&ws->slot.acc, lane);
        const long long t0 = clock64();
        const bool timed_out = run_job_mixed<G, false>(&ws->slot, J, 1, 0, status, lane);
        __syncwarp();
        if (lane == 0) wadd(&ws->slot.acc, kBusy, clock64() - t0);
        wacc_flush(&ws->slot.acc, J->totals, lane);
        if (timed_out) {                     // the launch's time limit: this warp is done
            if (lane == 0) {
                atomicOr(status, kStatusTimeout);
                if (J->jstat != nullptr) atomicOr(J->jstat, kStatusTimeout);
            }
            return;
        }
    }
}

// Served rounds: every warp works through the whole job table, two jobs at a
// time (run_job_mixed<G, true>), starting at a job of its own so that the
// warps spread over the table.
template <int kMinBlocks, bool G>
__global__ void __launch_bounds__(128, kMinBlocks) packets_mixed_multi(JobWork *jobs, int njobs, int *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    WarpSharedMulti *ws = reinterpret_cast<WarpSharedMulti *>(smem) + warp;
    if (njobs <= 0) return;
    run_job_mixed<G, true>(ws->slot, jobs, njobs, gw % njobs, status, lane);
}

}  // namespace

// Register budgets of the instantiations: variant v keeps kMinBlocks
// blocks of 128 threads resident per SM (more blocks = fewer registers per
// thread, possibly spilled); the autotuner picks per scene.  Variants
// kNumVariants .. 2 kNumVariants - 1 are the same budgets for scenes with
// general shapes (tori, cylinders, primitive frames).
constexpr int kVariantBlocks[kNumVariants] = {5, 4, 3};

cudaError_t launch_mixed(JobWork *jobs, int njobs, int *status, int blocks, int threads, cudaStream_t stream,
                        int variant)
{
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpShared);
    switch (variant) {
    case 1: packets_mixed<4, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 2: packets_mixed<3, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 3: packets_mixed<5, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 4: packets_mixed<4, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 5: packets_mixed<3, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    default: packets_mixed<5, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    }
    return cudaGetLastError();
}

// The served kernel: variant 0 / 1 = 5 / 4 resident blocks, plain shapes;
// 3 / 4 = the same for general shapes (the index space of launch_mixed).
cudaError_t launch_mixed_multi(JobWork *jobs, int njobs, int *status, int blocks, int threads, cudaStream_t stream,
                               int variant)
{
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpSharedMulti);
    switch (variant) {
    case 1: packets_mixed_multi<4, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 3: packets_mixed_multi<5, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 4: packets_mixed_multi<4, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    default: packets_mixed_multi<5, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    }
    return cudaGetLastError();
}

int occupancy_mixed_multi(int threads, int variant)
{
    int n = 0;
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpSharedMulti);
    switch (variant) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed_multi<4, false>, threads, sm); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed_multi<5, true>, threads, sm); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed_multi<4, true>, threads, sm); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed_multi<5, false>, threads, sm); break;
    }
    return n;
}

int occupancy_mixed(int threads, int variant)
{
    int n = 0;
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpShared);
    switch (variant) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<4, false>, threads, sm); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<3, false>, threads, sm); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<5, true>, threads, sm); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<4, true>, threads, sm); break;
    case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<3, true>, threads, sm); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_mixed<5, false>, threads, sm); break;
    }
    return n;
}

}  // namespace smcrt
