// smcrt_kernel.cuh -- persistent photon-packet kernel for sm_103a.
//
// One thread carries one photon packet; warps pull packet ids from the
// job's atomic cursor (warp-aggregated: one atomicAdd per refill, ranks
// from a ballot), so a lane whose packet terminates is refilled at the
// next iteration and the warp stays full until the job runs dry.
//
// Every loop iteration performs exactly ONE full scene SDF evaluation per
// lane (the dominant cost, Sec. 4 "having to evaluate every SDF each time
// the photon needs to be moved").  What the lane does with it depends on
// its phase:
//   TRACE  evaluate at p: bounding box exit, interaction or sphere-trace
//          step (Sec. 2.3, Fig. 2 right, Fig. 3; Eq. 1 for tau),
//   NRM    six probes p +/- h e_a of the nearest surface's SDF: central
//          differences for the normal (Sec. 1 "numerical differentiation"),
//   PROJ   (FP64) Newton projection onto the surface along the normal,
//   FAR    region on the far side of the surface,
//   NEAR   region on the near side; then Fresnel reflection or Snell
//          refraction if the refractive index changes (Sec. 2.3).
// Lanes at an interface therefore share the scene evaluation with lanes
// that are tracing, instead of running a divergent interface routine.
//
// The FP64 instantiation performs the same IEEE operations in the same
// order as the FP64 reference algorithm (compiled with -fmad=false), with
// ln and sin/cos written here from textbook series, so its integer tallies
// are bit-identical to the reference.  The mixed instantiation traces in
// FP32 and refines interfaces in FP64 only near grazing or critical
// incidence.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "smcrt_internal.h"

namespace smcrt {

#define SMCRT_FULL 0xffffffffu
// A branch a lane rarely takes (interfaces, launches, terminations, parking):
// the compiler places its code away from the hot path of the packet loop,
// which runs close to the instruction cache's capacity.
#define SMCRT_RARE(x) __builtin_expect(!!(x), 0)

// ---------------------------------------------------------------------------
// Philox4x32-10, from its definition (Salmon, Moraes, Dror & Shaw, SC'11):
// ten rounds of two 32x32 -> 64-bit products with multipliers 0xD2511F53 and
// 0xCD9E8D57, key bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    // two rounds per trip: the packet loop's code must fit the instruction
    // cache, and a fully unrolled generator is most of a kilobyte of it
#pragma unroll 2
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Packet stream: key (seed lo, seed hi); counter (event, 0, id lo, id hi).
struct Rng {
    uint32_t k0, k1, id_lo, id_hi, event;
    __device__ __forceinline__ uint4 next()
    {
        uint4 w = philox4x32_10(make_uint4(event, 0u, id_lo, id_hi), k0, k1);
        event += 1u;
        return w;
    }
};

// Uniforms in (0, 1]: FP64 uses the whole 32-bit word, FP32 its top 24 bits.
__device__ __forceinline__ double u01_64(uint32_t w) { return ((double)w + 1.0) * (1.0 / 4294967296.0); }
// FP32: the top 23 bits mapped to bin midpoints, (k + 1/2) 2^-23, strictly
// inside (0, 1) and unbiased (24 bits would not do: (2^24 - 1/2) 2^-24
// rounds to 1 in FP32).  The value 1 would put a square or disc source's
// packet exactly on the boundary of its footprint: where that edge lies in
// a scene face, such a packet crawled along the face at distance 0 (moving
// exactly parallel to it) until the step cap.
__device__ __forceinline__ float u01_32(uint32_t w) { return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f); }

// ---------------------------------------------------------------------------
// FP64 ln and sin/cos(2 pi t), written from the series (not libdevice):
// ln x = e ln2 + 2 atanh((m-1)/(m+1)) with m in (sqrt(1/2), sqrt(2)], atanh
// series to s^21; sin/cos by reduction to the nearest quarter turn and the
// Taylor series of sin to a^17, cos to a^16 on |a| <= pi/4.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double ln64(double x)
{
    const long long b = __double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    if (m > 1.4142135623730951) {
        m = m * 0.5;
        e = e + 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double z = s * s;
    double t = 1.0 / 21.0;
    t = t * z + 1.0 / 19.0;
    t = t * z + 1.0 / 17.0;
    t = t * z + 1.0 / 15.0;
    t = t * z + 1.0 / 13.0;
    t = t * z + 1.0 / 11.0;
    t = t * z + 1.0 / 9.0;
    t = t * z + 1.0 / 7.0;
    t = t * z + 1.0 / 5.0;
    t = t * z + 1.0 / 3.0;
    t = t * z + 1.0;
    return (double)e * 0.6931471805599453 + (2.0 * s) * t;
}

__device__ __forceinline__ void sincos2pi64(double t, double *sn, double *cs)
{
    const double q = floor(t * 4.0 + 0.5);
    const double f = t - q * 0.25;
    const double a = f * 6.283185307179586;
    const double z = a * a;
    double ps = 1.0 / 355687428096000.0;
    ps = ps * z - 1.0 / 1307674368000.0;
    ps = ps * z + 1.0 / 6227020800.0;
    ps = ps * z - 1.0 / 39916800.0;
    ps = ps * z + 1.0 / 362880.0;
    ps = ps * z - 1.0 / 5040.0;
    ps = ps * z + 1.0 / 120.0;
    ps = ps * z - 1.0 / 6.0;
    const double s = a + a * (z * ps);
    double pc = 1.0 / 20922789888000.0;
    pc = pc * z - 1.0 / 87178291200.0;
    pc = pc * z + 1.0 / 479001600.0;
    pc = pc * z - 1.0 / 3628800.0;
    pc = pc * z + 1.0 / 40320.0;
    pc = pc * z - 1.0 / 720.0;
    pc = pc * z + 1.0 / 24.0;
    pc = pc * z - 0.5;
    const double c = 1.0 + z * pc;
    switch (((int)q) & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
    }
}

// Fixed point: 2^-32 weight units.  FP64: round half to even like llrint.
__device__ __forceinline__ long long fx64(double x) { return __double2ll_rn(x * 4294967296.0); }
// FP32 (0 <= x < 2^31): x * 2^32 is exact (a power-of-two scale), then one
// hardware conversion to int64, round half to even (cheaper than shifting
// the mantissa in integer code, which cost the tally 7 % of the kernel).
__device__ __forceinline__ long long fx32(float x) { return __float2ll_rn(x * 4294967296.f); }

// ---------------------------------------------------------------------------
// Scene evaluation.  Instr.op packs op | (primitive kind << 8).
// The instruction stream, primitive kinds, FP32 primitive and region tables
// and region ranges are read with plain (generic) loads: a warp of the mixed
// kernel may stage them in its shared memory, and on global memory the plain
// loads measured 3.5 % faster than read-only-cache loads on the layered slab.
// ---------------------------------------------------------------------------
// dsoft: min |d| over soft regions (segment stepping), +inf if none.
struct Eval64 { double dmin, dstar, dsel, dbox, dsoft; int istar, region; };
struct Eval32 { float dmin, dstar, dsel, dbox, dsoft; int istar, region; };

__device__ __forceinline__ double box64(double x, double y, double z, double cx, double cy, double cz,
                                        double hx, double hy, double hz)
{
    const double qx = fabs(x - cx) - hx, qy = fabs(y - cy) - hy, qz = fabs(z - cz) - hz;
    const double mx = fmax(qx, 0.0), my = fmax(qy, 0.0), mz = fmax(qz, 0.0);
    const double outside = sqrt(mx * mx + my * my + mz * mz);
    const double inside = fmin(fmax(qx, fmax(qy, qz)), 0.0);
    return outside + inside;
}

__device__ __forceinline__ float box32(float x, float y, float z, float cx, float cy, float cz,
                                       float hx, float hy, float hz)
{
    const float qx = fabsf(x - cx) - hx, qy = fabsf(y - cy) - hy, qz = fabsf(z - cz) - hz;
    const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
    const float outside = sqrtf(__fmaf_rn(mx, mx, __fmaf_rn(my, my, mz * mz)));
    const float inside = fminf(fmaxf(qx, fmaxf(qy, qz)), 0.f);
    return outside + inside;
}

// Torus (kind 3) and capped cylinder (kind 4), out of line: they are rare,
// and inlined copies would cost the hot loop registers.
static __device__ __noinline__ double round64(int kind, const double *P, double x, double y, double z)
{
    const double dx = x - __ldg(P), dy = y - __ldg(P + 1), dz = z - __ldg(P + 2);
    if (kind == 3) {                     // torus about z: core circle distance - tube radius
        const double ring = sqrt(dx * dx + dy * dy) - __ldg(P + 3);
        return sqrt(ring * ring + dz * dz) - __ldg(P + 4);
    }
    const double a = sqrt(dx * dx + dy * dy) - __ldg(P + 3);   // capped cylinder along z
    const double b = fabs(dz) - __ldg(P + 4);
    const double ma = fmax(a, 0.0), mb = fmax(b, 0.0);
    return fmin(fmax(a, b), 0.0) + sqrt(ma * ma + mb * mb);
}

// Primitive distances in local coordinates (kind 0..4, Sec. 2.2 and the
// Fig. 1 basic shapes).  FP64: the reference's operations in its order.
// G = false: the scene has only spheres, boxes and capsules in scene
// coordinates (the kernels are instantiated for both cases, so plain
// scenes pay nothing for the general shapes).
template <bool G>
__device__ __forceinline__ double base64(int kind, const double *P, double x, double y, double z)
{
    if (kind == 0) {
        const double dx = x - __ldg(P), dy = y - __ldg(P + 1), dz = z - __ldg(P + 2);
        return sqrt(dx * dx + dy * dy + dz * dz) - __ldg(P + 3);
    }
    if (kind == 1)
        return box64(x, y, z, __ldg(P), __ldg(P + 1), __ldg(P + 2), __ldg(P + 3), __ldg(P + 4), __ldg(P + 5));
    if (!G || kind == 2) {
        const double pax = x - __ldg(P), pay = y - __ldg(P + 1), paz = z - __ldg(P + 2);
        const double bax = __ldg(P + 3), bay = __ldg(P + 4), baz = __ldg(P + 5);
        double t = (pax * bax + pay * bay + paz * baz) / __ldg(P + 7);
        t = fmin(fmax(t, 0.0), 1.0);
        const double dx = pax - bax * t, dy = pay - bay * t, dz = paz - baz * t;
        return sqrt(dx * dx + dy * dy + dz * dz) - __ldg(P + 6);
    }
    return round64(kind, P, x, y, z);
}

// A primitive in its frame (smcrt_xform): local point R^T (p - t) / s, the
// domain operation, the local distance scaled back by s and divided by the
// operation's Lipschitz bound.
static __device__ __noinline__ double xprim64(const DevScene &S, int kind, int i, double x, double y, double z)
{
    const double *X = S.xf64 + kXf64 * i;
    const double vx = x - __ldg(X + 9), vy = y - __ldg(X + 10), vz = z - __ldg(X + 11);
    const double s = __ldg(X + 12);
    double q0 = (__ldg(X) * vx + __ldg(X + 3) * vy + __ldg(X + 6) * vz) / s;
    double q1 = (__ldg(X + 1) * vx + __ldg(X + 4) * vy + __ldg(X + 7) * vz) / s;
    double q2 = (__ldg(X + 2) * vx + __ldg(X + 5) * vy + __ldg(X + 8) * vz) / s;
    const int op = (int)__ldg(X + 13);
    const double a0 = __ldg(X + 14), a1 = __ldg(X + 15), a2 = __ldg(X + 16), a3 = __ldg(X + 17);
    double L = 1.0;
    if (op == 1) {                       // elongate
        q0 = q0 - fmin(fmax(q0, -a0), a0);
        q1 = q1 - fmin(fmax(q1, -a1), a1);
        q2 = q2 - fmin(fmax(q2, -a2), a2);
    } else if (op == 2 || op == 3) {     // twist about z / bend in x-y
        const double rho = sqrt(q0 * q0 + q1 * q1);
        double sn, cs;
        sincos2pi64(a0 * (op == 2 ? q2 : q0), &sn, &cs);
        const double rx = cs * q0 - sn * q1;
        const double ry = sn * q0 + cs * q1;
        q0 = rx; q1 = ry;
        const double m = 6.283185307179586 * a0 * fmax(rho, a1);   // stretch bound of the map
        L = op == 2 ? 0.5 * (m + sqrt(m * m + 4.0)) : 1.0 + m;
    } else if (op == 4) {                // repetition: nearest copy
        if (a0 > 0.0) { double k = floor(q0 / a0 + 0.5); k = fmin(fmax(k, -a3), a3); q0 = q0 - a0 * k; }
        if (a1 > 0.0) { double k = floor(q1 / a1 + 0.5); k = fmin(fmax(k, -a3), a3); q1 = q1 - a1 * k; }
        if (a2 > 0.0) { double k = floor(q2 / a2 + 0.5); k = fmin(fmax(k, -a3), a3); q2 = q2 - a2 * k; }
    }
    return s * base64<true>(kind, S.p64 + 8 * i, q0, q1, q2) / L;
}

template <bool G>
__device__ __forceinline__ double prim64(const DevScene &S, int kind, int i, double x, double y, double z)
{
    if (G && (kind & kXformFlag)) return xprim64(S, kind & 0xf, i, x, y, z);
    return base64<G>(kind, S.p64 + 8 * i, x, y, z);
}

static __device__ __noinline__ float round32(int kind, const float4 *P, float x, float y, float z)
{
    const float4 A = (*(P)), B = (*(P + 1));
    const float dx = x - A.x, dy = y - A.y, dz = z - A.z;
    if (kind == 3) {
        const float ring = sqrtf(dx * dx + dy * dy) - A.w;
        return sqrtf(ring * ring + dz * dz) - B.x;
    }
    const float a = sqrtf(dx * dx + dy * dy) - A.w;
    const float b = fabsf(dz) - B.x;
    const float ma = fmaxf(a, 0.f), mb = fmaxf(b, 0.f);
    return fminf(fmaxf(a, b), 0.f) + sqrtf(ma * ma + mb * mb);
}

template <bool G>
__device__ __forceinline__ float base32(int kind, const float4 *P, float x, float y, float z)
{
    const float4 A = (*(P));
    if (kind == 0) {
        const float dx = x - A.x, dy = y - A.y, dz = z - A.z;
        return sqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz))) - A.w;
    }
    const float4 B = (*(P + 1));
    if (kind == 1) return box32(x, y, z, A.x, A.y, A.z, B.x, B.y, B.z);
    if (!G || kind == 2) {
        const float pax = x - A.x, pay = y - A.y, paz = z - A.z;
        float t = __fmaf_rn(pax, B.x, __fmaf_rn(pay, B.y, paz * B.z)) * B.w;
        t = fminf(fmaxf(t, 0.f), 1.f);
        const float dx = __fmaf_rn(-B.x, t, pax), dy = __fmaf_rn(-B.y, t, pay), dz = __fmaf_rn(-B.z, t, paz);
        return sqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz))) - A.w;
    }
    return round32(kind, P, x, y, z);
}

static __device__ __noinline__ float xprim32(const DevScene &S, int kind, int i, float x, float y, float z)
{
    const float4 *X = S.xf32 + kXf32 * i;
    const float4 R0 = __ldg(X), R1 = __ldg(X + 1), R2 = __ldg(X + 2), SC = __ldg(X + 3), A = __ldg(X + 4);
    const float vx = x - R0.w, vy = y - R1.w, vz = z - R2.w;
    float q0 = (R0.x * vx + R0.y * vy + R0.z * vz) * SC.y;
    float q1 = (R1.x * vx + R1.y * vy + R1.z * vz) * SC.y;
    float q2 = (R2.x * vx + R2.y * vy + R2.z * vz) * SC.y;
    const int op = (int)SC.z;
    float L = 1.f;
    if (op == 1) {
        q0 = q0 - fminf(fmaxf(q0, -A.x), A.x);
        q1 = q1 - fminf(fmaxf(q1, -A.y), A.y);
        q2 = q2 - fminf(fmaxf(q2, -A.z), A.z);
    } else if (op == 2 || op == 3) {
        const float rho = sqrtf(q0 * q0 + q1 * q1);
        float sn, cs;
        sincospif(2.f * A.x * (op == 2 ? q2 : q0), &sn, &cs);
        const float rx = cs * q0 - sn * q1;
        const float ry = sn * q0 + cs * q1;
        q0 = rx; q1 = ry;
        const float m = 6.2831853f * A.x * fmaxf(rho, A.y);
        L = op == 2 ? 0.5f * (m + sqrtf(m * m + 4.f)) : 1.f + m;
    } else if (op == 4) {
        if (A.x > 0.f) { float k = floorf(q0 / A.x + 0.5f); k = fminf(fmaxf(k, -A.w), A.w); q0 = q0 - A.x * k; }
        if (A.y > 0.f) { float k = floorf(q1 / A.y + 0.5f); k = fminf(fmaxf(k, -A.w), A.w); q1 = q1 - A.y * k; }
        if (A.z > 0.f) { float k = floorf(q2 / A.z + 0.5f); k = fminf(fmaxf(k, -A.w), A.w); q2 = q2 - A.z * k; }
    }
    return SC.x * base32<true>(kind, S.p32 + 2 * i, q0, q1, q2) / L;
}

template <bool G>
__device__ __forceinline__ float prim32(const DevScene &S, int kind, int i, float x, float y, float z)
{
    if (G && (kind & kXformFlag)) return xprim32(S, kind & 0xf, i, x, y, z);
    return base32<G>(kind, S.p32 + 2 * i, x, y, z);
}

// a = left (earlier) operand, b = right.  Smooth union: polynomial smooth
// minimum (the SDF literature cited with Fig. 1 e).
__device__ __forceinline__ double csg64(int op, double a, double b, double k)
{
    if (op == 1) return fmin(a, b);
    if (op == 3) return fmax(a, b);
    if (op == 4) return fmax(a, -b);
    double h = 0.5 + 0.5 * (b - a) / k;
    h = fmin(fmax(h, 0.0), 1.0);
    const double m = b * (1.0 - h) + a * h;
    return m - k * h * (1.0 - h);
}

__device__ __forceinline__ float csg32(int op, float a, float b, float kinv)
{
    if (op == 1) return fminf(a, b);
    if (op == 3) return fmaxf(a, b);
    if (op == 4) return fmaxf(a, -b);
    const float k = 1.0f / kinv;
    float h = 0.5f + 0.5f * (b - a) * kinv;
    h = fminf(fmaxf(h, 0.f), 1.f);
    const float m = b + (a - b) * h;
    return m - k * h * (1.f - h);
}

// Evaluate instructions [i0, i1) as a register-stack program; when `full`,
// record every region end (region, d_min, istar, and d of surface `sel`).
template <bool kFull, bool G>
__device__ __forceinline__ double run_prog64(const DevScene &S, int i0, int i1, double x, double y, double z,
                                             int sel, Eval64 *E)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int i = i0; i < i1; ++i) {
        const int4 ins = (*(reinterpret_cast<const int4 *>(S.instr) + i));
        const int op = ins.x & 0xff, kind = (ins.x >> 8) & 0xff;
        double v = 0.0;
        if (ins.y >= 0) v = prim64<G>(S, kind, ins.y, x, y, z);
        if (op == 0) {
            s3 = s2; s2 = s1; s1 = s0; s0 = v;
        } else {
            const double k = (op == 2) ? __ldg(S.k64 + i) : 0.0;
            if (ins.y >= 0) {
                s0 = csg64(op, s0, v, k);
            } else {
                s0 = csg64(op, s1, s0, k);
                s1 = s2; s2 = s3;
            }
        }
        if (kFull && ins.z >= 0) {
            const double d = s0;
            if (d < 0.0) E->region = ins.z;
            const double ad = fabs(d);
            if (ad < E->dmin) { E->dmin = ad; E->istar = ins.z; E->dstar = d; }
            if ((ins.x & kSoftRegionEnd) && ad < E->dsoft) E->dsoft = ad;
            if (ins.z == sel) E->dsel = d;
        }
    }
    return s0;
}

template <bool kFull, bool G>
__device__ __forceinline__ float run_prog32(const DevScene &S, int i0, int i1, float x, float y, float z,
                                            int sel, Eval32 *E)
{
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int i = i0; i < i1; ++i) {
        const int4 ins = (*(reinterpret_cast<const int4 *>(S.instr) + i));
        const int op = ins.x & 0xff, kind = (ins.x >> 8) & 0xff;
        float v = 0.f;
        if (ins.y >= 0) v = prim32<G>(S, kind, ins.y, x, y, z);
        if (op == 0) {
            s3 = s2; s2 = s1; s1 = s0; s0 = v;
        } else {
            const float kinv = __int_as_float(ins.w);
            if (ins.y >= 0) {
                s0 = csg32(op, s0, v, kinv);
            } else {
                s0 = csg32(op, s1, s0, kinv);
                s1 = s2; s2 = s3;
            }
        }
        if (kFull && ins.z >= 0) {
            const float d = s0;
            if (d < 0.f) E->region = ins.z;
            const float ad = fabsf(d);
            if (ad < E->dmin) { E->dmin = ad; E->istar = ins.z; E->dstar = d; }
            if ((ins.x & kSoftRegionEnd) && ad < E->dsoft) E->dsoft = ad;
            if (ins.z == sel) E->dsel = d;
        }
    }
    return s0;
}

// Full scene evaluation (Sec. 2.3): every region, then the bounding box.
template <bool G>
__device__ __forceinline__ Eval64 scene_eval64(const DevScene &S, double x, double y, double z, int sel)
{
    Eval64 E;
    E.dmin = __longlong_as_double(0x7ff0000000000000LL);
    E.dsoft = E.dmin;
    E.dstar = 0.0; E.dsel = 0.0; E.istar = -1; E.region = -1;
    run_prog64<true, G>(S, 0, S.ninstr, x, y, z, sel, &E);
    const double db = box64(x, y, z, S.bbc[0], S.bbc[1], S.bbc[2], S.bbh[0], S.bbh[1], S.bbh[2]);
    E.dbox = db;
    if (fabs(db) < E.dmin) { E.dmin = fabs(db); E.istar = -1; E.dstar = db; }
    if (sel == -1) E.dsel = db;
    return E;
}

// Value of the culled fold region at p: the fold over the primitives listed
// for p's cell, bounded by cull_rmax (every unlisted primitive is farther
// than R from the cell, so it cannot change the value below that bound).
__device__ __forceinline__ float culled_region32(const DevScene &S, float x, float y, float z)
{
    const int g = S.cull_g;
    const int cx = __float2int_rd((x - S.cull_lo[0]) * S.cull_inv_s[0]);
    const int cy = __float2int_rd((y - S.cull_lo[1]) * S.cull_inv_s[1]);
    const int cz = __float2int_rd((z - S.cull_lo[2]) * S.cull_inv_s[2]);
    if ((unsigned)cx >= (unsigned)g || (unsigned)cy >= (unsigned)g || (unsigned)cz >= (unsigned)g)
        return S.cull_rmax;
    const int c = (cz * g + cy) * g + cx;
    const int o0 = __ldg(S.cull_off + c), o1 = __ldg(S.cull_off + c + 1);
    if (o1 <= o0) return S.cull_rmax;
    int i = __ldg(S.cull_list + o0);
    float acc = prim32<false>(S, (*(S.pkind + i)), i, x, y, z);   // culled regions are plain
    for (int j = o0 + 1; j < o1; ++j) {
        i = __ldg(S.cull_list + j);
        acc = csg32(S.cull_op, acc, prim32<false>(S, (*(S.pkind + i)), i, x, y, z), S.cull_kinv);
    }
    return fminf(acc, S.cull_rmax);
}

__device__ __forceinline__ void region_end32(Eval32 *E, int r, float d, int sel, bool soft)
{
    if (d < 0.f) E->region = r;
    const float ad = fabsf(d);
    if (ad < E->dmin) { E->dmin = ad; E->istar = r; E->dstar = d; }
    if (soft && ad < E->dsoft) E->dsoft = ad;
    if (r == sel) E->dsel = d;
}

// One copy of the interpreter in the packet loop: the culled region's
// instructions [cb, ce) are replaced by its culled distance inside the same
// loop (each region's program is self-contained, so the stack left by the
// regions before it does not matter).  Code size counts here: the loop runs
// close to the instruction cache's capacity (measured on the layered slab:
// three interpreter copies 203.6 ms per 1e7 packets, one copy 184.4 ms).
template <bool G>
__device__ __forceinline__ Eval32 scene_eval32(const DevScene &S, float x, float y, float z, int sel)
{
    Eval32 E;
    E.dmin = __int_as_float(0x7f800000);
    E.dsoft = E.dmin;
    E.dstar = 0.f; E.dsel = 0.f; E.istar = -1; E.region = -1;
    int cb = S.ninstr, ce = S.ninstr;
    if (S.cull_region >= 0) {
        const int2 rr = (*(S.rrange + S.cull_region));
        cb = rr.x;
        ce = rr.y;
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int i = 0; i < S.ninstr; ++i) {
        if (i == cb) {
            // the culled region's distance bounds segment moves
            // isotropically (its primitives are not in seg_prims)
            region_end32(&E, S.cull_region, culled_region32(S, x, y, z), sel, true);
            i = ce - 1;
            continue;
        }
        const int4 ins = (*(reinterpret_cast<const int4 *>(S.instr) + i));
        const int op = ins.x & 0xff, kind = (ins.x >> 8) & 0xff;
        float v = 0.f;
        if (ins.y >= 0) v = prim32<G>(S, kind, ins.y, x, y, z);
        if (op == 0) {
            s3 = s2; s2 = s1; s1 = s0; s0 = v;
        } else {
            const float kinv = __int_as_float(ins.w);
            if (ins.y >= 0) {
                s0 = csg32(op, s0, v, kinv);
            } else {
                s0 = csg32(op, s1, s0, kinv);
                s1 = s2; s2 = s3;
            }
        }
        if (ins.z >= 0) region_end32(&E, ins.z, s0, sel, (ins.x & kSoftRegionEnd) != 0);
    }
    const float db = box32(x, y, z, S.bbc32[0], S.bbc32[1], S.bbc32[2], S.bbh32[0], S.bbh32[1], S.bbh32[2]);
    E.dbox = db;
    if (fabsf(db) < E.dmin) { E.dmin = fabsf(db); E.istar = -1; E.dstar = db; }
    if (sel == -1) E.dsel = db;
    return E;
}

// Value and analytic gradient of one primitive (FP32).  Sphere and capsule:
// unit vector from the nearest point of the centre / segment; box: outside,
// the normalised positive part of q = |p - c| - h with the signs of p - c;
// inside, the axis of the largest component of q.
__device__ __forceinline__ float prim_grad32(const DevScene &S, int kind, int i, float x, float y, float z,
                                             float &gx, float &gy, float &gz)
{
    const float4 A = (*(S.p32 + 2 * i));
    if (kind == 0) {
        const float dx = x - A.x, dy = y - A.y, dz = z - A.z;
        const float l = sqrtf(dx * dx + dy * dy + dz * dz);
        const float il = l > 0.f ? 1.f / l : 0.f;
        gx = dx * il; gy = dy * il; gz = dz * il;
        return l - A.w;
    }
    const float4 B = (*(S.p32 + 2 * i + 1));
    if (kind == 1) {
        const float px = x - A.x, py = y - A.y, pz = z - A.z;
        const float qx = fabsf(px) - B.x, qy = fabsf(py) - B.y, qz = fabsf(pz) - B.z;
        const float mx = fmaxf(qx, 0.f), my = fmaxf(qy, 0.f), mz = fmaxf(qz, 0.f);
        const float o = sqrtf(mx * mx + my * my + mz * mz);
        if (o > 0.f) {
            const float io = 1.f / o;
            gx = copysignf(mx * io, px); gy = copysignf(my * io, py); gz = copysignf(mz * io, pz);
            return o;
        }
        gx = gy = gz = 0.f;
        if (qx >= qy && qx >= qz) { gx = copysignf(1.f, px); return qx; }
        if (qy >= qz) { gy = copysignf(1.f, py); return qy; }
        gz = copysignf(1.f, pz);
        return qz;
    }
    const float pax = x - A.x, pay = y - A.y, paz = z - A.z;
    float t = (pax * B.x + pay * B.y + paz * B.z) * B.w;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float dx = pax - B.x * t, dy = pay - B.y * t, dz = paz - B.z * t;
    const float l = sqrtf(dx * dx + dy * dy + dz * dz);
    const float il = l > 0.f ? 1.f / l : 0.f;
    gx = dx * il; gy = dy * il; gz = dz * il;
    return l - A.w;
}

// CSG on (value, gradient) pairs: min / max / max(a, -b) select an operand's
// gradient; for the polynomial smooth minimum d/da = h and d/db = 1 - h.
__device__ __forceinline__ void csg_grad32(int op, float &a, float &ax, float &ay, float &az, float b, float bx,
                                           float by, float bz, float kinv)
{
    if (op == 1) {
        if (b < a) { a = b; ax = bx; ay = by; az = bz; }
    } else if (op == 3) {
        if (b > a) { a = b; ax = bx; ay = by; az = bz; }
    } else if (op == 4) {
        if (-b > a) { a = -b; ax = -bx; ay = -by; az = -bz; }
    } else {
        const float k = 1.0f / kinv;
        float h = 0.5f + 0.5f * (b - a) * kinv;
        h = fminf(fmaxf(h, 0.f), 1.f);
        const float m = b + (a - b) * h;
        a = m - k * h * (1.f - h);
        ax = h * ax + (1.f - h) * bx; ay = h * ay + (1.f - h) * by; az = h * az + (1.f - h) * bz;
    }
}

// Value and gradient of one surface's SDF (region program, or the bounding
// box for r = -1): used for analytic normals on short programs.
// Value and gradient of the culled region (the fold of union / smooth union
// over the cell's candidates, as culled_region32): the gradient of a smooth
// minimum is the h-weighted blend of its operands' gradients.  Only called
// within delta of the region's surface, where the fold is below the clamp.
__device__ __forceinline__ float grad_culled32(const DevScene &S, float x, float y, float z, float &gx, float &gy,
                                               float &gz)
{
    gx = gy = gz = 0.f;
    const int g = S.cull_g;
    const int cx = __float2int_rd((x - S.cull_lo[0]) * S.cull_inv_s[0]);
    const int cy = __float2int_rd((y - S.cull_lo[1]) * S.cull_inv_s[1]);
    const int cz = __float2int_rd((z - S.cull_lo[2]) * S.cull_inv_s[2]);
    if ((unsigned)cx >= (unsigned)g || (unsigned)cy >= (unsigned)g || (unsigned)cz >= (unsigned)g)
        return S.cull_rmax;
    const int c = (cz * g + cy) * g + cx;
    const int o0 = __ldg(S.cull_off + c), o1 = __ldg(S.cull_off + c + 1);
    if (o1 <= o0) return S.cull_rmax;
    int i = __ldg(S.cull_list + o0);
    float acc = prim_grad32(S, (*(S.pkind + i)), i, x, y, z, gx, gy, gz);
    for (int j = o0 + 1; j < o1; ++j) {
        i = __ldg(S.cull_list + j);
        float bx, by, bz;
        const float b = prim_grad32(S, (*(S.pkind + i)), i, x, y, z, bx, by, bz);
        csg_grad32(S.cull_op, acc, gx, gy, gz, b, bx, by, bz, S.cull_kinv);
    }
    if (!(acc < S.cull_rmax)) { gx = gy = gz = 0.f; return S.cull_rmax; }
    return acc;
}

static __device__ __noinline__ float grad_surface32(const DevScene &S, int r, float x, float y, float z, float &gx,
                                             float &gy, float &gz)
{
    if (r >= 0 && r == S.cull_region) return grad_culled32(S, x, y, z, gx, gy, gz);
    if (r < 0) {
        const float px = x - S.bbc32[0], py = y - S.bbc32[1], pz = z - S.bbc32[2];
        const float qx = fabsf(px) - S.bbh32[0], qy = fabsf(py) - S.bbh32[1], qz = fabsf(pz) - S.bbh32[2];
        gx = gy = gz = 0.f;
        if (qx >= qy && qx >= qz) { gx = copysignf(1.f, px); return qx; }
        if (qy >= qz) { gy = copysignf(1.f, py); return qy; }
        gz = copysignf(1.f, pz);
        return qz;
    }
    const int2 rr = (*(S.rrange + r));
    float v[kMaxStack], vx[kMaxStack], vy[kMaxStack], vz[kMaxStack];
    int sp = 0;
    for (int i = rr.x; i < rr.y; ++i) {
        const int4 ins = (*(reinterpret_cast<const int4 *>(S.instr) + i));
        const int op = ins.x & 0xff, kind = (ins.x >> 8) & 0xff;
        float a = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
        if (ins.y >= 0) a = prim_grad32(S, kind, ins.y, x, y, z, ax, ay, az);
        if (op == 0) {
            v[sp] = a; vx[sp] = ax; vy[sp] = ay; vz[sp] = az;
            ++sp;
        } else if (ins.y >= 0) {
            csg_grad32(op, v[sp - 1], vx[sp - 1], vy[sp - 1], vz[sp - 1], a, ax, ay, az, __int_as_float(ins.w));
        } else {
            --sp;
            csg_grad32(op, v[sp - 1], vx[sp - 1], vy[sp - 1], vz[sp - 1], v[sp], vx[sp], vy[sp], vz[sp],
                       __int_as_float(ins.w));
        }
    }
    gx = vx[0]; gy = vy[0]; gz = vz[0];
    return v[0];
}

// SDF of one surface in FP64 (region program, or the bounding box for -1).
template <bool G>
__device__ __forceinline__ double surface64(const DevScene &S, int r, double x, double y, double z)
{
    if (r < 0) return box64(x, y, z, S.bbc[0], S.bbc[1], S.bbc[2], S.bbh[0], S.bbh[1], S.bbh[2]);
    const int2 rr = (*(S.rrange + r));
    return run_prog64<false, G>(S, rr.x, rr.y, x, y, z, -2, nullptr);
}

// ---------------------------------------------------------------------------
// Segment stepping (scene option; Sec. 5 names segment tracing for packets
// moving nearly parallel to a surface).  Bound on the move along u: for each
// primitive of a region that is not soft, the distance along the ray until
// its |SDF| can fall to e = m + delta/2, m the sum of k/4 over its regions'
// smooth unions (a region's surface lies where some primitive has |d| <= m):
// spheres, boxes, capsules and capped cylinders grown by e from outside and
// shrunk by e from inside, tori from outside through the annular slab that
// holds the grown tube and from inside through a ball the shrunk tube holds,
// the same shapes placed by a frame without a domain operation, |d| - e
// otherwise; |d| - delta/2 for soft regions (dsoft); the
// exit of the bounding box shrunk by delta/2.  The caller moves
// max(d_min - delta/2, bound).  FP64: the reference's operations in its
// order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double seg_sphere64(const double *P, double d, double px, double py, double pz,
                                               double ux, double uy, double uz, double dh)
{
    const double rr = d > 0.0 ? __ldg(P + 3) + dh : __ldg(P + 3) - dh;
    const double ox = px - __ldg(P), oy = py - __ldg(P + 1), oz = pz - __ldg(P + 2);
    const double b = ox * ux + oy * uy + oz * uz;
    const double cc = ox * ox + oy * oy + oz * oz - rr * rr;
    const double disc = b * b - cc;
    double t;
    if (d > 0.0) {                       // outside: entry of the grown sphere (near root)
        if (b >= 0.0 || disc < 0.0) return __longlong_as_double(0x7ff0000000000000LL);
        t = cc / (sqrt(disc) - b);
    } else {                             // inside: exit of the shrunk sphere
        if (disc < 0.0) return 0.0;
        if (b > 0.0) t = -cc / (b + sqrt(disc));
        else t = sqrt(disc) - b;
    }
    return t > 0.0 ? t : 0.0;
}

__device__ __forceinline__ double seg_box64(double cx, double cy, double cz, double hx, double hy, double hz,
                                            double d, double px, double py, double pz, double ux, double uy,
                                            double uz, double dh)
{
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const double e = d > 0.0 ? dh : -dh;
    const double c[3] = {cx, cy, cz}, h[3] = {hx, hy, hz}, p[3] = {px, py, pz}, u[3] = {ux, uy, uz};
    double tn = -inf, tf = inf;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double lo = c[a] - (h[a] + e), hi = c[a] + (h[a] + e);
        if (u[a] != 0.0) {
            const double t0 = (lo - p[a]) / u[a], t1 = (hi - p[a]) / u[a];
            tn = fmax(tn, fmin(t0, t1));
            tf = fmin(tf, fmax(t0, t1));
        } else if (p[a] < lo || p[a] > hi) {
            return d > 0.0 ? inf : 0.0;
        }
    }
    if (d > 0.0) {                       // outside: entry of the grown box
        if (tn > tf || tf < 0.0) return inf;
        return tn > 0.0 ? tn : 0.0;
    }
    return tf > 0.0 ? tf : 0.0;          // inside: exit of the shrunk box
}

// Ray interval [t0, t1] inside the ball of radius rr whose centre is at
// p - o (t0 > t1: missed); the far root comes from the near one through the
// product of the roots.
__device__ __forceinline__ void ray_ball64(double ox, double oy, double oz, double rr, double ux, double uy,
                                           double uz, double &t0, double &t1)
{
    const double b = ox * ux + oy * uy + oz * uz;
    const double cc = ox * ox + oy * oy + oz * oz - rr * rr;
    const double disc = b * b - cc;
    t0 = __longlong_as_double(0x7ff0000000000000LL);
    t1 = -t0;
    if (disc < 0.0) return;
    const double sq = sqrt(disc);
    if (b > 0.0) {
        const double q = -(b + sq);
        t0 = q; t1 = cc / q;
    } else {
        const double q = sq - b;
        if (q > 0.0) { t1 = q; t0 = cc / q; }
        else { t0 = 0.0; t1 = 0.0; }
    }
}

// Ray interval inside the cylinder of radius rr about the axis a + s ba
// between the planes s = 0 and s = 1 (o = p - a, L2 = |ba|^2); the cross-axis
// parts of o and u are formed first.
__device__ __forceinline__ void ray_cylinder64(double ox, double oy, double oz, double bax, double bay,
                                               double baz, double L2, double rr, double ux, double uy,
                                               double uz, double &t0, double &t1)
{
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const double uw = ux * bax + uy * bay + uz * baz;
    const double ow = ox * bax + oy * bay + oz * baz;
    double lo = -inf, hi = inf;
    t0 = inf; t1 = -inf;
    if (uw != 0.0) {                     // between the end planes
        const double s0 = -ow / uw, s1 = (L2 - ow) / uw;
        lo = fmin(s0, s1); hi = fmax(s0, s1);
    } else if (ow < 0.0 || ow > L2) {
        return;
    }
    const double k = uw / L2, m = ow / L2;
    const double vx = ux - k * bax, vy = uy - k * bay, vz = uz - k * baz;
    const double wx = ox - m * bax, wy = oy - m * bay, wz = oz - m * baz;
    const double A = vx * vx + vy * vy + vz * vz;
    const double B = wx * vx + wy * vy + wz * vz;
    const double C = wx * wx + wy * wy + wz * wz - rr * rr;
    if (A > 0.0) {                       // A t^2 + 2 B t + C <= 0
        const double disc = B * B - A * C;
        if (disc < 0.0) return;
        const double sq = sqrt(disc);
        double c0, c1;
        if (B > 0.0) {
            const double q = -(B + sq);
            c0 = q / A; c1 = C / q;
        } else {
            const double q = sq - B;
            if (q > 0.0) { c1 = q / A; c0 = C / q; }
            else { c0 = 0.0; c1 = 0.0; }
        }
        lo = fmax(lo, c0); hi = fmin(hi, c1);
    } else if (C > 0.0) {
        return;
    }
    t0 = lo; t1 = hi;
}

// Capsule (convex: the cylinder between its end planes and the two end
// balls): from outside the earliest entry of a part of the grown capsule,
// from inside the latest exit from a part of the shrunk one.  Out of line in
// both precisions: inlined into the bound routine, its three quadratics cost
// scenes without capsules 7 % (the routine's registers and size).
static __device__ __noinline__ double seg_capsule64(const double *P, double d, double px, double py, double pz,
                                                double ux, double uy, double uz, double dh)
{
    const double rr = d > 0.0 ? __ldg(P + 6) + dh : __ldg(P + 6) - dh;
    const double ox = px - __ldg(P), oy = py - __ldg(P + 1), oz = pz - __ldg(P + 2);
    const double bax = __ldg(P + 3), bay = __ldg(P + 4), baz = __ldg(P + 5), L2 = __ldg(P + 7);
    double a0, a1, b0, b1, c0, c1;
    ray_ball64(ox, oy, oz, rr, ux, uy, uz, a0, a1);
    ray_ball64(ox - bax, oy - bay, oz - baz, rr, ux, uy, uz, b0, b1);
    ray_cylinder64(ox, oy, oz, bax, bay, baz, L2, rr, ux, uy, uz, c0, c1);
    double t;
    if (d > 0.0) {
        t = __longlong_as_double(0x7ff0000000000000LL);
        if (a0 <= a1 && a1 >= 0.0) t = fmin(t, a0);
        if (b0 <= b1 && b1 >= 0.0) t = fmin(t, b0);
        if (c0 <= c1 && c1 >= 0.0) t = fmin(t, c0);
    } else {
        t = 0.0;
        if (a0 <= a1) t = fmax(t, a1);
        if (b0 <= b1) t = fmax(t, b1);
        if (c0 <= c1) t = fmax(t, c1);
    }
    return t > 0.0 ? t : 0.0;
}

// Capped cylinder along z (radius P[3], half height P[4]): the slab cut by
// the cylinder, grown by e from outside, shrunk by e from inside.
static __device__ __noinline__ double seg_cylinder64(const double *P, double d, double px, double py, double pz,
                                                     double ux, double uy, double uz, double e)
{
    const double g = d > 0.0 ? e : -e;
    const double rr = __ldg(P + 3) + g, hh = __ldg(P + 4) + g;
    double t0, t1;
    ray_cylinder64(px - __ldg(P), py - __ldg(P + 1), pz - __ldg(P + 2) + hh, 0.0, 0.0, 2.0 * hh, 4.0 * hh * hh, rr,
                   ux, uy, uz, t0, t1);
    if (d > 0.0) {
        if (!(t0 <= t1) || t1 < 0.0) return __longlong_as_double(0x7ff0000000000000LL);
        return t0 > 0.0 ? t0 : 0.0;
    }
    if (!(t0 <= t1)) return 0.0;
    return t1 > 0.0 ? t1 : 0.0;
}

// Torus about z (major radius P[3], tube P[4]) from outside: the first point
// of the ray in the annular slab that holds the tube grown by e, and never
// less than d - e.  From inside the tube: the exit of the ball of radius
// r - e about the point of the core circle nearest p, which the tube shrunk
// by e holds (on the axis: |d| - e).
static __device__ __noinline__ double seg_torus64(const double *P, double d, double px, double py, double pz,
                                                  double ux, double uy, double uz, double e)
{
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    if (d < 0.0) {
        const double dx = px - __ldg(P), dy = py - __ldg(P + 1);
        const double rho = sqrt(dx * dx + dy * dy);
        if (!(rho > 0.0)) return -d - e;
        const double cx = __ldg(P) + __ldg(P + 3) * dx / rho, cy = __ldg(P + 1) + __ldg(P + 3) * dy / rho;
        const double rr = __ldg(P + 4) - e;
        const double ox = px - cx, oy = py - cy, oz = pz - __ldg(P + 2);
        const double b = ox * ux + oy * uy + oz * uz;
        const double cc = ox * ox + oy * oy + oz * oz - rr * rr;
        const double disc = b * b - cc;
        if (disc < 0.0) return 0.0;
        double t;
        if (b > 0.0) t = -cc / (b + sqrt(disc));
        else t = sqrt(disc) - b;
        return t > 0.0 ? t : 0.0;
    }
    const double R = __ldg(P + 3), rt = __ldg(P + 4) + e;
    const double ox = px - __ldg(P), oy = py - __ldg(P + 1), oz = pz - __ldg(P + 2) + rt;
    double a0, a1;
    ray_cylinder64(ox, oy, oz, 0.0, 0.0, 2.0 * rt, 4.0 * rt * rt, R + rt, ux, uy, uz, a0, a1);
    double lo = fmax(a0, 0.0);
    const double hi = a1;
    if (!(lo <= hi)) return inf;
    if (R - rt > 0.0) {                  // the hole is not in the slab
        double b0, b1;
        ray_cylinder64(ox, oy, oz, 0.0, 0.0, 2.0 * rt, 4.0 * rt * rt, R - rt, ux, uy, uz, b0, b1);
        if (b0 <= lo && lo < b1) lo = b1;
        if (!(lo < hi)) return inf;
    }
    return fmax(lo, d - e);
}

// A primitive placed by a frame without a domain operation: the local ray
// q + (t / s) w (q = R^T (p - t) / s, w = R^T u) and the local bound of d / s
// with margin e / s, times s; other frames keep the isotropic bound.
static __device__ __noinline__ double seg_xprim64(const DevScene &S, int kind, int i, double d, double px,
                                                  double py, double pz, double ux, double uy, double uz,
                                                  double e)
{
    const double *X = S.xf64 + kXf64 * i;
    if ((int)__ldg(X + 13) != 0) return fabs(d) - e;
    const double vx = px - __ldg(X + 9), vy = py - __ldg(X + 10), vz = pz - __ldg(X + 11);
    const double s = __ldg(X + 12);
    const double q0 = (__ldg(X) * vx + __ldg(X + 3) * vy + __ldg(X + 6) * vz) / s;
    const double q1 = (__ldg(X + 1) * vx + __ldg(X + 4) * vy + __ldg(X + 7) * vz) / s;
    const double q2 = (__ldg(X + 2) * vx + __ldg(X + 5) * vy + __ldg(X + 8) * vz) / s;
    const double w0 = __ldg(X) * ux + __ldg(X + 3) * uy + __ldg(X + 6) * uz;
    const double w1 = __ldg(X + 1) * ux + __ldg(X + 4) * uy + __ldg(X + 7) * uz;
    const double w2 = __ldg(X + 2) * ux + __ldg(X + 5) * uy + __ldg(X + 8) * uz;
    const double dl = d / s, el = e / s;
    const double *P = S.p64 + 8 * i;
    double t;
    if (kind == 0) t = seg_sphere64(P, dl, q0, q1, q2, w0, w1, w2, el);
    else if (kind == 1)
        t = seg_box64(__ldg(P), __ldg(P + 1), __ldg(P + 2), __ldg(P + 3), __ldg(P + 4), __ldg(P + 5), dl, q0, q1, q2,
                      w0, w1, w2, el);
    else if (kind == 2) t = seg_capsule64(P, dl, q0, q1, q2, w0, w1, w2, el);
    else if (kind == 3) t = seg_torus64(P, dl, q0, q1, q2, w0, w1, w2, el);
    else t = seg_cylinder64(P, dl, q0, q1, q2, w0, w1, w2, el);
    return s * t;
}

// The move bound: the bounding box's exit, the soft regions' isotropic
// bound, then each listed primitive with margin e = m + delta/2 (its
// regions' sum of k/4): 0 when |d| <= e, passed over when |d| - e cannot
// lower the bound so far, else its ray bound.
template <bool G>
static __device__ __noinline__ double segment_bound64(const DevScene &S, double dsoft, double dbox, double px,
                                                      double py, double pz, double ux, double uy, double uz)
{
    const double dh = 0.5 * S.delta;
    double t = fmin(seg_box64(S.bbc[0], S.bbc[1], S.bbc[2], S.bbh[0], S.bbh[1], S.bbh[2], dbox, px, py, pz, ux, uy,
                              uz, dh),
                    dsoft - dh);
    for (int j = 0; j < S.nseg; ++j) {
        const int i = __ldg(S.seg_prims + j);
        const int kind = (*(S.pkind + i));
        const double e = __ldg(S.seg_m64 + j) + dh;
        const double d = prim64<G>(S, kind, i, px, py, pz);
        if (!(fabs(d) > e)) return 0.0;
        if (fabs(d) - e >= t) continue;
        double b;
        if (kind == 0) {
            b = seg_sphere64(S.p64 + 8 * i, d, px, py, pz, ux, uy, uz, e);
        } else if (kind == 1) {
            const double *P = S.p64 + 8 * i;
            b = seg_box64(__ldg(P), __ldg(P + 1), __ldg(P + 2), __ldg(P + 3), __ldg(P + 4), __ldg(P + 5), d, px,
                          py, pz, ux, uy, uz, e);
        } else if (!G || kind == 2) {
            b = seg_capsule64(S.p64 + 8 * i, d, px, py, pz, ux, uy, uz, e);
        } else if (kind & kXformFlag) {
            b = seg_xprim64(S, kind & 0xf, i, d, px, py, pz, ux, uy, uz, e);
        } else if (kind == 3) {
            b = seg_torus64(S.p64 + 8 * i, d, px, py, pz, ux, uy, uz, e);
        } else {
            b = seg_cylinder64(S.p64 + 8 * i, d, px, py, pz, ux, uy, uz, e);
        }
        t = fmin(t, b);
    }
    return t;
}

// FP32 (mixed): the same bounds with reciprocal directions.
__device__ __forceinline__ float seg_sphere32(float4 A, float d, float px, float py, float pz, float ux, float uy,
                                              float uz, float dh)
{
    const float rr = d > 0.f ? A.w + dh : A.w - dh;
    const float ox = px - A.x, oy = py - A.y, oz = pz - A.z;
    const float b = ox * ux + oy * uy + oz * uz;
    const float cc = ox * ox + oy * oy + oz * oz - rr * rr;
    const float disc = b * b - cc;
    float t;
    if (d > 0.f) {
        if (b >= 0.f || disc < 0.f) return __int_as_float(0x7f800000);
        t = cc / (sqrtf(disc) - b);
    } else {
        if (disc < 0.f) return 0.f;
        t = b > 0.f ? -cc / (b + sqrtf(disc)) : sqrtf(disc) - b;
    }
    return t > 0.f ? t : 0.f;
}

__device__ __forceinline__ float seg_box32(float cx, float cy, float cz, float hx, float hy, float hz, float d,
                                           float px, float py, float pz, float ux, float uy, float uz, float iux,
                                           float iuy, float iuz, float dh)
{
    const float inf = __int_as_float(0x7f800000);
    const float e = d > 0.f ? dh : -dh;
    const float c[3] = {cx, cy, cz}, h[3] = {hx, hy, hz}, p[3] = {px, py, pz}, u[3] = {ux, uy, uz};
    const float iu[3] = {iux, iuy, iuz};
    float tn = -inf, tf = inf;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = c[a] - (h[a] + e), hi = c[a] + (h[a] + e);
        if (u[a] != 0.f) {
            const float t0 = (lo - p[a]) * iu[a], t1 = (hi - p[a]) * iu[a];
            tn = fmaxf(tn, fminf(t0, t1));
            tf = fminf(tf, fmaxf(t0, t1));
        } else if (p[a] < lo || p[a] > hi) {
            return d > 0.f ? inf : 0.f;
        }
    }
    if (d > 0.f) {
        if (tn > tf || tf < 0.f) return inf;
        return tn > 0.f ? tn : 0.f;
    }
    return tf > 0.f ? tf : 0.f;
}

__device__ __forceinline__ void ray_ball32(float ox, float oy, float oz, float rr, float ux, float uy, float uz,
                                           float &t0, float &t1)
{
    const float b = ox * ux + oy * uy + oz * uz;
    const float cc = ox * ox + oy * oy + oz * oz - rr * rr;
    const float disc = b * b - cc;
    t0 = __int_as_float(0x7f800000);
    t1 = -t0;
    if (disc < 0.f) return;
    const float sq = sqrtf(disc);
    if (b > 0.f) {
        const float q = -(b + sq);
        t0 = q; t1 = cc / q;
    } else {
        const float q = sq - b;
        if (q > 0.f) { t1 = q; t0 = cc / q; }
        else { t0 = 0.f; t1 = 0.f; }
    }
}

__device__ __forceinline__ void ray_cylinder32(float ox, float oy, float oz, float bax, float bay, float baz,
                                               float iL2, float rr, float ux, float uy, float uz, float &t0,
                                               float &t1)
{
    const float inf = __int_as_float(0x7f800000);
    const float L2 = bax * bax + bay * bay + baz * baz;
    const float uw = ux * bax + uy * bay + uz * baz;
    const float ow = ox * bax + oy * bay + oz * baz;
    float lo = -inf, hi = inf;
    t0 = inf; t1 = -inf;
    if (uw != 0.f) {
        const float s0 = -ow / uw, s1 = (L2 - ow) / uw;
        lo = fminf(s0, s1); hi = fmaxf(s0, s1);
    } else if (ow < 0.f || ow > L2) {
        return;
    }
    const float k = uw * iL2, m = ow * iL2;
    const float vx = ux - k * bax, vy = uy - k * bay, vz = uz - k * baz;
    const float wx = ox - m * bax, wy = oy - m * bay, wz = oz - m * baz;
    const float A = vx * vx + vy * vy + vz * vz;
    const float B = wx * vx + wy * vy + wz * vz;
    const float C = wx * wx + wy * wy + wz * wz - rr * rr;
    if (A > 0.f) {
        const float disc = B * B - A * C;
        if (disc < 0.f) return;
        const float sq = sqrtf(disc);
        float c0, c1;
        if (B > 0.f) {
            const float q = -(B + sq);
            c0 = q / A; c1 = C / q;
        } else {
            const float q = sq - B;
            if (q > 0.f) { c1 = q / A; c0 = C / q; }
            else { c0 = 0.f; c1 = 0.f; }
        }
        lo = fmaxf(lo, c0); hi = fminf(hi, c1);
    } else if (C > 0.f) {
        return;
    }
    t0 = lo; t1 = hi;
}

// FP32 capsule bound; the tables hold (a, r) and (b - a, 1 / |b - a|^2).
static __device__ __noinline__ float seg_capsule32(float4 A, float4 Bv, float d, float px, float py, float pz,
                                               float ux, float uy, float uz, float dh)
{
    const float rr = d > 0.f ? A.w + dh : A.w - dh;
    const float ox = px - A.x, oy = py - A.y, oz = pz - A.z;
    float a0, a1, b0, b1, c0, c1;
    ray_ball32(ox, oy, oz, rr, ux, uy, uz, a0, a1);
    ray_ball32(ox - Bv.x, oy - Bv.y, oz - Bv.z, rr, ux, uy, uz, b0, b1);
    ray_cylinder32(ox, oy, oz, Bv.x, Bv.y, Bv.z, Bv.w, rr, ux, uy, uz, c0, c1);
    float t;
    if (d > 0.f) {
        t = __int_as_float(0x7f800000);
        if (a0 <= a1 && a1 >= 0.f) t = fminf(t, a0);
        if (b0 <= b1 && b1 >= 0.f) t = fminf(t, b0);
        if (c0 <= c1 && c1 >= 0.f) t = fminf(t, c0);
    } else {
        t = 0.f;
        if (a0 <= a1) t = fmaxf(t, a1);
        if (b0 <= b1) t = fmaxf(t, b1);
        if (c0 <= c1) t = fmaxf(t, c1);
    }
    return t > 0.f ? t : 0.f;
}

// FP32 capped cylinder (kind 4) and torus (kind 3) bounds, the FP64 rules
// above; the tables hold (c, R or radius) and (tube radius or half height).
static __device__ __noinline__ float seg_round32(int kind, const float4 *P, float d, float px, float py, float pz,
                                                 float ux, float uy, float uz, float e)
{
    const float inf = __int_as_float(0x7f800000);
    const float4 A = (*(P)), B = (*(P + 1));
    if (kind == 3) {
        if (d < 0.f) {                   // inside: the ball about the nearest core-circle point
            const float dx = px - A.x, dy = py - A.y;
            const float rho = sqrtf(dx * dx + dy * dy);
            if (!(rho > 0.f)) return -d - e;
            const float cx = A.x + A.w * dx / rho, cy = A.y + A.w * dy / rho;
            const float rr = B.x - e;
            const float ox = px - cx, oy = py - cy, oz = pz - A.z;
            const float b = ox * ux + oy * uy + oz * uz;
            const float cc = ox * ox + oy * oy + oz * oz - rr * rr;
            const float disc = b * b - cc;
            if (disc < 0.f) return 0.f;
            const float t = b > 0.f ? -cc / (b + sqrtf(disc)) : sqrtf(disc) - b;
            return t > 0.f ? t : 0.f;
        }
        const float R = A.w, rt = B.x + e;
        const float ox = px - A.x, oy = py - A.y, oz = pz - A.z + rt;
        const float iL2 = 1.0f / (4.f * rt * rt);
        float a0, a1;
        ray_cylinder32(ox, oy, oz, 0.f, 0.f, 2.f * rt, iL2, R + rt, ux, uy, uz, a0, a1);
        float lo = fmaxf(a0, 0.f);
        const float hi = a1;
        if (!(lo <= hi)) return inf;
        if (R - rt > 0.f) {
            float b0, b1;
            ray_cylinder32(ox, oy, oz, 0.f, 0.f, 2.f * rt, iL2, R - rt, ux, uy, uz, b0, b1);
            if (b0 <= lo && lo < b1) lo = b1;
            if (!(lo < hi)) return inf;
        }
        return fmaxf(lo, d - e);
    }
    const float g = d > 0.f ? e : -e;
    const float rr = A.w + g, hh = B.x + g;
    float t0, t1;
    ray_cylinder32(px - A.x, py - A.y, pz - A.z + hh, 0.f, 0.f, 2.f * hh, 1.0f / (4.f * hh * hh), rr, ux, uy, uz,
                   t0, t1);
    if (d > 0.f) {
        if (!(t0 <= t1) || t1 < 0.f) return inf;
        return t0 > 0.f ? t0 : 0.f;
    }
    if (!(t0 <= t1)) return 0.f;
    return t1 > 0.f ? t1 : 0.f;
}

// FP32 placed primitive (frame without a domain operation).
static __device__ __noinline__ float seg_xprim32(const DevScene &S, int kind, int i, float d, float px, float py,
                                                 float pz, float ux, float uy, float uz, float e)
{
    const float4 *X = S.xf32 + kXf32 * i;
    const float4 R0 = __ldg(X), R1 = __ldg(X + 1), R2 = __ldg(X + 2), SC = __ldg(X + 3);
    if ((int)SC.z != 0) return fabsf(d) - e;
    const float vx = px - R0.w, vy = py - R1.w, vz = pz - R2.w;
    const float q0 = (R0.x * vx + R0.y * vy + R0.z * vz) * SC.y;
    const float q1 = (R1.x * vx + R1.y * vy + R1.z * vz) * SC.y;
    const float q2 = (R2.x * vx + R2.y * vy + R2.z * vz) * SC.y;
    const float w0 = R0.x * ux + R0.y * uy + R0.z * uz;
    const float w1 = R1.x * ux + R1.y * uy + R1.z * uz;
    const float w2 = R2.x * ux + R2.y * uy + R2.z * uz;
    const float dl = d * SC.y, el = e * SC.y;
    const float4 A = (*(S.p32 + 2 * i)), B = (*(S.p32 + 2 * i + 1));
    float t;
    if (kind == 0) t = seg_sphere32(A, dl, q0, q1, q2, w0, w1, w2, el);
    else if (kind == 1)
        t = seg_box32(A.x, A.y, A.z, B.x, B.y, B.z, dl, q0, q1, q2, w0, w1, w2, 1.0f / w0, 1.0f / w1, 1.0f / w2, el);
    else if (kind == 2) t = seg_capsule32(A, B, dl, q0, q1, q2, w0, w1, w2, el);
    else t = seg_round32(kind, S.p32 + 2 * i, dl, q0, q1, q2, w0, w1, w2, el);
    return SC.x * t;
}

// The move bound: the FP64 rule, with the culled region's distance (mixed)
// among the soft regions' isotropic bounds.  Measured on the vessel tree: a
// bound over the culled cell's candidates along the ray, or only the cell's
// exit, cut the steps per packet (132 to 117-118) but made each packet
// slower (cycles per packet +15 % with the cell's exit alone, +42 % with the
// candidates); most of the loss came with the longer, more uneven moves'
// tally (without a fluence grid the cell's exit alone cost 4 %).  The
// isotropic bound is kept.
template <bool G>
static __device__ __noinline__ float segment_bound32(const DevScene &S, float dsoft, float dbox, float px,
                                                     float py, float pz, float ux, float uy, float uz)
{
    const float dh = 0.5f * S.delta32;
    const float iux = 1.0f / ux, iuy = 1.0f / uy, iuz = 1.0f / uz;
    float t = fminf(seg_box32(S.bbc32[0], S.bbc32[1], S.bbc32[2], S.bbh32[0], S.bbh32[1], S.bbh32[2], dbox, px, py,
                              pz, ux, uy, uz, iux, iuy, iuz, dh),
                    dsoft - dh);
    for (int j = 0; j < S.nseg; ++j) {
        const int i = __ldg(S.seg_prims + j);
        const int kind = (*(S.pkind + i));
        const float e = __ldg(S.seg_m32 + j) + dh;
        const float d = prim32<G>(S, kind, i, px, py, pz);
        if (!(fabsf(d) > e)) return 0.f;
        if (fabsf(d) - e >= t) continue;
        float b;
        if (kind == 0) {
            b = seg_sphere32((*(S.p32 + 2 * i)), d, px, py, pz, ux, uy, uz, e);
        } else if (kind == 1) {
            const float4 A = (*(S.p32 + 2 * i)), B = (*(S.p32 + 2 * i + 1));
            b = seg_box32(A.x, A.y, A.z, B.x, B.y, B.z, d, px, py, pz, ux, uy, uz, iux, iuy, iuz, e);
        } else if (!G || kind == 2) {
            b = seg_capsule32((*(S.p32 + 2 * i)), (*(S.p32 + 2 * i + 1)), d, px, py, pz, ux, uy, uz, e);
        } else if (kind & kXformFlag) {
            b = seg_xprim32(S, kind & 0xf, i, d, px, py, pz, ux, uy, uz, e);
        } else {
            b = seg_round32(kind, S.p32 + 2 * i, d, px, py, pz, ux, uy, uz, e);
        }
        t = fminf(t, b);
    }
    return t;
}

// ---------------------------------------------------------------------------
// Track-length tally (Sec. 3.1-3.2): 3D DDA over the grid (Amanatides & Woo
// 1987), distance to each axis' next plane recomputed from the segment
// start; each piece adds round(w * piece * 2^32) to its voxel atomically.
// Per-axis state lives in scalars (no dynamically indexed arrays, which
// would be placed in local memory); ties advance x before y before z.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add(long long *a, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(a), (unsigned long long)v);
}

// FP64: the reference's arithmetic, operation for operation.
__device__ __forceinline__ bool clip64(double lo, double hi, double p, double u, double &tin, double &tout)
{
    if (u != 0.0) {
        const double t0 = (lo - p) / u;
        const double t1 = (hi - p) / u;
        tin = fmax(tin, fmin(t0, t1));
        tout = fmin(tout, fmax(t0, t1));
        return true;
    }
    return !(p < lo || p > hi);
}

__device__ __forceinline__ void dda_axis64(double lo, double dl, int n, double p, double u, double tin, int &i,
                                           double &tn)
{
    const double xa = p + tin * u;
    const double f = floor((xa - lo) / dl);
    i = (int)fmin(fmax(f, 0.0), (double)(n - 1));
    if (u > 0.0)
        tn = ((lo + (double)(i + 1) * dl) - p) / u;
    else if (u < 0.0)
        tn = ((lo + (double)i * dl) - p) / u;
    else
        tn = __longlong_as_double(0x7ff0000000000000LL);
}

static __device__ __noinline__ void tally64(const DevScene &S, long long *flu, double px, double py, double pz,
                                            double ux, double uy, double uz, double len, double w,
                                            unsigned *npieces)
{
    if (!(len > 0.0) || !(w > 0.0)) return;
    double tin = 0.0, tout = len;
    if (!clip64(S.g_lo[0], S.g_hi[0], px, ux, tin, tout)) return;
    if (!clip64(S.g_lo[1], S.g_hi[1], py, uy, tin, tout)) return;
    if (!clip64(S.g_lo[2], S.g_hi[2], pz, uz, tin, tout)) return;
    if (!(tin < tout)) return;
    const int nx = S.g_n[0], ny = S.g_n[1], nz = S.g_n[2];
    int ix, iy, iz;
    double tx, ty, tz;
    dda_axis64(S.g_lo[0], S.g_dl[0], nx, px, ux, tin, ix, tx);
    dda_axis64(S.g_lo[1], S.g_dl[1], ny, py, uy, tin, iy, ty);
    dda_axis64(S.g_lo[2], S.g_dl[2], nz, pz, uz, tin, iz, tz);
    double t = tin;
    int guard = nx + ny + nz + 3;
    while (guard-- > 0) {
        const int ax = (tx <= ty && tx <= tz) ? 0 : ((ty <= tz) ? 1 : 2);
        const double ta = ax == 0 ? tx : (ax == 1 ? ty : tz);
        const double tend = fmin(ta, tout);
        const double piece = tend - t;
        if (piece > 0.0) {
            const long long off = ((long long)iz * ny + iy) * nx + ix;
            red_add(flu + off, fx64(w * piece));
            *npieces += 1u;
            t = tend;
        }
        if (ta >= tout) break;
        if (ax == 0) {
            ix += ux > 0.0 ? 1 : -1;
            if (ix < 0 || ix >= nx) break;
            tx = ux > 0.0 ? ((S.g_lo[0] + (double)(ix + 1) * S.g_dl[0]) - px) / ux
                          : ((S.g_lo[0] + (double)ix * S.g_dl[0]) - px) / ux;
        } else if (ax == 1) {
            iy += uy > 0.0 ? 1 : -1;
            if (iy < 0 || iy >= ny) break;
            ty = uy > 0.0 ? ((S.g_lo[1] + (double)(iy + 1) * S.g_dl[1]) - py) / uy
                          : ((S.g_lo[1] + (double)iy * S.g_dl[1]) - py) / uy;
        } else {
            iz += uz > 0.0 ? 1 : -1;
            if (iz < 0 || iz >= nz) break;
            tz = uz > 0.0 ? ((S.g_lo[2] + (double)(iz + 1) * S.g_dl[2]) - pz) / uz
                          : ((S.g_lo[2] + (double)iz * S.g_dl[2]) - pz) / uz;
        }
    }
}

// FP32 (mixed): reciprocal directions, incremental voxel offset.
__device__ __forceinline__ bool clip32(float lo, float hi, float p, float iu, bool nz_, float &tin, float &tout)
{
    if (nz_) {
        const float t0 = (lo - p) * iu;
        const float t1 = (hi - p) * iu;
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
        return true;
    }
    return !(p < lo || p > hi);
}

__device__ __forceinline__ void tally32(const DevScene &S, long long *flu, float px, float py, float pz,
                                        float ux, float uy, float uz, float len, float w,
                                        unsigned *npieces)
{
    // FP32: the distance to the next plane of each axis advances by one
    // voxel's crossing time per step (no re-derivation from the segment
    // start), and the step is branch-free across the three axes, so lanes
    // of a warp stepping along different axes do not serialise.
    if (!(len > 0.f) || !(w > 0.f)) return;
    const float iux = 1.0f / ux, iuy = 1.0f / uy, iuz = 1.0f / uz;
    float tin = 0.f, tout = len;
    if (!clip32(S.g_lo32[0], S.g_hi32[0], px, iux, ux != 0.f, tin, tout)) return;
    if (!clip32(S.g_lo32[1], S.g_hi32[1], py, iuy, uy != 0.f, tin, tout)) return;
    if (!clip32(S.g_lo32[2], S.g_hi32[2], pz, iuz, uz != 0.f, tin, tout)) return;
    if (!(tin < tout)) return;
    const int nx = S.g_n[0], ny = S.g_n[1], nz = S.g_n[2];
    const float inf = __int_as_float(0x7f800000);
    const float lx = S.g_lo32[0], ly = S.g_lo32[1], lz = S.g_lo32[2];
    const float dx = S.g_dl32[0], dy = S.g_dl32[1], dz = S.g_dl32[2];
    int ix = min(max(__float2int_rd((__fmaf_rn(tin, ux, px) - lx) * S.g_idl32[0]), 0), nx - 1);
    int iy = min(max(__float2int_rd((__fmaf_rn(tin, uy, py) - ly) * S.g_idl32[1]), 0), ny - 1);
    int iz = min(max(__float2int_rd((__fmaf_rn(tin, uz, pz) - lz) * S.g_idl32[2]), 0), nz - 1);
    const int sx = ux > 0.f ? 1 : -1, sy = uy > 0.f ? 1 : -1, sz = uz > 0.f ? 1 : -1;
    float tx = ux != 0.f ? (__fmaf_rn((float)(ix + (sx > 0)), dx, lx) - px) * iux : inf;
    float ty = uy != 0.f ? (__fmaf_rn((float)(iy + (sy > 0)), dy, ly) - py) * iuy : inf;
    float tz = uz != 0.f ? (__fmaf_rn((float)(iz + (sz > 0)), dz, lz) - pz) * iuz : inf;
    const float tdx = ux != 0.f ? dx * fabsf(iux) : inf;
    const float tdy = uy != 0.f ? dy * fabsf(iuy) : inf;
    const float tdz = uz != 0.f ? dz * fabsf(iuz) : inf;
    long long off = ((long long)iz * ny + iy) * nx + ix;
    const long long ox = sx, oy = sy > 0 ? nx : -nx, oz = sz > 0 ? (long long)nx * ny : -(long long)nx * ny;
    // remaining planes along each axis before the grid ends
    const int rx = sx > 0 ? nx - 1 - ix : ix, ry = sy > 0 ? ny - 1 - iy : iy, rz = sz > 0 ? nz - 1 - iz : iz;
    int cx = 0, cy = 0, cz = 0;
    float t = tin;
    for (int guard = nx + ny + nz + 3; guard > 0; --guard) {
        const bool bx = tx <= ty && tx <= tz;
        const bool by = !bx && ty <= tz;
        const bool bz = !bx && !by;
        const float ta = fminf(tx, fminf(ty, tz));
        const float tend = fminf(ta, tout);
        const float piece = tend - t;
        if (piece > 0.f) {
            red_add(flu + off, fx32(w * piece));
            *npieces += 1u;
            t = tend;
        }
        if (ta >= tout) break;
        // step to the next voxel along the axis whose plane came first
        cx += bx; cy += by; cz += bz;
        if (cx > rx || cy > ry || cz > rz) break;
        off += bx ? ox : (by ? oy : oz);
        tx += bx ? tdx : 0.f;
        ty += by ? tdy : 0.f;
        tz += bz ? tdz : 0.f;
    }
}

// ---------------------------------------------------------------------------
// Orthonormal basis perpendicular to a unit vector: branchless construction
// of Duff et al., "Building an Orthonormal Basis, Revisited", JCGT 2017.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void onb64(double nx, double ny, double nz, double b1[3], double b2[3])
{
    const double sg = copysign(1.0, nz);
    const double a = -1.0 / (sg + nz);
    const double b = nx * ny * a;
    b1[0] = 1.0 + sg * nx * nx * a; b1[1] = sg * b; b1[2] = -sg * nx;
    b2[0] = b; b2[1] = sg + ny * ny * a; b2[2] = -ny;
}

__device__ __forceinline__ void onb32(float nx, float ny, float nz, float b1[3], float b2[3])
{
    const float sg = copysignf(1.f, nz);
    const float a = -1.f / (sg + nz);
    const float b = nx * ny * a;
    b1[0] = 1.f + sg * nx * nx * a; b1[1] = sg * b; b1[2] = -sg * nx;
    b2[0] = b; b2[1] = sg + ny * ny * a; b2[2] = -ny;
}

// ---------------------------------------------------------------------------
// Tally accumulators.  Frequent per-lane counters stay in registers; the
// rest are summed per warp in shared memory (slot i mirrors the i-th int64
// of smcrt_totals) and flushed to the job's totals when the warp leaves it.
// ---------------------------------------------------------------------------
enum TotSlot {
    kR = 0, kT, kA, kKilled, kGain, kPackets, kScat, kSteps, kEvals, kIntf, kFres, kPieces, kCap, kRefined,
    kBusy, kParked, kNumSlots = 16
};

struct WarpAcc {
    unsigned long long v[kNumSlots];
};

__device__ __forceinline__ void wadd(WarpAcc *a, int slot, long long x)
{
    if (x != 0) atomicAdd(&a->v[slot], (unsigned long long)x);
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(SMCRT_FULL, v, o);
    return v;
}

__device__ __forceinline__ void wacc_clear(WarpAcc *a, int lane)
{
    if (lane < kNumSlots) a->v[lane] = 0ull;
    __syncwarp();
}

__device__ __forceinline__ void wacc_flush(WarpAcc *a, smcrt_totals *t, int lane)
{
    __syncwarp();
    if (lane < kNumSlots) {
        const unsigned long long x = a->v[lane];
        if (x) red_add(reinterpret_cast<long long *>(t) + lane, (long long)x);
    }
    __syncwarp();
}

// Per-job constants of the warp's current job, kept in shared memory and
// read where used (volatile), so they do not occupy registers across the
// packet loop.
struct JobConst {
    unsigned long long flu, recs, end, begin, dfr;
    unsigned long long deadline;   // global timer (ns) after which the warp stops the job (0 = never)
    uint32_t k0, k1;
    int32_t din;
    uint32_t budget;          // park after this many clock() cycles (0 = never)
    uint32_t drain;           // ... or after this many once the warp has no more work (0 = budget)
};

// The GPU's global nanosecond timer (the same clock on every SM).
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device-side time limit of a launch, checked where a warp claims new
// packet ids (no cost in the packet loop itself): past the job's deadline
// the warp claims no more ids, the packets it holds finish as usual (each
// bounded by the step cap), and the warp returns.  The totals and the
// fluence then cover exactly the packets counted.
__device__ __forceinline__ bool past_deadline(const volatile JobConst *jc)
{
    const unsigned long long dl = jc->deadline;
    return dl != 0ull && globaltimer_ns() > dl;
}

__device__ __forceinline__ void jobconst_fill(volatile JobConst *jc, const JobWork *J)
{
    jc->flu = (unsigned long long)J->fluence;
    jc->recs = (unsigned long long)J->records;
    jc->end = J->end;
    jc->begin = J->begin;
    jc->dfr = (unsigned long long)J->defer;
    jc->k0 = (uint32_t)J->seed;
    jc->k1 = (uint32_t)(J->seed >> 32);
    jc->din = J->defer_in & 1;
    const long long b = J->defer != nullptr ? J->park_cycles : 0;
    jc->budget = (uint32_t)(b > 0x7fffffffLL ? 0x7fffffffLL : (b < 0 ? 0 : b));
    const long long dr = J->defer != nullptr && J->drain_cycles > 0 ? J->drain_cycles : b;
    jc->drain = (uint32_t)(dr > 0x7fffffffLL ? 0x7fffffffLL : (dr < 0 ? 0 : dr));
    jc->deadline = J->time_limit_ns > 0ull ? globaltimer_ns() + J->time_limit_ns : 0ull;
}

enum Phase { kTrace = 0, kNrm = 1, kProj = 2, kFar = 3, kNear = 4, kLaunch = 5 };

constexpr double kWRoulette = 1e-4;   // roulette threshold (MCML convention)
constexpr double kRouletteM = 10.0;   // survival 1/m, weight x m

}  // namespace smcrt
