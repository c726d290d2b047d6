// smcrt_internal.h -- structures shared by the host runtime (smcrt_api.cpp)
// and the two packet-kernel translation units (FP64 and mixed precision).
// Not part of the public C-ABI.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/smcrt.h"

namespace smcrt {

constexpr int kMaxStack = 4;      // CSG register stack depth on the device
constexpr int kMaxRegions = 64;
constexpr int kMaxPrims = 4096;
constexpr int kMaxGridSide = 1024;
constexpr int kMaxThreads = 128;
// Longest region program (instructions) whose normal the mixed kernel takes
// from the analytic SDF gradient; longer programs use six shared probes.
constexpr int kAnalyticNormalMaxInstr = 4;
// Fold regions with at least this many primitives get a culling grid.
constexpr int kCullMinPrims = 16;
// Cells per axis of the culling grid.  Finer cells list fewer candidates (the
// reach R is one cell): on the 64-capsule vessel scene 32 cells per axis
// beat 16 by 11 % with segment stepping and 22 % with sphere tracing.
constexpr int kCullGrid = 32;

// Device primitive kind: the smcrt_prim_kind, plus this bit when the
// primitive is evaluated in its own frame (smcrt_xform).  Instr.op carries
// it in bits 8..15, the DevScene.pkind table as is.
constexpr int32_t kXformFlag = 0x10;
constexpr int kXf64 = 20;   // doubles per primitive frame: R (9), t (3), s, op, a (4), 2 unused
constexpr int kXf32 = 5;    // float4 per primitive frame: R^T rows | t, (s, 1/s, op, 0), a

inline int32_t device_kind(const smcrt_prim &P) { return P.kind | (P.xform > 0 ? kXformFlag : 0); }

// The tables of primitive i: FP64 (8 doubles), FP32 (2 float4), and, when
// xd / xf are given and the primitive has a frame, the frame (kXf64 doubles,
// kXf32 float4).  Doubles are the caller's values or the reference's
// expressions (capsule: b - a and |b - a|^2), so the FP64 kernel computes
// with the same numbers as the oracle.
inline void fill_prim(const smcrt_scene *sc, int i, double *d, float4 *f, double *xd, float4 *xf)
{
    const smcrt_prim &P = sc->prims[i];
    for (int k = 0; k < 8; ++k) d[k] = 0.0;
    f[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    f[1] = f[0];
    if (P.kind == SMCRT_CAPSULE) {
        const double bax = P.p[3] - P.p[0], bay = P.p[4] - P.p[1], baz = P.p[5] - P.p[2];
        const double baba = bax * bax + bay * bay + baz * baz;
        d[0] = P.p[0]; d[1] = P.p[1]; d[2] = P.p[2];
        d[3] = bax; d[4] = bay; d[5] = baz; d[6] = P.p[6]; d[7] = baba;
        f[0] = make_float4((float)P.p[0], (float)P.p[1], (float)P.p[2], (float)P.p[6]);
        f[1] = make_float4((float)bax, (float)bay, (float)baz, (float)(1.0 / baba));
    } else if (P.kind == SMCRT_BOX) {
        for (int k = 0; k < 6; ++k) d[k] = P.p[k];
        f[0] = make_float4((float)P.p[0], (float)P.p[1], (float)P.p[2], 0.f);
        f[1] = make_float4((float)P.p[3], (float)P.p[4], (float)P.p[5], 0.f);
    } else if (P.kind == SMCRT_TORUS || P.kind == SMCRT_CYLINDER) {
        for (int k = 0; k < 5; ++k) d[k] = P.p[k];
        f[0] = make_float4((float)P.p[0], (float)P.p[1], (float)P.p[2], (float)P.p[3]);
        f[1] = make_float4((float)P.p[4], 0.f, 0.f, 0.f);
    } else {
        for (int k = 0; k < 4; ++k) d[k] = P.p[k];
        f[0] = make_float4((float)P.p[0], (float)P.p[1], (float)P.p[2], (float)P.p[3]);
    }
    if (xd == nullptr || xf == nullptr) return;
    for (int k = 0; k < kXf64; ++k) xd[k] = 0.0;
    for (int k = 0; k < kXf32; ++k) xf[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P.xform <= 0) return;
    const smcrt_xform &X = sc->xforms[P.xform - 1];
    for (int k = 0; k < 9; ++k) xd[k] = X.rot[k];
    for (int k = 0; k < 3; ++k) xd[9 + k] = X.t[k];
    xd[12] = X.s;
    xd[13] = (double)X.op;
    for (int k = 0; k < 4; ++k) xd[14 + k] = X.a[k];
    const double *R = X.rot;
    xf[0] = make_float4((float)R[0], (float)R[3], (float)R[6], (float)X.t[0]);
    xf[1] = make_float4((float)R[1], (float)R[4], (float)R[7], (float)X.t[1]);
    xf[2] = make_float4((float)R[2], (float)R[5], (float)R[8], (float)X.t[2]);
    xf[3] = make_float4((float)X.s, (float)(1.0 / X.s), (float)X.op, 0.f);
    xf[4] = make_float4((float)X.a[0], (float)X.a[1], (float)X.a[2], (float)X.a[3]);
}

// Primitives the mixed kernel's analytic normal and the culling grid handle:
// sphere, box, capsule in scene coordinates.
inline bool plain_prim(const smcrt_prim &P) { return P.kind <= SMCRT_CAPSULE && P.xform <= 0; }

// Segment stepping bounds a region by rays to its primitives, widened by a
// margin of k/4 per smooth union (a smooth union lies at most k/4 below
// min, and min, max and subtraction move by at most their operands'
// change, so the region's surface lies where some primitive has |d| <= the
// sum).  A region with more smooth unions than kSegMaxSmooth ("soft") keeps
// the isotropic bound |d| - delta/2; the last instruction of its program
// carries kSoftRegionEnd in Instr.op.
constexpr int kSegMaxSmooth = 8;
constexpr int32_t kSoftRegionEnd = 0x10000;

inline bool region_is_soft(const smcrt_scene *sc, int r)
{
    const smcrt_region &R = sc->regions[r];
    int n = 0;
    for (int i = 0; i < R.node_count; ++i)
        if (sc->nodes[R.node_begin + i].op == SMCRT_OP_SMOOTH_UNION) ++n;
    return n > kSegMaxSmooth;
}

// Sum of k/4 over region r's smooth unions, in program order (0: hard CSG).
inline double region_margin(const smcrt_scene *sc, int r)
{
    const smcrt_region &R = sc->regions[r];
    double m = 0.0;
    for (int i = 0; i < R.node_count; ++i)
        if (sc->nodes[R.node_begin + i].op == SMCRT_OP_SMOOTH_UNION) m = m + 0.25 * sc->nodes[R.node_begin + i].k;
    return m;
}

// The primitives whose offset surfaces bound a segment-stepping move: the
// distinct primitives of the regions that are not soft, in first-use order,
// each with the largest margin of those regions that use it.  skip_region
// (the mixed kernel's culled region) is left out: its culled distance
// bounds moves isotropically (ray bounds over all its primitives would undo
// the culling).  Writes at most kMaxPrims entries; no allocation.
inline int seg_entries(const smcrt_scene *sc, int32_t *out, double *margin, int skip_region = -1)
{
    uint64_t seen[kMaxPrims / 64] = {};
    int n = 0;
    for (int r = 0; r < sc->nregions; ++r) {
        if (r == skip_region || region_is_soft(sc, r)) continue;
        const smcrt_region &R = sc->regions[r];
        for (int i = 0; i < R.node_count; ++i) {
            const smcrt_csg_node &nd = sc->nodes[R.node_begin + i];
            if (nd.op != SMCRT_OP_PRIM || nd.prim < 0 || nd.prim >= kMaxPrims) continue;
            const uint64_t bit = 1ull << (nd.prim & 63);
            if (seen[nd.prim >> 6] & bit) continue;
            seen[nd.prim >> 6] |= bit;
            double m = 0.0;
            for (int r2 = 0; r2 < sc->nregions; ++r2) {
                if (r2 == skip_region || region_is_soft(sc, r2)) continue;
                const smcrt_region &Q = sc->regions[r2];
                for (int j = 0; j < Q.node_count; ++j)
                    if (sc->nodes[Q.node_begin + j].op == SMCRT_OP_PRIM && sc->nodes[Q.node_begin + j].prim == nd.prim) {
                        m = std::fmax(m, region_margin(sc, r2));
                        break;
                    }
            }
            margin[n] = m;
            out[n++] = nd.prim;
        }
    }
    return n;
}

// Device instruction (compiled CSG program).  op: 0 push primitive;
// 1 union, 2 smooth union, 3 intersect, 4 subtract.  prim >= 0 with a
// binary op means "combine the stack top (left) with this primitive
// (right)"; prim < 0 with a binary op combines the top two stack entries.
// region >= 0 marks the last instruction of that region's program.
struct Instr {
    int32_t op;
    int32_t prim;
    int32_t region;
    int32_t pad;
};

// Scene + source + grid of one plan as the kernels read them.  Lives in
// device memory; each warp stages a copy in shared memory when it starts
// on a job.  All double fields are computed on the host with the same
// expressions the FP64 reference uses, so the FP64 kernel sees identical
// values.
struct DevScene {
    // instruction stream and primitive tables (device pointers)
    const Instr *instr;
    const double *k64;        // smooth radius per instruction
    const float *kinv32;      // 1/k per instruction (FP32 path)
    const int32_t *pkind;     // per primitive: 0 sphere, 1 box, 2 capsule
    const double *p64;        // 8 per primitive (capsule: a, b-a, r, |b-a|^2)
    const float4 *p32;        // 2 per primitive (capsule: a|r, b-a|1/|b-a|^2)
    const int2 *rrange;       // per region: instruction [begin, end)
    const double *reg64;      // 8 per region: mu_a, mu_s, g, n, mu_t, albedo, 0, 0
    const float4 *reg32;      // per region: mu_t, albedo, g, n
    int32_t ninstr, nregions, nprims, precision;
    // bounding box as centre / half extent
    double bbc[3], bbh[3];
    float bbc32[3], bbh32[3];
    double delta, ambient_n;
    float delta32;            // FP32 surface threshold (>= 64 ulp of the scene extent)
    float ambient_n32;
    int32_t analytic_nrm;     // mixed mode: normals from the analytic SDF gradient (short programs)
    // Spatial culling of one long fold region (mixed mode only): a G^3 grid
    // of cells, each listing the region's primitives within distance R of
    // the cell; elsewhere the region's value is bounded by R - k/4.
    int32_t cull_region;      // -1: none
    int32_t cull_g;
    int32_t cull_op;          // 1 union, 2 smooth union
    float cull_lo[3], cull_inv_s[3];
    float cull_rmax;          // R (union) or R - k/4 (smooth union)
    float cull_kinv;
    const int32_t *cull_off;  // G^3 + 1 prefix offsets into cull_list
    const int32_t *cull_list; // primitive indices, in the region's fold order
    // Segment stepping (enum smcrt_stepping): the bounding primitives and
    // their margins (sum of k/4 over the smooth unions of their regions)
    const int32_t *seg_prims;
    const double *seg_m64;
    const float *seg_m32;
    int32_t stepping, nseg;
    // Primitive frames (kXf64 doubles / kXf32 float4 per primitive), null
    // when no primitive has one
    const double *xf64;
    const float4 *xf32;
    int32_t general;          // some primitive is a torus or cylinder or has a frame
    int32_t general_pad;
    float h32;                // FP32 central-difference step for normals
    int64_t max_steps;
    // source
    int32_t src_kind, pad0;
    double src_pos[3], src_dir[3], src_b1[3], src_b2[3], src_radius;
    float src_pos32[3], src_dir32[3], src_b132[3], src_b232[3], src_radius32;
    // grid (fluence voxels; n = 0 disables the tally)
    double g_lo[3], g_hi[3], g_dl[3];
    float g_lo32[3], g_hi32[3], g_dl32[3], g_idl32[3];
    int32_t g_n[3], pad1;
};

// A packet parked between serving rounds: its complete state at a trace
// boundary (FP32 values are stored widened, which round-trips exactly), so
// resuming it later continues the same arithmetic and the same random stream.
struct DeferState {
    double p[3], u[3], w, tau;
    long long pA, pG;
    uint32_t id_lo, id_hi, event, nsteps, pscat, pad[3];
};

// Per-job deferral lists, double-buffered by round parity: a round resumes
// the packets parked in list `in` and parks its own stragglers in 1 - in.
struct JobDefer {
    unsigned count[2];
    unsigned cursor[2];
    DeferState *buf[2];
    unsigned cap;
    unsigned overflow;       // stragglers that found the list full (kept running)
};

// Work descriptor of one job in a launch.  `next` is the packet-id cursor
// the warps claim from with atomicAdd.
struct JobWork {
    unsigned long long next;      // next packet id to hand out
    unsigned long long end;       // one past the last id
    unsigned long long begin;     // first id (records are indexed id - begin)
    unsigned long long seed;
    long long *fluence;           // device, may be null
    smcrt_totals *totals;         // device
    smcrt_packet_record *records; // device, may be null
    const DevScene *scene;        // device
    int32_t cancelled;            // host-set: stop handing out ids
    int32_t defer_in;             // list resumed in this launch (0 / 1)
    JobDefer *defer;              // device, may be null (no parking)
    long long park_cycles;        // > 0: park a packet after this many SM cycles in the launch
    long long drain_cycles;       // > 0 (served rounds): once its warp finds no job with work left,
                                  // park a packet after this many SM cycles in the launch
    int32_t stage;                // mixed kernel: stage the scene tables in shared memory
    int32_t stage_pad;
    int32_t *jstat;               // device, may be null: this job's own status word (bits OR-ed in)
    unsigned long long time_limit_ns;   // > 0: a warp stops this job that long after it started on it
};

// Kernel status word bits.
constexpr int kStatusBadJob = SMCRT_STATUS_BAD_JOB;
constexpr int kStatusStackOverflow = 2;
constexpr int kStatusTimeout = SMCRT_STATUS_TIMEOUT;

// Launch wrappers, one per translation unit; `variant` selects the register
// budget of the kernel instantiation (0 .. kNumVariants-1).
constexpr int kNumVariants = 3;
cudaError_t launch_fp64(JobWork *jobs, int njobs, int *status, int blocks, int threads,
                        cudaStream_t stream, int variant = 0);
cudaError_t launch_mixed(JobWork *jobs, int njobs, int *status, int blocks, int threads,
                         cudaStream_t stream, int variant = 0);
int occupancy_fp64(int threads, int variant = 0);
int occupancy_mixed(int threads, int variant = 0);
// Served rounds' mixed kernel, whose warps hold two jobs at a time (lanes
// refill from the next job instead of draining each): variant 0 / 1 = 5 / 4
// resident blocks of 128 threads, + kNumVariants for general shapes.
cudaError_t launch_mixed_multi(JobWork *jobs, int njobs, int *status, int blocks, int threads,
                               cudaStream_t stream, int variant = 0);
int occupancy_mixed_multi(int threads, int variant = 0);
cudaError_t launch_set_job(JobWork *dst, const JobWork &v, cudaStream_t stream);
// Field validation of scene / source / grid, without compiling or
// allocating (host runtime).
int validate_scene(const smcrt_scene *sc, const smcrt_source *src, const smcrt_grid *g);

// Round prologue: for each table entry with a deferral list, zero the
// resume cursor of its input list and the count of its output list.
cudaError_t launch_round_prologue(JobWork *jobs, int njobs, cudaStream_t stream);

}  // namespace smcrt
