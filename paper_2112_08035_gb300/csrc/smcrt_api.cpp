// smcrt_api.cpp -- host runtime behind the C-ABI of include/smcrt.h:
// validation, CSG compilation into the device instruction stream, plans,
// the one-shot run, the launch-shape autotuner and the continuously
// batched serving scheduler.
//
// Compiled as host C++ with -ffp-contract=off: the double constants it
// precomputes for the FP64 kernel (capsule |b-a|^2, bounding-box centre and
// half extent, mu_t, albedo, source basis, voxel size) use the expressions
// of the FP64 reference so both see identical values.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "smcrt_internal.h"

using namespace smcrt;

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
namespace {

#define CU(x)                                        \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return SMCRT_ERR_CUDA; \
    } while (0)

bool finite(double x) { return std::isfinite(x); }

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

float ulp_f32(float x)
{
    x = std::fabs(x);
    return std::nextafter(x, INFINITY) - x;
}

// Orthonormal basis perpendicular to unit n (Duff et al., JCGT 2017); same
// expression order as the FP64 reference.
void onb_host(const double n[3], double b1[3], double b2[3])
{
    const double sg = std::copysign(1.0, n[2]);
    const double a = -1.0 / (sg + n[2]);
    const double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sg * n[0] * n[0] * a;
    b1[1] = sg * b;
    b1[2] = -sg * n[0];
    b2[0] = b;
    b2[1] = sg + n[1] * n[1] * a;
    b2[2] = -n[1];
}

int validate(const smcrt_scene *sc, const smcrt_source *src, const smcrt_grid *g)
{
    if (!sc || !src || !g) return SMCRT_ERR_BAD_ARG;
    if (!sc->prims || !sc->nodes || !sc->regions) return SMCRT_ERR_BAD_ARG;
    if (sc->nprims < 1 || sc->nprims > kMaxPrims) return SMCRT_ERR_BAD_SCENE;
    if (sc->nregions < 1 || sc->nregions > kMaxRegions) return SMCRT_ERR_BAD_SCENE;
    if (sc->nnodes < 1) return SMCRT_ERR_BAD_SCENE;
    for (int i = 0; i < sc->nprims; ++i) {
        const smcrt_prim &p = sc->prims[i];
        for (int k = 0; k < 7; ++k)
            if (!finite(p.p[k])) return SMCRT_ERR_BAD_SCENE;
        if (p.kind == SMCRT_SPHERE) {
            if (!(p.p[3] > 0)) return SMCRT_ERR_BAD_SCENE;
        } else if (p.kind == SMCRT_BOX) {
            if (!(p.p[3] > 0 && p.p[4] > 0 && p.p[5] > 0)) return SMCRT_ERR_BAD_SCENE;
        } else if (p.kind == SMCRT_CAPSULE) {
            const double dx = p.p[3] - p.p[0], dy = p.p[4] - p.p[1], dz = p.p[5] - p.p[2];
            if (!(p.p[6] > 0) || !(dx * dx + dy * dy + dz * dz > 0)) return SMCRT_ERR_BAD_SCENE;
        } else if (p.kind == SMCRT_TORUS) {
            if (!(p.p[4] > 0 && p.p[3] > p.p[4])) return SMCRT_ERR_BAD_SCENE;
        } else if (p.kind == SMCRT_CYLINDER) {
            if (!(p.p[3] > 0 && p.p[4] > 0)) return SMCRT_ERR_BAD_SCENE;
        } else {
            return SMCRT_ERR_BAD_SCENE;
        }
        if (p.xform < 0 || p.xform > sc->nxforms) return SMCRT_ERR_BAD_SCENE;
    }
    if (sc->nxforms < 0 || sc->nxforms > kMaxPrims || (sc->nxforms > 0 && !sc->xforms)) return SMCRT_ERR_BAD_SCENE;
    for (int i = 0; i < sc->nxforms; ++i) {
        const smcrt_xform &X = sc->xforms[i];
        bool ok = finite(X.s) && X.s > 0 && X.op >= SMCRT_XF_NONE && X.op <= SMCRT_XF_REPEAT;
        for (int k = 0; k < 9; ++k) ok = ok && finite(X.rot[k]);
        for (int k = 0; k < 3; ++k) ok = ok && finite(X.t[k]);
        for (int k = 0; k < 4; ++k) ok = ok && finite(X.a[k]);
        if (!ok) return SMCRT_ERR_BAD_SCENE;
        for (int a = 0; a < 3; ++a)          // orthonormal columns
            for (int b = 0; b < 3; ++b) {
                const double dot = X.rot[a] * X.rot[b] + X.rot[3 + a] * X.rot[3 + b] + X.rot[6 + a] * X.rot[6 + b];
                if (!(std::fabs(dot - (a == b ? 1.0 : 0.0)) < 1e-9)) return SMCRT_ERR_BAD_SCENE;
            }
        const double *R = X.rot;
        const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                           R[2] * (R[3] * R[7] - R[4] * R[6]);
        if (!(det > 0)) return SMCRT_ERR_BAD_SCENE;
        if (X.op == SMCRT_XF_ELONGATE && !(X.a[0] >= 0 && X.a[1] >= 0 && X.a[2] >= 0)) return SMCRT_ERR_BAD_SCENE;
        if ((X.op == SMCRT_XF_TWIST || X.op == SMCRT_XF_BEND) && !(X.a[1] >= 0)) return SMCRT_ERR_BAD_SCENE;
        if (X.op == SMCRT_XF_REPEAT &&
            !(X.a[0] >= 0 && X.a[1] >= 0 && X.a[2] >= 0 && X.a[3] >= 0 && X.a[3] <= 1e6 &&
              X.a[3] == std::floor(X.a[3])))
            return SMCRT_ERR_BAD_SCENE;
    }
    for (int r = 0; r < sc->nregions; ++r) {
        const smcrt_region &R = sc->regions[r];
        if (R.node_count < 1 || R.node_begin < 0 || R.node_begin + R.node_count > sc->nnodes)
            return SMCRT_ERR_BAD_SCENE;
        if (!(R.mu_a >= 0 && R.mu_s >= 0 && finite(R.mu_a) && finite(R.mu_s))) return SMCRT_ERR_BAD_SCENE;
        if (!(R.g > -1 && R.g < 1)) return SMCRT_ERR_BAD_SCENE;
        if (!(R.n >= 1 && finite(R.n))) return SMCRT_ERR_BAD_SCENE;
    }
    if (!(sc->ambient_n >= 1 && finite(sc->ambient_n))) return SMCRT_ERR_BAD_SCENE;
    for (int a = 0; a < 3; ++a)
        if (!(sc->bbox_lo[a] < sc->bbox_hi[a]) || !finite(sc->bbox_lo[a]) || !finite(sc->bbox_hi[a]))
            return SMCRT_ERR_BAD_SCENE;
    if (!(sc->delta > 0 && finite(sc->delta))) return SMCRT_ERR_BAD_SCENE;
    if (sc->max_steps < 1 || sc->max_steps > (int64_t(1) << 31)) return SMCRT_ERR_BAD_SCENE;
    if (sc->stepping != SMCRT_STEP_SPHERE_TRACING && sc->stepping != SMCRT_STEP_SEGMENT) return SMCRT_ERR_BAD_SCENE;
    if (src->kind < SMCRT_SRC_PENCIL || src->kind > SMCRT_SRC_ISO_POINT) return SMCRT_ERR_BAD_SCENE;
    const double dl = std::sqrt(src->dir[0] * src->dir[0] + src->dir[1] * src->dir[1] + src->dir[2] * src->dir[2]);
    if (!(std::fabs(dl - 1.0) < 1e-9)) return SMCRT_ERR_BAD_SCENE;
    if ((src->kind == SMCRT_SRC_DISC || src->kind == SMCRT_SRC_SQUARE) && !(src->radius > 0))
        return SMCRT_ERR_BAD_SCENE;
    for (int a = 0; a < 3; ++a) {
        if (!finite(src->pos[a])) return SMCRT_ERR_BAD_SCENE;
        if (g->n[a] < 1 || g->n[a] > kMaxGridSide) return SMCRT_ERR_BAD_SCENE;
        if (!(g->lo[a] < g->hi[a]) || !finite(g->lo[a]) || !finite(g->hi[a])) return SMCRT_ERR_BAD_SCENE;
    }
    return SMCRT_OK;
}

// Postfix CSG -> device instruction stream.  A primitive immediately
// followed by a binary operator becomes one fused instruction that combines
// it with the stack top; the register stack depth must stay <= kMaxStack.
int compile(const smcrt_scene *sc, std::vector<Instr> &ins, std::vector<double> &k64, std::vector<int2> &rr)
{
    for (int r = 0; r < sc->nregions; ++r) {
        const smcrt_region &R = sc->regions[r];
        const smcrt_csg_node *nd = sc->nodes + R.node_begin;
        const int begin = (int)ins.size();
        int depth = 0;
        for (int i = 0; i < R.node_count; ++i) {
            const int op = nd[i].op;
            if (op == SMCRT_OP_PRIM) {
                const int p = nd[i].prim;
                if (p < 0 || p >= sc->nprims) return SMCRT_ERR_BAD_SCENE;
                const int kind = device_kind(sc->prims[p]);
                const bool fuse = depth >= 1 && i + 1 < R.node_count && nd[i + 1].op >= SMCRT_OP_UNION &&
                                  nd[i + 1].op <= SMCRT_OP_SUBTRACT;
                Instr in{};
                in.prim = p;
                in.region = -1;
                if (fuse) {
                    const int bop = nd[i + 1].op;
                    const double k = nd[i + 1].k;
                    if (bop == SMCRT_OP_SMOOTH_UNION && !(k > 0 && finite(k))) return SMCRT_ERR_BAD_SCENE;
                    in.op = bop | (kind << 8);
                    const float kinv = bop == SMCRT_OP_SMOOTH_UNION ? (float)(1.0 / k) : 0.f;
                    std::memcpy(&in.pad, &kinv, 4);
                    ins.push_back(in);
                    k64.push_back(bop == SMCRT_OP_SMOOTH_UNION ? k : 0.0);
                    ++i;  // operator consumed
                } else {
                    in.op = 0 | (kind << 8);
                    ins.push_back(in);
                    k64.push_back(0.0);
                    if (++depth > kMaxStack) return SMCRT_ERR_BAD_SCENE;
                }
            } else if (op >= SMCRT_OP_UNION && op <= SMCRT_OP_SUBTRACT) {
                if (depth < 2) return SMCRT_ERR_BAD_SCENE;
                const double k = nd[i].k;
                if (op == SMCRT_OP_SMOOTH_UNION && !(k > 0 && finite(k))) return SMCRT_ERR_BAD_SCENE;
                Instr in{};
                in.op = op;
                in.prim = -1;
                in.region = -1;
                const float kinv = op == SMCRT_OP_SMOOTH_UNION ? (float)(1.0 / k) : 0.f;
                std::memcpy(&in.pad, &kinv, 4);
                ins.push_back(in);
                k64.push_back(op == SMCRT_OP_SMOOTH_UNION ? k : 0.0);
                --depth;
            } else {
                return SMCRT_ERR_BAD_SCENE;
            }
        }
        if (depth != 1) return SMCRT_ERR_BAD_SCENE;
        ins.back().region = r;
        if (region_is_soft(sc, r)) ins.back().op |= kSoftRegionEnd;
        rr.push_back(make_int2(begin, (int)ins.size()));
    }
    return SMCRT_OK;
}

struct Timer {
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double s() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------------------------
// Context, plan, job
// ---------------------------------------------------------------------------
struct Job;

struct smcrt_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    double time_limit_s = 0.0;   // device time limit of smcrt_run and the default of new plans
    std::mutex tune_mu;
    struct Tuned { int blocks, threads, variant; };
    std::map<uint64_t, Tuned> tuned;  // scene shape -> launch shape

    // serving
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_job_id = 1;
    std::thread sched;
    bool stop = false;
    bool sched_started = false;
    int sched_error = 0;   // the scheduler could not set up: every job fails with this
    int64_t launches = 0;
    int64_t running = 0;
    size_t mem_in_use = 0;
    std::vector<std::shared_ptr<Job>> to_release;   // waited jobs whose device memory can go
};

struct smcrt_plan {
    smcrt_ctx *ctx = nullptr;
    int precision = SMCRT_MIXED;
    void *dbuf = nullptr;
    DevScene *dscene = nullptr;
    DevScene host{};
    JobWork *djobs = nullptr;  // ring of launch descriptors
    int ring = 64, ring_pos = 0;
    int *dstatus = nullptr;
    int blocks = 0, threads = 0, variant = 0;
    int stage = 0;             // mixed: stage the scene tables in shared memory
    double time_limit_s = 0.0; // device time limit of a launch (0 = none)
    size_t cells = 0;
    size_t dbytes = 0;
    uint64_t shape_key = 0;
};

namespace {

// Kernel instantiation of a plan: its register variant, in the general-shape
// family when the scene has tori, cylinders or primitive frames.
int kvariant(const smcrt_plan *pl) { return pl->variant + (pl->host.general ? kNumVariants : 0); }

int occupancy(int precision, int threads, int variant)
{
    return precision == SMCRT_FP64 ? occupancy_fp64(threads, variant) : occupancy_mixed(threads, variant);
}

cudaError_t launch_kernel(int precision, JobWork *jobs, int njobs, int *status, int blocks, int threads,
                          cudaStream_t s, int variant)
{
    return precision == SMCRT_FP64 ? launch_fp64(jobs, njobs, status, blocks, threads, s, variant)
                                   : launch_mixed(jobs, njobs, status, blocks, threads, s, variant);
}

// Register budgets measured fastest at full size on GB300 (see the design
// notes): mixed 96 registers x 5 blocks/SM, FP64 146 registers x 3 blocks/SM.
int default_variant(int precision) { return precision == SMCRT_FP64 ? 1 : 0; }

uint64_t shape_key(const smcrt_scene *sc, int precision, const smcrt_grid *g)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)precision);
    mix((uint64_t)sc->stepping);
    mix((uint64_t)sc->nxforms);
    mix((uint64_t)sc->nprims);
    mix((uint64_t)sc->nregions);
    mix((uint64_t)sc->nnodes);
    for (int i = 0; i < sc->nprims; ++i) mix((uint64_t)sc->prims[i].kind);
    mix((uint64_t)g->n[0] * 1315423911ull + (uint64_t)g->n[1] * 2654435761ull + (uint64_t)g->n[2]);
    return h;
}

// A region whose program is a left fold of one operator (union or smooth
// union, one k) over primitives: returns the primitives in fold order.
bool fold_region(const smcrt_scene *sc, int r, int *op, double *k, std::vector<int> *prims)
{
    const smcrt_region &R = sc->regions[r];
    const smcrt_csg_node *nd = sc->nodes + R.node_begin;
    if (R.node_count < 3 || (R.node_count - 1) % 2 != 0 || nd[0].op != SMCRT_OP_PRIM) return false;
    if (nd[0].prim < 0 || nd[0].prim >= sc->nprims || !plain_prim(sc->prims[nd[0].prim])) return false;
    prims->clear();
    prims->push_back(nd[0].prim);
    int o = -1;
    double kk = 0.0;
    for (int i = 1; i + 1 < R.node_count; i += 2) {
        const int bop = nd[i + 1].op;
        if (nd[i].op != SMCRT_OP_PRIM || (bop != SMCRT_OP_UNION && bop != SMCRT_OP_SMOOTH_UNION)) return false;
        if (nd[i].prim < 0 || nd[i].prim >= sc->nprims || !plain_prim(sc->prims[nd[i].prim]))
            return false;   // the grid bounds spheres, boxes, capsules
        if (o < 0) {
            o = bop;
            kk = bop == SMCRT_OP_SMOOTH_UNION ? nd[i + 1].k : 0.0;
        } else if (bop != o || (bop == SMCRT_OP_SMOOTH_UNION && nd[i + 1].k != kk)) {
            return false;
        }
        prims->push_back(nd[i].prim);
    }
    *op = o;
    *k = kk;
    return true;
}

struct CullGrid {
    int region = -1, g = 0, op = 0;
    float lo[3] = {0, 0, 0}, inv_s[3] = {0, 0, 0}, rmax = 0, kinv = 0;
    std::vector<int32_t> off, list;
};

// Uniform grid over the longest fold region (>= kCullMinPrims primitives):
// each cell lists the primitives whose bounding box lies within R' of the
// cell (R' = 1.05 R plus 1% of a cell, covering FP32 cell-index rounding);
// the grid extends R beyond every primitive, so outside it and for unlisted
// primitives the region's distance exceeds R; the kernel bounds the value
// by R (union) or R - k/4 (smooth union, which lies at most k/4 below min).
void build_cull(const smcrt_scene *sc, CullGrid &cg)
{
    int best = -1, bop = 0;
    double bk = 0.0;
    std::vector<int> prims, bprims;
    for (int r = 0; r < sc->nregions; ++r) {
        int op;
        double k;
        if (fold_region(sc, r, &op, &k, &prims) && (int)prims.size() >= kCullMinPrims &&
            (best < 0 || prims.size() > bprims.size())) {
            best = r; bop = op; bk = k; bprims = prims;
        }
    }
    if (best < 0) return;
    const int n = (int)bprims.size();
    std::vector<double> plo(3 * n), phi(3 * n);
    double blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = 0; j < n; ++j) {
        const smcrt_prim &P = sc->prims[bprims[j]];
        for (int a = 0; a < 3; ++a) {
            double lo, hi;
            if (P.kind == SMCRT_SPHERE) { lo = P.p[a] - P.p[3]; hi = P.p[a] + P.p[3]; }
            else if (P.kind == SMCRT_BOX) { lo = P.p[a] - P.p[3 + a]; hi = P.p[a] + P.p[3 + a]; }
            else {
                lo = std::min(P.p[a], P.p[3 + a]) - P.p[6];
                hi = std::max(P.p[a], P.p[3 + a]) + P.p[6];
            }
            plo[3 * j + a] = lo; phi[3 * j + a] = hi;
            blo[a] = std::min(blo[a], lo); bhi[a] = std::max(bhi[a], hi);
        }
    }
    const int G = kCullGrid;
    const double ext = std::max(bhi[0] - blo[0], std::max(bhi[1] - blo[1], bhi[2] - blo[2]));
    const double R = std::max(ext / G, bop == SMCRT_OP_SMOOTH_UNION ? 4.0 * bk : 0.0);
    double glo[3], s[3];
    for (int a = 0; a < 3; ++a) {
        glo[a] = blo[a] - R;
        s[a] = (bhi[a] + R - glo[a]) / G;
    }
    const double smax = std::max(s[0], std::max(s[1], s[2]));
    const double Rl = 1.05 * std::max(R, smax) + 0.01 * smax;
    cg.off.assign((size_t)G * G * G + 1, 0);
    cg.list.clear();
    for (int cz = 0; cz < G; ++cz)
        for (int cy = 0; cy < G; ++cy)
            for (int cx = 0; cx < G; ++cx) {
                const int c = (cz * G + cy) * G + cx;
                const double clo[3] = {glo[0] + cx * s[0], glo[1] + cy * s[1], glo[2] + cz * s[2]};
                cg.off[c] = (int32_t)cg.list.size();
                for (int j = 0; j < n; ++j) {
                    double d2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        const double gap = std::max(0.0, std::max(clo[a] - phi[3 * j + a], plo[3 * j + a] - (clo[a] + s[a])));
                        d2 += gap * gap;
                    }
                    if (d2 <= Rl * Rl) cg.list.push_back(bprims[j]);
                }
            }
    cg.off[(size_t)G * G * G] = (int32_t)cg.list.size();
    cg.region = best;
    cg.g = G;
    cg.op = bop;
    cg.kinv = bop == SMCRT_OP_SMOOTH_UNION ? (float)(1.0 / bk) : 0.f;
    cg.rmax = (float)(bop == SMCRT_OP_SMOOTH_UNION ? R - 0.25 * bk : R);
    for (int a = 0; a < 3; ++a) {
        cg.lo[a] = (float)glo[a];
        cg.inv_s[a] = (float)(1.0 / s[a]);
    }
}

// Validate, compile and upload a plan.  With a stream (the serving
// scheduler) the scene buffer is allocated and filled stream-ordered, no
// device-wide synchronisation happens, and no launch ring is created.
int build_plan(smcrt_ctx *ctx, const smcrt_scene *sc, const smcrt_source *src, const smcrt_grid *g,
               int32_t precision, smcrt_plan **out, cudaStream_t serving_stream = nullptr)
{
    int rc = validate(sc, src, g);
    if (rc) return rc;
    if (precision != SMCRT_FP64 && precision != SMCRT_MIXED) return SMCRT_ERR_BAD_ARG;
    std::vector<Instr> ins;
    std::vector<double> k64;
    std::vector<int2> rr;
    rc = compile(sc, ins, k64, rr);
    if (rc) return rc;
    const int np = sc->nprims, nr = sc->nregions, ni = (int)ins.size();

    std::vector<int32_t> pkind(np);
    std::vector<double> p64((size_t)np * 8, 0.0);
    std::vector<float4> p32((size_t)np * 2, make_float4(0, 0, 0, 0));
    const bool has_xf = sc->nxforms > 0;
    std::vector<double> xf64(has_xf ? (size_t)np * kXf64 : 0);
    std::vector<float4> xf32(has_xf ? (size_t)np * kXf32 : 0);
    for (int i = 0; i < np; ++i) {
        pkind[i] = device_kind(sc->prims[i]);
        fill_prim(sc, i, &p64[(size_t)8 * i], &p32[(size_t)2 * i], has_xf ? &xf64[(size_t)kXf64 * i] : nullptr,
                  has_xf ? &xf32[(size_t)kXf32 * i] : nullptr);
    }
    std::vector<double> reg64((size_t)nr * 8, 0.0);
    std::vector<float4> reg32((size_t)nr * 2);
    for (int r = 0; r < nr; ++r) {
        const smcrt_region &R = sc->regions[r];
        const double mu_t = R.mu_a + R.mu_s;
        const double albedo = mu_t > 0.0 ? R.mu_s / mu_t : 0.0;
        double *d = &reg64[(size_t)8 * r];
        d[0] = R.mu_a; d[1] = R.mu_s; d[2] = R.g; d[3] = R.n; d[4] = mu_t; d[5] = albedo;
        reg32[2 * r] = make_float4((float)mu_t, mu_t > 0 ? (float)(1.0 / mu_t) : 0.f, (float)albedo, (float)R.g);
        reg32[2 * r + 1] = make_float4((float)R.n, (float)R.mu_a, (float)R.mu_s, 0.f);
    }

    // one device buffer: [DevScene | instr | k64 | pkind | p64 | p32 | rrange | reg64 | reg32]
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align16(off + bytes); return o; };
    const size_t o_scene = take(sizeof(DevScene));
    const size_t o_ins = take(sizeof(Instr) * ni);
    const size_t o_k64 = take(sizeof(double) * ni);
    const size_t o_kind = take(sizeof(int32_t) * np);
    const size_t o_p64 = take(sizeof(double) * 8 * np);
    const size_t o_p32 = take(sizeof(float4) * 2 * np);
    const size_t o_rr = take(sizeof(int2) * nr);
    const size_t o_r64 = take(sizeof(double) * 8 * nr);
    const size_t o_r32 = take(sizeof(float4) * 2 * nr);
    CullGrid cg;
    if (precision == SMCRT_MIXED) build_cull(sc, cg);
    const size_t o_coff = take(sizeof(int32_t) * cg.off.size());
    const size_t o_clist = take(sizeof(int32_t) * cg.list.size());
    std::vector<int32_t> segp(sc->stepping == SMCRT_STEP_SEGMENT ? kMaxPrims : 0);
    std::vector<double> segm(segp.size());
    // the culled region bounds segment moves by its (culled) distance, like a
    // soft region: ray bounds over all its primitives would undo the culling
    const int nseg = segp.empty() ? 0 : seg_entries(sc, segp.data(), segm.data(), cg.region);
    std::vector<float> segm32(nseg);
    for (int j = 0; j < nseg; ++j) segm32[j] = (float)segm[j];
    const size_t o_seg = take(sizeof(int32_t) * nseg);
    const size_t o_segm64 = take(sizeof(double) * nseg);
    const size_t o_segm32 = take(sizeof(float) * nseg);
    const size_t o_xf64 = take(sizeof(double) * xf64.size());
    const size_t o_xf32 = take(sizeof(float4) * xf32.size());
    const size_t total = off;

    std::unique_ptr<smcrt_plan> pl(new smcrt_plan());
    pl->ctx = ctx;
    pl->precision = precision;
    pl->variant = default_variant(precision);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return SMCRT_ERR_CUDA;
    if (serving_stream) {
        if (cudaMallocAsync(&pl->dbuf, total, serving_stream) != cudaSuccess) return SMCRT_ERR_NO_MEMORY;
    } else if (cudaMalloc(&pl->dbuf, total) != cudaSuccess) {
        return SMCRT_ERR_NO_MEMORY;
    }
    pl->dbytes = total;
    char *base = (char *)pl->dbuf;
    DevScene &H = pl->host;
    std::memset(&H, 0, sizeof H);
    H.instr = (const Instr *)(base + o_ins);
    H.k64 = (const double *)(base + o_k64);
    H.kinv32 = nullptr;
    H.pkind = (const int32_t *)(base + o_kind);
    H.p64 = (const double *)(base + o_p64);
    H.p32 = (const float4 *)(base + o_p32);
    H.rrange = (const int2 *)(base + o_rr);
    H.reg64 = (const double *)(base + o_r64);
    H.reg32 = (const float4 *)(base + o_r32);
    H.ninstr = ni;
    H.nregions = nr;
    H.nprims = np;
    H.precision = precision;
    float rmax = 0.f;
    for (int a = 0; a < 3; ++a) {
        H.bbc[a] = (sc->bbox_lo[a] + sc->bbox_hi[a]) * 0.5;
        H.bbh[a] = (sc->bbox_hi[a] - sc->bbox_lo[a]) * 0.5;
        H.bbc32[a] = (float)H.bbc[a];
        H.bbh32[a] = (float)H.bbh[a];
        rmax = std::max(rmax, (float)std::max(std::fabs(sc->bbox_lo[a]), std::fabs(sc->bbox_hi[a])));
    }
    H.delta = sc->delta;
    H.ambient_n = sc->ambient_n;
    H.ambient_n32 = (float)sc->ambient_n;
    H.cull_region = cg.region;
    H.cull_g = cg.g;
    H.cull_op = cg.op;
    for (int a = 0; a < 3; ++a) {
        H.cull_lo[a] = cg.lo[a];
        H.cull_inv_s[a] = cg.inv_s[a];
    }
    H.cull_rmax = cg.rmax;
    H.cull_kinv = cg.kinv;
    H.cull_off = cg.region >= 0 ? (const int32_t *)(base + o_coff) : nullptr;
    H.cull_list = cg.region >= 0 ? (const int32_t *)(base + o_clist) : nullptr;
    H.stepping = sc->stepping;
    H.nseg = nseg;
    H.seg_prims = nseg > 0 ? (const int32_t *)(base + o_seg) : nullptr;
    H.seg_m64 = nseg > 0 ? (const double *)(base + o_segm64) : nullptr;
    H.seg_m32 = nseg > 0 ? (const float *)(base + o_segm32) : nullptr;
    H.xf64 = has_xf ? (const double *)(base + o_xf64) : nullptr;
    H.xf32 = has_xf ? (const float4 *)(base + o_xf32) : nullptr;
    for (int i = 0; i < np; ++i) H.general = H.general || !plain_prim(sc->prims[i]);
    {   // analytic normals when every region's program is short and made of
        // spheres, boxes and capsules in scene coordinates
        // (the culled region counts as short: its gradient folds over the
        // cell's few candidates)
        int longest = 0;
        bool plain = true;
        for (int r = 0; r < nr; ++r)
            if (r != cg.region) longest = std::max(longest, rr[r].y - rr[r].x);
        for (int i = 0; i < np; ++i) plain = plain && plain_prim(sc->prims[i]);
        H.analytic_nrm = longest <= kAnalyticNormalMaxInstr && plain ? 1 : 0;
    }
    // The plain mixed instantiation leaves the six-probe normal out of its
    // loop (smaller loop: 4.6 % on the layered slab); a mixed scene whose
    // normals need the probes runs the general one, whose plain-shape
    // arithmetic is the same.
    if (precision == SMCRT_MIXED && !H.analytic_nrm) H.general = 1;
    H.delta32 = std::max((float)sc->delta, 64.f * ulp_f32(rmax));
    H.h32 = 32.f * H.delta32;
    H.max_steps = sc->max_steps;
    H.src_kind = src->kind;
    onb_host(src->dir, H.src_b1, H.src_b2);
    for (int a = 0; a < 3; ++a) {
        H.src_pos[a] = src->pos[a];
        H.src_dir[a] = src->dir[a];
        H.src_pos32[a] = (float)src->pos[a];
        H.src_dir32[a] = (float)src->dir[a];
        H.src_b132[a] = (float)H.src_b1[a];
        H.src_b232[a] = (float)H.src_b2[a];
        H.g_lo[a] = g->lo[a];
        H.g_hi[a] = g->hi[a];
        H.g_dl[a] = (g->hi[a] - g->lo[a]) / (double)g->n[a];
        H.g_lo32[a] = (float)g->lo[a];
        H.g_hi32[a] = (float)g->hi[a];
        H.g_dl32[a] = (float)H.g_dl[a];
        H.g_idl32[a] = (float)(1.0 / H.g_dl[a]);
        H.g_n[a] = g->n[a];
    }
    H.src_radius = src->radius;
    H.src_radius32 = (float)src->radius;

    std::vector<char> hb(total, 0);
    std::memcpy(hb.data() + o_scene, &H, sizeof H);
    std::memcpy(hb.data() + o_ins, ins.data(), sizeof(Instr) * ni);
    std::memcpy(hb.data() + o_k64, k64.data(), sizeof(double) * ni);
    std::memcpy(hb.data() + o_kind, pkind.data(), sizeof(int32_t) * np);
    std::memcpy(hb.data() + o_p64, p64.data(), sizeof(double) * 8 * np);
    std::memcpy(hb.data() + o_p32, p32.data(), sizeof(float4) * 2 * np);
    std::memcpy(hb.data() + o_rr, rr.data(), sizeof(int2) * nr);
    std::memcpy(hb.data() + o_r64, reg64.data(), sizeof(double) * 8 * nr);
    std::memcpy(hb.data() + o_r32, reg32.data(), sizeof(float4) * 2 * nr);
    if (!cg.off.empty()) std::memcpy(hb.data() + o_coff, cg.off.data(), sizeof(int32_t) * cg.off.size());
    if (!cg.list.empty()) std::memcpy(hb.data() + o_clist, cg.list.data(), sizeof(int32_t) * cg.list.size());
    if (nseg > 0) {
        std::memcpy(hb.data() + o_seg, segp.data(), sizeof(int32_t) * nseg);
        std::memcpy(hb.data() + o_segm64, segm.data(), sizeof(double) * nseg);
        std::memcpy(hb.data() + o_segm32, segm32.data(), sizeof(float) * nseg);
    }
    if (has_xf) {
        std::memcpy(hb.data() + o_xf64, xf64.data(), sizeof(double) * xf64.size());
        std::memcpy(hb.data() + o_xf32, xf32.data(), sizeof(float4) * xf32.size());
    }
    pl->dscene = (DevScene *)(base + o_scene);
    pl->cells = (size_t)g->n[0] * g->n[1] * g->n[2];
    if (serving_stream) {
        // pageable source: staged before the call returns, so hb may go
        if (cudaMemcpyAsync(pl->dbuf, hb.data(), total, cudaMemcpyHostToDevice, serving_stream) != cudaSuccess) {
            cudaFreeAsync(pl->dbuf, serving_stream);
            return SMCRT_ERR_CUDA;
        }
        *out = pl.release();
        return SMCRT_OK;
    }
    if (cudaMemcpy(pl->dbuf, hb.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(pl->dbuf);
        return SMCRT_ERR_CUDA;
    }
    if (cudaMalloc(&pl->djobs, sizeof(JobWork) * pl->ring) != cudaSuccess) {
        cudaFree(pl->dbuf);
        return SMCRT_ERR_NO_MEMORY;
    }
    if (cudaMalloc(&pl->dstatus, sizeof(int)) != cudaSuccess || cudaMemset(pl->dstatus, 0, sizeof(int)) != cudaSuccess) {
        cudaFree(pl->dbuf);
        cudaFree(pl->djobs);
        return SMCRT_ERR_NO_MEMORY;
    }
    pl->cells = (size_t)g->n[0] * g->n[1] * g->n[2];
    pl->shape_key = shape_key(sc, precision, g);
    pl->time_limit_s = ctx->time_limit_s;
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        auto it = ctx->tuned.find(pl->shape_key);
        if (it != ctx->tuned.end()) {
            pl->blocks = it->second.blocks;
            pl->threads = it->second.threads;
            pl->variant = it->second.variant % kNumVariants;
            pl->stage = it->second.variant / kNumVariants;
        }
    }
    *out = pl.release();
    return SMCRT_OK;
}

void default_launch(const smcrt_plan *pl, int &blocks, int &threads)
{
    threads = pl->threads > 0 ? pl->threads : 128;
    blocks = pl->blocks;
    if (blocks <= 0) {
        const int occ = std::max(1, occupancy(pl->precision, threads, kvariant(pl)));
        blocks = pl->ctx->sm_count * occ;
    }
}

int plan_launch_impl(smcrt_plan *pl, uint64_t id_begin, uint64_t n, uint64_t seed, int64_t *flu,
                     smcrt_totals *tot, smcrt_packet_record *rec, cudaStream_t s, int blocks, int threads)
{
    JobWork jw{};
    jw.next = id_begin;
    jw.end = id_begin + n;
    jw.begin = id_begin;
    jw.seed = seed;
    jw.fluence = (long long *)flu;
    jw.totals = tot;
    jw.records = rec;
    jw.scene = pl->dscene;
    jw.cancelled = 0;
    jw.stage = pl->precision == SMCRT_MIXED ? pl->stage : 0;
    jw.time_limit_ns = pl->time_limit_s > 0.0 ? (unsigned long long)std::llround(pl->time_limit_s * 1e9) : 0ull;
    JobWork *slot = pl->djobs + pl->ring_pos;
    pl->ring_pos = (pl->ring_pos + 1) % pl->ring;
    if (launch_set_job(slot, jw, s) != cudaSuccess) return SMCRT_ERR_CUDA;
    if (launch_kernel(pl->precision, slot, 1, pl->dstatus, blocks, threads, s, kvariant(pl)) != cudaSuccess)
        return SMCRT_ERR_CUDA;
    return SMCRT_OK;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// Serving: job state and scheduler
// ---------------------------------------------------------------------------
struct Job {
    uint64_t id = 0;
    // host copies of the request
    std::vector<smcrt_prim> prims;
    std::vector<smcrt_csg_node> nodes;
    std::vector<smcrt_region> regions;
    std::vector<smcrt_xform> xforms;
    smcrt_scene scene{};
    smcrt_source source{};
    smcrt_grid grid{};
    uint64_t npackets = 0, seed = 0;
    int precision = SMCRT_MIXED;
    // device resources while admitted
    smcrt_plan *plan = nullptr;
    int64_t *dflu = nullptr;
    JobDefer *ddefer = nullptr;   // parked-packet lists (two) and their header
    int slot = -1;                // index into the device totals array
    size_t bytes = 0;
    uint64_t cursor = 0;          // next packet id to schedule
    double cost = 0;              // measured warp-cycles per packet (0 = unknown)
    int64_t admit_round = 0;      // first round index that can carry this job
    int64_t last_round = -1;      // last round index that carried its ids
    bool admitted = false, done = false, cancelled = false, released = false;
    int status = SMCRT_OK;
    smcrt_totals totals{};
    double t_submit = 0, t_done = 0;
};

namespace {

constexpr int kMaxSlots = 64;
constexpr int kRoundsInFlight = 2;
constexpr double kRoundSeconds = 0.008;   // target device time of one round
constexpr double kParkSeconds = 0.004;    // device time a packet may run per round before it is parked
constexpr double kDrainSeconds = 0.0005;  // ... once its warp has no more work, in rounds with new ids
constexpr double kTailSeconds = 0.05;     // ... in rounds of parked packets only, with no job waiting
// Parked packets per list and job: at least one per lane of the served
// kernels' launches (the tuned mixed shapes hold up to about 1e5 lanes on
// 152 SMs).  At a round's end nearly every lane holds a packet younger than
// its lifetime (1.5 ms on the layered slab under full load); a packet that
// finds the list full keeps running, and the round then waits for the
// longest of them (measured with 65,536 entries: 11 ms rounds for 8 ms of
// work, the list full every round).
constexpr unsigned kDeferCap = 131072;

size_t job_bytes(const smcrt_grid &g)
{
    return (size_t)g.n[0] * g.n[1] * g.n[2] * 8 + 65536 + 2 * sizeof(DeferState) * (size_t)kDeferCap;
}

void free_job_device(Job &j, cudaStream_t st)
{
    if (j.plan) {
        cudaFreeAsync(j.plan->dbuf, st);
        delete j.plan;
        j.plan = nullptr;
    }
    if (j.dflu) cudaFreeAsync(j.dflu, st);
    j.dflu = nullptr;
    if (j.ddefer) cudaFreeAsync(j.ddefer, st);
    j.ddefer = nullptr;
}

// One allocation: JobDefer header, then its two lists.
int alloc_defer(Job &j, cudaStream_t st)
{
    const size_t hdr = (sizeof(JobDefer) + 255) & ~size_t(255);
    const size_t bytes = hdr + 2 * sizeof(DeferState) * kDeferCap;
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) return SMCRT_ERR_NO_MEMORY;
    JobDefer h{};
    h.buf[0] = (DeferState *)((char *)p + hdr);
    h.buf[1] = h.buf[0] + kDeferCap;
    h.cap = kDeferCap;
    // pageable source: staged before the call returns
    if (cudaMemcpyAsync(p, &h, sizeof h, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaFreeAsync(p, st);
        return SMCRT_ERR_CUDA;
    }
    j.ddefer = (JobDefer *)p;
    return SMCRT_OK;
}

// The scheduler thread.  Each round is one replay of a captured CUDA graph:
//   [job tables H2D] -> fork -> {mixed kernel | FP64 kernel} -> join ->
//   [all job totals D2H into pinned memory]
// with up to two rounds in flight.  A round gives every admitted job a
// quantum of packet ids sized by processor sharing: each job gets an equal
// share of the round's warp-cycles, converted to packets with the job's
// measured cost (busy cycles per packet from earlier rounds), so short jobs
// finish within one round while long ones keep progressing.  Jobs join at the
// next round after admission; completion is read from the totals snapshot.
void scheduler(smcrt_ctx *ctx)
{
    // Setup: every call is checked; on a failure the scheduler fails all jobs
    // with the error instead of running rounds on missing buffers.
    // SMCRT_FAULT_SCHEDULER_SETUP (any value) makes the first allocation
    // report failure: host-side injection for the error-path tests.
    int setup_rc = SMCRT_OK;
    const bool inject = std::getenv("SMCRT_FAULT_SCHEDULER_SETUP") != nullptr;
    auto chk = [&](cudaError_t e, int rc) {
        if (e != cudaSuccess && setup_rc == SMCRT_OK) setup_rc = rc;
    };
    chk(cudaSetDevice(ctx->device), SMCRT_ERR_CUDA);
    cudaStream_t st = nullptr, st2 = nullptr;
    chk(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), SMCRT_ERR_CUDA);
    chk(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking), SMCRT_ERR_CUDA);
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    chk(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming), SMCRT_ERR_CUDA);
    chk(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming), SMCRT_ERR_CUDA);
    // Status words: one per round buffer for the launch (cleared by the
    // round's graph before its kernels run), and one per job slot (cleared
    // when a job is admitted to the slot), both read back with the totals:
    // a job that the kernel flags fails alone, and no flag outlives its round.
    int *d_status = nullptr;     // [kRoundsInFlight]
    int32_t *d_jstat = nullptr;  // [kMaxSlots]
    smcrt_totals *d_tot = nullptr;
    chk(inject ? cudaErrorMemoryAllocation : cudaMalloc(&d_status, sizeof(int) * kRoundsInFlight),
        SMCRT_ERR_NO_MEMORY);
    if (d_status) chk(cudaMemset(d_status, 0, sizeof(int) * kRoundsInFlight), SMCRT_ERR_CUDA);
    chk(cudaMalloc(&d_jstat, sizeof(int32_t) * kMaxSlots), SMCRT_ERR_NO_MEMORY);
    if (d_jstat) chk(cudaMemset(d_jstat, 0, sizeof(int32_t) * kMaxSlots), SMCRT_ERR_CUDA);
    chk(cudaMalloc(&d_tot, sizeof(smcrt_totals) * kMaxSlots), SMCRT_ERR_NO_MEMORY);
    if (d_tot) chk(cudaMemset(d_tot, 0, sizeof(smcrt_totals) * kMaxSlots), SMCRT_ERR_CUDA);
    // Launch shape of the served kernels.  The mixed jobs run in the kernel
    // whose warps hold two jobs at a time (launch_mixed_multi); its register
    // variant, threads and blocks are chosen by timing trials on the first
    // mixed job served (tune_served below) before the graphs are captured;
    // until then, and for FP64, the defaults.
    int threads_m = 128, variant_m = 0;
    int blocks_m = ctx->sm_count * std::max(1, occupancy_mixed_multi(threads_m, variant_m));
    const int threads_d = 128;
    const int blocks_d = ctx->sm_count * std::max(1, occupancy_fp64(threads_d, default_variant(SMCRT_FP64)));
    bool tuned_served = false;
    int clk_khz = 1900000;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ctx->device);
    // warp-cycles one round can spend (the mixed kernel's resident warps)
    auto round_cycles = [&] { return (double)blocks_m * (threads_m / 32) * clk_khz * 1e3 * kRoundSeconds; };
    const long long park_cycles = (long long)(clk_khz * 1e3 * kParkSeconds);
    const long long drain_cycles = (long long)(clk_khz * 1e3 * kDrainSeconds);
    const long long tail_cycles = (long long)(clk_khz * 1e3 * kTailSeconds);
    // SMCRT_FAULT_BAD_JOB=<job id>: that job's round-table entry gets no
    // scene, which the kernels report as a bad job (host-side injection for
    // the status tests; no GPU fault is involved).
    uint64_t bad_job = 0;
    if (const char *bj = std::getenv("SMCRT_FAULT_BAD_JOB")) bad_job = std::strtoull(bj, nullptr, 10);

    struct Buf {
        JobWork *h_tab = nullptr, *d_tab = nullptr;   // [2 * kMaxSlots]: mixed table, then FP64 table
        smcrt_totals *h_tot = nullptr;                // totals snapshot taken at the end of the round
        int32_t *h_stat = nullptr;                    // [1 + kMaxSlots]: the round's status, then each slot's
        cudaGraphExec_t graph = nullptr;     // plain scenes only
        cudaGraphExec_t graph_g = nullptr;   // kernels for scenes with general shapes
        cudaEvent_t ev = nullptr, ev0 = nullptr;
        bool busy = false;
        int64_t idx = -1;
        int njobs = 0;
        uint64_t quanta = 0;
        double t_launch = 0;
    } buf[kRoundsInFlight];
    const bool trace = std::getenv("SMCRT_TRACE") != nullptr;
    for (auto &b : buf) {
        if (setup_rc != SMCRT_OK) break;
        chk(cudaMallocHost(&b.h_tab, sizeof(JobWork) * 2 * kMaxSlots), SMCRT_ERR_NO_MEMORY);
        chk(cudaMalloc(&b.d_tab, sizeof(JobWork) * 2 * kMaxSlots), SMCRT_ERR_NO_MEMORY);
        chk(cudaMallocHost(&b.h_tot, sizeof(smcrt_totals) * kMaxSlots), SMCRT_ERR_NO_MEMORY);
        chk(cudaMallocHost(&b.h_stat, sizeof(int32_t) * (1 + kMaxSlots)), SMCRT_ERR_NO_MEMORY);
        chk(cudaEventCreate(&b.ev), SMCRT_ERR_CUDA);
        chk(cudaEventCreate(&b.ev0), SMCRT_ERR_CUDA);
        if (setup_rc != SMCRT_OK) break;
        std::memset(b.h_tab, 0, sizeof(JobWork) * 2 * kMaxSlots);
        std::memset(b.h_stat, 0, sizeof(int32_t) * (1 + kMaxSlots));
    }

    // Capture each buffer's round graphs with the current launch shape.
    auto capture = [&]() -> int {
        for (int bi = 0; bi < kRoundsInFlight; ++bi) {
            Buf &b = buf[bi];
            for (int gen = 0; gen < 2; ++gen) {
                const int off = gen ? kNumVariants : 0;
                cudaGraph_t g;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SMCRT_ERR_CUDA;
                cudaMemsetAsync(d_status + bi, 0, sizeof(int), st);
                cudaMemcpyAsync(b.d_tab, b.h_tab, sizeof(JobWork) * 2 * kMaxSlots, cudaMemcpyHostToDevice, st);
                launch_round_prologue(b.d_tab, 2 * kMaxSlots, st);
                cudaEventRecord(ev_fork, st);
                cudaStreamWaitEvent(st2, ev_fork, 0);
                launch_mixed_multi(b.d_tab, kMaxSlots, d_status + bi, blocks_m, threads_m, st, variant_m + off);
                launch_fp64(b.d_tab + kMaxSlots, kMaxSlots, d_status + bi, blocks_d, threads_d, st2,
                            default_variant(SMCRT_FP64) + off);
                cudaEventRecord(ev_join, st2);
                cudaStreamWaitEvent(st, ev_join, 0);
                cudaMemcpyAsync(b.h_tot, d_tot, sizeof(smcrt_totals) * kMaxSlots, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(b.h_stat, d_status + bi, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(b.h_stat + 1, d_jstat, sizeof(int32_t) * kMaxSlots, cudaMemcpyDeviceToHost, st);
                if (cudaStreamEndCapture(st, &g) != cudaSuccess) return SMCRT_ERR_CUDA;
                cudaGraphExec_t &ge = gen ? b.graph_g : b.graph;
                if (ge) cudaGraphExecDestroy(ge);
                ge = nullptr;
                const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return SMCRT_ERR_CUDA;
            }
        }
        return SMCRT_OK;
    };
    if (setup_rc == SMCRT_OK) setup_rc = capture();

    // Timing trials of the served mixed kernel on one job's scene (scratch
    // tallies, ids from 0 with the job's seed, whatever the job's own size):
    // register variant x threads x resident blocks, as smcrt_plan_autotune
    // does for a plan.  A trial gives every lane a few packets (4e5 packets,
    // about 8 ms on the layered slab), so it times throughput rather than
    // one packet's lifetime.  Results do not depend on the choice (every
    // variant computes the same bits).
    auto tune_served = [&](const Job &j) {
        const uint64_t trial = 400000;
        const size_t cells = (size_t)j.grid.n[0] * j.grid.n[1] * j.grid.n[2];
        void *flu = nullptr, *tot = nullptr, *tab = nullptr, *tst = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaMallocAsync(&flu, cells * 8, st) == cudaSuccess &&
                  cudaMallocAsync(&tot, sizeof(smcrt_totals), st) == cudaSuccess &&
                  cudaMallocAsync(&tab, sizeof(JobWork), st) == cudaSuccess &&
                  cudaMallocAsync(&tst, sizeof(int), st) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
        const int off = j.plan->host.general ? kNumVariants : 0;
        float best = 1e30f;
        for (int v = 0; ok && v < 2; ++v) {
            for (int t : {64, 128}) {
                const int occ = occupancy_mixed_multi(t, v + off);
                if (occ < 1) continue;
                for (int mult : {1, 2}) {
                    const int b = ctx->sm_count * occ * mult;
                    JobWork w{};
                    w.next = 0;
                    w.end = trial;
                    w.begin = 0;
                    w.seed = j.seed;
                    w.fluence = (long long *)flu;
                    w.totals = (smcrt_totals *)tot;
                    w.scene = j.plan->dscene;
                    cudaMemsetAsync(flu, 0, cells * 8, st);
                    cudaMemsetAsync(tot, 0, sizeof(smcrt_totals), st);
                    if (launch_set_job((JobWork *)tab, w, st) != cudaSuccess) { ok = false; break; }
                    cudaEventRecord(e0, st);
                    if (launch_mixed_multi((JobWork *)tab, 1, (int *)tst, b, t, st, v + off) != cudaSuccess) {
                        ok = false;
                        break;
                    }
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { ok = false; break; }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) {
                        best = ms;
                        variant_m = v;
                        threads_m = t;
                        blocks_m = b;
                    }
                }
                if (!ok) break;
            }
        }
        if (flu) cudaFreeAsync(flu, st);
        if (tot) cudaFreeAsync(tot, st);
        if (tab) cudaFreeAsync(tab, st);
        if (tst) cudaFreeAsync(tst, st);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
        if (trace)
            std::fprintf(stderr, "[smcrt] served kernel tuned on job %llu: variant %d threads %d blocks %d\n",
                         (unsigned long long)j.id, variant_m, threads_m, blocks_m);
        return ok;
    };

    if (setup_rc != SMCRT_OK) {
        // fail every queued job, and every later one, until the context ends
        std::unique_lock<std::mutex> lk(ctx->mu);
        ctx->sched_error = setup_rc;
        for (;;) {
            while (!ctx->queue.empty()) {
                auto j = ctx->queue.front();
                ctx->queue.pop_front();
                j->status = setup_rc;
                j->done = true;
                j->t_done = now_s();
            }
            ctx->to_release.clear();
            ctx->cv_done.notify_all();
            if (ctx->stop) break;
            ctx->cv_work.wait(lk, [&] { return ctx->stop || !ctx->queue.empty(); });
        }
    }

    std::vector<std::shared_ptr<Job>> active;   // admitted, not yet complete
    std::vector<int> free_slots;
    for (int i = kMaxSlots - 1; i >= 0; --i) free_slots.push_back(i);
    int cur = 0;
    int64_t issued = 0, completed = -1;

    auto is_cancelled = [&](const std::shared_ptr<Job> &j) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        return j->cancelled;
    };
    auto complete = [&](const std::shared_ptr<Job> &j, const smcrt_totals *t, int status) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (t) j->totals = *t;
        j->status = status;
        j->done = true;
        j->t_done = now_s();
        ctx->running -= 1;
        free_slots.push_back(j->slot);
        ctx->cv_done.notify_all();
    };

    for (; setup_rc == SMCRT_OK;) {
        // ---- admission (FIFO, by slots and device memory) and releases
        std::vector<std::shared_ptr<Job>> newly, released;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            const bool idle = active.empty() && !buf[0].busy && !buf[1].busy;
            if (idle && ctx->queue.empty() && ctx->to_release.empty()) {
                if (ctx->stop) break;
                ctx->cv_work.wait(lk, [&] { return ctx->stop || !ctx->queue.empty() || !ctx->to_release.empty(); });
                if (ctx->stop && ctx->queue.empty() && ctx->to_release.empty()) break;
            }
            released.swap(ctx->to_release);
            while (!ctx->queue.empty() && (int)free_slots.size() > (int)newly.size()) {
                auto j = ctx->queue.front();
                if (ctx->mem_in_use + j->bytes > ctx->budget && !(active.empty() && newly.empty())) break;
                ctx->queue.pop_front();
                if (j->cancelled) {
                    j->status = SMCRT_ERR_CANCELLED;
                    j->done = true;
                    j->t_done = now_s();
                    ctx->cv_done.notify_all();
                    continue;
                }
                ctx->mem_in_use += j->bytes;
                ctx->running += 1;
                j->admitted = true;
                newly.push_back(j);
            }
        }
        for (auto &j : released) free_job_device(*j, st);
        for (auto &j : newly) {
            int rc = build_plan(ctx, &j->scene, &j->source, &j->grid, j->precision, &j->plan, st);
            const size_t fb = (size_t)j->grid.n[0] * j->grid.n[1] * j->grid.n[2] * 8;
            if (rc == SMCRT_OK && cudaMallocAsync(&j->dflu, fb, st) != cudaSuccess) rc = SMCRT_ERR_NO_MEMORY;
            if (rc == SMCRT_OK) rc = alloc_defer(*j, st);
            j->slot = free_slots.back();
            free_slots.pop_back();
            j->admit_round = issued;     // snapshots of earlier rounds do not describe this job
            if (rc == SMCRT_OK) {
                cudaMemsetAsync(j->dflu, 0, fb, st);
                cudaMemsetAsync(d_tot + j->slot, 0, sizeof(smcrt_totals), st);
                cudaMemsetAsync(d_jstat + j->slot, 0, sizeof(int32_t), st);
                active.push_back(j);
            } else {
                free_job_device(*j, st);
                {
                    std::lock_guard<std::mutex> lk(ctx->mu);
                    ctx->mem_in_use -= std::min(ctx->mem_in_use, j->bytes);
                    j->admitted = false;
                }
                complete(j, nullptr, rc);
            }
        }

        // ---- reap the buffer we are about to refill
        Buf &B = buf[cur];
        if (B.busy) {
            cudaEventSynchronize(B.ev);
            B.busy = false;
            completed = B.idx;
            if (trace) {
                float ms = 0;
                cudaEventElapsedTime(&ms, B.ev0, B.ev);
                long long parked = 0;
                for (auto &j : active) parked += B.h_tot[j->slot].parked;
                std::fprintf(stderr, "[smcrt] round %lld jobs %d quanta %llu gpu %.3f ms wall %.3f ms parked %lld\n",
                             (long long)B.idx, B.njobs, (unsigned long long)B.quanta, ms,
                             1e3 * (now_s() - B.t_launch), parked);
            }
            // the round's launch status: bits that name no job fail the jobs
            // the round carried; a job's own status word fails that job alone
            const int rstat = B.h_stat[0] & ~kStatusBadJob;
            std::vector<std::shared_ptr<Job>> still;
            for (auto &j : active) {
                if (B.idx < j->admit_round) {
                    still.push_back(j);
                    continue;
                }
                const smcrt_totals &t = B.h_tot[j->slot];
                if (t.packets > 0 && t.busy_cycles > 0) j->cost = (double)t.busy_cycles / (double)t.packets;
                const bool drained = j->last_round <= completed;
                const bool failed = B.h_stat[1 + j->slot] != 0 || (rstat != 0 && j->last_round >= B.idx);
                if (failed) {
                    complete(j, &t, SMCRT_ERR_DEVICE);
                } else if ((uint64_t)t.packets >= j->npackets) {
                    complete(j, &t, SMCRT_OK);
                } else if (drained && is_cancelled(j)) {
                    complete(j, &t, SMCRT_ERR_CANCELLED);
                } else {
                    still.push_back(j);
                }
            }
            active.swap(still);
        }

        // ---- the next round: processor-sharing quanta over runnable jobs
        std::memset(B.h_tab, 0, sizeof(JobWork) * 2 * kMaxSlots);
        std::vector<std::shared_ptr<Job>> runnable, keep;
        for (auto &j : active) {
            if (is_cancelled(j)) {
                if (j->last_round <= completed) {   // nothing in flight: done now
                    complete(j, nullptr, SMCRT_ERR_CANCELLED);
                    continue;
                }
            } else {
                runnable.push_back(j);   // new ids and/or parked packets
            }
            keep.push_back(j);
        }
        active.swap(keep);
        if (runnable.empty()) {
            if (buf[1 - cur].busy) cur = 1 - cur;   // reap the other round next
            continue;
        }
        if (!tuned_served) {
            // the first mixed job served sets the served kernel's launch shape
            const Job *first = nullptr;
            for (auto &j : runnable)
                if (j->precision == SMCRT_MIXED) { first = j.get(); break; }
            if (first != nullptr) {
                cudaStreamSynchronize(st);   // no round in flight while the graphs are replaced
                tuned_served = true;
                if (tune_served(*first)) {
                    const int rc = capture();
                    if (rc != SMCRT_OK) {
                        // keep serving with the default shape captured at set-up
                        variant_m = 0;
                        threads_m = 128;
                        blocks_m = ctx->sm_count * std::max(1, occupancy_mixed_multi(threads_m, variant_m));
                        if (capture() != SMCRT_OK) {
                            for (auto &j : active) complete(j, nullptr, SMCRT_ERR_CUDA);
                            active.clear();
                            std::lock_guard<std::mutex> lk(ctx->mu);
                            ctx->sched_error = SMCRT_ERR_CUDA;
                            break;
                        }
                    }
                }
            }
        }
        double known = 0;
        int nk = 0;
        int nfresh = 0;
        for (auto &j : runnable) {
            if (j->cost > 0) { known += j->cost; ++nk; }
            if (j->cursor < j->npackets) ++nfresh;
        }
        const double dflt = nk ? known / nk : 2.0e5;
        // A round of parked packets only (every id claimed), with no job
        // waiting for admission: its packets are the last of their jobs, and
        // parking them again after 4 ms only repeats near-empty rounds
        // (measured: fifteen 4 ms rounds of a few hundred packets at the end
        // of a 40-job batch), so they run up to 50 ms.
        bool waiting = false;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            waiting = !ctx->queue.empty();
        }
        const long long budget = nfresh == 0 && !waiting ? tail_cycles : park_cycles;
        const double share = round_cycles() / (double)std::max(1, nfresh);
        int nm = 0, nd = 0;
        bool general = false;
        for (auto &j : runnable) {
            general = general || j->plan->host.general;
            const double c = j->cost > 0 ? j->cost : dflt;
            uint64_t q = (uint64_t)std::max(2048.0, share / c);
            if (!(j->cost > 0)) q = std::min<uint64_t>(q, 16384);   // unmeasured: a short first quantum
            q = std::min<uint64_t>(q, j->npackets - j->cursor);
            JobWork w{};
            w.next = j->cursor;
            w.end = j->cursor + q;
            w.begin = 0;
            w.seed = j->seed;
            w.fluence = (long long *)j->dflu;
            w.totals = d_tot + j->slot;
            w.records = nullptr;
            w.scene = j->id == bad_job ? nullptr : j->plan->dscene;
            w.cancelled = 0;
            w.park_cycles = budget;
            // a round with new ids ends soon after they run out; a round of
            // parked packets only lets them run the full budget
            w.drain_cycles = nfresh > 0 ? drain_cycles : budget;
            w.jstat = d_jstat + j->slot;
            w.defer = j->ddefer;
            w.defer_in = (int32_t)(issued & 1);
            w.stage = 0;   // the served kernels read the scene tables from global memory
            j->cursor += q;
            j->last_round = issued;
            if (j->precision == SMCRT_FP64) B.h_tab[kMaxSlots + nd++] = w;
            else B.h_tab[nm++] = w;
        }
        B.njobs = (int)runnable.size();
        B.quanta = 0;
        for (int k = 0; k < nm; ++k) B.quanta += B.h_tab[k].end - B.h_tab[k].next;
        for (int k = 0; k < nd; ++k) B.quanta += B.h_tab[kMaxSlots + k].end - B.h_tab[kMaxSlots + k].next;
        B.t_launch = now_s();
        cudaEventRecord(B.ev0, st);
        cudaGraphLaunch(general ? B.graph_g : B.graph, st);
        cudaEventRecord(B.ev, st);
        B.busy = true;
        B.idx = issued++;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->launches += 1;
        }
        cur = 1 - cur;
    }
    {   // a scheduler that stopped on an error fails what is still queued
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->sched_error != SMCRT_OK && setup_rc == SMCRT_OK) {
            while (!ctx->queue.empty()) {
                auto j = ctx->queue.front();
                ctx->queue.pop_front();
                j->status = ctx->sched_error;
                j->done = true;
                j->t_done = now_s();
            }
            ctx->cv_done.notify_all();
        }
    }
    // shut down: wait for rounds, free everything still held
    if (st) cudaStreamSynchronize(st);
    for (auto &j : active) free_job_device(*j, st);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        for (auto &j : ctx->to_release) free_job_device(*j, st);
        ctx->to_release.clear();
        for (auto &kv : ctx->jobs) free_job_device(*kv.second, st);   // done but never waited
    }
    if (st) cudaStreamSynchronize(st);
    for (auto &b : buf) {
        if (b.graph) cudaGraphExecDestroy(b.graph);
        if (b.graph_g) cudaGraphExecDestroy(b.graph_g);
        if (b.ev) cudaEventDestroy(b.ev);
        if (b.ev0) cudaEventDestroy(b.ev0);
        if (b.h_tab) cudaFreeHost(b.h_tab);
        if (b.h_tot) cudaFreeHost(b.h_tot);
        if (b.h_stat) cudaFreeHost(b.h_stat);
        if (b.d_tab) cudaFree(b.d_tab);
    }
    if (d_jstat) cudaFree(d_jstat);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (d_tot) cudaFree(d_tot);
    if (d_status) cudaFree(d_status);
    if (st2) cudaStreamDestroy(st2);
    if (st) cudaStreamDestroy(st);
}

void start_scheduler(smcrt_ctx *ctx)
{
    if (!ctx->sched_started) {
        ctx->sched = std::thread(scheduler, ctx);
        ctx->sched_started = true;
    }
}

}  // namespace

namespace smcrt {
// Field validation of scene / source / grid (no compilation, no allocation).
int validate_scene(const smcrt_scene *sc, const smcrt_source *src, const smcrt_grid *g)
{
    return validate(sc, src, g);
}
}  // namespace smcrt

extern "C" {

int smcrt_version(void) { return 10000; }

const char *smcrt_strerror(int code)
{
    switch (code) {
    case SMCRT_OK: return "ok";
    case SMCRT_ERR_BAD_ARG: return "bad argument";
    case SMCRT_ERR_BAD_SCENE: return "invalid scene, source or grid";
    case SMCRT_ERR_NO_MEMORY: return "out of memory or over the device memory budget";
    case SMCRT_ERR_CUDA: return "CUDA runtime error";
    case SMCRT_ERR_TIMEOUT: return "timed out";
    case SMCRT_ERR_CANCELLED: return "cancelled";
    case SMCRT_ERR_NOT_FOUND: return "unknown job";
    case SMCRT_ERR_DEVICE: return "kernel reported an error";
    default: return "unknown status";
    }
}

int smcrt_validate(const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid, int32_t *ninstr)
{
    int rc = validate(scene, source, grid);
    if (rc) return rc;
    std::vector<Instr> ins;
    std::vector<double> k64;
    std::vector<int2> rr;
    rc = compile(scene, ins, k64, rr);
    if (rc) return rc;
    if (ninstr) *ninstr = (int32_t)ins.size();
    return SMCRT_OK;
}

int smcrt_create(smcrt_ctx **out, int device, size_t budget)
{
    if (!out) return SMCRT_ERR_BAD_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SMCRT_ERR_BAD_ARG;
    CU(cudaSetDevice(device));
    std::unique_ptr<smcrt_ctx> c(new smcrt_ctx());
    c->device = device;
    CU(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
    size_t fr = 0, tot = 0;
    CU(cudaMemGetInfo(&fr, &tot));
    c->budget = budget ? budget : (size_t)(0.8 * (double)fr);
    *out = c.release();
    return SMCRT_OK;
}

int smcrt_destroy(smcrt_ctx *ctx)
{
    if (!ctx) return SMCRT_ERR_BAD_ARG;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv_work.notify_all();
    if (ctx->sched_started) ctx->sched.join();
    delete ctx;
    return SMCRT_OK;
}

int smcrt_plan_create(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source,
                      const smcrt_grid *grid, int32_t precision, smcrt_plan **out)
{
    if (!ctx || !out) return SMCRT_ERR_BAD_ARG;
    return build_plan(ctx, scene, source, grid, precision, out);
}

int smcrt_plan_destroy(smcrt_plan *pl)
{
    if (!pl) return SMCRT_ERR_BAD_ARG;
    cudaSetDevice(pl->ctx->device);
    cudaDeviceSynchronize();
    cudaFree(pl->dbuf);
    cudaFree(pl->djobs);
    cudaFree(pl->dstatus);
    delete pl;
    return SMCRT_OK;
}

int smcrt_plan_set_launch(smcrt_plan *pl, int32_t blocks, int32_t threads)
{
    if (!pl || blocks < 0 || threads < 0 || threads > kMaxThreads || (threads % 32) != 0) return SMCRT_ERR_BAD_ARG;
    pl->blocks = blocks;
    pl->threads = threads;
    return SMCRT_OK;
}

int smcrt_plan_launch(smcrt_plan *pl, uint64_t id_begin, uint64_t npackets, uint64_t seed, int64_t *fluence_dev,
                      smcrt_totals *totals_dev, smcrt_packet_record *records_dev, void *stream)
{
    if (!pl || !totals_dev) return SMCRT_ERR_BAD_ARG;
    if (npackets == 0) return SMCRT_OK;
    if (id_begin + npackets < id_begin) return SMCRT_ERR_BAD_ARG;
    int blocks, threads;
    default_launch(pl, blocks, threads);
    return plan_launch_impl(pl, id_begin, npackets, seed, fluence_dev, totals_dev, records_dev,
                            (cudaStream_t)stream, blocks, threads);
}

int smcrt_plan_set_variant(smcrt_plan *pl, int32_t variant)
{
    const int nv = pl && pl->precision == SMCRT_MIXED ? 2 * kNumVariants : kNumVariants;
    if (!pl || variant < 0 || variant >= nv) return SMCRT_ERR_BAD_ARG;
    pl->variant = variant % kNumVariants;
    pl->stage = variant / kNumVariants;
    return SMCRT_OK;
}

int smcrt_plan_status(smcrt_plan *pl, int32_t *status)
{
    if (!pl || !status) return SMCRT_ERR_BAD_ARG;
    int v = 0;
    CU(cudaMemcpy(&v, pl->dstatus, sizeof v, cudaMemcpyDeviceToHost));
    CU(cudaMemset(pl->dstatus, 0, sizeof(int)));
    *status = v;
    return SMCRT_OK;
}

int smcrt_plan_set_time_limit(smcrt_plan *pl, double seconds)
{
    if (!pl || !(seconds >= 0.0) || !std::isfinite(seconds)) return SMCRT_ERR_BAD_ARG;
    pl->time_limit_s = seconds;
    return SMCRT_OK;
}

int smcrt_set_time_limit(smcrt_ctx *ctx, double seconds)
{
    if (!ctx || !(seconds >= 0.0) || !std::isfinite(seconds)) return SMCRT_ERR_BAD_ARG;
    ctx->time_limit_s = seconds;
    return SMCRT_OK;
}

int smcrt_plan_autotune(smcrt_plan *pl, uint64_t trial, int32_t *blocks_out, int32_t *threads_out,
                        int32_t *variant_out)
{
    if (!pl || trial == 0) return SMCRT_ERR_BAD_ARG;
    CU(cudaSetDevice(pl->ctx->device));
    int64_t *flu = nullptr;
    smcrt_totals *tot = nullptr;
    if (cudaMalloc(&flu, pl->cells * 8) != cudaSuccess) return SMCRT_ERR_NO_MEMORY;
    if (cudaMalloc(&tot, sizeof(smcrt_totals)) != cudaSuccess) {
        cudaFree(flu);
        return SMCRT_ERR_NO_MEMORY;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bb = 0, bt = 0, bv = 0;
    const int thread_opts[] = {64, 128};
    const int saved_variant = pl->variant, saved_stage = pl->stage;
    int rc = SMCRT_OK;
    // register variant x (mixed) scene tables read from global memory or
    // staged in shared memory; public variant = register variant + 3 * stage
    const int nv = pl->precision == SMCRT_MIXED ? 2 * kNumVariants : kNumVariants;
    for (int pv = 0; pv < nv && rc == SMCRT_OK; ++pv) {
        const int v = pv % kNumVariants;
        pl->variant = v;
        pl->stage = pv / kNumVariants;
        for (int t : thread_opts) {
            const int occ = occupancy(pl->precision, t, v);
            if (occ < 1) continue;
            for (int mult : {1, 2}) {
                const int b = pl->ctx->sm_count * occ * mult;
                float ms_best = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    cudaMemsetAsync(flu, 0, pl->cells * 8, 0);
                    cudaMemsetAsync(tot, 0, sizeof(smcrt_totals), 0);
                    cudaEventRecord(e0, 0);
                    rc = plan_launch_impl(pl, 0, trial, 12345, flu, tot, nullptr, 0, b, t);
                    cudaEventRecord(e1, 0);
                    if (rc != SMCRT_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                        rc = SMCRT_ERR_CUDA;
                        break;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms_best = std::min(ms_best, ms);
                }
                if (rc != SMCRT_OK) break;
                if (ms_best < best) {
                    best = ms_best;
                    bb = b;
                    bt = t;
                    bv = pv;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(flu);
    cudaFree(tot);
    if (rc != SMCRT_OK) {
        pl->variant = saved_variant;
        pl->stage = saved_stage;
        return rc;
    }
    pl->blocks = bb;
    pl->threads = bt;
    pl->variant = bv % kNumVariants;
    pl->stage = bv / kNumVariants;
    {
        std::lock_guard<std::mutex> lk(pl->ctx->tune_mu);
        pl->ctx->tuned[pl->shape_key] = {bb, bt, bv};
    }
    if (blocks_out) *blocks_out = bb;
    if (threads_out) *threads_out = bt;
    if (variant_out) *variant_out = bv;
    return SMCRT_OK;
}

int smcrt_run(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid,
              uint64_t npackets, uint64_t seed, int32_t precision, int64_t *fluence_out, smcrt_totals *totals_out)
{
    if (!ctx || !totals_out) return SMCRT_ERR_BAD_ARG;
    smcrt_plan *pl = nullptr;
    int rc = build_plan(ctx, scene, source, grid, precision, &pl);
    if (rc) return rc;
    const size_t fb = pl->cells * 8;
    int64_t *dflu = nullptr;
    smcrt_totals *dtot = nullptr;
    const bool dev_out = fluence_out && is_device_ptr(fluence_out);
    rc = SMCRT_OK;
    if (fluence_out) {
        if (dev_out) dflu = fluence_out;
        else if (cudaMalloc(&dflu, fb) != cudaSuccess) rc = SMCRT_ERR_NO_MEMORY;
    }
    if (rc == SMCRT_OK && cudaMalloc(&dtot, sizeof(smcrt_totals)) != cudaSuccess) rc = SMCRT_ERR_NO_MEMORY;
    if (rc == SMCRT_OK) {
        if (dflu && cudaMemsetAsync(dflu, 0, fb, 0) != cudaSuccess) rc = SMCRT_ERR_CUDA;
        if (cudaMemsetAsync(dtot, 0, sizeof(smcrt_totals), 0) != cudaSuccess) rc = SMCRT_ERR_CUDA;
    }
    if (rc == SMCRT_OK && npackets > 0) {
        int blocks, threads;
        default_launch(pl, blocks, threads);
        rc = plan_launch_impl(pl, 0, npackets, seed, dflu, dtot, nullptr, 0, blocks, threads);
    }
    smcrt_totals t{};
    if (rc == SMCRT_OK) {
        if (cudaMemcpy(&t, dtot, sizeof t, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SMCRT_ERR_CUDA;
        else if (fluence_out && !dev_out && cudaMemcpy(fluence_out, dflu, fb, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = SMCRT_ERR_CUDA;
    }
    int32_t ks = 0;
    if (rc == SMCRT_OK && smcrt_plan_status(pl, &ks) == SMCRT_OK && ks)
        rc = (ks & kStatusTimeout) ? SMCRT_ERR_TIMEOUT : SMCRT_ERR_DEVICE;
    if (rc == SMCRT_OK) *totals_out = t;
    if (dflu && !dev_out) cudaFree(dflu);
    if (dtot) cudaFree(dtot);
    smcrt_plan_destroy(pl);
    return rc;
}

int smcrt_submit(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid,
                 uint64_t npackets, uint64_t seed, int32_t precision, uint64_t *job_id)
{
    if (!ctx || !job_id) return SMCRT_ERR_BAD_ARG;
    if (precision != SMCRT_FP64 && precision != SMCRT_MIXED) return SMCRT_ERR_BAD_ARG;
    int rc = validate(scene, source, grid);
    if (rc) return rc;
    std::vector<Instr> ins;
    std::vector<double> k64;
    std::vector<int2> rr;
    rc = compile(scene, ins, k64, rr);
    if (rc) return rc;
    auto j = std::make_shared<Job>();
    j->prims.assign(scene->prims, scene->prims + scene->nprims);
    j->nodes.assign(scene->nodes, scene->nodes + scene->nnodes);
    j->regions.assign(scene->regions, scene->regions + scene->nregions);
    if (scene->nxforms > 0) j->xforms.assign(scene->xforms, scene->xforms + scene->nxforms);
    j->scene = *scene;
    j->scene.prims = j->prims.data();
    j->scene.nodes = j->nodes.data();
    j->scene.regions = j->regions.data();
    j->scene.xforms = scene->nxforms > 0 ? j->xforms.data() : nullptr;
    j->source = *source;
    j->grid = *grid;
    j->npackets = npackets;
    j->seed = seed;
    j->precision = precision;
    j->t_submit = now_s();
    j->bytes = job_bytes(*grid);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->sched_error) return ctx->sched_error;
        if (j->bytes > ctx->budget) return SMCRT_ERR_NO_MEMORY;
        j->id = ctx->next_job_id++;
        ctx->jobs[j->id] = j;
        if (npackets == 0) {
            j->done = true;
            j->t_done = j->t_submit;
        } else {
            ctx->queue.push_back(j);
        }
        *job_id = j->id;
        start_scheduler(ctx);
    }
    ctx->cv_work.notify_all();
    return SMCRT_OK;
}

int smcrt_poll(smcrt_ctx *ctx, uint64_t job_id, int32_t *done)
{
    if (!ctx || !done) return SMCRT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(job_id);
    if (it == ctx->jobs.end()) return SMCRT_ERR_NOT_FOUND;
    *done = it->second->done ? 1 : 0;
    return SMCRT_OK;
}

int smcrt_wait(smcrt_ctx *ctx, uint64_t job_id, double timeout_s, int64_t *fluence_out, smcrt_totals *totals_out,
               double *latency_s)
{
    if (!ctx) return SMCRT_ERR_BAD_ARG;
    std::shared_ptr<Job> j;
    {
        std::unique_lock<std::mutex> lk(ctx->mu);
        auto it = ctx->jobs.find(job_id);
        if (it == ctx->jobs.end()) return SMCRT_ERR_NOT_FOUND;
        j = it->second;
        auto pred = [&] { return j->done; };
        if (timeout_s < 0) {
            ctx->cv_done.wait(lk, pred);
        } else if (!ctx->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
            return SMCRT_ERR_TIMEOUT;
        }
        ctx->jobs.erase(job_id);
    }
    int rc = j->status;
    cudaSetDevice(ctx->device);
    if (rc == SMCRT_OK) {
        if (fluence_out && j->dflu) {
            const size_t fb = (size_t)j->grid.n[0] * j->grid.n[1] * j->grid.n[2] * 8;
            if (cudaMemcpy(fluence_out, j->dflu, fb, cudaMemcpyDefault) != cudaSuccess) rc = SMCRT_ERR_CUDA;
        } else if (fluence_out && j->npackets == 0) {
            std::memset(fluence_out, 0, (size_t)j->grid.n[0] * j->grid.n[1] * j->grid.n[2] * 8);
        }
        if (totals_out) *totals_out = j->totals;
    }
    if (latency_s) *latency_s = j->t_done - j->t_submit;
    if (j->admitted) {   // the scheduler frees the device memory, stream-ordered
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->mem_in_use -= std::min(ctx->mem_in_use, j->bytes);
            j->admitted = false;
            ctx->to_release.push_back(j);
        }
        ctx->cv_work.notify_all();
    }
    return rc;
}

int smcrt_cancel(smcrt_ctx *ctx, uint64_t job_id)
{
    if (!ctx) return SMCRT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(job_id);
    if (it == ctx->jobs.end()) return SMCRT_ERR_NOT_FOUND;
    it->second->cancelled = true;
    return SMCRT_OK;
}

int smcrt_serving_stats(smcrt_ctx *ctx, int64_t *queued, int64_t *running, int64_t *launches)
{
    if (!ctx) return SMCRT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (queued) *queued = (int64_t)ctx->queue.size();
    if (running) *running = ctx->running;
    if (launches) *launches = ctx->launches;
    return SMCRT_OK;
}

}  // extern "C"
