/*
 * smcrt.h -- C-ABI of the GB300 photon-packet propagation library.
 *
 * The library propagates photon packets through turbid media whose geometry
 * is a set of signed distance functions (SDFs) combined by constructive
 * solid geometry (CSG), as in signedMCRT (McMillan, Bruce & Dholakia,
 * "Meshless Monte Carlo Radiation Transfer Method for Curved Geometries
 * using Signed Distance Functions"):
 *   - Sec. 2.1, Eq. 1: optical depth tau = -ln(xi), free path tau / mu_t;
 *   - Sec. 2.2, Eq. 2-3 and Fig. 1: SDF primitives and CSG operations;
 *   - Sec. 2.3, Fig. 2 (right) and Fig. 3: sphere tracing to the nearest
 *     surface, threshold delta, Fresnel reflection / Snell refraction with
 *     the normal from the SDF gradient, bounding box as volume of interest;
 *   - Sec. 3.1: Henyey-Greenstein scattering; absorption weighting with
 *     Russian roulette (the paper reuses its earlier codes' routines);
 *   - Sec. 3.1-3.2: fluence tallied in rectangular voxel bins.
 *
 * Units: lengths in cm, coefficients in cm^-1.  Every tally is a signed
 * 64-bit fixed-point number in units of 2^-32 packet weight (fluence: weight
 * x path length in cm), accumulated with integer atomics, so results do not
 * depend on execution order and are bit-reproducible.
 *
 * Conventions for every function:
 *   - return value: SMCRT_OK (0) or a negative SMCRT_ERR_* code; on error
 *     no output is written and no job is created;
 *   - host structs passed in are read during the call only; the caller
 *     keeps ownership;
 *   - "device pointer" means memory of the context's CUDA device (for
 *     example a torch CUDA tensor's data_ptr()); "host or device" pointers
 *     are classified with cudaPointerGetAttributes;
 *   - a context is used from one host thread at a time, except that
 *     smcrt_submit / smcrt_poll / smcrt_wait / smcrt_cancel may be called
 *     from any thread (the serving queue is internally locked).
 */
#ifndef SMCRT_H
#define SMCRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SMCRT_OK 0
#define SMCRT_ERR_BAD_ARG -1      /* null pointer, zero size, unknown enum */
#define SMCRT_ERR_BAD_SCENE -2    /* scene / source / grid failed validation */
#define SMCRT_ERR_NO_MEMORY -3    /* device or host allocation failed, or over budget */
#define SMCRT_ERR_CUDA -4         /* a CUDA runtime call failed */
#define SMCRT_ERR_TIMEOUT -5      /* smcrt_wait timed out (job keeps running), or a launch's
                                     device time limit expired (smcrt_set_time_limit) */
#define SMCRT_ERR_CANCELLED -6    /* job was cancelled */
#define SMCRT_ERR_NOT_FOUND -7    /* unknown job id */
#define SMCRT_ERR_DEVICE -8       /* kernel reported an error status word */

/* ---- bits of the kernels' status word (smcrt_plan_status) ------------- */
#define SMCRT_STATUS_BAD_JOB 1    /* a launch descriptor without scene or totals, or a scene
                                     that needs the general-shape kernel */
#define SMCRT_STATUS_TIMEOUT 4    /* the launch's device time limit expired */

/* ---- scene description (Sec. 2.2-2.3) ---------------------------------- */
enum smcrt_prim_kind {
    SMCRT_SPHERE = 0,   /* p = {cx, cy, cz, r}: |x - c| - r (Eq. 2-3) */
    SMCRT_BOX = 1,      /* p = {cx, cy, cz, hx, hy, hz}: exact box distance */
    SMCRT_CAPSULE = 2,  /* p = {ax, ay, az, bx, by, bz, r}: segment distance - r */
    SMCRT_TORUS = 3,    /* p = {cx, cy, cz, R, r}, 0 < r < R: ring about the z axis
                         * through c; distance to the core circle - r (Fig. 1 basic shapes) */
    SMCRT_CYLINDER = 4  /* p = {cx, cy, cz, r, h}: capped cylinder along z through c,
                         * radius r, half height h; exact distance */
};

/* Domain operation applied to a primitive's local coordinates (Sec. 2.2:
 * SDFs "can easily be translated, rotated, twisted and scaled"; Fig. 1
 * i, o, p, q).  Operations that stretch space divide the distance by their
 * Lipschitz bound, so it never exceeds the true distance (Sec. 5 on
 * non-bounded SDFs). */
enum smcrt_domain_op {
    SMCRT_XF_NONE = 0,
    SMCRT_XF_ELONGATE = 1,  /* a[0..2] >= 0: q - clamp(q, -a, a) (exact outside) */
    SMCRT_XF_TWIST = 2,     /* (x, y) rotated by 2 pi a[0] z (a[0] turns per unit length);
                             * a[1] >= 0 the radius the shape reaches from the axis.  With
                             * m = 2 pi a[0] max(rho, a[1]) the distance is divided by
                             * (m + sqrt(m^2 + 4)) / 2, the map's largest stretch */
    SMCRT_XF_BEND = 3,      /* (x, y) rotated by 2 pi a[0] x; a[1] as for twist; divided
                             * by 1 + m */
    SMCRT_XF_REPEAT = 4     /* a[0..2] >= 0 periods (0 = not repeated), a[3] >= 0 integer
                             * copies each way: nearest copy; exact for a shape centred
                             * at the local origin and inside its cell */
};

/* Frame of a primitive: the point with local coordinates l sits at
 * s R l + t.  The distance is s * d_local(op(R^T (x - t) / s)) / L. */
typedef struct {
    double rot[9];      /* R, row-major, orthonormal with det +1 (1e-9) */
    double t[3];        /* translation (cm) */
    double s;           /* uniform scale, > 0 */
    int32_t op;         /* enum smcrt_domain_op */
    int32_t reserved;   /* must be 0 */
    double a[4];        /* parameters of op */
} smcrt_xform;

enum smcrt_op {         /* postfix CSG program nodes (Sec. 2.2, Fig. 1 e-h) */
    SMCRT_OP_PRIM = 0,          /* push primitive `prim` */
    SMCRT_OP_UNION = 1,         /* min(a, b) */
    SMCRT_OP_SMOOTH_UNION = 2,  /* polynomial smooth minimum with radius k > 0 */
    SMCRT_OP_INTERSECT = 3,     /* max(a, b) */
    SMCRT_OP_SUBTRACT = 4       /* max(a, -b): a minus b */
};

typedef struct {
    int32_t kind;       /* enum smcrt_prim_kind */
    int32_t xform;      /* 0: p in scene coordinates; k > 0: p in the frame xforms[k - 1] */
    double p[7];        /* parameters, see smcrt_prim_kind */
} smcrt_prim;

typedef struct {
    int32_t op;         /* enum smcrt_op */
    int32_t prim;       /* primitive index for SMCRT_OP_PRIM, else ignored */
    double k;           /* smoothing radius (cm) for SMCRT_OP_SMOOTH_UNION */
} smcrt_csg_node;

/* One optical region: its SDF is the value of nodes[node_begin ..
 * node_begin+node_count) evaluated as a postfix program (binary operators
 * take the earlier operand as a, the later as b).  A point belongs to the
 * highest-index region whose SDF is negative there, else to the ambient
 * medium (mu_a = mu_s = 0, n = ambient_n).  Sec. 2.3: "Each SDF has its
 * own set of optical properties". */
typedef struct {
    int32_t node_begin;
    int32_t node_count;
    double mu_a;        /* absorption coefficient, >= 0 */
    double mu_s;        /* scattering coefficient, >= 0 */
    double g;           /* Henyey-Greenstein anisotropy, in (-1, 1) */
    double n;           /* refractive index, >= 1 */
} smcrt_region;

/* How a packet's move between scene evaluations is bounded. */
enum smcrt_stepping {
    /* Sphere tracing (Sec. 2.3, Fig. 3): move d_min - delta/2, the distance
     * to the nearest surface less half the threshold. */
    SMCRT_STEP_SPHERE_TRACING = 0,
    /* Segment stepping (Sec. 5 names segment tracing for packets moving
     * nearly parallel to a surface): move max(d_min - delta/2, B), where B
     * bounds the move along the packet's own direction.  Each primitive of
     * a region with at most eight smooth unions takes the margin
     * e = M + delta/2, M the sum of k/4 over the smooth unions of the
     * regions that use it (0 for hard CSG: union, intersection,
     * subtraction); its bound is the distance along the ray until |d| can
     * reach e: spheres, boxes, capsules and capped cylinders grown by e
     * from outside and shrunk by e from inside, tori from outside (through
     * the annular slab that holds the grown tube) and from inside (through
     * the ball of radius r - e about the nearest point of the core circle),
     * the same shapes placed by a frame without a domain operation;
     * |d| - e for domain operations.  Regions with more than eight smooth unions
     * take |d| - delta/2 (in mixed precision so does a union of 16 or more
     * primitives, which is evaluated through a grid of per-cell candidate
     * lists); the bounding box takes its exit distance less delta/2.  The
     * move stops delta/2 short of the first surface it would reach, and the
     * interface handling is unchanged.  Same transport, fewer steps. */
    SMCRT_STEP_SEGMENT = 1
};

typedef struct {
    const smcrt_prim *prims;       /* host array of nprims */
    int32_t nprims;                /* 1 .. 4096 */
    const smcrt_csg_node *nodes;   /* host array of nnodes */
    int32_t nnodes;
    const smcrt_region *regions;   /* host array of nregions */
    int32_t nregions;              /* 1 .. 64; postfix stack depth <= 4 */
    double ambient_n;              /* refractive index outside all regions */
    double bbox_lo[3];             /* bounding box: the volume of interest; */
    double bbox_hi[3];             /* leaving it terminates a packet (Sec. 2.3) */
    double delta;                  /* surface threshold delta (cm), > 0 */
    int64_t max_steps;             /* per-packet step cap (grazing guard), > 0 */
    int32_t stepping;              /* enum smcrt_stepping */
    int32_t reserved;              /* must be 0 */
    const smcrt_xform *xforms;     /* host array of nxforms (may be NULL if 0) */
    int32_t nxforms;               /* 0 .. 4096 */
    int32_t reserved2;             /* must be 0 */
} smcrt_scene;

enum smcrt_source_kind {
    SMCRT_SRC_PENCIL = 0,     /* all packets start at pos heading dir */
    SMCRT_SRC_DISC = 1,       /* uniform over a disc of `radius` about pos, normal dir */
    SMCRT_SRC_SQUARE = 2,     /* uniform over a square of half side `radius` about pos */
    SMCRT_SRC_ISO_POINT = 3   /* isotropic directions from pos */
};

typedef struct {
    int32_t kind;        /* enum smcrt_source_kind */
    int32_t reserved;    /* must be 0 */
    double pos[3];
    double dir[3];       /* unit vector; also splits escapes into R (u.dir < 0) and T */
    double radius;
} smcrt_source;

/* Fluence grid: n[0] x n[1] x n[2] rectangular voxels over [lo, hi],
 * stored [z][y][x] with x fastest (Sec. 3.1-3.2 rectangular bins). */
typedef struct {
    double lo[3];
    double hi[3];
    int32_t n[3];        /* each 1 .. 1024 */
    int32_t reserved;    /* must be 0 */
} smcrt_grid;

enum smcrt_precision {
    SMCRT_FP64 = 0,   /* every step in FP64, bit-identical to the FP64 reference */
    SMCRT_MIXED = 1   /* FP32 tracing/scattering; FP64 interface refinement near
                         grazing and critical incidence; exact int64 tallies */
};

/* Totals of one run, all int64.  R, T, A, killed, gain are fixed point
 * (2^-32 weight units): R + T + A + killed - gain = packets * 2^32 up to
 * one half unit per deposit.  The rest are event counts. */
typedef struct {
    int64_t R;            /* escaped with u.dir < 0 (reflected) */
    int64_t T;            /* escaped otherwise (transmitted) */
    int64_t A;            /* absorbed (implicit capture, w mu_a / mu_t per interaction) */
    int64_t killed;       /* removed by roulette or the step cap */
    int64_t gain;         /* added by roulette survivors */
    int64_t packets;      /* packets completed */
    int64_t scatters;     /* interactions */
    int64_t steps;        /* sphere-tracing iterations */
    int64_t scene_evals;  /* full scene SDF evaluations (all phases) */
    int64_t interfaces;   /* index-boundary arrivals (Sec. 2.3, d_sdf < delta) */
    int64_t fresnel;      /* of which with a refractive-index change */
    int64_t pieces;       /* voxel deposits */
    int64_t max_steps_hit;/* packets stopped by the step cap */
    int64_t refined;      /* mixed mode: interfaces refined in FP64 */
    int64_t busy_cycles;  /* SM clock cycles warps spent on this job (summed over warps) */
    int64_t parked;       /* serving: times a packet was parked at a round's time budget */
} smcrt_totals;

/* Optional per-packet record (debugging and per-packet parity). */
typedef struct {
    int64_t R, T, A, killed, gain, scatters, steps, reserved;
} smcrt_packet_record;

typedef struct smcrt_ctx smcrt_ctx;
typedef struct smcrt_plan smcrt_plan;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`.  device_mem_budget bounds the
 * device memory the serving queue may hold for admitted jobs (0 = 80% of
 * the free memory at creation).  *out receives the context. */
int smcrt_create(smcrt_ctx **out, int device, size_t device_mem_budget);

/* Wait for outstanding work, free every device buffer, destroy ctx. */
int smcrt_destroy(smcrt_ctx *ctx);

/* Static string for a status code. */
const char *smcrt_strerror(int code);

/* Library version as major*10000 + minor*100 + patch. */
int smcrt_version(void);

/* Validate scene/source/grid and compile the CSG programs without touching
 * a device (Sec. 2.2-2.3 scene model).  *ninstr (may be NULL) receives the
 * length of the compiled instruction stream.  Returns OK, BAD_ARG or
 * BAD_SCENE.  Needs no context and no GPU. */
int smcrt_validate(const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid,
                   int32_t *ninstr);

/* ---- plans: a validated, compiled, device-resident scene --------------- */

/* Validate scene/source/grid, compile the CSG programs into the device
 * instruction stream of the chosen precision and upload it.  *out owns the
 * device copy until smcrt_plan_destroy.  Errors: BAD_ARG, BAD_SCENE,
 * NO_MEMORY, CUDA. */
int smcrt_plan_create(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source,
                      const smcrt_grid *grid, int32_t precision, smcrt_plan **out);

int smcrt_plan_destroy(smcrt_plan *plan);

/* Launch configuration of the persistent packet kernel: blocks (0 = SM
 * count x resident blocks per SM) and threads per block (a multiple of 32,
 * 32 .. 128; 0 = tuned default).  Other values return BAD_ARG. */
int smcrt_plan_set_launch(smcrt_plan *plan, int32_t blocks, int32_t threads);

/* Asynchronously propagate packets [id_begin, id_begin + npackets) with
 * Philox key `seed` on CUDA stream `stream` (a cudaStream_t; NULL = legacy
 * default stream).  fluence_dev (device pointer, n[0]*n[1]*n[2] int64, may
 * be NULL for no grid tally) and totals_dev (device pointer to one
 * smcrt_totals) are ACCUMULATED into -- zero them first for a fresh run.
 * records_dev (device pointer to npackets records, or NULL) receives one
 * record per packet, indexed by id - id_begin.  Packet ids are independent
 * (counter-based RNG), so a job split into id blocks gives the same tallies
 * as one launch. */
int smcrt_plan_launch(smcrt_plan *plan, uint64_t id_begin, uint64_t npackets, uint64_t seed,
                      int64_t *fluence_dev, smcrt_totals *totals_dev,
                      smcrt_packet_record *records_dev, void *stream);

/* Register budget of the packet kernel: variant 0, 1, 2 keep 5/4/3 (mixed)
 * or 4/3/2 (FP64) blocks of 128 threads resident per SM; fewer resident
 * blocks give each thread more registers (no spilling) at lower occupancy.
 * MIXED plans also take 3, 4, 5: the same budgets with each warp staging
 * the scene's instruction stream and FP32 tables in shared memory (when
 * they fit 4 KiB).  Results do not depend on the variant. */
int smcrt_plan_set_variant(smcrt_plan *plan, int32_t variant);

/* Read back the kernel's device error word for the plan's last launches
 * (0 = none; SMCRT_STATUS_* bits) and clear it. */
int smcrt_plan_status(smcrt_plan *plan, int32_t *status);

/* Device time limit of the plan's later launches (seconds; 0 = none, the
 * default is the context's, smcrt_set_time_limit).  Each warp of the packet
 * kernel reads the GPU's global nanosecond timer when it claims new packet
 * ids; once the limit has passed since it started on the launch it claims no
 * more, lets the packets it holds finish (each bounded by the step cap) and
 * returns, and the kernel sets SMCRT_STATUS_TIMEOUT in the status word.  The
 * totals and the fluence then cover exactly the packets that completed
 * (totals.packets of them; R + T + A + killed - gain closes over those).
 * The paper has no counterpart: this bounds a launch's time on the device.
 * Errors: BAD_ARG for a negative or non-finite value. */
int smcrt_plan_set_time_limit(smcrt_plan *plan, double seconds);

/* The context's device time limit (seconds, 0 = none): applied to smcrt_run,
 * which then returns SMCRT_ERR_TIMEOUT (and writes nothing) when it expires,
 * and the default of plans created afterwards.  Serving rounds are bounded by
 * their own budgets and do not use it. */
int smcrt_set_time_limit(smcrt_ctx *ctx, double seconds);

/* Time the candidate launch shapes (register-budget variant x, for MIXED
 * plans, scene tables in global or shared memory x threads per block x
 * resident blocks) on a short trial run of this plan and keep the
 * fastest; the choice is cached per scene shape in the context and applied
 * to later plans of the same shape.  Trial tallies go to scratch buffers.
 * *blocks / *threads / *variant (may be NULL) receive the choice. */
int smcrt_plan_autotune(smcrt_plan *plan, uint64_t trial_packets, int32_t *blocks,
                        int32_t *threads, int32_t *variant);

/* ---- launch without device allocation ---------------------------------- */

/* The packet launch of smcrt_plan_launch, for callers that must not
 * allocate device memory: for example a host application whose own memory
 * pool reserves the device up front and forbids other cudaMalloc calls, or
 * a latency-critical loop in which an allocation (which can synchronise the
 * device) is not allowed.  The paper has no counterpart; this is a property
 * of the library's interface, not of the method.
 *
 * Needs no context: it runs on the current CUDA device and on `stream` (a
 * cudaStream_t, NULL = legacy default stream), asynchronously.  All the
 * scratch it needs -- the compiled scene, the launch descriptor and the
 * kernel's status word -- lives in one fixed device array of 64 KiB inside
 * the library, held by every device that loads the library until the process
 * exits.  Scenes are limited accordingly: at most 128 primitives, 256 CSG
 * nodes and 16 regions (larger ones return SMCRT_ERR_NO_MEMORY; invalid ones
 * SMCRT_ERR_BAD_SCENE or SMCRT_ERR_BAD_ARG).  It calls no cudaMalloc or
 * cudaFree and allocates no host memory: the scene is compiled into a fixed
 * host buffer (calls from several host threads take turns on it) and reaches
 * the device array in the launch arguments of small copy kernels, so nothing
 * reads the caller's or the library's host memory after the call returns.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call shares the one array and leaves its contents
 * behind: the status word is cleared by each call, the rest is overwritten.
 * Calls whose work overlaps on the GPU race on the array -- order them on one
 * stream or wait between them.
 *
 * Arguments as smcrt_plan_launch: packets [id_begin, id_begin + npackets)
 * with key `seed`; fluence_dev (may be NULL) and totals_dev are device
 * pointers the results are ACCUMULATED into (zero them first).  Results are
 * identical to a plan launch of the same scene, ids and seed, except in
 * MIXED precision for scenes with a union or smooth-union region of 16 or
 * more primitives: a plan evaluates that region through a spatial cell list
 * (a different, equally valid distance bound away from the surface), this
 * call evaluates it in full, so the two agree statistically, not bit for
 * bit. */
int smcrt_run_noalloc(const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid,
                      uint64_t id_begin, uint64_t npackets, uint64_t seed, int32_t precision,
                      int64_t *fluence_dev, smcrt_totals *totals_dev, void *stream);

/* ---- one-shot synchronous run ------------------------------------------ */

/* Plan, launch and wait: packets [0, npackets), key `seed`.  fluence_out
 * (host or device, n[0]*n[1]*n[2] int64, may be NULL) and totals_out (host)
 * are OVERWRITTEN with this run's tallies.  Host-to-device and
 * device-to-host copies happen inside the call. */
int smcrt_run(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source,
              const smcrt_grid *grid, uint64_t npackets, uint64_t seed, int32_t precision,
              int64_t *fluence_out, smcrt_totals *totals_out);

/* ---- serving: continuously batched jobs ------------------------------- */

/* Queue a job (same arguments as smcrt_run).  Jobs are admitted to device
 * slots in arrival order as slots and device memory (fluence grid + scene)
 * free up; all admitted jobs share each persistent launch, which runs
 * under a captured CUDA graph.  *job_id receives a handle.  Errors:
 * BAD_ARG, BAD_SCENE, NO_MEMORY (the job alone exceeds the budget). */
int smcrt_submit(smcrt_ctx *ctx, const smcrt_scene *scene, const smcrt_source *source,
                 const smcrt_grid *grid, uint64_t npackets, uint64_t seed, int32_t precision,
                 uint64_t *job_id);

/* *done = 1 when the job's results are ready (or it failed), else 0. */
int smcrt_poll(smcrt_ctx *ctx, uint64_t job_id, int32_t *done);

/* Block until the job completes or timeout_s elapses (< 0: forever).
 * Copies the fluence (host pointer, may be NULL) and totals (host, may be
 * NULL), then releases the job.  Returns TIMEOUT (job kept), CANCELLED,
 * DEVICE, or OK.  *latency_s (may be NULL) receives submit-to-completion
 * wall time. */
int smcrt_wait(smcrt_ctx *ctx, uint64_t job_id, double timeout_s, int64_t *fluence_out,
               smcrt_totals *totals_out, double *latency_s);

/* Stop issuing new packets of the job; its result becomes CANCELLED. */
int smcrt_cancel(smcrt_ctx *ctx, uint64_t job_id);

/* Serving counters: jobs queued, running, launches issued so far. */
int smcrt_serving_stats(smcrt_ctx *ctx, int64_t *queued, int64_t *running, int64_t *launches);

/* Measured ceilings of this GPU for the packet kernel's roofline (the paper
 * has no counterpart; Sec. 3.2 reports CPU timings only):
 *   fp32_flops        FP32 FMA throughput (an FMA counts 2 flops) of a
 *                     kernel of eight independent FMA chains per thread;
 *   atomics_distinct  int64 atomic adds per second to scattered addresses
 *                     of a 64 MiB table (the fluence tally's access);
 *   atomics_hot       the same to 32 addresses (a beam's hottest voxels).
 * scratch_dev: caller-owned device memory of at least 64 MiB, overwritten.
 * Synchronous; runs on a private stream of `device`.  Returns
 * SMCRT_ERR_BAD_ARG for null pointers or a smaller scratch. */
int smcrt_microbench(int device, void *scratch_dev, size_t scratch_bytes, double *fp32_flops,
                     double *atomics_distinct, double *atomics_hot);

#ifdef __cplusplus
}
#endif

#endif /* SMCRT_H */
