// smcrt_k64.cu -- plain FP64 packet kernel (compiled with -fmad=false).
//
// Every floating-point step is an IEEE double operation in the order of the
// reference algorithm (Sec. 2.3 sphere tracing and interface handling,
// Eq. 1 free path, Sec. 3.1 HG scattering), so the int64 tallies equal the
// FP64 CPU reference bit for bit for any packet count.
#include "smcrt_kernel.cuh"

namespace smcrt {

namespace {

__device__ __forceinline__ double hg_cos64(double g, double xi)
{   // Henyey-Greenstein inverse CDF (Sec. 3.1); isotropic for |g| < 1e-6
    double c;
    if (fabs(g) < 1e-6) {
        c = 2.0 * xi - 1.0;
    } else {
        const double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
        c = (1.0 + g * g - t * t) / (2.0 * g);
    }
    return fmin(fmax(c, -1.0), 1.0);
}

__device__ __forceinline__ void normalise64(double &x, double &y, double &z)
{
    const double l = sqrt(x * x + y * y + z * z);
    x = x / l;
    y = y / l;
    z = z / l;
}

__device__ __forceinline__ void scatter64(double &ux, double &uy, double &uz, double ct, double xi_phi)
{
    const double st = sqrt((1.0 - ct) * (1.0 + ct));
    double sp, cp;
    sincos2pi64(xi_phi, &sp, &cp);
    double b1[3], b2[3];
    onb64(ux, uy, uz, b1, b2);
    const double a1 = st * cp, a2 = st * sp;
    double vx = a1 * b1[0] + a2 * b2[0] + ct * ux;
    double vy = a1 * b1[1] + a2 * b2[1] + ct * uy;
    double vz = a1 * b1[2] + a2 * b2[2] + ct * uz;
    normalise64(vx, vy, vz);
    ux = vx; uy = vy; uz = vz;
}

__device__ __forceinline__ double region_n64(const DevScene &S, int r)
{
    return r < 0 ? S.ambient_n : __ldg(S.reg64 + 8 * r + 3);
}

struct WarpShared {
    DevScene S;
    WarpAcc acc;
    JobConst jc;
};

// Same iteration structure as the mixed kernel (refill, one scene
// evaluation, classify, one tally site, one Philox call, consumers), with
// every floating-point operation the reference algorithm's, in its order:
// the oracle's run of a packet is a sequence of the same IEEE operations on
// the same values, so its tallies come out bit for bit.
template <bool G>
__device__ bool run_job_fp64(const DevScene &S, WarpAcc *wa, const volatile JobConst *jc, JobWork *J,
                             int lane)
{
    const double delta = S.delta;

    bool alive = false, retired = false;
    double px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0, w = 0, tau = 0;
    double qx = 0, qy = 0, qz = 0;       // NRM: gradient; PROJ / FAR / NEAR: surface point
    double nx = 0, ny = 0, nz = 0, cdot = 0, fplus = 0, dstar = 0;
    int phase = kTrace, sub = 0, istar = -1, reg = -1, rfar = -1;
    int nsteps = 0;
    unsigned pscat = 0, npieces = 0;
    long long pA = 0, pG = 0;
    uint32_t id_lo = 0, id_hi = 0, event = 0;
    uint32_t t_acq = 0;
    bool timed_out = false;              // the launch's time limit stopped the refills

    for (;;) {
        // ---- 1. refill: this job's parked packets first, then new ids
        {
            unsigned need = __ballot_sync(SMCRT_FULL, !alive && !retired);
            JobDefer *const dfr = (JobDefer *)jc->dfr;
            const int din = jc->din;
            if (need && dfr != nullptr) {
                const int leader = __ffs(need) - 1;
                unsigned base = 0u, avail = 0u;
                if (lane == leader) {
                    // the counter also counts packets that found the list full
                    // (they kept running): only the first `cap` entries exist
                    avail = min(*(volatile unsigned *)&dfr->count[din], dfr->cap);
                    base = atomicAdd(&dfr->cursor[din], (unsigned)__popc(need));
                }
                base = __shfl_sync(SMCRT_FULL, base, leader);
                avail = __shfl_sync(SMCRT_FULL, avail, leader);
                if (!alive && !retired) {
                    const unsigned k = base + (unsigned)__popc(need & ((1u << lane) - 1u));
                    if (k < avail) {
                        const DeferState &d = dfr->buf[din][k];
                        px = (double)d.p[0]; py = (double)d.p[1]; pz = (double)d.p[2];
                        ux = (double)d.u[0]; uy = (double)d.u[1]; uz = (double)d.u[2];
                        w = (double)d.w; tau = (double)d.tau;
                        pA = d.pA; pG = d.pG;
                        id_lo = d.id_lo; id_hi = d.id_hi; event = d.event;
                        nsteps = (int)d.nsteps; pscat = d.pscat;
                        phase = kTrace;
                        t_acq = (uint32_t)clock();
                        alive = true;
                    }
                }
                need = __ballot_sync(SMCRT_FULL, !alive && !retired);
            }
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

        // ---- 2. the scene evaluation of this iteration
        const double ee = 2.0 * delta * (cdot > 0.0 ? 1.0 : -1.0);
        double ex = px, ey = py, ez = pz;
        int sel = -2;
        if (phase == kNrm) {
            const double hh = (sub & 1) ? -delta : delta;
            const int a = sub >> 1;
            if (a == 0) ex = px + hh; else if (a == 1) ey = py + hh; else ez = pz + hh;
            sel = istar;
        } else if (phase == kProj) {
            ex = qx; ey = qy; ez = qz;
            sel = istar;
        } else if (phase == kFar) {
            ex = qx + ee * nx; ey = qy + ee * ny; ez = qz + ee * nz;
        } else if (phase == kNear) {
            ex = qx - ee * nx; ey = qy - ee * ny; ez = qz - ee * nz;
        }
        const Eval64 E = scene_eval64<G>(S, ex, ey, ez, sel);
        {
            const unsigned ev = __ballot_sync(SMCRT_FULL, alive && phase != kLaunch);
            if (lane == 0) wadd(wa, kEvals, __popc(ev));
        }

        // ---- 3. classify
        bool move = false, fresnel = false, iter_done = false;
        bool seg_step = false;                 // a tracing move that segment stepping may lengthen
        bool fin = false;                      // the packet ends this iteration
        long long fin_R = 0, fin_T = 0, fin_K = 0;
        double L = 0.0, R = 1.0, ct = 0.0, n1 = 0.0, n2 = 0.0;
        if (alive) {
            if (phase == kTrace) {
                if (E.dbox > 0.0) {                      // outside the volume of interest
                    {                                          // leaves the volume: R or T
                        const long long v = fx64(w);
                        if (ux * S.src_dir[0] + uy * S.src_dir[1] + uz * S.src_dir[2] < 0.0) fin_R = v; else fin_T = v;
                        fin = true;
                        alive = false;
                    }
                } else {
                    reg = E.region;
                    if (E.dmin < delta) {                // on a boundary: find its normal
                        istar = E.istar;
                        dstar = E.dstar;
                        phase = kNrm;
                        sub = 0;
                    } else {
                        L = E.dmin - 0.5 * delta;        // stop short of the surface
                        move = true;
                        seg_step = S.stepping == SMCRT_STEP_SEGMENT;
                    }
                }
            } else if (phase == kNrm) {
                const double f = E.dsel;
                if ((sub & 1) == 0) {
                    fplus = f;
                } else {
                    const double gg = fplus - f;
                    const int a = sub >> 1;
                    if (a == 0) qx = gg; else if (a == 1) qy = gg; else qz = gg;
                }
                if (++sub == 6) {
                    const double l2 = qx * qx + qy * qy + qz * qz;
                    bool approaching = false;
                    if (l2 > 0.0) {
                        const double l = sqrt(l2);
                        nx = qx / l; ny = qy / l; nz = qz / l;
                        cdot = ux * nx + uy * ny + uz * nz;
                        approaching = (cdot > 0.0 && dstar < 0.0) || (cdot < 0.0 && dstar >= 0.0);
                    }
                    if (!approaching) {
                        L = delta;                       // forced step along u
                        move = true;
                    } else if (istar < 0) {
                        {                                          // leaves the volume: R or T
                        const long long v = fx64(w);
                        if (ux * S.src_dir[0] + uy * S.src_dir[1] + uz * S.src_dir[2] < 0.0) fin_R = v; else fin_T = v;
                        fin = true;
                        alive = false;
                    }                        // outward through the bounding box
                    } else {
                        wadd(wa, kIntf, 1);
                        qx = px; qy = py; qz = pz;
                        phase = kProj;
                        sub = 0;
                    }
                }
            } else if (phase == kProj) {
                const double dq = E.dsel;
                if (fabs(dq) <= delta * 1e-3) {
                    phase = kFar;
                } else {
                    qx = qx - dq * nx; qy = qy - dq * ny; qz = qz - dq * nz;
                    if (++sub == 3) phase = kFar;
                }
            } else if (phase == kFar) {
                rfar = E.region;
                phase = kNear;
            } else if (phase == kNear) {
                n1 = region_n64(S, E.region);
                n2 = region_n64(S, rfar);
                if (n1 == n2) {
                    px = qx + ee * nx; py = qy + ee * ny; pz = qz + ee * nz;
                    phase = kTrace;
                    iter_done = true;
                } else {
                    wadd(wa, kFres, 1);
                    fresnel = true;
                    const double ci = fabs(cdot);
                    const double eta = n1 / n2;
                    const double st2 = eta * eta * ((1.0 - ci) * (1.0 + ci));
                    if (st2 < 1.0) {
                        ct = sqrt(1.0 - st2);
                        const double rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
                        const double rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
                        R = 0.5 * (rs * rs + rp * rp);
                    }
                }
            }
        }

        // ---- 4. move: interaction point or sphere-trace step, one tally site
        bool interact = false;
        if (move) {
            double mu_t = 0.0;
            if (reg >= 0) mu_t = __ldg(S.reg64 + 8 * reg + 4);
            interact = mu_t > 0.0 && tau < mu_t * L;
            if (seg_step && !interact) {           // segment stepping: a longer move along u
                L = fmax(L, segment_bound64<G>(S, E.dsoft, E.dbox, px, py, pz, ux, uy, uz));
                interact = mu_t > 0.0 && tau < mu_t * L;
            }
            const double seg = interact ? tau / mu_t : L;
            long long *const flu = (long long *)jc->flu;
            if (flu) tally64(S, flu, px, py, pz, ux, uy, uz, seg, w, &npieces);
            px = px + seg * ux; py = py + seg * uy; pz = pz + seg * uz;
            if (!interact) tau = tau - mu_t * L;
            phase = kTrace;
            iter_done = true;
        }

        // ---- 5. one Philox call for every lane that draws this iteration
        const bool draws = alive && (phase == kLaunch || interact || (fresnel && R < 1.0));
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (__any_sync(SMCRT_FULL, draws)) {
            r = philox4x32_10(make_uint4(event, 0u, id_lo, id_hi), jc->k0, jc->k1);
            if (draws) event += 1u;
        }

        // ---- 6. consumers
        if (alive && phase == kLaunch) {                 // photon release
            const double x0 = u01_64(r.x), x1 = u01_64(r.y), x3 = u01_64(r.w);
            px = S.src_pos[0]; py = S.src_pos[1]; pz = S.src_pos[2];
            ux = S.src_dir[0]; uy = S.src_dir[1]; uz = S.src_dir[2];
            if (S.src_kind == 1 || S.src_kind == 2) {
                double c1, c2;
                if (S.src_kind == 1) {
                    const double rho = S.src_radius * sqrt(x0);
                    double sn, cs;
                    sincos2pi64(x1, &sn, &cs);
                    c1 = rho * cs;
                    c2 = rho * sn;
                } else {
                    c1 = S.src_radius * (2.0 * x0 - 1.0);
                    c2 = S.src_radius * (2.0 * x1 - 1.0);
                }
                px = S.src_pos[0] + c1 * S.src_b1[0] + c2 * S.src_b2[0];
                py = S.src_pos[1] + c1 * S.src_b1[1] + c2 * S.src_b2[1];
                pz = S.src_pos[2] + c1 * S.src_b1[2] + c2 * S.src_b2[2];
            } else if (S.src_kind == 3) {
                const double ctt = 2.0 * x0 - 1.0;
                const double st = sqrt((1.0 - ctt) * (1.0 + ctt));
                double sn, cs;
                sincos2pi64(x1, &sn, &cs);
                ux = st * cs; uy = st * sn; uz = ctt;
            }
            tau = -ln64(x3);
            w = 1.0;
            nsteps = 0; pA = 0; pG = 0; pscat = 0;
            phase = kTrace;
        }
        if (interact) {                                  // implicit capture, HG, roulette
            const double *RG = S.reg64 + 8 * reg;
            const double wn = w * __ldg(RG + 5);
            pA += fx64(w - wn);
            w = wn;
            scatter64(ux, uy, uz, hg_cos64(__ldg(RG + 2), u01_64(r.x)), u01_64(r.y));
            pscat += 1u;
            if (w < kWRoulette) {
                if (u01_64(r.z) <= 1.0 / kRouletteM) {
                    pG += fx64(w * (kRouletteM - 1.0));
                    w = w * kRouletteM;
                } else {
                    fin_K = fx64(w);
                    fin = true;
                    alive = false;
                }
            }
            tau = -ln64(u01_64(r.w));
        }
        if (fresnel) {                                   // Fresnel reflection / Snell refraction
            const bool reflect = R < 1.0 ? (u01_64(r.x) <= R) : true;
            if (reflect) {
                const double c2 = 2.0 * cdot;
                ux = ux - c2 * nx; uy = uy - c2 * ny; uz = uz - c2 * nz;
                normalise64(ux, uy, uz);
                px = qx - ee * nx; py = qy - ee * ny; pz = qz - ee * nz;
            } else {
                const double eta = n1 / n2;
                const double ci = fabs(cdot);
                const double k = (cdot > 0.0 ? 1.0 : -1.0) * (eta * ci - ct);
                ux = eta * ux - k * nx; uy = eta * uy - k * ny; uz = eta * uz - k * nz;
                normalise64(ux, uy, uz);
                px = qx + ee * nx; py = qy + ee * ny; pz = qz + ee * nz;
            }
            phase = kTrace;
            iter_done = true;
        }
        if (iter_done && alive) {
            nsteps += 1;
            if (nsteps >= S.max_steps) {
                wadd(wa, kCap, 1);
                fin_K = fx64(w);
                fin = true;
                alive = false;
            }
        }
        // ---- a terminated packet: one bookkeeping site per iteration
        if (fin) {
            wadd(wa, kR, fin_R); wadd(wa, kT, fin_T); wadd(wa, kKilled, fin_K);
            wadd(wa, kA, pA); wadd(wa, kGain, pG); wadd(wa, kScat, pscat); wadd(wa, kSteps, nsteps);
            wadd(wa, kPackets, 1);
            smcrt_packet_record *const recs = (smcrt_packet_record *)jc->recs;
            if (recs) {
                smcrt_packet_record r;
                r.R = fin_R; r.T = fin_T; r.A = pA; r.killed = fin_K; r.gain = pG;
                r.scatters = pscat; r.steps = nsteps; r.reserved = 0;
                const unsigned long long id = ((unsigned long long)id_hi << 32) | id_lo;
                recs[id - jc->begin] = r;
            }
        }
        // ---- park a straggler at a trace boundary (serving rounds only)
        if (alive && phase == kTrace && jc->budget > 0u && (uint32_t)clock() - t_acq > jc->budget) {
            JobDefer *const dfr = (JobDefer *)jc->dfr;
            const int din = jc->din;
            const unsigned k = atomicAdd(&dfr->count[1 - din], 1u);
            if (k < dfr->cap) {
                DeferState &d = dfr->buf[1 - din][k];
                d.p[0] = px; d.p[1] = py; d.p[2] = pz;
                d.u[0] = ux; d.u[1] = uy; d.u[2] = uz;
                d.w = w; d.tau = tau;
                d.pA = pA; d.pG = pG;
                d.id_lo = id_lo; d.id_hi = id_hi; d.event = event;
                d.nsteps = (uint32_t)nsteps; d.pscat = pscat;
                wadd(wa, kParked, 1);
                alive = false;
            } else {
                atomicAdd(&dfr->overflow, 1u);
                t_acq = (uint32_t)clock() + 0x7fffffffu;   // list full: run on (one retry per ~1 s)
            }
        }
    }
    const long long pc = warp_sum((long long)npieces);
    if (lane == 0) wadd(wa, kPieces, pc);
    return timed_out;
}

template <int kMinBlocks, bool G>
__global__ void __launch_bounds__(128, kMinBlocks) packets_fp64(JobWork *jobs, int njobs, int *status)
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
        long long *d8 = reinterpret_cast<long long *>(&ws->S);
        for (int i = lane; i < (int)(sizeof(DevScene) / 8); i += 32) d8[i] = s8[i];
        if (!G && ws->S.general) {           // a scene with general shapes needs the G instantiation
            if (lane == 0) {
                atomicOr(status, kStatusBadJob);
                if (J->jstat != nullptr) atomicOr(J->jstat, kStatusBadJob);
            }
            continue;
        }
        if (lane == 0) jobconst_fill(&ws->jc, J);
        wacc_clear(&ws->acc, lane);
        const long long t0 = clock64();
        const bool timed_out = run_job_fp64<G>(ws->S, &ws->acc, &ws->jc, J, lane);
        __syncwarp();
        if (lane == 0) wadd(&ws->acc, kBusy, clock64() - t0);
        wacc_flush(&ws->acc, J->totals, lane);
        if (timed_out) {                     // the launch's time limit: this warp is done
            if (lane == 0) {
                atomicOr(status, kStatusTimeout);
                if (J->jstat != nullptr) atomicOr(J->jstat, kStatusTimeout);
            }
            return;
        }
    }
}

}  // namespace

// Register budgets of the instantiations: variant v keeps kMinBlocks
// blocks of 128 threads resident per SM (more blocks = fewer registers per
// thread, possibly spilled); the autotuner picks per scene.
constexpr int kVariantBlocks[kNumVariants] = {4, 3, 2};

cudaError_t launch_fp64(JobWork *jobs, int njobs, int *status, int blocks, int threads, cudaStream_t stream,
                        int variant)
{
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpShared);
    switch (variant) {   // kNumVariants and up: the same budgets for scenes with general shapes
    case 1: packets_fp64<3, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 2: packets_fp64<2, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 3: packets_fp64<4, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 4: packets_fp64<3, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    case 5: packets_fp64<2, true><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    default: packets_fp64<4, false><<<blocks, threads, sm, stream>>>(jobs, njobs, status); break;
    }
    return cudaGetLastError();
}

int occupancy_fp64(int threads, int variant)
{
    int n = 0;
    const size_t sm = (size_t)(threads / 32) * sizeof(WarpShared);
    switch (variant) {
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<3, false>, threads, sm); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<2, false>, threads, sm); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<4, true>, threads, sm); break;
    case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<3, true>, threads, sm); break;
    case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<2, true>, threads, sm); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, packets_fp64<4, false>, threads, sm); break;
    }
    return n;
}

}  // namespace smcrt
