// smcrt_noalloc.cu -- smcrt_run_noalloc: the single-job packet launch with
// all of its scratch in one file-scope device array, for callers that may
// not allocate device memory (see include/smcrt.h).
//
// The scratch holds the launch descriptor, the kernel's status word and the
// compiled scene image.  Host code cannot use the array's name as a device
// address: the address is looked up once per device with
// cudaGetSymbolAddress and cached.  Every call shares the array and leaves
// its contents behind, so calls that overlap on the GPU race with one another.
// The image is written into the array by small copy kernels that carry it in
// their launch arguments, so the call reads no host memory after it returns.
#include <cmath>
#include <cstring>
#include <mutex>

#include "smcrt_internal.h"

namespace smcrt {

namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;   // stated maximum scratch size
constexpr int kNoAllocMaxPrims = 128;
constexpr int kNoAllocMaxNodes = 256;
constexpr int kNoAllocMaxRegions = 16;
constexpr int kNoAllocMaxDevices = 64;

// The scratch: [JobWork][status][pad to 256][DevScene image + tables].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

unsigned char *g_scratch_addr[kNoAllocMaxDevices] = {};
std::mutex g_scratch_mu;

// Host staging of the scene image: one file-scope buffer, used under
// g_image_mu from the start of the image build until the last copy kernel
// has been launched.  The image reaches the device as the parameters of
// copy kernels (below): launch arguments are copied when the kernel is
// launched, so the buffer is free again as soon as the launches return and
// no copy reads host memory later.
alignas(16) unsigned char g_image[kNoAllocScratchBytes];
std::mutex g_image_mu;

// Bytes of the image carried by one copy kernel's parameters.
constexpr int kChunkBytes = 8192;
struct ImageChunk {
    uint32_t nwords;          // 16-byte words in this chunk
    uint32_t pad[3];
    uint4 w[kChunkBytes / 16];
};

__global__ void __launch_bounds__(256) copy_image_chunk(uint4 *dst, const ImageChunk c)
{
    for (uint32_t k = threadIdx.x; k < c.nwords; k += blockDim.x) dst[k] = c.w[k];
}

constexpr size_t kJobOff = 0;
constexpr size_t kStatusOff = 256;
constexpr size_t kImageOff = 512;

size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

float ulp32(float x)
{
    x = std::fabs(x);
    return std::nextafter(x, INFINITY) - x;
}

// The same checks as the plan path, and the same precomputed doubles
// (same expressions), with every table in fixed-size arrays.
int build_image(const smcrt_scene *sc, const smcrt_source *src, const smcrt_grid *g, int precision,
                unsigned char *dev_base, unsigned char *img, size_t *used)
{
    if (!sc || !src || !g || !sc->prims || !sc->nodes || !sc->regions) return SMCRT_ERR_BAD_ARG;
    if (precision != SMCRT_FP64 && precision != SMCRT_MIXED) return SMCRT_ERR_BAD_ARG;
    if (sc->nprims < 1 || sc->nregions < 1 || sc->nnodes < 1) return SMCRT_ERR_BAD_SCENE;
    if (sc->nprims > kNoAllocMaxPrims || sc->nnodes > kNoAllocMaxNodes || sc->nregions > kNoAllocMaxRegions)
        return SMCRT_ERR_NO_MEMORY;   // beyond the fixed scratch
    const int vrc = validate_scene(sc, src, g);   // field checks only: no allocation
    if (vrc != SMCRT_OK) return vrc;

    // Postfix CSG -> instruction stream in fixed arrays, with the checks and
    // the fusion rule of the plan compiler (a primitive followed by a binary
    // operator combines with the stack top; register stack depth <= 4).
    Instr ins[kNoAllocMaxNodes];
    double k64[kNoAllocMaxNodes];
    int2 rr[kNoAllocMaxRegions];
    int ni = 0;
    for (int r = 0; r < sc->nregions; ++r) {
        const smcrt_region &R = sc->regions[r];
        const smcrt_csg_node *nd = sc->nodes + R.node_begin;
        const int begin = ni;
        int depth = 0;
        for (int i = 0; i < R.node_count; ++i) {
            const int op = nd[i].op;
            Instr in{};
            in.region = -1;
            float kinv = 0.f;
            double k = 0.0;
            if (op == SMCRT_OP_PRIM) {
                const int p = nd[i].prim;
                if (p < 0 || p >= sc->nprims) return SMCRT_ERR_BAD_SCENE;
                const int kind = device_kind(sc->prims[p]);
                const bool fuse = depth >= 1 && i + 1 < R.node_count && nd[i + 1].op >= SMCRT_OP_UNION &&
                                  nd[i + 1].op <= SMCRT_OP_SUBTRACT;
                in.prim = p;
                if (fuse) {
                    const int bop = nd[i + 1].op;
                    in.op = bop | (kind << 8);
                    if (bop == SMCRT_OP_SMOOTH_UNION) {
                        k = nd[i + 1].k;
                        if (!(k > 0 && std::isfinite(k))) return SMCRT_ERR_BAD_SCENE;
                        kinv = (float)(1.0 / k);
                    }
                    ++i;
                } else {
                    in.op = 0 | (kind << 8);
                    if (++depth > kMaxStack) return SMCRT_ERR_BAD_SCENE;
                }
            } else if (op >= SMCRT_OP_UNION && op <= SMCRT_OP_SUBTRACT) {
                if (depth < 2) return SMCRT_ERR_BAD_SCENE;
                in.op = op;
                in.prim = -1;
                if (op == SMCRT_OP_SMOOTH_UNION) {
                    k = nd[i].k;
                    if (!(k > 0 && std::isfinite(k))) return SMCRT_ERR_BAD_SCENE;
                    kinv = (float)(1.0 / k);
                }
                --depth;
            } else {
                return SMCRT_ERR_BAD_SCENE;
            }
            if (ni >= kNoAllocMaxNodes) return SMCRT_ERR_NO_MEMORY;
            std::memcpy(&in.pad, &kinv, 4);
            ins[ni] = in;
            k64[ni] = k;
            ++ni;
        }
        if (depth != 1) return SMCRT_ERR_BAD_SCENE;
        ins[ni - 1].region = r;
        if (region_is_soft(sc, r)) ins[ni - 1].op |= kSoftRegionEnd;
        rr[r] = make_int2(begin, ni);
    }
    const int np = sc->nprims, nr = sc->nregions;

    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = a16(off + b); return o; };
    const size_t o_scene = take(sizeof(DevScene));
    const size_t o_ins = take(sizeof(Instr) * ni);
    const size_t o_k64 = take(sizeof(double) * ni);
    const size_t o_kind = take(sizeof(int32_t) * np);
    const size_t o_p64 = take(sizeof(double) * 8 * np);
    const size_t o_p32 = take(sizeof(float4) * 2 * np);
    const size_t o_rr = take(sizeof(int2) * nr);
    const size_t o_r64 = take(sizeof(double) * 8 * nr);
    const size_t o_r32 = take(sizeof(float4) * 2 * nr);
    int32_t segp[kMaxPrims];
    double segm[kMaxPrims];
    const int nseg = sc->stepping == SMCRT_STEP_SEGMENT ? seg_entries(sc, segp, segm) : 0;
    const size_t o_seg = take(sizeof(int32_t) * nseg);
    const size_t o_segm64 = take(sizeof(double) * nseg);
    const size_t o_segm32 = take(sizeof(float) * nseg);
    const bool has_xf = sc->nxforms > 0;
    const size_t o_xf64 = take(has_xf ? sizeof(double) * kXf64 * np : 0);
    const size_t o_xf32 = take(has_xf ? sizeof(float4) * kXf32 * np : 0);
    if (kImageOff + off > kNoAllocScratchBytes) return SMCRT_ERR_NO_MEMORY;
    std::memset(img, 0, off);

    int32_t *pkind = (int32_t *)(img + o_kind);
    double *p64 = (double *)(img + o_p64);
    float4 *p32 = (float4 *)(img + o_p32);
    double *xf64 = has_xf ? (double *)(img + o_xf64) : nullptr;
    float4 *xf32 = has_xf ? (float4 *)(img + o_xf32) : nullptr;
    for (int i = 0; i < np; ++i) {
        pkind[i] = device_kind(sc->prims[i]);
        fill_prim(sc, i, p64 + 8 * i, p32 + 2 * i, has_xf ? xf64 + kXf64 * i : nullptr,
                  has_xf ? xf32 + kXf32 * i : nullptr);
    }
    double *reg64 = (double *)(img + o_r64);
    float4 *reg32 = (float4 *)(img + o_r32);
    for (int r = 0; r < nr; ++r) {
        const smcrt_region &R = sc->regions[r];
        const double mu_t = R.mu_a + R.mu_s;
        const double albedo = mu_t > 0.0 ? R.mu_s / mu_t : 0.0;
        double *d = reg64 + 8 * r;
        d[0] = R.mu_a; d[1] = R.mu_s; d[2] = R.g; d[3] = R.n; d[4] = mu_t; d[5] = albedo;
        reg32[2 * r] = make_float4((float)mu_t, mu_t > 0 ? (float)(1.0 / mu_t) : 0.f, (float)albedo, (float)R.g);
        reg32[2 * r + 1] = make_float4((float)R.n, (float)R.mu_a, (float)R.mu_s, 0.f);
    }
    std::memcpy(img + o_ins, ins, sizeof(Instr) * ni);
    std::memcpy(img + o_k64, k64, sizeof(double) * ni);
    std::memcpy(img + o_rr, rr, sizeof(int2) * nr);
    if (nseg > 0) {
        std::memcpy(img + o_seg, segp, sizeof(int32_t) * nseg);
        std::memcpy(img + o_segm64, segm, sizeof(double) * nseg);
        float *m32 = (float *)(img + o_segm32);
        for (int j = 0; j < nseg; ++j) m32[j] = (float)segm[j];
    }

    unsigned char *base = dev_base + kImageOff;   // device addresses of the tables
    DevScene H;
    std::memset(&H, 0, sizeof H);
    H.instr = (const Instr *)(base + o_ins);
    H.k64 = (const double *)(base + o_k64);
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
        rmax = std::fmax(rmax, (float)std::fmax(std::fabs(sc->bbox_lo[a]), std::fabs(sc->bbox_hi[a])));
    }
    H.delta = sc->delta;
    H.ambient_n = sc->ambient_n;
    H.ambient_n32 = (float)sc->ambient_n;
    H.cull_region = -1;   // no culling grid in the fixed scratch
    H.stepping = sc->stepping;
    H.nseg = nseg;
    H.seg_prims = nseg > 0 ? (const int32_t *)(base + o_seg) : nullptr;
    H.seg_m64 = nseg > 0 ? (const double *)(base + o_segm64) : nullptr;
    H.seg_m32 = nseg > 0 ? (const float *)(base + o_segm32) : nullptr;
    H.xf64 = has_xf ? (const double *)(base + o_xf64) : nullptr;
    H.xf32 = has_xf ? (const float4 *)(base + o_xf32) : nullptr;
    for (int i = 0; i < np; ++i) H.general = H.general || !plain_prim(sc->prims[i]);
    {
        int longest = 0;
        bool plain = true;
        for (int i = 0; i < np; ++i) plain = plain && plain_prim(sc->prims[i]);
        for (int r = 0; r < nr; ++r) longest = (rr[r].y - rr[r].x) > longest ? (rr[r].y - rr[r].x) : longest;
        if (!plain) longest = kAnalyticNormalMaxInstr + 1;   // probe normals for other shapes and frames
        H.analytic_nrm = longest <= kAnalyticNormalMaxInstr ? 1 : 0;
    }
    // probe normals run in the general mixed instantiation (the plain one
    // leaves them out)
    if (precision == SMCRT_MIXED && !H.analytic_nrm) H.general = 1;
    H.delta32 = std::fmax((float)sc->delta, 64.f * ulp32(rmax));
    H.h32 = 32.f * H.delta32;
    H.max_steps = sc->max_steps;
    H.src_kind = src->kind;
    {   // basis perpendicular to the source direction (Duff et al., JCGT 2017)
        const double *n = src->dir;
        const double sg = std::copysign(1.0, n[2]);
        const double a = -1.0 / (sg + n[2]);
        const double b = n[0] * n[1] * a;
        H.src_b1[0] = 1.0 + sg * n[0] * n[0] * a;
        H.src_b1[1] = sg * b;
        H.src_b1[2] = -sg * n[0];
        H.src_b2[0] = b;
        H.src_b2[1] = sg + n[1] * n[1] * a;
        H.src_b2[2] = -n[1];
    }
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
    std::memcpy(img + o_scene, &H, sizeof H);
    *used = off;
    return SMCRT_OK;
}

// Device address of the scratch on the current device; looked up once per
// device (the first call on a device does this set-up).
int scratch_address(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return SMCRT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return SMCRT_ERR_CUDA;
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return SMCRT_OK;
}

}  // namespace

}  // namespace smcrt

using namespace smcrt;

extern "C" int smcrt_run_noalloc(const smcrt_scene *scene, const smcrt_source *source, const smcrt_grid *grid,
                                 uint64_t id_begin, uint64_t npackets, uint64_t seed, int32_t precision,
                                 int64_t *fluence_dev, smcrt_totals *totals_dev, void *stream)
{
    if (!totals_dev) return SMCRT_ERR_BAD_ARG;
    if (id_begin + npackets < id_begin) return SMCRT_ERR_BAD_ARG;
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SMCRT_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // tori, cylinders, frames (and, in mixed precision, probe normals): the
    // general instantiation, as the image's scene header records
    bool general = false;
    {
        std::lock_guard<std::mutex> lk(g_image_mu);
        size_t used = 0;
        rc = build_image(scene, source, grid, precision, base, g_image, &used);
        if (rc != SMCRT_OK) return rc;
        general = reinterpret_cast<const DevScene *>(g_image)->general != 0;
        if (npackets == 0) return SMCRT_OK;
        // the image (a multiple of 16 bytes), chunk by chunk, in the copy
        // kernels' launch arguments
        static ImageChunk chunk;   // guarded by g_image_mu
        for (size_t o = 0; o < used; o += kChunkBytes) {
            const size_t nb = used - o < (size_t)kChunkBytes ? used - o : (size_t)kChunkBytes;
            chunk.nwords = (uint32_t)(nb / 16);
            std::memcpy(chunk.w, g_image + o, nb);
            copy_image_chunk<<<1, 256, 0, s>>>((uint4 *)(base + kImageOff + o), chunk);
            if (cudaGetLastError() != cudaSuccess) return SMCRT_ERR_CUDA;
        }
    }
    // a cleared status word; the descriptor goes in by value
    if (cudaMemsetAsync(base + kStatusOff, 0, sizeof(int), s) != cudaSuccess) return SMCRT_ERR_CUDA;
    JobWork jw{};
    jw.next = id_begin;
    jw.end = id_begin + npackets;
    jw.begin = id_begin;
    jw.seed = seed;
    jw.fluence = (long long *)fluence_dev;
    jw.totals = totals_dev;
    jw.records = nullptr;
    jw.scene = (const DevScene *)(base + kImageOff);
    JobWork *dj = (JobWork *)(base + kJobOff);
    if (launch_set_job(dj, jw, s) != cudaSuccess) return SMCRT_ERR_CUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SMCRT_ERR_CUDA;
    const int threads = 128;
    const int variant = (precision == SMCRT_FP64 ? 1 : 0) + (general ? kNumVariants : 0);
    const int occ = precision == SMCRT_FP64 ? occupancy_fp64(threads, variant) : occupancy_mixed(threads, variant);
    const int blocks = sms * (occ > 0 ? occ : 1);
    const cudaError_t e = precision == SMCRT_FP64
                              ? launch_fp64(dj, 1, (int *)(base + kStatusOff), blocks, threads, s, variant)
                              : launch_mixed(dj, 1, (int *)(base + kStatusOff), blocks, threads, s, variant);
    return e == cudaSuccess ? SMCRT_OK : SMCRT_ERR_CUDA;
}
