// static_render.cu -- curast_render_static: the rasterizer for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time loops that are not allowed
// to allocate (an allocation can synchronize the device and take
// milliseconds), and plug-ins whose host hands out device memory only
// through its own pools or reserves all of it up front.  This entry point
// renders up to kStaticMaxInstances instances of one mesh into one view with
// no context and no allocation: every buffer the pipeline needs besides the
// caller's inputs and outputs (frame tables, counters, the stage-1 -> 2 and
// stage-2 -> 3 queues) lives in one file-scope __device__ array.
#include <cmath>
#include <cstring>
#include <mutex>

#include "curast.h"
#include "internal.h"

namespace curast {
namespace {

constexpr int kStaticMaxInstances = CURAST_STATIC_MAX_INSTANCES;
constexpr uint64_t kStaticQ1 = 1ull << 16;    // queue-1 entries (16 B each); overflow is rasterized in place
constexpr uint64_t kStaticQ2 = 1ull << 14;    // queue-2 tile parts (56 B each); overflow likewise

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffHdr = 0;
constexpr size_t kOffView = al(kOffHdr + sizeof(FrameHdr));
constexpr size_t kOffMesh = al(kOffView + sizeof(ViewDev));
constexpr size_t kOffSeg = al(kOffMesh + sizeof(MeshDev));
constexpr size_t kOffRound = al(kOffSeg + sizeof(SegDev));
constexpr size_t kOffCtr = al(kOffRound + sizeof(RoundDev));
constexpr size_t kOffErr = al(kOffCtr + sizeof(Counters));
constexpr size_t kOffPairs = al(kOffErr + sizeof(unsigned));
constexpr size_t kOffQ1 = al(kOffPairs + kStaticMaxInstances * sizeof(PairDev));
constexpr size_t kOffQ2 = al(kOffQ1 + kStaticQ1 * sizeof(Q1Entry));
constexpr size_t kScratchBytes = al(kOffQ2 + kStaticQ2 * sizeof(Q2Entry));   // about 2 MB

// The scratch every call shares.  Every GPU that loads the library holds one
// copy of it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Everything a frame needs, passed by value to the one-block set-up kernel.
struct StaticFrame {
    FrameHdr hdr;
    ViewDev view;
    MeshDev mesh;
    SegDev seg;
    RoundDev round;
    int n;
    float mv[kStaticMaxInstances][12];
    uint64_t base[kStaticMaxInstances];
};

// Writes the frame tables into the scratch and zeroes its counters (they
// keep the previous call's values otherwise).
__global__ void k_static_setup(StaticFrame s) {
    unsigned char *g = g_static_scratch;
    const int t = threadIdx.x;
    if (t < s.n) {
        PairDev p;
        for (int q = 0; q < 12; ++q) p.mv[q] = s.mv[t][q];
        for (int q = 0; q < 12; ++q) p.fn[q] = 0.0f;
        for (int q = 0; q < 4; ++q) p.fk[q] = 0.0f;
        for (int q = 0; q < 3; ++q) p.fs[q] = 0.0f;
        p.nlo = -INFINITY;    // nor a near-plane cull
        p.wsafe = INFINITY;   // no conservative cull: every triangle takes the exact path
        p.win = 0.0f;
        p.base = s.base[t];
        p.view = 0;
        p.mesh = 0;
        reinterpret_cast<PairDev *>(g + kOffPairs)[t] = p;
    }
    if (t == 0) {
        *reinterpret_cast<FrameHdr *>(g + kOffHdr) = s.hdr;
        *reinterpret_cast<ViewDev *>(g + kOffView) = s.view;
        *reinterpret_cast<MeshDev *>(g + kOffMesh) = s.mesh;
        *reinterpret_cast<SegDev *>(g + kOffSeg) = s.seg;
        *reinterpret_cast<RoundDev *>(g + kOffRound) = s.round;
        *reinterpret_cast<unsigned *>(g + kOffErr) = 0u;
    }
    unsigned long long *c = reinterpret_cast<unsigned long long *>(g + kOffCtr);
    for (size_t i = t; i < sizeof(Counters) / sizeof(unsigned long long); i += blockDim.x) c[i] = 0ull;
}

// Per-device set-up: the scratch's device address and the launch shape.
// It is marked done only when it succeeded, so a failed first call (a
// transient error) is retried by the next call instead of failing every
// later call on that device.
struct DeviceSetup {
    bool done = false;
    unsigned char *scratch = nullptr;
    LaunchShape shape{};
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// In host code g_static_scratch names a host-side stand-in, not device
// memory: the kernels get the address cudaGetSymbolAddress returns for the
// current device.
cudaError_t device_setup(int dev, DeviceSetup **out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.done) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        LaunchShape sh{};
        if ((e = query_launch_shape(&sh, dev)) != cudaSuccess) return e;
        d.scratch = static_cast<unsigned char *>(p);
        d.shape = sh;
        d.done = true;
    }
    *out = &d;
    return cudaSuccess;
}

bool affine_static(const float *m) { return m && m[12] == 0.0f && m[13] == 0.0f && m[14] == 0.0f && m[15] == 1.0f; }

}  // namespace
}  // namespace curast

using namespace curast;

extern "C" curast_status curast_render_static(const float *pos, uint64_t V, const uint32_t *idx, uint64_t T,
                                              const float *models, int n_instances, const float view[16],
                                              const float proj[16], int W, int H, uint64_t *vis,
                                              curast_stream stream) {
    if (!view || !proj || !vis || (V > 0 && !pos) || (T > 0 && !idx)) return CURAST_ERR_INVALID_ARG;
    if (n_instances < 1 || n_instances > kStaticMaxInstances) return CURAST_ERR_TOO_LARGE;
    if (V > 0xFFFFFFFFull || T > 0xFFFFFFFFull) return CURAST_ERR_TOO_LARGE;
    if ((uint64_t)n_instances * T > kIdMask) return CURAST_ERR_ID_SPACE_OVERFLOW;
    if (W < 1 || H < 1 || W > 16384 || H > 16384) return CURAST_ERR_INVALID_ARG;
    if (!affine_static(view)) return CURAST_ERR_NOT_AFFINE;
    for (int i = 0; models && i < n_instances; ++i)
        if (!affine_static(models + 16 * i)) return CURAST_ERR_NOT_AFFINE;
    // the projection vector of Eq. 2 and the near plane (as curast_render)
    if (proj[1] != 0.0f || proj[2] != 0.0f || proj[3] != 0.0f || proj[4] != 0.0f || proj[6] != 0.0f ||
        proj[7] != 0.0f || proj[8] != 0.0f || proj[9] != 0.0f || proj[12] != 0.0f || proj[13] != 0.0f ||
        proj[14] != -1.0f || proj[15] != 0.0f)
        return CURAST_ERR_BAD_CAMERA;
    const float nearv = (float)((double)proj[11] / ((double)proj[10] - 1.0));
    if (!(proj[0] > 0.0f) || !(proj[5] > 0.0f) || !(nearv > 0.0f) || !std::isfinite(nearv)) return CURAST_ERR_BAD_CAMERA;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CURAST_ERR_CUDA;
    DeviceSetup *ds = nullptr;
    cudaError_t e = device_setup(dev, &ds);
    if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDeviceFunction) return CURAST_ERR_NOT_BUILT;
    if (e != cudaSuccess) return CURAST_ERR_CUDA;
    unsigned char *g = ds->scratch;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    StaticFrame fr;
    std::memset(&fr, 0, sizeof(fr));
    fr.n = n_instances;
    const float ident[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    for (int i = 0; i < n_instances; ++i) {
        const float *m = models ? models + 16 * i : ident;
        for (int r = 0; r < 3; ++r)      // view * model in double, rounded once (as curast_render)
            for (int c = 0; c < 4; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) acc = acc + (double)view[4 * r + k] * (double)m[4 * k + c];
                fr.mv[i][4 * r + c] = (float)acc;
            }
        fr.base[i] = (uint64_t)i * T;
    }
    const uint64_t per_item = 256ull * 4;
    fr.hdr.n_batches = T ? (T + per_item - 1) / per_item : 0;
    fr.hdr.n_segs = T ? 1u : 0u;
    fr.hdr.n_views = 1;
    fr.hdr.n_rounds = 1;
    fr.round.b0 = 0;                      // one round over every item; no bitmap (fused stage 1)
    fr.round.b1 = fr.hdr.n_batches;
    fr.view.fx = proj[0];
    fr.view.fy = proj[5];
    fr.view.nearv = nearv;
    fr.view.hw = 0.5f * (float)W;
    fr.view.hh = 0.5f * (float)H;
    fr.view.W = W;
    fr.view.H = H;
    fr.view.tile0 = 0;
    fr.view.ntx = 0;
    fr.view.vis = vis;
    fr.mesh.pos = pos;
    fr.mesh.idx = idx;
    fr.mesh.rgba = nullptr;
    fr.mesh.V = V;
    fr.mesh.T = T;
    fr.seg.mesh = 0;
    fr.seg.pair0 = 0;
    fr.seg.npairs = (uint32_t)n_instances;
    fr.seg.T = T;
    fr.seg.batch0 = 0;

    FrameDev f;
    f.hdr = reinterpret_cast<const FrameHdr *>(g + kOffHdr);
    f.views = reinterpret_cast<const ViewDev *>(g + kOffView);
    f.pairs = reinterpret_cast<const PairDev *>(g + kOffPairs);
    f.segs = reinterpret_cast<const SegDev *>(g + kOffSeg);
    f.meshes = reinterpret_cast<const MeshDev *>(g + kOffMesh);
    f.q1 = reinterpret_cast<Q1Entry *>(g + kOffQ1);
    f.q2 = reinterpret_cast<Q2Entry *>(g + kOffQ2);
    f.rounds = reinterpret_cast<const RoundDev *>(g + kOffRound);
    f.bits = nullptr;   // no survivor bitmap: the fused cull kernel runs the exact path itself
    f.ctr = reinterpret_cast<Counters *>(g + kOffCtr);
    f.err = reinterpret_cast<unsigned *>(g + kOffErr);
    f.q1_cap = kStaticQ1;
    f.q2_cap = kStaticQ2;
    f.s1_max = 128;
    f.s2_max = 4096;
    f.tile_log2 = 6;
    f.tpt = 4;
    fastdiv_consts(8u * f.tpt, f.g_m, f.g_s);
    f.group_min = 0;
    f.s3_ray = 0;
    f.check = 1;
    f.stats = 0;
    f.s3_bin = 0;     // stage 3 writes straight to the buffer (no tile bins in the scratch)
    f.n_tiles = 0;
    f.tile_cnt = f.tile_start = f.tile_fill = f.part_sorted = nullptr;
    f.units = nullptr;

    const bool inst = n_instances > 1;
    const int sms = ds->shape.num_sms;
    k_static_setup<<<1, 32, 0, s>>>(fr);
    if ((e = cudaGetLastError()) != cudaSuccess) return CURAST_ERR_CUDA;
    if ((e = launch_clear(vis, (uint64_t)W * (uint64_t)H, s)) != cudaSuccess) return CURAST_ERR_CUDA;
    if ((e = launch_stage1(f, inst, 1, 0, sms * ds->shape.stage1_blocks_per_sm[inst ? 1 : 0][1], true, s)) !=
        cudaSuccess)
        return CURAST_ERR_CUDA;
    if ((e = launch_stage2(f, sms * ds->shape.stage2_blocks_per_sm, s)) != cudaSuccess) return CURAST_ERR_CUDA;
    if ((e = launch_stage3(f, sms * ds->shape.stage3_blocks_per_sm, s)) != cudaSuccess) return CURAST_ERR_CUDA;
    return CURAST_OK;
}
