// runtime.cu -- host runtime behind include/curast.h.
//
// Frame setup follows Section 4 ("On the host side, before launching the
// rasterization stages"): per (instance, view) frustum culling against the
// mesh bounds, the list of meshes with their transformation matrices, the
// exclusive prefix sum of triangle counts for the global ids, and a copy of
// all of it to the GPU; then the stage kernels are enqueued.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "curast.h"
#include "internal.h"

using namespace curast;

namespace {

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        release();
        size_t c = std::max<size_t>(n, 16);
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), c * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; return e; }
        cap = c;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

template <class T>
struct PinBuf {
    T *p = nullptr;
    size_t cap = 0;
    cudaError_t reserve(size_t n) {
        if (n <= cap) return cudaSuccess;
        release();
        size_t c = std::max<size_t>(n, 16);
        cudaError_t e = cudaMallocHost(reinterpret_cast<void **>(&p), c * sizeof(T));
        if (e != cudaSuccess) { p = nullptr; return e; }
        cap = c;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
    }
};

struct MeshRec {
    const float *pos;
    const uint32_t *idx;
    const uint8_t *rgba;
    uint64_t V, T;
    bool bounded;
    double lo[3], hi[3];
    // Section 4.6 encoding, owned by the context (comp)
    bool comp = false;
    uint32_t *cidx = nullptr;
    uint16_t *qpos = nullptr;
    uint32_t *gflag = nullptr;            // grid flags of the 128-triangle groups (k_grid_flags)
    uint64_t cwords = 0;
    uint32_t bits = 0, imin = 0;
    float clo[3] = {0, 0, 0}, cstep[3] = {0, 0, 0};
    // texture (borrowed): per-vertex uv and an RGBA8 mip chain
    const float *uv = nullptr;
    const uint8_t *tex = nullptr;
    int32_t tex_log2 = 0;
};

struct InstRec {
    uint32_t mesh;
    float model[16];
};

struct Cam {
    float fx, fy, nearv;
};

// The projection vector of Eq. 2 from a symmetric perspective matrix.
curast_status parse_camera(const float *p, Cam *c) {
    if (!p) return CURAST_ERR_INVALID_ARG;
    if (p[1] != 0.0f || p[2] != 0.0f || p[3] != 0.0f || p[4] != 0.0f || p[6] != 0.0f || p[7] != 0.0f ||
        p[8] != 0.0f || p[9] != 0.0f || p[12] != 0.0f || p[13] != 0.0f || p[14] != -1.0f || p[15] != 0.0f)
        return CURAST_ERR_BAD_CAMERA;
    const double nd = (double)p[11] / ((double)p[10] - 1.0);
    const float nearv = (float)nd;
    if (!(p[0] > 0.0f) || !(p[5] > 0.0f) || !(nearv > 0.0f) || !std::isfinite(nearv)) return CURAST_ERR_BAD_CAMERA;
    c->fx = p[0];
    c->fy = p[5];
    c->nearv = nearv;
    return CURAST_OK;
}

bool affine(const float *m) { return m && m[12] == 0.0f && m[13] == 0.0f && m[14] == 0.0f && m[15] == 1.0f; }

// view * model, each entry accumulated over k = 0..3 in double (products of
// two floats are exact there) and rounded to FP32 once.
void model_view(const float *view, const float *model, float *mv) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc = acc + (double)view[4 * r + k] * (double)model[4 * k + c];
            mv[4 * r + c] = (float)acc;
        }
}

// Conservative per-(instance, view) frustum test on the mesh bounds: the
// instance is skipped only when all 8 bound corners lie beyond the same
// plane (near, or a screen edge widened by 0.1%) by a margin far above the
// FP32 rounding of the per-vertex transform, so no skipped instance could
// have covered a pixel centre.
bool instance_visible(const float *mv, const MeshRec &m, const Cam &cam) {
    if (!m.bounded) return true;
    const double eps = 1e-3;
    bool all_near = true, all_l = true, all_r = true, all_b = true, all_t = true;
    for (int k = 0; k < 8; ++k) {
        const double p[3] = {(k & 1) ? m.hi[0] : m.lo[0], (k & 2) ? m.hi[1] : m.lo[1], (k & 4) ? m.hi[2] : m.lo[2]};
        double v[3], a[3];
        for (int r = 0; r < 3; ++r) {
            v[r] = mv[4 * r + 3];
            a[r] = std::fabs((double)mv[4 * r + 3]);
            for (int j = 0; j < 3; ++j) {
                v[r] += (double)mv[4 * r + j] * p[j];
                a[r] += std::fabs((double)mv[4 * r + j] * p[j]);
            }
        }
        const double cx = cam.fx * v[0], cy = cam.fy * v[1], cw = -v[2];
        const double e = 1e-4 * (cam.fx * a[0] + cam.fy * a[1] + a[2]) + 1e-30;
        all_near = all_near && (cam.nearv - cw > e);
        all_r = all_r && (cx - (1 + eps) * cw > e);
        all_l = all_l && (-cx - (1 + eps) * cw > e);
        all_t = all_t && (cy - (1 + eps) * cw > e);
        all_b = all_b && (-cy - (1 + eps) * cw > e);
    }
    return !(all_near || all_l || all_r || all_b || all_t);
}

// Constants of the conservative tiny-triangle cull of one (instance, view).
// The estimate X'_f = (fn_x . p) / (fn_w . p) uses FMA rows and an
// approximate reciprocal; the exact path is the FP32 sequence of the
// projection (Eq. 2) and the snap.  Forward error analysis of both, with
// S_r = sum_j |m_rj a_j| + |m_r3| (a_j the largest |coordinate| of the mesh
// bounds), bounds their distance by max(1/w) (ka + kb |X'|) + kc |X'| + kd
// pixels (the terms are listed below).  wsafe keeps the exact depth of every
// vertex above the near plane.
void fast_constants(PairDev &p, const MeshRec &m, const ViewDev &v) {
    std::memset(p.fn, 0, sizeof(p.fn));
    std::memset(p.fk, 0, sizeof(p.fk));
    std::memset(p.fs, 0, sizeof(p.fs));
    p.nlo = -INFINITY;
    p.wsafe = INFINITY;
    p.win = 0.0f;
    if (!m.bounded) return;
    // u: FP32 unit roundoff; rho: relative error assumed for rcp.approx.ftz.f32
    // (8x the documented one ulp)
    const double u = std::ldexp(1.0, -24), rho = std::ldexp(1.0, -20);
    double amax[3], S[3];
    for (int j = 0; j < 3; ++j) amax[j] = std::max(std::fabs(m.lo[j]), std::fabs(m.hi[j]));
    for (int r = 0; r < 3; ++r) {
        S[r] = std::fabs((double)p.mv[4 * r + 3]);
        for (int j = 0; j < 3; ++j) S[r] += std::fabs((double)p.mv[4 * r + j]) * amax[j];
    }
    const double hw = v.hw, hh = v.hh, fx = v.fx, fy = v.fy;
    const double ax = hw * fx, bx = hw - 0.5, ay = hh * fy, by = hh - 0.5;
    for (int j = 0; j < 4; ++j) {
        const double wr = -(double)p.mv[8 + j];
        p.fn[j] = (float)(ax * (double)p.mv[j] + bx * wr);
        p.fn[4 + j] = (float)(ay * (double)p.mv[4 + j] + by * wr);
        p.fn[8 + j] = (float)wr;
    }
    // Near plane: the w row holds the exact path's own coefficients, negated,
    // so the FMA estimate and the exact path's w (three products and sums
    // without FMA) are each within 3.01 u S_z of the true value; a vertex
    // whose estimate lies below near - 8 u S_z is beyond the near plane in
    // the exact path, and a triangle with all three there is dropped by it.
    {
        const double nl = (double)v.nearv - 8 * u * S[2];
        float f = (float)nl;
        if ((double)f > nl) f = std::nextafter(f, -INFINITY);
        p.nlo = f;
    }
    // Error budget per coordinate (pixels), exact path plus estimate:
    //   (9.002u a S_axis + 4.001u b S_z + 4.001u h S_z + 7.002u (|X'| + 1) S_z) / w
    //   + (|X'| + 1)(rho + 7.01u) + 5.01u (h + 1) + 1/512 (the snap),
    // with 1/w <= max(1/w~) (1 + 4u S_z / wsafe) / (1 - rho) for the estimated w~.
    double ws = v.nearv * (1 + 1e-3) + 8 * u * S[2];
    const double F = 1.01 * (1 + 4 * u * S[2] / ws) / (1 - rho);
    const double kax = 9.002 * ax * S[0] + 4.001 * bx * S[2] + 4.001 * hw * S[2] + 7.002 * S[2];
    const double kay = 9.002 * ay * S[1] + 4.001 * by * S[2] + 4.001 * hh * S[2] + 7.002 * S[2];
    const double ka = F * u * std::max(kax, kay);
    const double kb = F * u * 7.002 * S[2];
    const double kc = 1.01 * (rho + 7.01 * u);
    const double kd = 1.01 * (5.01 * u * (std::max(hw, hh) + 1) + rho + 7.01 * u) + 1.0 / 512;
    // The test applies where w > wsafe and |X'|, |Y'| < win = 100 min(W/2,
    // H/2).  wsafe is raised until the margin stays below 20 min(W/2, H/2)
    // there (the reciprocal may read 1 + rho high), so every exact vertex of a
    // tested triangle has |X'|, |Y'| < 120 min(W/2, H/2): well inside the
    // guard band (|X - W/2| <= 128 W/2, likewise for Y), where the exact path
    // snaps it and never clips.  The bound is linear in |X'| and holds at any
    // size of the margin; a margin of many pixels only culls less.
    const double hm = std::min(hw, hh);
    const double win = 100.0 * hm;
    const double room = 20.0 * hm - kc * win - kd;
    if (!(room > 0.0)) return;
    ws = std::max(ws, 1.01 * (1 + rho) * (ka + kb * win) / room);
    if (!std::isfinite(ka) || !std::isfinite(ws) || ka > 1e30 || ws > 1e30) return;
    // round the constants up (the window down) so the float copies stay conservative
    p.fk[0] = (float)(ka * (1 + 1e-6));
    p.fk[1] = (float)(kb * (1 + 1e-6));
    p.fk[2] = (float)(kc * (1 + 1e-6));
    p.fk[3] = (float)(kd * (1 + 1e-6));
    // the rows' magnitude over the mesh bounds is at most ax S_0 + bx S_2,
    // ay S_1 + by S_2 and S_2; 2^-19 of it covers the rounding of the group
    // test's box arithmetic (centre, half extent, row sums: a few u each)
    p.fs[0] = (float)(std::ldexp(ax * S[0] + bx * S[2], -19) * (1 + 1e-6));
    p.fs[1] = (float)(std::ldexp(ay * S[1] + by * S[2], -19) * (1 + 1e-6));
    p.fs[2] = (float)(std::ldexp(S[2], -19) * (1 + 1e-6));
    p.wsafe = (float)(ws * (1 + 1e-6));
    p.win = (float)win;
}

// Whether the near-plane test of the stage-1 cull could fire for a pair: w is
// affine in the position, so its smallest value over the mesh bounds is at
// a corner; when that (in double) clears near by 16 u S_z, every vertex's
// estimated w lies above the pair's nlo and the test never drops anything.
bool may_reach_near(const PairDev &p, const MeshRec &m, const Cam &cam) {
    if (!(p.nlo > -INFINITY)) return false;           // the test is off for this pair
    const double u = std::ldexp(1.0, -24);
    double S = std::fabs((double)p.mv[11]), wmin = INFINITY;
    for (int j = 0; j < 3; ++j) S += std::fabs((double)p.mv[8 + j]) * std::max(std::fabs(m.lo[j]), std::fabs(m.hi[j]));
    for (int k = 0; k < 8; ++k) {
        double w = -(double)p.mv[11];
        for (int j = 0; j < 3; ++j) w -= (double)p.mv[8 + j] * ((k >> j) & 1 ? m.hi[j] : m.lo[j]);
        wmin = std::min(wmin, w);
    }
    return !(wmin > (double)cam.nearv + 16 * u * S);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

curast_config default_config() {
    curast_config c;
    std::memset(&c, 0, sizeof(c));
    c.stage1_max_pixels = 128;
    c.stage2_max_pixels = 4096;
    c.tile_log2 = 6;
    c.stage1_tri_per_thread = 4;
    c.pairs_per_segment = 64;
    c.queue1_capacity = 1ull << 22;
    c.queue2_capacity = 1ull << 21;
    c.stage1_bitmap_bytes = 1ull << 32;
    c.stage1_group_min_pairs = 2;
    c.stage1_vertex_reuse = 0;
    c.stage3_tile_buffer = 0;
    c.check_indices = 1;
    c.collect_stats = 0;
    return c;
}

}  // namespace

struct curast_ctx {
    int device = 0;
    curast_config cfg;
    LaunchShape shape;
    cudaStream_t aux = nullptr;           // private stream for synchronous set-up work

    std::vector<MeshRec> meshes;
    std::vector<InstRec> insts;
    std::vector<uint64_t> base{0};        // exclusive prefix sum, n_inst + 1 entries
    std::vector<std::vector<uint32_t>> mesh_insts;
    bool inst_dirty = true, meshes_dirty = true;

    DevBuf<MeshDev> d_meshes;
    DevBuf<uint64_t> d_base;
    DevBuf<uint32_t> d_inst_mesh;
    DevBuf<float> d_inst_mv;
    PinBuf<float> h_inst_mv;
    cudaEvent_t ev_inst_mv = nullptr;

    // frame tables: [hdr | views | segs | pairs], one device and one pinned copy
    DevBuf<unsigned char> d_tab;
    PinBuf<unsigned char> h_tab;
    size_t cap_views = 0, cap_segs = 0, cap_pairs = 0;
    cudaEvent_t ev_tab = nullptr;
    std::vector<ViewDev> hv;
    std::vector<PairDev> hp;
    std::vector<SegDev> hs;
    FrameHdr hdr{};
    bool instanced = false;
    bool near_needed = true;              // some pair's mesh bounds reach the near plane

    DevBuf<Q1Entry> d_q1;
    DevBuf<uint32_t> d_bits;              // survivor bitmap of one stage-1 round
    std::vector<RoundDev> rounds;
    std::vector<char> round_comp;         // the round's meshes are compressed
    DevBuf<Q2Entry> d_q2;
    DevBuf<uint32_t> d_sorted;            // queue-2 indices in tile order (binned stage 3)
    DevBuf<uint32_t> d_tiles;             // per tile: count | start (+1) | fill
    DevBuf<uint2> d_units;                // stage-3 units: (tile, first part), up to 8 parts each
    uint32_t n_tiles = 0;
    Counters *d_ctr = nullptr;
    unsigned *d_err = nullptr;
    float *d_aabb = nullptr;              // 256*6 scratch + 6 result
    unsigned long long *d_diff = nullptr;

    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_recorded = false;

    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gkey;
};

namespace {

curast_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CURAST_OK;
    if (e == cudaErrorMemoryAllocation) return CURAST_ERR_OUT_OF_MEMORY;
    if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorInvalidDeviceFunction) return CURAST_ERR_NOT_BUILT;
    std::fprintf(stderr, "curast: CUDA error %s (%s)\n", cudaGetErrorName(e), cudaGetErrorString(e));
    return CURAST_ERR_CUDA;
}

#define CU(x)                                           \
    do {                                                \
        cudaError_t e_ = (x);                           \
        if (e_ != cudaSuccess) return cuda_status(e_);  \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

void invalidate_graph(curast_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey.clear();
}

curast_status sync_scene(curast_ctx *c, cudaStream_t s) {
    if (c->meshes_dirty) {
        std::vector<MeshDev> md(c->meshes.size());
        for (size_t i = 0; i < md.size(); ++i) {
            const MeshRec &r = c->meshes[i];
            md[i] = MeshDev{};
            md[i].pos = r.pos;
            md[i].idx = r.idx;
            md[i].rgba = r.rgba;
            md[i].V = r.V;
            md[i].T = r.T;
            md[i].uv = r.uv;
            md[i].tex = r.tex;
            md[i].tex_log2 = r.tex_log2;
            if (r.comp) {
                md[i].cidx = r.cidx;
                md[i].qpos = r.qpos;
                md[i].gflag = r.gflag;
                md[i].bits = r.bits;
                md[i].mask = r.bits >= 32 ? ~0u : (1u << r.bits) - 1u;
                md[i].imin = r.imin;
                for (int a = 0; a < 3; ++a) {
                    md[i].lo[a] = r.clo[a];
                    md[i].step[a] = r.cstep[a];
                }
            }
        }
        const bool grow = md.size() > c->d_meshes.cap;
        CU(c->d_meshes.reserve(std::max<size_t>(md.size(), 1)));
        if (grow) invalidate_graph(c);
        if (!md.empty()) CU(cudaMemcpyAsync(c->d_meshes.p, md.data(), md.size() * sizeof(MeshDev), cudaMemcpyHostToDevice, s));
        c->meshes_dirty = false;
    }
    if (c->inst_dirty) {
        const size_t n = c->insts.size();
        CU(c->d_base.reserve(n + 1));
        CU(c->d_inst_mesh.reserve(std::max<size_t>(n, 1)));
        std::vector<uint32_t> im(n);
        for (size_t i = 0; i < n; ++i) im[i] = c->insts[i].mesh;
        CU(cudaMemcpyAsync(c->d_base.p, c->base.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
        if (n) CU(cudaMemcpyAsync(c->d_inst_mesh.p, im.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        c->mesh_insts.assign(c->meshes.size(), {});
        for (size_t i = 0; i < n; ++i) c->mesh_insts[c->insts[i].mesh].push_back((uint32_t)i);
        c->inst_dirty = false;
    }
    return CURAST_OK;
}

curast_status make_view(const curast_view &v, ViewDev *out) {
    if (v.W < 1 || v.H < 1 || v.W > 16384 || v.H > 16384 || !v.vis) return CURAST_ERR_INVALID_ARG;
    if (!affine(v.view)) return CURAST_ERR_NOT_AFFINE;
    Cam cam;
    curast_status st = parse_camera(v.proj, &cam);
    if (st != CURAST_OK) return st;
    out->fx = cam.fx;
    out->fy = cam.fy;
    out->nearv = cam.nearv;
    out->hw = 0.5f * (float)v.W;
    out->hh = 0.5f * (float)v.H;
    out->W = v.W;
    out->H = v.H;
    out->tile0 = 0;
    out->ntx = 0;
    out->vis = v.vis;
    return CURAST_OK;
}

// Builds the frame tables for the given views; only_mesh < 0 = all meshes.
curast_status build_frame(curast_ctx *c, const curast_view *views, int nv, long only_mesh) {
    c->hv.assign((size_t)nv, ViewDev{});
    std::vector<Cam> cams((size_t)nv);
    for (int v = 0; v < nv; ++v) {
        curast_status st = make_view(views[v], &c->hv[v]);
        if (st != CURAST_OK) return st;
        cams[v] = Cam{c->hv[v].fx, c->hv[v].fy, c->hv[v].nearv};
    }
    c->hp.clear();
    c->hs.clear();
    c->near_needed = false;
    const uint64_t per_item = 256ull * c->cfg.stage1_tri_per_thread;
    const size_t m0 = only_mesh < 0 ? 0 : (size_t)only_mesh;
    const size_t m1 = only_mesh < 0 ? c->meshes.size() : (size_t)only_mesh + 1;
    for (size_t m = m0; m < m1; ++m) {
        const MeshRec &mr = c->meshes[m];
        if (mr.T == 0) continue;
        const size_t first = c->hp.size();
        for (uint32_t i : c->mesh_insts[m]) {
            for (int v = 0; v < nv; ++v) {
                PairDev p;
                model_view(views[v].view, c->insts[i].model, p.mv);
                if (!instance_visible(p.mv, mr, cams[v])) continue;
                p.base = c->base[i];
                p.view = (uint32_t)v;
                p.mesh = (uint32_t)m;
                fast_constants(p, mr, c->hv[v]);
                if (c->cfg.stage1_exact_all) p.wsafe = INFINITY, p.nlo = -INFINITY;   // no conservative cull
                c->near_needed = c->near_needed || may_reach_near(p, mr, cams[v]);
                c->hp.push_back(p);
            }
        }
        const size_t np = c->hp.size() - first;
        for (size_t k = 0; k < np; k += c->cfg.pairs_per_segment) {
            SegDev s;
            s.mesh = (uint32_t)m;
            s.pair0 = (uint32_t)(first + k);
            s.npairs = (uint32_t)std::min<size_t>(c->cfg.pairs_per_segment, np - k);
            s.pad = 0;
            s.T = mr.T;
            s.batch0 = 0;
            c->hs.push_back(s);
        }
    }
    // uncompressed meshes first, then compressed ones (rounds hold one kind, so
    // each runs the cull kernel built for it); within each, heavy work items
    // (many pairs) first so the tail of the persistent loop is light
    std::stable_sort(c->hs.begin(), c->hs.end(), [c](const SegDev &a, const SegDev &b) {
        const bool ca = c->meshes[a.mesh].comp, cb = c->meshes[b.mesh].comp;
        if (ca != cb) return cb;
        return a.npairs > b.npairs;
    });
    // survivor-bitmap words: per item, npairs x (per_item / 32)
    const uint64_t G = per_item / 32;
    uint64_t nb = 0, nw = 0;
    c->instanced = false;
    for (SegDev &s : c->hs) {
        s.batch0 = nb;
        s.word0 = nw;
        const uint64_t items = (s.T + per_item - 1) / per_item;
        nb += items;
        nw += items * s.npairs * G;
        c->instanced = c->instanced || s.npairs > 1;
    }
    // rounds: runs of items whose bitmap fits the configured size (grown
    // when the frame would need more than kMaxRounds rounds; one round more
    // may start where the meshes turn from uncompressed to compressed)
    uint64_t cap = std::max<uint64_t>(c->cfg.stage1_bitmap_bytes / 4, 64 * G);
    cap = std::max<uint64_t>(cap, (nw + kMaxRounds - 3) / (kMaxRounds - 2) + 64 * G);
    c->rounds.clear();
    c->round_comp.clear();
    RoundDev cur{0, 0, 0, 0};
    bool cur_comp = false;
    for (const SegDev &s : c->hs) {
        const uint64_t items = (s.T + per_item - 1) / per_item, wpi = s.npairs * G;
        const bool comp = c->meshes[s.mesh].comp;
        if (comp != cur_comp && cur.b1 > cur.b0) {           // a round holds one kind of mesh
            c->rounds.push_back(cur);
            c->round_comp.push_back(cur_comp);
            cur = RoundDev{cur.b1, cur.b1, cur.w1, cur.w1};
        }
        cur_comp = comp;
        uint64_t done = 0;
        while (done < items) {
            uint64_t room = (cap - (cur.w1 - cur.w0)) / wpi;
            if (room == 0) {
                c->rounds.push_back(cur);
                c->round_comp.push_back(cur_comp);
                cur = RoundDev{cur.b1, cur.b1, cur.w1, cur.w1};
                room = cap / wpi;
            }
            const uint64_t take = std::min(room, items - done);
            cur.b1 += take;
            cur.w1 += take * wpi;
            done += take;
        }
    }
    if (cur.b1 > cur.b0 || c->rounds.empty()) {
        c->rounds.push_back(cur);
        c->round_comp.push_back(cur_comp);
    }
    if (c->rounds.size() > (size_t)kMaxRounds) return CURAST_ERR_INVALID_ARG;   // unreachable by the cap above
    uint64_t maxw = 1;
    for (const RoundDev &r : c->rounds) maxw = std::max(maxw, r.w1 - r.w0);
    CU(c->d_bits.reserve(maxw));
    // stage-3 tiles of every view, numbered view by view, row by row
    {
        const uint64_t ts = 1ull << c->cfg.tile_log2;
        uint64_t nt = 0;
        for (ViewDev &v : c->hv) {
            v.tile0 = (uint32_t)nt;
            v.ntx = (uint32_t)(((uint64_t)v.W + ts - 1) / ts);
            nt += (uint64_t)v.ntx * (((uint64_t)v.H + ts - 1) / ts);
        }
        if (nt >= (1ull << 31)) return CURAST_ERR_INVALID_ARG;
        c->n_tiles = (uint32_t)nt;
        if (c->cfg.stage3_tile_buffer) {
            CU(c->d_tiles.reserve(3 * nt + 1));
            // a tile of c parts makes ceil(c / 8) units
            CU(c->d_units.reserve(nt + c->cfg.queue2_capacity / 8 + 1));
        }
    }
    c->hdr.n_batches = nb;
    c->hdr.n_segs = (uint32_t)c->hs.size();
    c->hdr.n_views = (uint32_t)nv;
    c->hdr.n_rounds = (uint32_t)c->rounds.size();
    c->hdr.pad = 0;
    return CURAST_OK;
}

constexpr size_t kRoundsOff = 256;                                        // RoundDev[kMaxRounds]
constexpr size_t kHdrBytes = kRoundsOff + kMaxRounds * sizeof(RoundDev);   // 2304

size_t off_views(const curast_ctx *) { return kHdrBytes; }
size_t off_segs(const curast_ctx *c) { return align_up(kHdrBytes + c->cap_views * sizeof(ViewDev), 256); }
size_t off_pairs(const curast_ctx *c) { return align_up(off_segs(c) + c->cap_segs * sizeof(SegDev), 256); }
size_t tab_bytes(const curast_ctx *c) { return off_pairs(c) + c->cap_pairs * sizeof(PairDev); }

curast_status upload_frame(curast_ctx *c, cudaStream_t s) {
    if (c->hv.size() > c->cap_views || c->hs.size() > c->cap_segs || c->hp.size() > c->cap_pairs) {
        CU(cudaEventSynchronize(c->ev_tab));
        c->cap_views = std::max<size_t>(c->hv.size(), std::max<size_t>(2 * c->cap_views, 8));
        c->cap_segs = std::max<size_t>(c->hs.size(), std::max<size_t>(2 * c->cap_segs, 256));
        c->cap_pairs = std::max<size_t>(c->hp.size(), std::max<size_t>(2 * c->cap_pairs, 256));
        c->d_tab.release();
        c->h_tab.release();
        CU(c->d_tab.reserve(tab_bytes(c)));
        CU(c->h_tab.reserve(tab_bytes(c)));
        invalidate_graph(c);
    }
    // the pinned staging copy may still feed the previous frame's upload
    CU(cudaEventSynchronize(c->ev_tab));
    unsigned char *h = c->h_tab.p;
    std::memcpy(h, &c->hdr, sizeof(FrameHdr));
    std::memcpy(h + kRoundsOff, c->rounds.data(), c->rounds.size() * sizeof(RoundDev));
    std::memcpy(h + off_views(c), c->hv.data(), c->hv.size() * sizeof(ViewDev));
    std::memcpy(h + off_segs(c), c->hs.data(), c->hs.size() * sizeof(SegDev));
    std::memcpy(h + off_pairs(c), c->hp.data(), c->hp.size() * sizeof(PairDev));
    const size_t n1 = off_views(c) + c->hv.size() * sizeof(ViewDev);
    CU(cudaMemcpyAsync(c->d_tab.p, h, n1, cudaMemcpyHostToDevice, s));
    if (!c->hs.empty())
        CU(cudaMemcpyAsync(c->d_tab.p + off_segs(c), h + off_segs(c), c->hs.size() * sizeof(SegDev),
                           cudaMemcpyHostToDevice, s));
    if (!c->hp.empty())
        CU(cudaMemcpyAsync(c->d_tab.p + off_pairs(c), h + off_pairs(c), c->hp.size() * sizeof(PairDev),
                           cudaMemcpyHostToDevice, s));
    CU(cudaEventRecord(c->ev_tab, s));
    return CURAST_OK;
}

FrameDev make_frame_dev(const curast_ctx *c) {
    FrameDev f;
    f.hdr = reinterpret_cast<const FrameHdr *>(c->d_tab.p);
    f.views = reinterpret_cast<const ViewDev *>(c->d_tab.p + off_views(c));
    f.segs = reinterpret_cast<const SegDev *>(c->d_tab.p + off_segs(c));
    f.pairs = reinterpret_cast<const PairDev *>(c->d_tab.p + off_pairs(c));
    f.meshes = c->d_meshes.p;
    f.q1 = c->d_q1.p;
    f.q2 = c->d_q2.p;
    f.rounds = reinterpret_cast<const RoundDev *>(c->d_tab.p + kRoundsOff);
    f.bits = c->d_bits.p;
    f.ctr = c->d_ctr;
    f.err = c->d_err;
    f.q1_cap = c->cfg.queue1_capacity;
    f.q2_cap = c->cfg.queue2_capacity;
    f.s1_max = c->cfg.stage1_max_pixels;
    f.s2_max = c->cfg.stage2_max_pixels;
    f.tile_log2 = c->cfg.tile_log2;
    f.tpt = c->cfg.stage1_tri_per_thread;
    fastdiv_consts(8u * f.tpt, f.g_m, f.g_s);
    f.group_min = c->cfg.stage1_group_min_pairs;
    f.s3_ray = c->cfg.stage3_raycast;
    f.check = c->cfg.check_indices;
    f.stats = c->cfg.collect_stats;
    f.s3_bin = c->cfg.stage3_tile_buffer;
    f.n_tiles = c->n_tiles;
    f.tile_cnt = f.tile_start = f.tile_fill = f.part_sorted = nullptr;
    f.units = nullptr;
    if (f.s3_bin) {
        f.tile_cnt = c->d_tiles.p;
        f.tile_start = f.tile_cnt + c->n_tiles;
        f.tile_fill = f.tile_start + c->n_tiles + 1;
        f.part_sorted = c->d_sorted.p;
        f.units = c->d_units.p;
    }
    return f;
}

// clear (optional) -> reset counters -> stage 1 (cull, exact) -> stage 2 -> stage 3
curast_status enqueue_stages(curast_ctx *c, bool clear, bool timing, cudaStream_t s) {
    const FrameDev f = make_frame_dev(c);
    const int sms = c->shape.num_sms;
    if (timing) CU(cudaEventRecord(c->ev[0], s));
    if (clear)
        for (const ViewDev &v : c->hv) CU(launch_clear(v.vis, (uint64_t)v.W * (uint64_t)v.H, s));
    CU(cudaMemsetAsync(c->d_ctr, 0, sizeof(Counters), s));
    if (f.s3_bin && c->n_tiles) CU(cudaMemsetAsync(f.tile_cnt, 0, (size_t)c->n_tiles * sizeof(uint32_t), s));
    if (timing) CU(cudaEventRecord(c->ev[1], s));
    // stage 1 round by round: the cull fills the survivor bitmap, the exact
    // kernel empties it (ev[2] falls after the last round's cull)
    const uint32_t nr = (uint32_t)c->rounds.size();
    for (uint32_t r = 0; r < nr; ++r) {
        const int variant = c->round_comp[r] ? 2 : (!c->instanced && c->cfg.stage1_vertex_reuse ? 3 : 0);
        CU(launch_stage1(f, c->instanced, variant, r, sms * c->shape.stage1_blocks_per_sm[c->instanced ? 1 : 0][variant],
                         c->near_needed, s));
        if (timing && r + 1 == nr) CU(cudaEventRecord(c->ev[2], s));
        CU(launch_stage1_exact(f, r, sms * c->shape.stage1x_blocks_per_sm, s));
    }
    if (timing) CU(cudaEventRecord(c->ev[3], s));
    CU(launch_stage2(f, sms * c->shape.stage2_blocks_per_sm, s));
    if (timing) CU(cudaEventRecord(c->ev[4], s));
    if (f.s3_bin)
        CU(launch_stage3_binned(f, sms * 4, sms * c->shape.stage3t_blocks_per_sm[c->cfg.tile_log2 - 4], s));
    else
        CU(launch_stage3(f, sms * c->shape.stage3_blocks_per_sm, s));
    if (timing) CU(cudaEventRecord(c->ev[5], s));
    c->ev_recorded = c->ev_recorded || timing;
    return CURAST_OK;
}

curast_status render_views(curast_ctx *c, const curast_view *views, int nv, long only_mesh, bool clear, bool graph,
                           cudaStream_t s) {
    DeviceGuard g(c->device);
    curast_status st = sync_scene(c, s);
    if (st != CURAST_OK) return st;
    st = build_frame(c, views, nv, only_mesh);
    if (st != CURAST_OK) return st;
    st = upload_frame(c, s);
    if (st != CURAST_OK) return st;
    if (!graph) return enqueue_stages(c, clear, true, s);
    std::vector<uint64_t> key = {(uint64_t)nv, (uint64_t)c->instanced, (uint64_t)clear,
                                 (uint64_t)(uintptr_t)c->d_tab.p, (uint64_t)(uintptr_t)c->d_meshes.p,
                                 (uint64_t)(uintptr_t)c->d_bits.p, (uint64_t)c->rounds.size(),
                                 (uint64_t)(uintptr_t)c->d_tiles.p, (uint64_t)(uintptr_t)c->d_sorted.p,
                                 (uint64_t)(uintptr_t)c->d_units.p};
    for (char rc : c->round_comp) key.push_back((uint64_t)rc);
    for (int v = 0; v < nv; ++v) {
        key.push_back((uint64_t)views[v].W);
        key.push_back((uint64_t)views[v].H);
        key.push_back((uint64_t)(uintptr_t)views[v].vis);
    }
    if (!c->gexec || key != c->gkey) {
        invalidate_graph(c);
        cudaStream_t cs;
        CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue_stages(c, clear, false, cs);
            e = cudaStreamEndCapture(cs, &gr);
        }
        if (e == cudaSuccess && st == CURAST_OK) e = cudaGraphInstantiate(&c->gexec, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cs);
        if (st != CURAST_OK) return st;
        CU(e);
        c->gkey = key;
    }
    CU(cudaGraphLaunch(c->gexec, s));
    return CURAST_OK;
}

curast_status upload_inst_mv(curast_ctx *c, const float *view, cudaStream_t s) {
    const size_t n = c->insts.size();
    CU(cudaEventSynchronize(c->ev_inst_mv));
    CU(c->h_inst_mv.reserve(12 * std::max<size_t>(n, 1)));
    CU(c->d_inst_mv.reserve(12 * std::max<size_t>(n, 1)));
    for (size_t i = 0; i < n; ++i) model_view(view, c->insts[i].model, c->h_inst_mv.p + 12 * i);
    if (n) CU(cudaMemcpyAsync(c->d_inst_mv.p, c->h_inst_mv.p, 12 * n * sizeof(float), cudaMemcpyHostToDevice, s));
    CU(cudaEventRecord(c->ev_inst_mv, s));
    return CURAST_OK;
}

curast_status shade_setup(curast_ctx *c, const float *view, const float *proj, int W, int H, const uint64_t *vis,
                          ShadeArgs *a, cudaStream_t s) {
    if (!vis || W < 1 || H < 1 || W > 16384 || H > 16384) return CURAST_ERR_INVALID_ARG;
    if (!affine(view)) return CURAST_ERR_NOT_AFFINE;
    Cam cam;
    curast_status st = parse_camera(proj, &cam);
    if (st != CURAST_OK) return st;
    st = sync_scene(c, s);
    if (st != CURAST_OK) return st;
    st = upload_inst_mv(c, view, s);
    if (st != CURAST_OK) return st;
    std::memset(a, 0, sizeof(*a));
    a->vis = vis;
    a->W = W;
    a->H = H;
    a->fx = cam.fx;
    a->fy = cam.fy;
    a->inst_mv = c->d_inst_mv.p;
    a->base = c->d_base.p;
    a->inst_mesh = c->d_inst_mesh.p;
    a->meshes = c->d_meshes.p;
    a->n_inst = (int)c->insts.size();
    return CURAST_OK;
}

curast_status alloc_queues(curast_ctx *c) {
    c->d_q1.release();
    c->d_q2.release();
    c->d_sorted.release();
    CU(c->d_q1.reserve(std::max<uint64_t>(c->cfg.queue1_capacity, 1)));
    CU(c->d_q2.reserve(std::max<uint64_t>(c->cfg.queue2_capacity, 1)));
    CU(c->d_sorted.reserve(std::max<uint64_t>(c->cfg.queue2_capacity, 1)));
    invalidate_graph(c);
    return CURAST_OK;
}

curast_status compute_bounds(curast_ctx *c, MeshRec &m) {
    m.bounded = false;
    if (m.V == 0) return CURAST_OK;
    // the positions may have been written by work on any stream
    CU(cudaDeviceSynchronize());
    CU(launch_aabb(m.pos, m.V, c->d_aabb, c->d_aabb + 256 * 6, c->aux));
    float b[6];
    CU(cudaMemcpyAsync(b, c->d_aabb + 256 * 6, sizeof(b), cudaMemcpyDeviceToHost, c->aux));
    CU(cudaStreamSynchronize(c->aux));
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        ok = ok && std::isfinite(b[k]) && std::isfinite(b[3 + k]) && b[k] <= b[3 + k];
        m.lo[k] = b[k];
        m.hi[k] = b[3 + k];
    }
    m.bounded = ok;
    return CURAST_OK;
}

int index_bits(uint32_t span) {
    int b = 0;
    while (b < 32 && (1ull << b) < (uint64_t)span + 1) ++b;
    return b;
}

void free_compressed(MeshRec &m) {
    if (m.cidx) cudaFree(m.cidx);
    if (m.qpos) cudaFree(m.qpos);
    if (m.gflag) cudaFree(m.gflag);
    m.cidx = nullptr;
    m.qpos = nullptr;
    m.gflag = nullptr;
}

// Section 4.6 encoding of an uploaded mesh into context-owned buffers (see
// CURAST_MESH_COMPRESSED); m.lo / m.hi hold the bounds of the positions.
curast_status compress_mesh(curast_ctx *c, MeshRec &m) {
    uint32_t imin = 0, imax = 0;
    if (m.T > 0) {
        unsigned init[2] = {~0u, 0u}, mm[2];
        CU(cudaMemcpyAsync(c->d_aabb, init, sizeof(init), cudaMemcpyHostToDevice, c->aux));
        CU(launch_minmax_u32(m.idx, 3 * m.T, reinterpret_cast<unsigned *>(c->d_aabb), c->aux));
        CU(cudaMemcpyAsync(mm, c->d_aabb, sizeof(mm), cudaMemcpyDeviceToHost, c->aux));
        CU(cudaStreamSynchronize(c->aux));
        imin = mm[0];
        imax = mm[1];
        if (imax >= m.V) return CURAST_ERR_INDEX_OUT_OF_RANGE;
    }
    m.bits = (uint32_t)index_bits(imax - imin);
    m.imin = imin;
    // words of the stream, then padding: the cull reads one word ahead and
    // rounds its copies up to 16 bytes
    m.cwords = ((3 * m.T * m.bits + 31) >> 5) + 8;
    double lo[3], size[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = m.bounded ? (double)(float)m.lo[a] : 0.0;
        size[a] = m.bounded ? (double)(float)m.hi[a] - lo[a] : 0.0;
        m.clo[a] = (float)lo[a];
        m.cstep[a] = (float)(size[a] / 65535.0);
    }
    uint32_t *w = nullptr;
    uint16_t *q = nullptr;
    CU(cudaMalloc(reinterpret_cast<void **>(&w), m.cwords * sizeof(uint32_t)));
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&q), std::max<uint64_t>(3 * m.V, 8) * sizeof(uint16_t));
    if (e != cudaSuccess) {
        cudaFree(w);
        return e == cudaErrorMemoryAllocation ? CURAST_ERR_OUT_OF_MEMORY : CURAST_ERR_CUDA;
    }
    m.cidx = w;
    m.qpos = q;
    const uint64_t gwords = ((m.T + 127) / 128 + 31) / 32;
    if (gwords) {
        e = cudaMalloc(reinterpret_cast<void **>(&m.gflag), gwords * sizeof(uint32_t));
        if (e != cudaSuccess) {
            m.gflag = nullptr;
            free_compressed(m);
            return e == cudaErrorMemoryAllocation ? CURAST_ERR_OUT_OF_MEMORY : CURAST_ERR_CUDA;
        }
    }
    cudaError_t e1 = cudaMemsetAsync(w, 0, m.cwords * sizeof(uint32_t), c->aux);
    if (e1 == cudaSuccess && m.T) e1 = launch_pack_indices(m.idx, 3 * m.T, imin, m.bits, w, m.cwords - 8, c->aux);
    if (e1 == cudaSuccess && gwords) e1 = launch_grid_flags(m.idx, m.T, m.V, m.gflag, gwords, c->aux);
    if (e1 == cudaSuccess && m.V) e1 = launch_quantize_positions(m.pos, m.V, lo, size, q, c->aux);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(c->aux);
    if (e1 != cudaSuccess) {
        free_compressed(m);
        return CURAST_ERR_CUDA;
    }
    m.comp = true;
    m.pos = nullptr;      // the caller's buffers are no longer read
    m.idx = nullptr;
    // bounds of the decoded positions fma(q, step, lo), q <= 65535, for culling
    for (int a = 0; a < 3; ++a) {
        m.lo[a] = (double)m.clo[a] - 1e-6 * std::fabs((double)m.clo[a]);
        m.hi[a] = (double)m.clo[a] + 65535.0 * (double)m.cstep[a];
        m.hi[a] += 1e-6 * std::fabs(m.hi[a]);
    }
    return CURAST_OK;
}

bool valid_config(const curast_config &c) {
    return c.stage1_max_pixels >= 1 && c.stage1_max_pixels <= 1024 && c.stage2_max_pixels >= 32 &&
           c.tile_log2 >= 4 && c.tile_log2 <= 7 && c.stage1_tri_per_thread >= 1 && c.stage1_tri_per_thread <= 4 &&
           c.pairs_per_segment >= 1 && c.pairs_per_segment <= 64 && c.queue1_capacity >= 1 &&
           c.queue2_capacity >= 1 && c.queue1_capacity <= (1ull << 32) && c.queue2_capacity <= (1ull << 32) &&
           c.stage1_bitmap_bytes >= (1ull << 12) && c.stage1_bitmap_bytes <= (1ull << 36) &&
           c.stage1_group_min_pairs <= 64 && c.stage3_raycast <= 1 && c.stage1_exact_all <= 1 &&
           c.stage1_vertex_reuse <= 1 && c.stage3_tile_buffer <= 1 && c.reserved == 0;
}

}  // namespace

// ================================================================== C ABI ===
extern "C" {

const char *curast_status_string(curast_status s) {
    switch (s) {
    case CURAST_OK: return "ok";
    case CURAST_ERR_INVALID_ARG: return "invalid argument";
    case CURAST_ERR_OUT_OF_MEMORY: return "out of device memory";
    case CURAST_ERR_ID_SPACE_OVERFLOW: return "more than 2^36-1 triangles over all instances";
    case CURAST_ERR_INDEX_OUT_OF_RANGE: return "a vertex index was out of range";
    case CURAST_ERR_DEVICE_TIMEOUT: return "a device wait timed out";
    case CURAST_ERR_CUDA: return "CUDA runtime error";
    case CURAST_ERR_NOT_AFFINE: return "matrix is not affine";
    case CURAST_ERR_BAD_CAMERA: return "projection is not a symmetric perspective matrix";
    case CURAST_ERR_NOT_BUILT: return "no kernel image for this device";
    case CURAST_ERR_TOO_LARGE: return "exceeds a fixed capacity of the no-allocation render";
    default: return "unknown status";
    }
}

curast_status curast_create(curast_ctx **out, int device) {
    if (!out) return CURAST_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    CU(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(device);
    curast_ctx *c = new (std::nothrow) curast_ctx();
    if (!c) return CURAST_ERR_OUT_OF_MEMORY;
    c->device = device;
    c->cfg = default_config();
    curast_status st = CURAST_OK;
    cudaError_t e = query_launch_shape(&c->shape, device);
    if (e != cudaSuccess) st = cuda_status(e);
    if (st == CURAST_OK && c->shape.stage1_blocks_per_sm[0][0] < 1) st = CURAST_ERR_NOT_BUILT;
    if (st == CURAST_OK) st = cuda_status(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
    if (st == CURAST_OK) st = cuda_status(cudaMalloc(reinterpret_cast<void **>(&c->d_ctr), sizeof(Counters)));
    if (st == CURAST_OK) st = cuda_status(cudaMalloc(reinterpret_cast<void **>(&c->d_err), sizeof(unsigned)));
    if (st == CURAST_OK) st = cuda_status(cudaMemset(c->d_err, 0, sizeof(unsigned)));
    if (st == CURAST_OK) st = cuda_status(cudaMemset(c->d_ctr, 0, sizeof(Counters)));
    if (st == CURAST_OK) st = cuda_status(cudaMalloc(reinterpret_cast<void **>(&c->d_aabb), (256 * 6 + 6) * sizeof(float)));
    if (st == CURAST_OK) st = cuda_status(cudaMalloc(reinterpret_cast<void **>(&c->d_diff), sizeof(unsigned long long)));
    for (int k = 0; k < 6 && st == CURAST_OK; ++k) st = cuda_status(cudaEventCreate(&c->ev[k]));
    if (st == CURAST_OK) st = cuda_status(cudaEventCreateWithFlags(&c->ev_tab, cudaEventDisableTiming));
    if (st == CURAST_OK) st = cuda_status(cudaEventCreateWithFlags(&c->ev_inst_mv, cudaEventDisableTiming));
    if (st == CURAST_OK) st = alloc_queues(c);
    if (st == CURAST_OK) st = cuda_status(c->d_base.reserve(1));
    if (st != CURAST_OK) {
        curast_destroy(c);
        return st;
    }
    *out = c;
    return CURAST_OK;
}

void curast_destroy(curast_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    invalidate_graph(c);
    for (MeshRec &m : c->meshes) free_compressed(m);
    c->d_meshes.release();
    c->d_base.release();
    c->d_inst_mesh.release();
    c->d_inst_mv.release();
    c->h_inst_mv.release();
    c->d_tab.release();
    c->h_tab.release();
    c->d_q1.release();
    c->d_q2.release();
    c->d_sorted.release();
    c->d_tiles.release();
    c->d_units.release();
    c->d_bits.release();
    if (c->d_ctr) cudaFree(c->d_ctr);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_aabb) cudaFree(c->d_aabb);
    if (c->d_diff) cudaFree(c->d_diff);
    for (cudaEvent_t &e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->ev_tab) cudaEventDestroy(c->ev_tab);
    if (c->ev_inst_mv) cudaEventDestroy(c->ev_inst_mv);
    if (c->aux) cudaStreamDestroy(c->aux);
    delete c;
}

curast_status curast_get_config(const curast_ctx *c, curast_config *out) {
    if (!c || !out) return CURAST_ERR_INVALID_ARG;
    *out = c->cfg;
    return CURAST_OK;
}

curast_status curast_set_config(curast_ctx *c, const curast_config *cfg) {
    if (!c || !cfg || !valid_config(*cfg)) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    const bool requeue = cfg->queue1_capacity != c->cfg.queue1_capacity ||
                         cfg->queue2_capacity != c->cfg.queue2_capacity;
    CU(cudaDeviceSynchronize());
    c->cfg = *cfg;
    invalidate_graph(c);
    if (requeue) return alloc_queues(c);
    return CURAST_OK;
}

curast_status curast_upload_mesh(curast_ctx *c, const float *pos, uint64_t V, const uint32_t *idx, uint64_t T,
                                 const uint8_t *rgba8, uint32_t flags, uint32_t *mesh_id) {
    if (!c || !mesh_id || (flags & ~CURAST_MESH_COMPRESSED)) return CURAST_ERR_INVALID_ARG;
    if ((V > 0 && !pos) || (T > 0 && !idx) || V > 0xFFFFFFFFull || T > 0xFFFFFFFFull) return CURAST_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(pos) & 3) || (reinterpret_cast<uintptr_t>(idx) & 3) ||
        (reinterpret_cast<uintptr_t>(rgba8) & 3))
        return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    MeshRec m;
    m.pos = pos;
    m.idx = idx;
    m.rgba = rgba8;
    m.V = V;
    m.T = T;
    curast_status st = compute_bounds(c, m);
    if (st != CURAST_OK) return st;
    if (flags & CURAST_MESH_COMPRESSED) {
        st = compress_mesh(c, m);
        if (st != CURAST_OK) return st;
    }
    c->meshes.push_back(m);
    c->meshes_dirty = true;
    c->inst_dirty = true;
    *mesh_id = (uint32_t)(c->meshes.size() - 1);
    return CURAST_OK;
}

curast_status curast_update_mesh(curast_ctx *c, uint32_t mesh_id, const float *pos, const uint32_t *idx,
                                 const uint8_t *rgba8) {
    if (!c || mesh_id >= c->meshes.size()) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    MeshRec &m = c->meshes[mesh_id];
    if (m.comp && (pos || idx)) return CURAST_ERR_INVALID_ARG;
    if (pos) m.pos = pos;
    if (idx) m.idx = idx;
    if (rgba8) m.rgba = rgba8;
    curast_status st = compute_bounds(c, m);
    if (st != CURAST_OK) return st;
    c->meshes_dirty = true;
    return CURAST_OK;
}

curast_status curast_get_mesh_info(const curast_ctx *c, uint32_t mesh_id, curast_mesh_info *out) {
    if (!c || !out || mesh_id >= c->meshes.size()) return CURAST_ERR_INVALID_ARG;
    const MeshRec &m = c->meshes[mesh_id];
    std::memset(out, 0, sizeof(*out));
    out->V = m.V;
    out->T = m.T;
    out->compressed = m.comp ? 1u : 0u;
    if (m.comp) {
        out->index_bits = m.bits;
        out->index_min = m.imin;
        for (int a = 0; a < 3; ++a) {
            out->pos_lo[a] = m.clo[a];
            out->pos_step[a] = m.cstep[a];
        }
        out->geometry_bytes = ((3 * m.T * m.bits + 31) >> 5) * 4 + 6 * m.V;
        out->packed_indices = m.cidx;
        out->quantized_positions = m.qpos;
        out->grid_flags = m.gflag;
    } else {
        out->geometry_bytes = 12 * m.T + 12 * m.V;
    }
    return CURAST_OK;
}

curast_status curast_add_instance(curast_ctx *c, uint32_t mesh_id, const float model[16], uint32_t *instance_id) {
    if (!c || !model || mesh_id >= c->meshes.size()) return CURAST_ERR_INVALID_ARG;
    if (!affine(model)) return CURAST_ERR_NOT_AFFINE;
    const uint64_t total = c->base.back() + c->meshes[mesh_id].T;
    if (total > kIdMask) return CURAST_ERR_ID_SPACE_OVERFLOW;
    InstRec r;
    r.mesh = mesh_id;
    std::memcpy(r.model, model, sizeof(r.model));
    c->insts.push_back(r);
    c->base.push_back(total);
    c->inst_dirty = true;
    if (instance_id) *instance_id = (uint32_t)(c->insts.size() - 1);
    return CURAST_OK;
}

curast_status curast_clear_instances(curast_ctx *c) {
    if (!c) return CURAST_ERR_INVALID_ARG;
    c->insts.clear();
    c->base.assign(1, 0);
    c->inst_dirty = true;
    return CURAST_OK;
}

curast_status curast_clear(uint64_t *vis, uint64_t n, curast_stream stream) {
    if (!vis && n) return CURAST_ERR_INVALID_ARG;
    CU(launch_clear(vis, n, static_cast<cudaStream_t>(stream)));
    return CURAST_OK;
}

curast_status curast_render(curast_ctx *c, const float view[16], const float proj[16], int W, int H, uint64_t *vis,
                            curast_stream stream) {
    if (!c || !view || !proj) return CURAST_ERR_INVALID_ARG;
    curast_view v;
    std::memcpy(v.view, view, sizeof(v.view));
    std::memcpy(v.proj, proj, sizeof(v.proj));
    v.W = W;
    v.H = H;
    v.vis = vis;
    return render_views(c, &v, 1, -1, true, false, static_cast<cudaStream_t>(stream));
}

curast_status curast_render_mesh(curast_ctx *c, uint32_t mesh_id, const float view[16], const float proj[16], int W,
                                 int H, uint64_t *vis, curast_stream stream) {
    if (!c || !view || !proj || mesh_id >= c->meshes.size()) return CURAST_ERR_INVALID_ARG;
    curast_view v;
    std::memcpy(v.view, view, sizeof(v.view));
    std::memcpy(v.proj, proj, sizeof(v.proj));
    v.W = W;
    v.H = H;
    v.vis = vis;
    return render_views(c, &v, 1, (long)mesh_id, false, false, static_cast<cudaStream_t>(stream));
}

curast_status curast_render_batch(curast_ctx *c, const curast_view *views, int n_views, int use_graph,
                                  curast_stream stream) {
    if (!c || !views || n_views < 1 || n_views > 65536) return CURAST_ERR_INVALID_ARG;
    return render_views(c, views, n_views, -1, true, use_graph != 0, static_cast<cudaStream_t>(stream));
}

curast_status curast_resolve(curast_ctx *c, const float view[16], const float proj[16], int W, int H,
                             const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, curast_stream stream) {
    if (!c) return CURAST_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rgba_f32) & 15) || (reinterpret_cast<uintptr_t>(rgba8) & 3))
        return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ShadeArgs a;
    curast_status st = shade_setup(c, view, proj, W, H, vis, &a, s);
    if (st != CURAST_OK) return st;
    a.rgba_f32 = rgba_f32;
    a.rgba8 = rgba8;
    CU(launch_resolve(a, s));
    return CURAST_OK;
}

curast_status curast_set_mesh_texture(curast_ctx *c, uint32_t mesh_id, const float *uv, const uint8_t *texels,
                                     int log2_size) {
    if (!c || mesh_id >= c->meshes.size()) return CURAST_ERR_INVALID_ARG;
    MeshRec &m = c->meshes[mesh_id];
    if (!texels) {
        m.uv = nullptr;
        m.tex = nullptr;
        m.tex_log2 = 0;
    } else {
        if ((!uv && m.V > 0) || log2_size < 0 || log2_size > 15) return CURAST_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(uv) & 7) || (reinterpret_cast<uintptr_t>(texels) & 3))
            return CURAST_ERR_INVALID_ARG;
        m.uv = uv;
        m.tex = texels;
        m.tex_log2 = log2_size;
    }
    c->meshes_dirty = true;
    return CURAST_OK;
}

curast_status curast_resolve_textured(curast_ctx *c, const float view[16], const float proj[16], int W, int H,
                                      const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, uint8_t *level,
                                      curast_stream stream) {
    if (!c) return CURAST_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rgba_f32) & 15) || (reinterpret_cast<uintptr_t>(rgba8) & 3))
        return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ShadeArgs a;
    curast_status st = shade_setup(c, view, proj, W, H, vis, &a, s);
    if (st != CURAST_OK) return st;
    a.rgba_f32 = rgba_f32;
    a.rgba8 = rgba8;
    a.level = level;
    CU(launch_resolve_textured(a, s));
    return CURAST_OK;
}

curast_status curast_resolve_ss(curast_ctx *c, const float view[16], const float proj[16], int W, int H, int ss,
                                const uint64_t *vis, float *rgba_f32, uint8_t *rgba8, curast_stream stream) {
    if (!c || ss < 1 || ss > 8 || W < 1 || H < 1 || W > 16384 / ss || H > 16384 / ss) return CURAST_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(rgba_f32) & 15) || (reinterpret_cast<uintptr_t>(rgba8) & 3))
        return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ShadeArgs a;
    curast_status st = shade_setup(c, view, proj, ss * W, ss * H, vis, &a, s);
    if (st != CURAST_OK) return st;
    a.rgba_f32 = rgba_f32;
    a.rgba8 = rgba8;
    a.ss = ss;
    CU(launch_resolve_ss(a, W, H, s));
    return CURAST_OK;
}

curast_status curast_interpolate(curast_ctx *c, uint32_t mesh_id, const float *pos, const float view[16],
                                 const float proj[16], int W, int H, const uint64_t *vis, const float *attr, int C,
                                 float *out, curast_stream stream) {
    if (!c || mesh_id >= c->meshes.size() || !attr || !out || C < 1 || C > 16) return CURAST_ERR_INVALID_ARG;
    if (c->meshes[mesh_id].comp) return CURAST_ERR_INVALID_ARG;     // no differentiable path
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ShadeArgs a;
    curast_status st = shade_setup(c, view, proj, W, H, vis, &a, s);
    if (st != CURAST_OK) return st;
    a.mesh = mesh_id;
    a.pos = pos;
    a.attr = attr;
    a.C = C;
    a.out = out;
    CU(launch_interpolate(a, s));
    return CURAST_OK;
}

curast_status curast_interpolate_backward(curast_ctx *c, uint32_t mesh_id, const float *pos, const float view[16],
                                          const float proj[16], int W, int H, const uint64_t *vis, const float *attr,
                                          int C, const float *grad_out, float *grad_attr, float *grad_pos,
                                          curast_stream stream) {
    if (!c || mesh_id >= c->meshes.size() || !attr || !grad_out || C < 1 || C > 16) return CURAST_ERR_INVALID_ARG;
    if (c->meshes[mesh_id].comp) return CURAST_ERR_INVALID_ARG;     // no differentiable path
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ShadeArgs a;
    curast_status st = shade_setup(c, view, proj, W, H, vis, &a, s);
    if (st != CURAST_OK) return st;
    a.mesh = mesh_id;
    a.pos = pos;
    a.attr = attr;
    a.C = C;
    a.grad_out = grad_out;
    a.grad_attr = grad_attr;
    a.grad_pos = grad_pos;
    CU(launch_interpolate_backward(a, s));
    return CURAST_OK;
}

curast_status curast_sync(curast_ctx *c, curast_stream stream, curast_stats *stats) {
    if (!c) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    CU(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    Counters h;
    unsigned err = 0;
    CU(cudaMemcpyAsync(&h, c->d_ctr, sizeof(h), cudaMemcpyDeviceToHost, c->aux));
    CU(cudaMemcpyAsync(&err, c->d_err, sizeof(err), cudaMemcpyDeviceToHost, c->aux));
    CU(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->aux));
    CU(cudaStreamSynchronize(c->aux));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->triangles_in = h.stats[kStatIn];
        stats->culled_clip = h.stats[kStatClip];
        stats->culled_backface = h.stats[kStatBack];
        stats->culled_tiny = h.stats[kStatTiny];
        stats->stage1_rasterized = h.stats[kStatS1];
        stats->queued_stage2 = h.q1_count;
        stats->stage2_rasterized = h.stats[kStatS2];
        stats->queued_stage3 = h.q2_count;
        stats->queue1_overflow = h.overflow1;
        stats->queue2_overflow = h.overflow2;
        stats->exact_path = h.stats[kStatFast];
        stats->device_error = err;
    }
    if (err & kErrTimeout) return CURAST_ERR_DEVICE_TIMEOUT;
    return (err & kErrIndex) ? CURAST_ERR_INDEX_OUT_OF_RANGE : CURAST_OK;
}

curast_status curast_last_frame(const curast_ctx *c, curast_frame_info *out) {
    if (!c || !out) return CURAST_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->pairs = c->hp.size();
    out->segments = c->hs.size();
    out->work_items = c->hdr.n_batches;
    out->rounds = c->rounds.size();
    std::vector<char> seen(c->meshes.size(), 0);
    for (const PairDev &p : c->hp) {
        out->triangles += c->meshes[p.mesh].T;
        if (!seen[p.mesh]) {
            seen[p.mesh] = 1;
            out->unique_triangles += c->meshes[p.mesh].T;
            out->unique_vertices += c->meshes[p.mesh].V;
        }
    }
    return CURAST_OK;
}

curast_status curast_stage_times(curast_ctx *c, float out[5]) {
    if (!c || !out) return CURAST_ERR_INVALID_ARG;
    if (!c->ev_recorded) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    CU(cudaEventSynchronize(c->ev[5]));
    for (int k = 0; k < 5; ++k) CU(cudaEventElapsedTime(&out[k], c->ev[k], c->ev[k + 1]));
    return CURAST_OK;
}

curast_status curast_autotune(curast_ctx *c, const curast_view *views, int n_views, curast_stream stream,
                              curast_config *chosen) {
    if (!c || !views || n_views < 1) return CURAST_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const curast_config base = c->cfg;
    // reference output of the current configuration
    uint64_t total = 0;
    for (int v = 0; v < n_views; ++v) total += (uint64_t)views[v].W * (uint64_t)views[v].H;
    uint64_t *ref = nullptr;
    CU(cudaMalloc(reinterpret_cast<void **>(&ref), total * sizeof(uint64_t)));
    curast_status st = render_views(c, views, n_views, -1, true, false, s);
    uint64_t off = 0;
    for (int v = 0; v < n_views && st == CURAST_OK; ++v) {
        const uint64_t n = (uint64_t)views[v].W * (uint64_t)views[v].H;
        st = cuda_status(cudaMemcpyAsync(ref + off, views[v].vis, n * 8, cudaMemcpyDeviceToDevice, s));
        off += n;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == CURAST_OK) st = cuda_status(cudaEventCreate(&e0));
    if (st == CURAST_OK) st = cuda_status(cudaEventCreate(&e1));
    auto measure = [&](const curast_config &cand, float *ms, bool *exact) -> curast_status {
        curast_status r = curast_set_config(c, &cand);
        if (r != CURAST_OK) return r;
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            CU(cudaEventRecord(e0, s));
            r = render_views(c, views, n_views, -1, true, false, s);
            if (r != CURAST_OK) return r;
            CU(cudaEventRecord(e1, s));
            CU(cudaEventSynchronize(e1));
            float t = 0.0f;
            CU(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t);
        }
        CU(cudaMemsetAsync(c->d_diff, 0, sizeof(unsigned long long), s));
        uint64_t o = 0;
        for (int v = 0; v < n_views; ++v) {
            const uint64_t n = (uint64_t)views[v].W * (uint64_t)views[v].H;
            CU(launch_count_diff(views[v].vis, ref + o, n, c->d_diff, s));
            o += n;
        }
        unsigned long long diff = 0;
        CU(cudaMemcpyAsync(&diff, c->d_diff, sizeof(diff), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        *ms = best;
        *exact = diff == 0;
        return CURAST_OK;
    };
    curast_config best = base;
    float best_ms = 1e30f;
    bool exact = true;
    if (st == CURAST_OK) st = measure(base, &best_ms, &exact);
    // coordinate descent over the batch shape, the two stage thresholds, the
    // tile size, the pairs a work item loops over and the group test's
    // threshold (none of them changes the buffer; a candidate that did would
    // be rejected below)
    const uint32_t tpts[] = {1, 2, 4};
    const uint32_t s1s[] = {32, 64, 128, 256};
    const uint32_t s2s[] = {1024, 4096, 16384};
    const uint32_t tiles[] = {5, 6, 7};
    const uint32_t ppss[] = {16, 32, 64};
    const uint32_t groups[] = {0, 2, 8};
    for (int dim = 0; dim < 6 && st == CURAST_OK; ++dim) {
        const int n = dim == 1 ? 4 : 3;
        for (int k = 0; k < n && st == CURAST_OK; ++k) {
            curast_config cand = best;
            if (dim == 0) cand.stage1_tri_per_thread = tpts[k];
            if (dim == 1) cand.stage1_max_pixels = s1s[k];
            if (dim == 2) cand.stage2_max_pixels = s2s[k];
            if (dim == 3) cand.tile_log2 = tiles[k];
            if (dim == 4) cand.pairs_per_segment = ppss[k];
            if (dim == 5) cand.stage1_group_min_pairs = groups[k];
            if (std::memcmp(&cand, &best, sizeof(cand)) == 0) continue;
            float ms = 0.0f;
            bool ok = false;
            st = measure(cand, &ms, &ok);
            if (st == CURAST_OK && ok && ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(ref);
    curast_status st2 = curast_set_config(c, st == CURAST_OK ? &best : &base);
    if (st == CURAST_OK) st = st2;
    if (st == CURAST_OK && chosen) *chosen = best;
    return st;
}

}  // extern "C"
