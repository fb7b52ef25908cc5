// raster.cu -- clear, stage 1, stage 2 and stage 3 kernels (Sections 4.1-4.3).
#include "internal.h"

namespace curast {

// ------------------------------------------------------------------ clear --
// Section 4.1: the framebuffer starts each frame at the empty word (all
// ones, larger than any fragment).  16-byte stores, grid-stride.
__global__ void __launch_bounds__(256) k_clear(uint64_t *vis, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool aligned = (reinterpret_cast<uintptr_t>(vis) & 15) == 0;
    if (aligned) {
        ulonglong2 *v2 = reinterpret_cast<ulonglong2 *>(vis);
        const uint64_t n2 = n / 2;
        for (uint64_t k = i; k < n2; k += stride) v2[k] = make_ulonglong2(kEmpty, kEmpty);
        if (i == 0 && (n & 1)) vis[n - 1] = kEmpty;
    } else {
        for (uint64_t k = i; k < n; k += stride) vis[k] = kEmpty;
    }
}

// ----------------------------------------------------- whole-triangle path --
// Clips, snaps and fan-rasterizes one triangle with the pixel loop split as
// (start, stride) -- used by a single thread when queue 1 is full.
__device__ __noinline__ void raster_triangle_general(const CV c[3], const ViewDev &vw, uint64_t id, int start,
                                                     int stride) {
    CV poly[kMaxPoly];
    const int n = clip_polygon(c, vw.nearv, poly);
    if (n < 3) return;
    int X[kMaxPoly], Y[kMaxPoly];
    float iz[kMaxPoly];
    for (int k = 0; k < n; ++k) snap(poly[k], vw.hw, vw.hh, X[k], Y[k], iz[k]);
    for (int j = 1; j + 1 < n; ++j) {
        SubTri s;
        s.X[0] = X[0]; s.X[1] = X[j]; s.X[2] = X[j + 1];
        s.Y[0] = Y[0]; s.Y[1] = Y[j]; s.Y[2] = Y[j + 1];
        s.iz[0] = iz[0]; s.iz[1] = iz[j]; s.iz[2] = iz[j + 1];
        s.id = id;
        if (!setup_subtri(s, vw.W, vw.H)) continue;
        raster_range(s, s.x0, s.x1, s.y0, s.y1, start, stride, vw.vis, vw.W);
    }
}

// The triangle of global id `id` under pair `pidx` in view space, set up for
// the ray cast of stage 3; false when an index is out of range.
__device__ __forceinline__ bool ray_tri_of(const FrameDev &f, uint32_t pidx, uint64_t id, RayTri &R) {
    const PairDev &pr = f.pairs[pidx];
    const MeshDev &mesh = f.meshes[pr.mesh];
    const uint64_t t = id - pr.base;
    float3 v[3];
    for (int k = 0; k < 3; ++k) {
        const uint32_t vi = mesh_index(mesh, 3 * t + k);
        if (vi >= mesh.V) return false;
        float p[3];
        mesh_vertex(mesh, vi, p[0], p[1], p[2]);
        v[k] = view_space(pr.mv, p);
    }
    R = ray_setup(v[0], v[1], v[2]);
    return true;
}

// Snapped bbox of a clipped polygon as a pixel-centre range on the screen;
// returns the number of pixel centres (0 when there are none).
__device__ __forceinline__ int64_t poly_range(const int *X, const int *Y, int n, int W, int H, int &x0, int &x1,
                                              int &y0, int &y1) {
    int mnx = X[0], mxx = X[0], mny = Y[0], mxy = Y[0];
    for (int k = 1; k < n; ++k) {
        mnx = min(mnx, X[k]); mxx = max(mxx, X[k]);
        mny = min(mny, Y[k]); mxy = max(mxy, Y[k]);
    }
    centre_range(mnx, mxx, W, x0, x1);
    centre_range(mny, mxy, H, y0, y1);
    if (x0 > x1 || y0 > y1) return 0;
    return (int64_t)(x1 - x0 + 1) * (int64_t)(y1 - y0 + 1);
}

__device__ __forceinline__ void stat_add(const FrameDev &f, int k, unsigned long long v) {
    if (f.stats && v) atomicAdd(&f.ctr->stats[k], v);
}

// clip-space vertices of triangle t of a mesh under pair p (from global memory)
__device__ __forceinline__ void load_clip(const FrameDev &f, const MeshDev &mesh, uint32_t pidx, uint64_t t,
                                          const ViewDev &vw, CV c[3]) {
    const float *mv = f.pairs[pidx].mv;
    for (int k = 0; k < 3; ++k) {
        float x, y, z;
        mesh_vertex(mesh, mesh_index(mesh, 3 * t + k), x, y, z);
        c[k] = to_clip(mv, x, y, z, vw.fx, vw.fy);
    }
}

// queue 1 is full: the thread clips and rasterizes its triangle itself.
// (Out-of-line helpers take the frame and the mesh by pointer into parameter
// or global memory: a struct passed by value, or a reference to a local,
// would be copied to local memory on every call.)
__device__ __noinline__ void q1_overflow(const FrameDev *fp, uint64_t id, uint32_t pidx, const MeshDev *mesh,
                                         uint64_t t) {
    const FrameDev &f = *fp;
    atomicAdd(&f.ctr->overflow1, 1ull);
    const ViewDev &vw = f.views[f.pairs[pidx].view];
    CV c[3];
    load_clip(f, *mesh, pidx, t, vw, c);
    raster_triangle_general(c, vw, id, 0, 1);
}

// The same in the ray-cast mode, with its stage-2 decision: a visible bbox
// over s2_max pixel centres takes the ray cast, here by this thread alone.
// (A function of its own: the fixed-point kernels never reach it, and its
// frame does not weigh on their register allocation.)
__device__ __noinline__ void q1_overflow_ray(const FrameDev *fp, uint64_t id, uint32_t pidx, const MeshDev *mesh,
                                             uint64_t t) {
    const FrameDev &f = *fp;
    atomicAdd(&f.ctr->overflow1, 1ull);
    const ViewDev &vw = f.views[f.pairs[pidx].view];
    CV c[3];
    load_clip(f, *mesh, pidx, t, vw, c);
    {
        CV poly[kMaxPoly];
        const int n = clip_polygon(c, vw.nearv, poly);
        if (n < 3) return;
        int X[kMaxPoly], Y[kMaxPoly];
        float iz[kMaxPoly];
        for (int k = 0; k < n; ++k) snap(poly[k], vw.hw, vw.hh, X[k], Y[k], iz[k]);
        int x0, x1, y0, y1;
        if (poly_range(X, Y, n, vw.W, vw.H, x0, x1, y0, y1) > (int64_t)f.s2_max) {
            RayTri R;
            if (ray_tri_of(f, pidx, id, R)) ray_range(R, x0, x1, y0, y1, 0, 1, vw, id);
            return;
        }
    }
    raster_triangle_general(c, vw, id, 0, 1);
}

// Warp-aggregated append to queue 1 (ballot + popc + one atomicAdd per warp).
// Lanes whose slot lies beyond the capacity rasterize their triangle in place.
// f must live in parameter or global memory (its address is passed on).
template <bool RAY>
__device__ __forceinline__ void q1_append(const FrameDev &f, bool want, uint64_t id, uint32_t pidx,
                                          const MeshDev *mesh, uint64_t t) {
    const unsigned active = __activemask();
    const unsigned m = __ballot_sync(active, want);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&f.ctr->q1_count, (unsigned long long)__popc(m));
    base = __shfl_sync(active, base, leader);
    if (!want) return;
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    if (slot < f.q1_cap) {
        Q1Entry e;
        e.id = id;
        e.pair = pidx;
        e.pad = 0;
        f.q1[slot] = e;
    } else {
        if (RAY) q1_overflow_ray(&f, id, pidx, mesh, t);
        else q1_overflow(&f, id, pidx, mesh, t);
    }
}

// ---------------------------------------------------------------- stage 1 --
// Small-triangle rasterizer of Section 4.1: one thread per triangle, y outer
// / x inner over the bounding box with incrementally updated edge functions.
// int32 is exact here because both bbox extents are below 2^14 subpixels,
// so |E| < 2^30 at every visited sample.
__device__ __forceinline__ void raster_small(const int X[3], const int Y[3], const float iz[3], int64_t A, int x0,
                                             int x1, int y0, int y1, uint64_t id, uint64_t *vis, int W) {
    const int px0 = 256 * x0 + 128, py0 = 256 * y0 + 128;
    // edge k runs from vertex k+1 to vertex k+2
    const int ax0 = X[1], ay0 = Y[1], dx0 = X[2] - X[1], dy0 = Y[2] - Y[1];
    const int ax1 = X[2], ay1 = Y[2], dx1 = X[0] - X[2], dy1 = Y[0] - Y[2];
    const int ax2 = X[0], ay2 = Y[0], dx2 = X[1] - X[0], dy2 = Y[1] - Y[0];
    int e0 = dx0 * (py0 - ay0) - dy0 * (px0 - ax0);
    int e1 = dx1 * (py0 - ay1) - dy1 * (px0 - ax1);
    int e2 = dx2 * (py0 - ay2) - dy2 * (px0 - ax2);
    const int b0 = (dy0 < 0 || (dy0 == 0 && dx0 < 0)) ? 0 : 1;
    const int b1 = (dy1 < 0 || (dy1 == 0 && dx1 < 0)) ? 0 : 1;
    const int b2 = (dy2 < 0 || (dy2 == 0 && dx2 < 0)) ? 0 : 1;
    const float fA = __ll2float_rn(A);
    for (int y = y0; y <= y1; ++y) {
        int r0 = e0, r1 = e1, r2 = e2;
        uint64_t *row = vis + (size_t)y * (size_t)W;
        for (int x = x0; x <= x1; ++x) {
            if (((r0 - b0) | (r1 - b1) | (r2 - b2)) >= 0) {
                float s = __fadd_rn(__fadd_rn(__fmul_rn(__int2float_rn(r0), iz[0]), __fmul_rn(__int2float_rn(r1), iz[1])),
                                    __fmul_rn(__int2float_rn(r2), iz[2]));
                float depth = __fdiv_rn(fA, s);
                uint64_t key = ((uint64_t)(__float_as_uint(depth) >> 3) << 36) | (id & kIdMask);
                depth_min(row, (size_t)x, key);
            }
            r0 -= dy0 * 256; r1 -= dy1 * 256; r2 -= dy2 * 256;
        }
        e0 += dx0 * 256; e1 += dx1 * 256; e2 += dx2 * 256;
    }
}

// Per-vertex record of one (instance, view): the snapped screen position and
// 1/depth, or X = INT_MIN with Y = the clip outcode when the vertex lies
// outside the near plane or the guard band.
struct Rec { int X, Y; float iz; };
constexpr int kOutside = (int)0x80000000;

__device__ __forceinline__ Rec make_rec(CV c, const ViewDev &vw) {
    Rec r;
    // Inside every plane, decided without the five plane values: w >= near,
    // |x| <= 128 w and |y| <= 128 w give the same answers as the signs of
    // w - near, x + 128 w, ... (a sum of two finite floats rounds to zero only
    // when it is zero; no flush to zero here), NaN fails both forms, and an
    // infinite 128 w takes the full outcode (inf - inf is NaN there).
    const float gw = __fmul_rn(kGuard, c.w);
    const bool inside = (c.w >= vw.nearv) & (gw < INFINITY) & (fabsf(c.x) <= gw) & (fabsf(c.y) <= gw);
    const unsigned oc = inside ? 0u : outcode(c, vw.nearv);
    if (oc) {
        r.X = kOutside;
        r.Y = (int)oc;
        r.iz = 0.0f;
    } else {
        snap(c, vw.hw, vw.hh, r.X, r.Y, r.iz);
    }
    return r;
}

enum Class { kDrop = 0, kQueue = 1, kSmall = 2 };

// Cull tests of one triangle of one (instance, view) from its vertex records:
// beyond one clip plane -> drop; crossing the near plane or the guard band
// -> stage 2 (clipping); back-facing or degenerate -> drop; bbox without a
// pixel centre on screen (frustum and tiny-triangle cull) -> drop; bbox over
// the stage-1 limit -> stage 2; else rasterize here.
__device__ __forceinline__ int classify(const FrameDev &f, const Rec r[3], const ViewDev &vw, int &x0, int &x1,
                                        int &y0, int &y1, int64_t &A, unsigned &stat) {
    if (r[0].X == kOutside || r[1].X == kOutside || r[2].X == kOutside) {
        const unsigned o0 = r[0].X == kOutside ? (unsigned)r[0].Y : 0u;
        const unsigned o1 = r[1].X == kOutside ? (unsigned)r[1].Y : 0u;
        const unsigned o2 = r[2].X == kOutside ? (unsigned)r[2].Y : 0u;
        if (o0 & o1 & o2) { stat = kStatClip; return kDrop; }
        return kQueue;
    }
    A = (int64_t)(r[1].X - r[0].X) * (int64_t)(r[2].Y - r[0].Y) - (int64_t)(r[2].X - r[0].X) * (int64_t)(r[1].Y - r[0].Y);
    if (A <= 0) { stat = kStatBack; return kDrop; }
    const int minX = min(r[0].X, min(r[1].X, r[2].X)), maxX = max(r[0].X, max(r[1].X, r[2].X));
    const int minY = min(r[0].Y, min(r[1].Y, r[2].Y)), maxY = max(r[0].Y, max(r[1].Y, r[2].Y));
    // pixel centres 256 x + 128 inside [min, max] (arithmetic shifts are
    // floor divisions), clamped to the screen
    x0 = max(-((128 - minX) >> 8), 0);
    x1 = min((maxX - 128) >> 8, vw.W - 1);
    y0 = max(-((128 - minY) >> 8), 0);
    y1 = min((maxY - 128) >> 8, vw.H - 1);
    if (x0 > x1 || y0 > y1) { stat = kStatTiny; return kDrop; }
    if (maxX - minX >= (1 << 14) || maxY - minY >= (1 << 14)) return kQueue;
    if ((uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1)) > f.s1_max) return kQueue;
    return kSmall;
}

#include "stage1.cuh"
#include "stage1_win.cuh"

// ---------------------------------------------------------------- stage 2 --
// Section 4.2: one warp per queued triangle.  The triangle is clipped
// (Sutherland-Hodgman, near plane and guard band) and fan-triangulated;
// sub-triangles with a bbox of at most s2_max pixels are rasterized by the
// warp with the 1D pixel loop, larger ones are split along tile boundaries
// into stage-3 parts.
__device__ __forceinline__ void q2_append(const FrameDev &f, bool want, const SubTri &s, uint32_t view, int tx,
                                          int ty, const ViewDev &vw) {
    const unsigned active = __activemask();
    const unsigned m = __ballot_sync(active, want);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&f.ctr->q2_count, (unsigned long long)__popc(m));
    base = __shfl_sync(active, base, leader);
    if (!want) return;
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    if (slot < f.q2_cap) {
        Q2Entry e;
        for (int k = 0; k < 3; ++k) { e.X[k] = s.X[k]; e.Y[k] = s.Y[k]; e.iz[k] = s.iz[k]; }
        e.view = view;
        e.id = s.id;
        e.tx = (uint32_t)tx;
        e.ty = (uint32_t)ty;
        e.pair = 0;
        e.ray = 0;
        f.q2[slot] = e;
        if (f.s3_bin) atomicAdd(&f.tile_cnt[vw.tile0 + (uint32_t)ty * vw.ntx + (uint32_t)tx], 1u);
    } else {
        atomicAdd(&f.ctr->overflow2, 1ull);
        const int ts = 1 << f.tile_log2;
        raster_range(s, max(s.x0, tx * ts), min(s.x1, tx * ts + ts - 1), max(s.y0, ty * ts),
                     min(s.y1, ty * ts + ts - 1), 0, 1, vw.vis, vw.W);
    }
}

// The same for one tile of a triangle that takes the ray-cast stage 3: the
// entry names the triangle (id, pair) and its visible pixel range.
__device__ __forceinline__ void q2_append_ray(const FrameDev &f, bool want, uint64_t id, uint32_t pidx, uint32_t view,
                                              int x0, int x1, int y0, int y1, int tx, int ty, const ViewDev &vw) {
    const unsigned active = __activemask();
    const unsigned m = __ballot_sync(active, want);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&f.ctr->q2_count, (unsigned long long)__popc(m));
    base = __shfl_sync(active, base, leader);
    if (!want) return;
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    if (slot < f.q2_cap) {
        Q2Entry e;
        e.X[0] = x0; e.X[1] = x1; e.X[2] = 0;
        e.Y[0] = y0; e.Y[1] = y1; e.Y[2] = 0;
        e.iz[0] = e.iz[1] = e.iz[2] = 0.0f;
        e.view = view;
        e.id = id;
        e.tx = (uint32_t)tx;
        e.ty = (uint32_t)ty;
        e.pair = pidx;
        e.ray = 1;
        f.q2[slot] = e;
        if (f.s3_bin) atomicAdd(&f.tile_cnt[vw.tile0 + (uint32_t)ty * vw.ntx + (uint32_t)tx], 1u);
    } else {
        atomicAdd(&f.ctr->overflow2, 1ull);
        const int ts = 1 << f.tile_log2;
        RayTri R;
        if (ray_tri_of(f, pidx, id, R))
            ray_range(R, max(x0, tx * ts), min(x1, tx * ts + ts - 1), max(y0, ty * ts), min(y1, ty * ts + ts - 1), 0,
                      1, vw, id);
    }
}

__global__ void __launch_bounds__(256) k_stage2(FrameDev f) {
    const int lane = threadIdx.x & 31;
    const unsigned long long total = *((volatile unsigned long long *)&f.ctr->q1_count);
    const unsigned long long n = total < f.q1_cap ? total : f.q1_cap;
    unsigned long long n_s2 = 0, n_parts = 0;
    for (;;) {
        unsigned long long i = 0;
        if (lane == 0) i = atomicAdd(&f.ctr->q1_next, 1ull);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= n) break;
        const Q1Entry e = f.q1[i];
        const PairDev &pr = f.pairs[e.pair];
        const ViewDev vw = f.views[pr.view];
        const MeshDev mesh = f.meshes[pr.mesh];
        CV c[3];
        load_clip(f, mesh, e.pair, e.id - pr.base, vw, c);
        CV poly[kMaxPoly];
        int np;
        if ((outcode(c[0], vw.nearv) | outcode(c[1], vw.nearv) | outcode(c[2], vw.nearv)) == 0) {
            // inside every plane: Sutherland-Hodgman would return it unchanged
            poly[0] = c[0]; poly[1] = c[1]; poly[2] = c[2];
            np = 3;
        } else {
            np = clip_polygon(c, vw.nearv, poly);
        }
        if (np < 3) continue;
        int X[kMaxPoly], Y[kMaxPoly];
        float iz[kMaxPoly];
        for (int k = 0; k < np; ++k) snap(poly[k], vw.hw, vw.hh, X[k], Y[k], iz[k]);
        if (f.s3_ray) {
            // the paper's stage 3: a triangle whose visible bbox holds more
            // than s2_max pixel centres is ray cast over that range, in tiles
            int x0, x1, y0, y1;
            const int64_t cnt = poly_range(X, Y, np, vw.W, vw.H, x0, x1, y0, y1);
            if (cnt == 0) continue;
            if (cnt > (int64_t)f.s2_max) {
                const int tl = (int)f.tile_log2;
                const int tx0 = x0 >> tl, tx1 = x1 >> tl, ty0 = y0 >> tl, ty1 = y1 >> tl;
                const int ntx = tx1 - tx0 + 1;
                const int nt = ntx * (ty1 - ty0 + 1);
                for (int kb = 0; kb < nt; kb += 32) {
                    const int k = kb + lane;
                    const bool want = k < nt;
                    const int tx = tx0 + (want ? k % ntx : 0), ty = ty0 + (want ? k / ntx : 0);
                    q2_append_ray(f, want, e.id, e.pair, pr.view, x0, x1, y0, y1, tx, ty, vw);
                    n_parts += want;
                }
                continue;
            }
        }
        for (int j = 1; j + 1 < np; ++j) {
            SubTri s;
            s.X[0] = X[0]; s.X[1] = X[j]; s.X[2] = X[j + 1];
            s.Y[0] = Y[0]; s.Y[1] = Y[j]; s.Y[2] = Y[j + 1];
            s.iz[0] = iz[0]; s.iz[1] = iz[j]; s.iz[2] = iz[j + 1];
            s.id = e.id;
            if (!setup_subtri(s, vw.W, vw.H)) continue;
            const int64_t cnt = (int64_t)(s.x1 - s.x0 + 1) * (int64_t)(s.y1 - s.y0 + 1);
            if (cnt <= (int64_t)f.s2_max) {
                raster_range<4>(s, s.x0, s.x1, s.y0, s.y1, lane, 32, vw.vis, vw.W);
                n_s2 += (lane == 0);
            } else {
                const int tl = (int)f.tile_log2;
                const int tx0 = s.x0 >> tl, tx1 = s.x1 >> tl, ty0 = s.y0 >> tl, ty1 = s.y1 >> tl;
                const int ntx = tx1 - tx0 + 1;
                const int nt = ntx * (ty1 - ty0 + 1);
                for (int kb = 0; kb < nt; kb += 32) {
                    const int k = kb + lane;
                    const bool want = k < nt;
                    const int tx = tx0 + (want ? k % ntx : 0), ty = ty0 + (want ? k / ntx : 0);
                    q2_append(f, want, s, pr.view, tx, ty, vw);
                    n_parts += want;
                }
            }
        }
    }
    if (f.stats) {
        stat_add(f, kStatS2, n_s2);
        stat_add(f, kStatParts, n_parts);
    }
}

// ---------------------------------------------------------------- stage 3 --
// Section 4.3: one block per tile part; its threads walk the tile's pixels
// (restricted to the sub-triangle's bbox) line by line -- with edge
// functions, or, in the ray-cast mode, with the paper's view-space pixel
// rays against the whole (unclipped) triangle.
__global__ void __launch_bounds__(256) k_stage3(FrameDev f) {
    __shared__ unsigned long long s_i;
    const unsigned long long total = *((volatile unsigned long long *)&f.ctr->q2_count);
    const unsigned long long n = total < f.q2_cap ? total : f.q2_cap;
    const int ts = 1 << f.tile_log2;
    for (;;) {
        if (threadIdx.x == 0) s_i = atomicAdd(&f.ctr->q2_next, 1ull);
        __syncthreads();
        const unsigned long long i = s_i;
        __syncthreads();
        if (i >= n) break;
        const Q2Entry e = f.q2[i];
        const ViewDev vw = f.views[e.view];
        if (e.ray) {
            RayTri R;
            if (!ray_tri_of(f, e.pair, e.id, R)) continue;
            const int x0 = max(e.X[0], (int)e.tx * ts), x1 = min(e.X[1], (int)e.tx * ts + ts - 1);
            const int y0 = max(e.Y[0], (int)e.ty * ts), y1 = min(e.Y[1], (int)e.ty * ts + ts - 1);
            if (x0 > x1 || y0 > y1) continue;
            ray_range(R, x0, x1, y0, y1, threadIdx.x, blockDim.x, vw, e.id);
            continue;
        }
        SubTri s;
        for (int k = 0; k < 3; ++k) { s.X[k] = e.X[k]; s.Y[k] = e.Y[k]; s.iz[k] = e.iz[k]; }
        s.id = e.id;
        if (!setup_subtri(s, vw.W, vw.H)) continue;
        const int x0 = max(s.x0, (int)e.tx * ts), x1 = min(s.x1, (int)e.tx * ts + ts - 1);
        const int y0 = max(s.y0, (int)e.ty * ts), y1 = min(s.y1, (int)e.ty * ts + ts - 1);
        if (x0 > x1 || y0 > y1) continue;
        raster_range(s, x0, x1, y0, y1, threadIdx.x, blockDim.x, vw.vis, vw.W);
    }
}

// ------------------------------------------------------- binned stage 3 --
// Section 4.3 with the tile framebuffer in shared memory: the parts stage 2
// queued are sorted by tile (stage 2 counts them per tile; one block scans
// the counts; a scatter pass writes the part indices in tile order) and cut
// into units of at most kUnitParts parts of one tile.  A block takes one
// unit at a time: it keeps the tile's words in shared memory, applies all of
// the unit's parts there, and then writes each pixel they covered to the
// visibility buffer with one global atomic minimum.  The minimum is
// order-independent, so the buffer is the same as with k_stage3.
constexpr int kUnitParts = 8;

// Shared memory of k_stage3_tiles: one 64-bit word per pixel of a tile.
size_t stage3_tile_smem(uint32_t tile_log2) { return (size_t)8 << (2 * tile_log2); }

// One block of kScanThreads: tile_start = exclusive prefix sum of tile_cnt
// (tile_start[n_tiles] = the total), tile_fill = tile_start, and the units
// (tile, first part) of every tile, ceil(count / kUnitParts) each (their
// number in ctr->s3_tiles).
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_bin_scan(FrameDev f) {
    __shared__ uint32_t wsum[kScanThreads / 32], wnu[kScanThreads / 32];
    const uint32_t n = f.n_tiles;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t chunk = (n + kScanThreads - 1) / kScanThreads;
    const uint32_t b = min(n, (uint32_t)t * chunk), e = min(n, b + chunk);
    uint32_t sum = 0, nu = 0;
    for (uint32_t g = b; g < e; ++g) {
        const uint32_t c = f.tile_cnt[g];
        sum += c;
        nu += (c + kUnitParts - 1) / kUnitParts;
    }
    // block-wide exclusive scans of sum and nu
    uint32_t is = sum, iu = nu;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, is, o), c = __shfl_up_sync(0xffffffffu, iu, o);
        if (lane >= o) is += a, iu += c;
    }
    if (lane == 31) wsum[warp] = is, wnu[warp] = iu;
    __syncthreads();
    if (warp == 0) {
        uint32_t a = wsum[lane], c = wnu[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, a, o), y = __shfl_up_sync(0xffffffffu, c, o);
            if (lane >= o) a += x, c += y;
        }
        wsum[lane] = a;
        wnu[lane] = c;
    }
    __syncthreads();
    uint32_t run = is - sum + (warp ? wsum[warp - 1] : 0u);
    uint32_t at = iu - nu + (warp ? wnu[warp - 1] : 0u);
    for (uint32_t g = b; g < e; ++g) {
        const uint32_t c = f.tile_cnt[g];
        f.tile_start[g] = run;
        f.tile_fill[g] = run;
        for (uint32_t q = 0; q < c; q += kUnitParts) f.units[at++] = make_uint2(g, run + q);
        run += c;
    }
    if (t == kScanThreads - 1) {
        f.tile_start[n] = run;
        f.ctr->s3_tiles = at;
    }
}

// Queue-2 part indices into tile order.
__global__ void __launch_bounds__(256) k_bin_scatter(FrameDev f) {
    const unsigned long long total = *((volatile unsigned long long *)&f.ctr->q2_count);
    const unsigned long long n = total < f.q2_cap ? total : f.q2_cap;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const Q2Entry &e = f.q2[i];
        const ViewDev &vw = f.views[e.view];
        const uint32_t g = vw.tile0 + e.ty * vw.ntx + e.tx;
        f.part_sorted[atomicAdd(&f.tile_fill[g], 1u)] = (uint32_t)i;
    }
}

// One part of a unit, set up once for all of the unit's threads.
struct PartRec {
    SubTri s;                // fixed-point rule; s.x0..s.y1: the pixel range clamped to the tile
    RayTri R;                // ray-cast parts
    int ray;
};

// Thread t of the block owns the pixels (t mod ts, t / ts + k 256 / ts),
// k = 0 .. ts^2 / 256 - 1, of the tile (tile-local coordinates; ts >= 16),
// and only it touches their words, so the minimum there needs no atomic.
// For every part of the unit the thread walks its own pixels inside the
// part's range -- one column, every (256 / ts)-th row -- with the edge
// functions stepped from row to row; then it writes each of its covered
// pixels once to the visibility buffer and resets the word.
__global__ void __launch_bounds__(256) k_stage3_tiles(FrameDev f) {
    extern __shared__ __align__(16) unsigned long long tw[];     // the tile's words
    __shared__ PartRec pr[kUnitParts];
    __shared__ unsigned long long s_i;
    const int tl = (int)f.tile_log2, ts = 1 << tl;
    const unsigned long long nunit = *((volatile unsigned long long *)&f.ctr->s3_tiles);
    const int n_views = (int)f.hdr->n_views;
    const int tid = threadIdx.x;
    const int lx = tid & (ts - 1), ly0 = tid >> tl, dyr = 256 >> tl;   // my column, first row, row step
    for (int i = tid; i < ts * ts; i += 256) tw[i] = kEmpty;     // (each thread's own pixels)
    for (;;) {
        if (tid == 0) s_i = atomicAdd(&f.ctr->s3_next, 1ull);
        __syncthreads();
        const unsigned long long k = s_i;
        if (k >= nunit) break;
        const uint2 u = f.units[k];
        const uint32_t g = u.x, p0 = u.y, p1 = min(p0 + (uint32_t)kUnitParts, f.tile_start[g + 1]);
        const int np = (int)(p1 - p0);
        int v = 0;
        while (v + 1 < n_views && f.views[v + 1].tile0 <= g) ++v;
        const ViewDev &vw = f.views[v];
        const uint32_t lt = g - vw.tile0;
        const int ty = (int)(lt / vw.ntx), tx = (int)(lt - (uint32_t)ty * vw.ntx);
        const int bx = tx * ts, by = ty * ts;
        if (tid < np) {
            const Q2Entry e = f.q2[f.part_sorted[p0 + tid]];
            PartRec &P = pr[tid];
            int x0 = 1, x1 = 0, y0 = 1, y1 = 0;
            P.ray = (int)e.ray;
            SubTri s;
            if (e.ray) {
                if (ray_tri_of(f, e.pair, e.id, P.R)) {
                    x0 = max(e.X[0], bx); x1 = min(e.X[1], bx + ts - 1);
                    y0 = max(e.Y[0], by); y1 = min(e.Y[1], by + ts - 1);
                }
            } else {
                for (int c = 0; c < 3; ++c) { s.X[c] = e.X[c]; s.Y[c] = e.Y[c]; s.iz[c] = e.iz[c]; }
                s.id = e.id;
                if (setup_subtri(s, vw.W, vw.H)) {
                    x0 = max(s.x0, bx); x1 = min(s.x1, bx + ts - 1);
                    y0 = max(s.y0, by); y1 = min(s.y1, by + ts - 1);
                }
            }
            s.id = e.id;
            s.x0 = x0 - bx; s.x1 = x1 - bx; s.y0 = y0 - by; s.y1 = y1 - by;   // tile-local, empty if x0 > x1
            P.s = s;
        }
        __syncthreads();
        int ux0 = ts, ux1 = -1, uy0 = ts, uy1 = -1;                     // union of the ranges
        for (int j = 0; j < np; ++j) {
            const int rx0 = pr[j].s.x0, rx1 = pr[j].s.x1, ry0 = pr[j].s.y0, ry1 = pr[j].s.y1;
            if (rx0 > rx1 || ry0 > ry1) continue;
            ux0 = min(ux0, rx0); ux1 = max(ux1, rx1); uy0 = min(uy0, ry0); uy1 = max(uy1, ry1);
            if (lx < rx0 || lx > rx1) continue;                          // not my column
            // my first row in range: ly0 + k dyr >= ry0
            int y = ly0 + (ry0 > ly0 ? ((ry0 - ly0 + dyr - 1) / dyr) * dyr : 0);
            if (y > ry1) continue;
            const int x = bx + lx;
            if (pr[j].ray) {
                const RayTri R = pr[j].R;
                const uint64_t id = pr[j].s.id;
                for (; y <= ry1; y += dyr) {
                    uint64_t key;
                    if (ray_key(R, x, by + y, vw, id, key) && key < tw[(y << tl) + lx]) tw[(y << tl) + lx] = key;
                }
            } else {
                const SubTri s = pr[j].s;
                const int64_t px = 256 * (int64_t)x + 128, py = 256 * (int64_t)(by + y) + 128;
                // edge k from vertex k+1 to vertex k+2, stepped by dyr rows
                const int64_t dx0 = (int64_t)(s.X[2] - s.X[1]), dy0 = (int64_t)(s.Y[2] - s.Y[1]);
                const int64_t dx1 = (int64_t)(s.X[0] - s.X[2]), dy1 = (int64_t)(s.Y[0] - s.Y[2]);
                const int64_t dx2 = (int64_t)(s.X[1] - s.X[0]), dy2 = (int64_t)(s.Y[1] - s.Y[0]);
                int64_t E0 = dx0 * (py - s.Y[1]) - dy0 * (px - s.X[1]);
                int64_t E1 = dx1 * (py - s.Y[2]) - dy1 * (px - s.X[2]);
                int64_t E2 = dx2 * (py - s.Y[0]) - dy2 * (px - s.X[0]);
                const int64_t st = 256 * (int64_t)dyr;
                const int64_t b0 = s.bias & 1u, b1 = (s.bias >> 1) & 1u, b2 = (s.bias >> 2) & 1u;
                for (; y <= ry1; y += dyr) {
                    if (((E0 - b0) | (E1 - b1) | (E2 - b2)) >= 0) {
                        const uint64_t key = frag_key(E0, E1, E2, s.A, s.iz, s.id);
                        if (key < tw[(y << tl) + lx]) tw[(y << tl) + lx] = key;
                    }
                    E0 += dx0 * st; E1 += dx1 * st; E2 += dx2 * st;
                }
            }
        }
        // one global atomic minimum per covered pixel of mine, resetting the
        // word (each thread reads and resets only its own pixels; the barrier
        // at the top of the loop orders pr[] and s_i)
        if (ux0 <= ux1 && lx >= ux0 && lx <= ux1) {
            int y = ly0 + (uy0 > ly0 ? ((uy0 - ly0 + dyr - 1) / dyr) * dyr : 0);
            for (; y <= uy1; y += dyr) {
                const uint64_t key = tw[(y << tl) + lx];
                if (key != kEmpty) {
                    depth_test_write(vw.vis, (size_t)(by + y) * (size_t)vw.W + (size_t)(bx + lx), key);
                    tw[(y << tl) + lx] = kEmpty;
                }
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------- compare --
__global__ void k_count_diff(const uint64_t *a, const uint64_t *b, uint64_t n, unsigned long long *out) {
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        c += a[i] != b[i];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------------ mesh bounds --
// Axis-aligned bounds of a mesh's positions (for per-instance frustum
// culling on the host): per-block partial min/max, then one block folds them.
constexpr int kAabbBlocks = 256;

__global__ void __launch_bounds__(256) k_aabb_partial(const float *pos, uint64_t V, float *part) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < 3; ++k) {
            const float v = pos[3 * i + k];
            lo[k] = fminf(lo[k], v);
            hi[k] = fmaxf(hi[k], v);
        }
    __shared__ float s[6][256];
    for (int k = 0; k < 3; ++k) { s[k][threadIdx.x] = lo[k]; s[3 + k][threadIdx.x] = hi[k]; }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fminf(s[k][threadIdx.x], s[k][threadIdx.x + w]);
                s[3 + k][threadIdx.x] = fmaxf(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_aabb_final(const float *part, int n, float *out) {
    if (threadIdx.x >= 6) return;
    const int k = threadIdx.x;
    float v = k < 3 ? INFINITY : -INFINITY;
    for (int b = 0; b < n; ++b) v = k < 3 ? fminf(v, part[6 * b + k]) : fmaxf(v, part[6 * b + k]);
    out[k] = v;
}

// -------------------------------------------------------------- launchers --
template <bool INST, bool FUSED, bool COMP, bool NEAR = true>
cudaError_t stage1_shape(int *blocks) {
    const size_t sm = stage1_smem_bytes<INST, FUSED>();
    cudaError_t e = cudaFuncSetAttribute(k_stage1<INST, FUSED, COMP, NEAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_stage1<INST, FUSED, COMP, NEAR>, s1::kThreads, sm);
}

cudaError_t query_launch_shape(LaunchShape *o, int device) {
    cudaError_t e = cudaDeviceGetAttribute(&o->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    if ((e = stage1_shape<false, false, false>(&o->stage1_blocks_per_sm[0][0])) != cudaSuccess) return e;
    {   // the forms without the near-plane test run at the same shape
        int b = 0;
        if ((e = stage1_shape<false, false, false, false>(&b)) != cudaSuccess) return e;
        if ((e = stage1_shape<false, false, true, false>(&b)) != cudaSuccess) return e;
        if ((e = stage1_shape<true, false, false, false>(&b)) != cudaSuccess) return e;
        if ((e = stage1_shape<true, false, true, false>(&b)) != cudaSuccess) return e;
    }
    if ((e = stage1_shape<false, true, false>(&o->stage1_blocks_per_sm[0][1])) != cudaSuccess) return e;
    if ((e = stage1_shape<false, false, true>(&o->stage1_blocks_per_sm[0][2])) != cudaSuccess) return e;
    if ((e = stage1_shape<true, false, false>(&o->stage1_blocks_per_sm[1][0])) != cudaSuccess) return e;
    if ((e = stage1_shape<true, true, false>(&o->stage1_blocks_per_sm[1][1])) != cudaSuccess) return e;
    if ((e = stage1_shape<true, false, true>(&o->stage1_blocks_per_sm[1][2])) != cudaSuccess) return e;
    {
        const size_t sw = stage1_win_smem_bytes();
        e = cudaFuncSetAttribute(k_stage1_win, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sw);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage1_blocks_per_sm[0][3], k_stage1_win, s1::kThreads, sw);
        if (e != cudaSuccess) return e;
        o->stage1_blocks_per_sm[1][3] = o->stage1_blocks_per_sm[0][3];
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage1x_blocks_per_sm, k_stage1_exact<false>,
                                                      32 * s1::kExactWarps, 0);

    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage2_blocks_per_sm, k_stage2, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage3_blocks_per_sm, k_stage3, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_stage3_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage3_tile_smem(7));
    if (e != cudaSuccess) return e;
    for (int t = 4; t <= 7; ++t) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage3t_blocks_per_sm[t - 4], k_stage3_tiles, 256,
                                                          stage3_tile_smem((uint32_t)t));
        if (e != cudaSuccess) return e;
    }
    return e;
}

cudaError_t launch_clear(uint64_t *vis, uint64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n / 2 + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) blocks = 1;
    k_clear<<<(unsigned)blocks, 256, 0, s>>>(vis, n);
    return cudaGetLastError();
}

cudaError_t launch_stage1(const FrameDev &f, bool instanced, int variant, uint32_t r, int blocks, bool near,
                          cudaStream_t s) {
    const size_t s0 = stage1_smem_bytes<false, false>(), s1f = stage1_smem_bytes<false, true>();
    const size_t i0 = stage1_smem_bytes<true, false>(), i1f = stage1_smem_bytes<true, true>();
    if (instanced) {
        if (variant == 1) k_stage1<true, true, false><<<blocks, s1::kThreads, i1f, s>>>(f, r);
        else if (variant == 2 && near) k_stage1<true, false, true, true><<<blocks, s1::kThreads, i0, s>>>(f, r);
        else if (variant == 2) k_stage1<true, false, true, false><<<blocks, s1::kThreads, i0, s>>>(f, r);
        else if (near) k_stage1<true, false, false, true><<<blocks, s1::kThreads, i0, s>>>(f, r);
        else k_stage1<true, false, false, false><<<blocks, s1::kThreads, i0, s>>>(f, r);
    } else {
        if (variant == 3) k_stage1_win<<<blocks, s1::kThreads, stage1_win_smem_bytes(), s>>>(f, r);
        else if (variant == 1) k_stage1<false, true, false><<<blocks, s1::kThreads, s1f, s>>>(f, r);
        else if (variant == 2 && near) k_stage1<false, false, true, true><<<blocks, s1::kThreads, s0, s>>>(f, r);
        else if (variant == 2) k_stage1<false, false, true, false><<<blocks, s1::kThreads, s0, s>>>(f, r);
        else if (near) k_stage1<false, false, false, true><<<blocks, s1::kThreads, s0, s>>>(f, r);
        else k_stage1<false, false, false, false><<<blocks, s1::kThreads, s0, s>>>(f, r);
    }
    return cudaGetLastError();
}

cudaError_t launch_stage1_exact(const FrameDev &f, uint32_t r, int blocks, cudaStream_t s) {
    if (f.s3_ray) k_stage1_exact<true><<<blocks, 32 * s1::kExactWarps, 0, s>>>(f, r);
    else k_stage1_exact<false><<<blocks, 32 * s1::kExactWarps, 0, s>>>(f, r);
    return cudaGetLastError();
}

cudaError_t launch_stage2(const FrameDev &f, int blocks, cudaStream_t s) {
    k_stage2<<<blocks, 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_stage3(const FrameDev &f, int blocks, cudaStream_t s) {
    k_stage3<<<blocks, 256, 0, s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_stage3_binned(const FrameDev &f, int scatter_blocks, int tile_blocks, cudaStream_t s) {
    k_bin_scan<<<1, kScanThreads, 0, s>>>(f);
    k_bin_scatter<<<scatter_blocks, 256, 0, s>>>(f);
    k_stage3_tiles<<<tile_blocks, 256, stage3_tile_smem(f.tile_log2), s>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_aabb(const float *pos, uint64_t V, float *scratch, float *out6, cudaStream_t s) {
    k_aabb_partial<<<kAabbBlocks, 256, 0, s>>>(pos, V, scratch);
    k_aabb_final<<<1, 32, 0, s>>>(scratch, kAabbBlocks, out6);
    return cudaGetLastError();
}

cudaError_t launch_count_diff(const uint64_t *a, const uint64_t *b, uint64_t n, unsigned long long *out,
                              cudaStream_t s) {
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    if (blocks == 0) blocks = 1;
    k_count_diff<<<(unsigned)blocks, 256, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace curast
