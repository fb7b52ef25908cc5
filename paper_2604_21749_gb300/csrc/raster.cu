// raster.cu -- clear, stage 1, stage 2 and stage 3 kernels (Section 3.1-3.3).
#include <cooperative_groups.h>

#include "internal.h"

namespace curast {

// ------------------------------------------------------------------ clear --
// Section 3.1: the framebuffer starts each frame at the empty word (all
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
// (start, stride) -- used by a single thread when a queue is full (stride 1)
// and by stage 2 (one warp per triangle, stride 32).
__device__ void raster_triangle_general(const CV c[3], const ViewDev &vw, uint64_t id, int start, int stride) {
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

__device__ __forceinline__ void stat_add(const FrameDev &f, int k, unsigned long long v) {
    if (f.stats && v) atomicAdd(&f.ctr->stats[k], v);
}

// Warp-aggregated append to queue 1 (ballot + popc + one atomicAdd per warp).
// Lanes whose slot lies beyond the capacity rasterize their triangle in place.
__device__ __forceinline__ void q1_append(const FrameDev &f, bool want, uint64_t id, uint32_t pair, const CV c[3],
                                          const ViewDev &vw) {
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
        e.pair = pair;
        e.pad = 0;
        f.q1[slot] = e;
    } else {
        atomicAdd(&f.ctr->overflow1, 1ull);
        raster_triangle_general(c, vw, id, 0, 1);
    }
}

// ---------------------------------------------------------------- stage 1 --
// Small-triangle rasterizer of Section 3.1: one thread per triangle, y outer
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
                depth_test_write(row, (size_t)x, key);
            }
            r0 -= dy0 * 256; r1 -= dy1 * 256; r2 -= dy2 * 256;
        }
        e0 += dx0 * 256; e1 += dx1 * 256; e2 += dx2 * 256;
    }
}

enum Class { kDrop = 0, kQueue = 1, kSmall = 2 };

// Transform, clip classification, snap, backface / frustum / tiny culls of
// one triangle for one (instance, view) pair; returns what to do with it.
struct Classified {
    int X[3], Y[3];
    float iz[3];
    int64_t A;
    int x0, x1, y0, y1;
};

__device__ __forceinline__ int classify(const FrameDev &f, const CV c[3], const ViewDev &vw, Classified &o,
                                        unsigned &stat_mask) {
    const unsigned o0 = outcode(c[0], vw.nearv), o1 = outcode(c[1], vw.nearv), o2 = outcode(c[2], vw.nearv);
    if (o0 & o1 & o2) { stat_mask = 1u << kStatClip; return kDrop; }      // wholly beyond one plane
    if (o0 | o1 | o2) return kQueue;                                        // crosses near/guard: stage 2 clips
#pragma unroll
    for (int k = 0; k < 3; ++k) snap(c[k], vw.hw, vw.hh, o.X[k], o.Y[k], o.iz[k]);
    const int64_t A = (int64_t)(o.X[1] - o.X[0]) * (int64_t)(o.Y[2] - o.Y[0]) -
                      (int64_t)(o.X[2] - o.X[0]) * (int64_t)(o.Y[1] - o.Y[0]);
    if (A <= 0) { stat_mask = 1u << kStatBack; return kDrop; }              // backface or degenerate
    const int minX = min(o.X[0], min(o.X[1], o.X[2])), maxX = max(o.X[0], max(o.X[1], o.X[2]));
    const int minY = min(o.Y[0], min(o.Y[1], o.Y[2])), maxY = max(o.Y[0], max(o.Y[1], o.Y[2]));
    // pixel centres 256 x + 128 inside [min, max], clamped to the screen;
    // an empty range is the frustum cull and the tiny-triangle cull at once
    const int x0 = max((int)ceil_div256((int64_t)minX - 128), 0);
    const int x1 = min((int)floor_div256((int64_t)maxX - 128), vw.W - 1);
    const int y0 = max((int)ceil_div256((int64_t)minY - 128), 0);
    const int y1 = min((int)floor_div256((int64_t)maxY - 128), vw.H - 1);
    if (x0 > x1 || y0 > y1) { stat_mask = 1u << kStatTiny; return kDrop; }
    if (maxX - minX >= (1 << 14) || maxY - minY >= (1 << 14)) return kQueue;
    if ((uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1)) > f.s1_max) return kQueue;
    o.A = A;
    o.x0 = x0; o.x1 = x1; o.y0 = y0; o.y1 = y1;
    return kSmall;
}

// Persistent stage-1 kernel (Section 3.1 "Looping Through Batches"): a
// fixed set of blocks grabs work items from a global counter until none are
// left.  A work item is blockDim * tpt consecutive triangles of one segment
// (a mesh and a run of its (instance, view) pairs); each thread loads its
// triangle's indices and positions once and rasterizes it for every pair of
// the segment (Section 3.5, extended to several views).  The next grab is
// issued one item ahead so its latency hides behind the current item.
template <bool INSTANCED>
__global__ void __launch_bounds__(256) k_stage1(FrameDev f) {
    __shared__ unsigned long long s_b;
    __shared__ SegDev s_seg;
    const unsigned tid = threadIdx.x;
    unsigned long long pre = 0;
    int segidx = 0;
    const uint64_t n_batches = f.hdr->n_batches;
    const int n_segs = (int)f.hdr->n_segs;
    auto find_segment = [&](unsigned long long b) {
        // batches only grow for one block, so search forward (galloping)
        int lo = segidx, step = 1, hi;
        while (true) {
            hi = lo + step;
            if (hi >= n_segs || f.segs[hi].batch0 > b) break;
            lo = hi;
            step <<= 1;
        }
        if (hi > n_segs) hi = n_segs;
        while (hi - lo > 1) {              // invariant: batch0[lo] <= b < batch0[hi]
            const int mid = (lo + hi) >> 1;
            if (f.segs[mid].batch0 <= b) lo = mid; else hi = mid;
        }
        segidx = lo;
        s_seg = f.segs[lo];
    };
    if (tid == 0) {
        const unsigned long long b = atomicAdd(&f.ctr->work, 1ull);
        s_b = b;
        if (b < n_batches) find_segment(b);
        pre = atomicAdd(&f.ctr->work, 1ull);
    }
    __syncthreads();
    const uint64_t per_item = (uint64_t)blockDim.x * f.tpt;
    for (;;) {
        const unsigned long long b = s_b;
        if (b >= n_batches) break;
        const SegDev seg = s_seg;
        const MeshDev mesh = f.meshes[seg.mesh];
        const uint64_t t0 = (b - seg.batch0) * per_item;
        unsigned long long n_in = 0, n_clip = 0, n_back = 0, n_tiny = 0, n_s1 = 0;
        for (uint32_t k = 0; k < f.tpt; ++k) {
            const uint64_t t = t0 + (uint64_t)k * blockDim.x + tid;
            if (t >= seg.T) break;
            const uint32_t *ip = mesh.idx + 3 * t;
            const uint32_t i0 = __ldg(ip), i1 = __ldg(ip + 1), i2 = __ldg(ip + 2);
            if (f.check && (i0 >= mesh.V || i1 >= mesh.V || i2 >= mesh.V)) {
                atomicOr(f.err, kErrIndex);
                continue;
            }
            const float *q0 = mesh.pos + 3 * (uint64_t)i0, *q1 = mesh.pos + 3 * (uint64_t)i1,
                        *q2 = mesh.pos + 3 * (uint64_t)i2;
            const float x0 = __ldg(q0), y0 = __ldg(q0 + 1), z0 = __ldg(q0 + 2);
            const float x1 = __ldg(q1), y1 = __ldg(q1 + 1), z1 = __ldg(q1 + 2);
            const float x2 = __ldg(q2), y2 = __ldg(q2 + 1), z2 = __ldg(q2 + 2);
            const uint32_t np = INSTANCED ? seg.npairs : 1u;
            for (uint32_t pi = 0; pi < np; ++pi) {
                const uint32_t pidx = seg.pair0 + pi;
                const PairDev &pr = f.pairs[pidx];
                const ViewDev &vw = f.views[pr.view];
                float mv[12];
#pragma unroll
                for (int j = 0; j < 12; ++j) mv[j] = pr.mv[j];
                const float fx = vw.fx, fy = vw.fy;
                CV c[3];
                c[0] = to_clip(mv, x0, y0, z0, fx, fy);
                c[1] = to_clip(mv, x1, y1, z1, fx, fy);
                c[2] = to_clip(mv, x2, y2, z2, fx, fy);
                Classified o;
                unsigned sm = 0;
                const int cls = classify(f, c, vw, o, sm);
                const uint64_t id = pr.base + t;
                q1_append(f, cls == kQueue, id, pidx, c, vw);
                if (cls == kSmall) raster_small(o.X, o.Y, o.iz, o.A, o.x0, o.x1, o.y0, o.y1, id, vw.vis, vw.W);
                if (f.stats) {
                    n_in += 1;
                    n_clip += (sm >> kStatClip) & 1u;
                    n_back += (sm >> kStatBack) & 1u;
                    n_tiny += (sm >> kStatTiny) & 1u;
                    n_s1 += cls == kSmall;
                }
            }
        }
        if (f.stats) {
            stat_add(f, kStatIn, n_in);
            stat_add(f, kStatClip, n_clip);
            stat_add(f, kStatBack, n_back);
            stat_add(f, kStatTiny, n_tiny);
            stat_add(f, kStatS1, n_s1);
        }
        __syncthreads();
        if (tid == 0) {
            s_b = pre;
            if (pre < n_batches) {
                find_segment(pre);
                pre = atomicAdd(&f.ctr->work, 1ull);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- stage 2 --
// Section 3.2: one warp per queued triangle.  The triangle is clipped
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
        f.q2[slot] = e;
    } else {
        atomicAdd(&f.ctr->overflow2, 1ull);
        const int ts = 1 << f.tile_log2;
        raster_range(s, max(s.x0, tx * ts), min(s.x1, tx * ts + ts - 1), max(s.y0, ty * ts),
                     min(s.y1, ty * ts + ts - 1), 0, 1, vw.vis, vw.W);
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
        const uint64_t t = e.id - pr.base;
        float mv[12];
        for (int j = 0; j < 12; ++j) mv[j] = pr.mv[j];
        CV c[3];
        for (int k = 0; k < 3; ++k) {
            const uint32_t vi = mesh.idx[3 * t + k];
            const float *q = mesh.pos + 3 * (uint64_t)vi;
            c[k] = to_clip(mv, q[0], q[1], q[2], vw.fx, vw.fy);
        }
        CV poly[kMaxPoly];
        const int np = clip_polygon(c, vw.nearv, poly);
        if (np < 3) continue;
        int X[kMaxPoly], Y[kMaxPoly];
        float iz[kMaxPoly];
        for (int k = 0; k < np; ++k) snap(poly[k], vw.hw, vw.hh, X[k], Y[k], iz[k]);
        for (int j = 1; j + 1 < np; ++j) {
            SubTri s;
            s.X[0] = X[0]; s.X[1] = X[j]; s.X[2] = X[j + 1];
            s.Y[0] = Y[0]; s.Y[1] = Y[j]; s.Y[2] = Y[j + 1];
            s.iz[0] = iz[0]; s.iz[1] = iz[j]; s.iz[2] = iz[j + 1];
            s.id = e.id;
            if (!setup_subtri(s, vw.W, vw.H)) continue;
            const int64_t cnt = (int64_t)(s.x1 - s.x0 + 1) * (int64_t)(s.y1 - s.y0 + 1);
            if (cnt <= (int64_t)f.s2_max) {
                raster_range(s, s.x0, s.x1, s.y0, s.y1, lane, 32, vw.vis, vw.W);
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
// Section 3.3: one block per tile part; its threads walk the tile's pixels
// (restricted to the sub-triangle's bbox) line by line.
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

cudaError_t launch_aabb(const float *pos, uint64_t V, float *scratch, float *out6, cudaStream_t s) {
    k_aabb_partial<<<kAabbBlocks, 256, 0, s>>>(pos, V, scratch);
    k_aabb_final<<<1, 32, 0, s>>>(scratch, kAabbBlocks, out6);
    return cudaGetLastError();
}

// -------------------------------------------------------------- launchers --
cudaError_t query_launch_shape(LaunchShape *o, int device) {
    cudaError_t e = cudaDeviceGetAttribute(&o->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage1_blocks_per_sm[0], k_stage1<false>, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage1_blocks_per_sm[1], k_stage1<true>, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage2_blocks_per_sm, k_stage2, 256, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o->stage3_blocks_per_sm, k_stage3, 256, 0);
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

cudaError_t launch_stage1(const FrameDev &f, bool instanced, int blocks, cudaStream_t s) {
    if (instanced) k_stage1<true><<<blocks, 256, 0, s>>>(f);
    else k_stage1<false><<<blocks, 256, 0, s>>>(f);
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

cudaError_t launch_count_diff(const uint64_t *a, const uint64_t *b, uint64_t n, unsigned long long *out,
                              cudaStream_t s) {
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    if (blocks == 0) blocks = 1;
    k_count_diff<<<(unsigned)blocks, 256, 0, s>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace curast
