// stage1_win.cuh -- the single-pair stage-1 cull with vertex windows in
// shared memory, included by raster.cu after stage1.cuh.
//
// Section 6 of the paper proposes transforming a cluster's vertices once
// into shared memory and then running one thread per triangle.  Here the
// cluster is the work item: its index triples arrive by TMA as in k_stage1,
// the producer warp reads them, finds the one or two contiguous vertex
// ranges ("windows") they reference -- on row-major grid meshes an item of
// 1024 triangles touches two runs of about 513 vertices -- and copies those
// ranges into shared memory with TMA as well.  The consumer warps then
//   phase 1: transform every window vertex once into the range of pixel
//            centres it could reach, its estimate widened by the error bound
//            of the conservative cull (win_range), packed in 8 bytes;
//   phase 2: run one thread per triangle: three lookups in the window, the
//            union of the three ranges, the pixel-centre test, one ballot per
//            32 triangles.
// Indices outside the windows (items that straddle mesh rows, unstructured
// meshes) are transformed by the thread itself from global memory with the
// same arithmetic.  The bound is the one fast_cull2 applies, taken per
// vertex (each vertex with its own 1/w and |X'|, |Y'|, as the error analysis
// is stated), so the cull is conservative: every (triangle, pair) the exact
// path could rasterize stays in the survivor bitmap.
#pragma once

namespace s1w {
using s1::kConsumers;
using s1::kConsumerWarps;
using s1::kItem;
constexpr int kNI = 3;              // index slots (TMA of index triples)
constexpr int kNV = 2;              // vertex-window slots
constexpr int kWinCap = 1040;       // window vertices per slot: one range, or two of kWinCap / 2
constexpr int kWinHalf = kWinCap / 2;
constexpr int kBlocks = 3;          // blocks per SM

struct WinDesc {
    uint32_t b0, n0;                // window 0: vertices [b0, b0 + n0), local 0..n0
    uint32_t b1, n1;                // window 1: vertices [b1, b1 + n1), local n0..n0 + n1
};

struct Smem {
    uint32_t idx[kNI][3 * kItem];
    float win[kNV][3 * kWinCap];    // raw x, y, z; then X', Y', 1/w in place
    FastPair fp[kNI];
    MeshDev mesh[kNI];
    s1::Desc desc[kNI];
    WinDesc wd[kNV];
    uint64_t ifull[kNI], iempty[kNI], vfull[kNV], vempty[kNV];
};
}  // namespace s1w

size_t stage1_win_smem_bytes() { return sizeof(s1w::Smem); }

// The conservative cull of one vertex (the error analysis behind the margin
// is per vertex and coordinate): the FMA rows of the pair give X'w, Y'w and
// w, rcp.approx gives 1/w, X' = (X'w)(1/w), and the exact snapped X' lies
// within m = (1/w)(ka + kb a) + kc a + kd of the estimate, a = max(|X'|,
// |Y'|), wherever w > wsafe and a < win.  The pixel centres (the integers
// 0..W-1 in X') the vertex could reach are then ceil(X' - m) .. floor(X' +
// m); clamped to [0, W] and [-1, W - 1] they fit 16 bits.  The result packs
// (x lo, y lo) and (x hi, y hi) as signed 16-bit pairs; a vertex outside the
// region where the bound holds gets the whole screen, so that no triangle
// using it is ever culled.  A triangle is culled when the union of its
// vertices' ranges holds no pixel centre on one axis -- then no exact
// snapped bbox of it can hold one either, which is the exact path's own
// tiny-and-off-screen cull.
__device__ __forceinline__ uint2 win_range(const float4 &rx, const float4 &ry, const float4 &rw, const float4 &k4,
                                           const float4 &lim, float x, float y, float z) {
    const float xw = __fmaf_rn(rx.x, x, __fmaf_rn(rx.y, y, __fmaf_rn(rx.z, z, rx.w)));
    const float yw = __fmaf_rn(ry.x, x, __fmaf_rn(ry.y, y, __fmaf_rn(ry.z, z, ry.w)));
    const float w = __fmaf_rn(rw.x, x, __fmaf_rn(rw.y, y, __fmaf_rn(rw.z, z, rw.w)));
    const float q = rcp_approx(w);
    const float X = __fmul_rn(xw, q), Y = __fmul_rn(yw, q);
    const float a = fmaxf(fabsf(X), fabsf(Y));
    const float m = __fmaf_rn(q, __fmaf_rn(k4.y, a, k4.x), __fmaf_rn(k4.z, a, k4.w));
    const int W1 = (int)lim.z, H1 = (int)lim.w;          // last pixel centre
    int xl = 0, xh = W1, yl = 0, yh = H1;
    if ((w > lim.x) & (a < lim.y)) {
        xl = min(max(__float2int_ru(__fsub_rn(X, m)), 0), W1 + 1);
        xh = max(min(__float2int_rd(__fadd_rn(X, m)), W1), -1);
        yl = min(max(__float2int_ru(__fsub_rn(Y, m)), 0), H1 + 1);
        yh = max(min(__float2int_rd(__fadd_rn(Y, m)), H1), -1);
    }
    return make_uint2(((uint32_t)xl & 0xFFFFu) | ((uint32_t)yl << 16), ((uint32_t)xh & 0xFFFFu) | ((uint32_t)yh << 16));
}

// Signed 16-bit pair minimum and maximum (one instruction on sm_90 and later).
__device__ __forceinline__ uint32_t min_s16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_s16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// A triangle from its vertices' packed ranges: culled when on one axis the
// smallest low end exceeds the largest high end (max(lo, hi) != hi).
__device__ __forceinline__ bool win_culled(uint2 a, uint2 b, uint2 c) {
    const uint32_t lo = min_s16x2(min_s16x2(a.x, b.x), c.x);
    const uint32_t hi = max_s16x2(max_s16x2(a.y, b.y), c.y);
    return max_s16x2(lo, hi) != hi;
}

// AND of v over the 256 consumer threads, with a barrier among them (named
// barrier 1; the producer warp does not take part).
__device__ __forceinline__ bool consumers_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(s1::kConsumers)
        : "memory");
    return r != 0;
}

// Producer: windows of item jp (its index copy was issued one grab earlier):
// waits for the indices, scans them for their smallest and largest vertex,
// chooses the windows, and copies them into vertex slot jp % kNV.  An index
// range that fits kWinCap vertices becomes one window; otherwise the two ends
// get kWinHalf vertices each.  Windows start on 4-vertex boundaries (48 B,
// a multiple of TMA's 16) and stay below V rounded down to 4; windows that
// would serve fewer than half of a sample of the item's index words are
// dropped.
__device__ __forceinline__ bool win_stage(const FrameDev &f, s1w::Smem &S, uint32_t jp, uint32_t n,
                                          const MeshDev &mesh) {
    using namespace s1w;
    const int lane = threadIdx.x & 31;
    const int s = jp % kNI, vs = jp % kNV;
    if (!mbar_wait(&S.ifull[s], (jp / kNI) & 1u)) return false;
    const uint32_t *ix = S.idx[s];
    const uint32_t nw = 3 * n;
    // 16-byte loads, unrolled so that a lane's loads are in flight together
    const uint4 *ix4 = reinterpret_cast<const uint4 *>(ix);
    const uint32_t nw4 = nw >> 2;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll 8
    for (uint32_t w = lane; w < nw4; w += 32) {
        const uint4 v = ix4[w];
        lo = min(lo, min(min(v.x, v.y), min(v.z, v.w)));
        hi = max(hi, max(max(v.x, v.y), max(v.z, v.w)));
    }
    for (uint32_t w = 4 * nw4 + lane; w < nw; w += 32) {
        lo = min(lo, ix[w]);
        hi = max(hi, ix[w]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    WinDesc wd{0u, 0u, 0u, 0u};
    const uint64_t vf = mesh.V & ~(uint64_t)3;                         // copies stay below this vertex
    const bool aligned = (reinterpret_cast<uintptr_t>(mesh.pos) & 15) == 0;
    if (aligned && n > 0 && (uint64_t)lo < vf) {
        const uint64_t a0 = (uint64_t)(lo & ~3u);
        const uint64_t top = min(((uint64_t)hi + 4) & ~(uint64_t)3, vf);  // one past the last window vertex
        if ((uint64_t)hi - a0 + 1 <= (uint64_t)kWinCap) {
            wd.b0 = (uint32_t)a0;
            wd.n0 = (uint32_t)(top - a0);
        } else {
            const uint64_t e0 = min(a0 + (uint64_t)kWinHalf, vf);
            wd.b0 = (uint32_t)a0;
            wd.n0 = (uint32_t)(e0 - a0);
            const uint64_t b1 = max(top >= (uint64_t)kWinHalf ? top - (uint64_t)kWinHalf : (uint64_t)0, e0);
            wd.b1 = (uint32_t)b1;
            wd.n1 = top > b1 ? (uint32_t)(top - b1) : 0u;
        }
        // a sample of 32 index words spread over the item: windows that
        // would serve fewer than half of them are not worth their copy
        const uint32_t v = ix[(uint32_t)(((uint64_t)lane * nw) >> 5)];
        const unsigned hit = __ballot_sync(0xffffffffu, (v - wd.b0 < wd.n0) | (v - wd.b1 < wd.n1));
        if (__popc(hit) < 16) wd = WinDesc{0u, 0u, 0u, 0u};
    }
    if (jp >= (uint32_t)kNV && !mbar_wait(&S.vempty[vs], ((jp / kNV) - 1) & 1u)) return false;
    if (lane == 0) {
        S.wd[vs] = wd;
        const uint32_t bytes = 12u * (wd.n0 + wd.n1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&S.vfull[vs], bytes);
        if (wd.n0) bulk_copy_g2s(S.win[vs], mesh.pos + 3 * (uint64_t)wd.b0, 12u * wd.n0, &S.vfull[vs]);
        if (wd.n1) bulk_copy_g2s(S.win[vs] + 3 * wd.n0, mesh.pos + 3 * (uint64_t)wd.b1, 12u * wd.n1, &S.vfull[vs]);
    } else {
        mbar_arrive(&S.vfull[vs]);
    }
    return true;
}

// Producer warp: work grabs as in stage1_producer (Section 4.1 "Looping
// Through Batches"), the TMA copy of each item's index triples, and one grab
// later the item's vertex windows.
__device__ __forceinline__ void win_producer(const FrameDev &f, s1w::Smem &S, const RoundDev &rd, uint32_t r,
                                             int n_segs, uint64_t per_item, uint32_t G) {
    using namespace s1w;
    const int lane = threadIdx.x & 31;
    unsigned long long next = 0;
    int segidx = 0;
    unsigned long long seg_end = 0;
    SegDev seg{};
    bool have = false;
    uint32_t prev_n = 0;
    uint32_t cur_mesh = ~0u, cur_pair = ~0u;         // segment of the last item whose constants were loaded
    if (lane == 0) next = rd.b0 + atomicAdd(&f.ctr->work[r], 1ull);
    for (uint32_t j = 0;; ++j) {
        const int s = j % kNI;
        if (j >= (uint32_t)kNI && !mbar_wait(&S.iempty[s], ((j / kNI) - 1) & 1u)) {
            if (lane == 0) atomicOr(f.err, kErrTimeout);
            return;
        }
        s1::Desc d{};
        if (lane == 0) {
            const unsigned long long b = next;
            d.b = b;
            if (b < rd.b1) {
                next = rd.b0 + atomicAdd(&f.ctr->work[r], 1ull);
                if (!have || b >= seg_end) {          // galloping forward search: grabs only grow
                    int lo = segidx, step = 1, hi;
                    while (true) {
                        hi = lo + step;
                        if (hi >= n_segs || f.segs[hi].batch0 > b) break;
                        lo = hi;
                        step <<= 1;
                    }
                    if (hi > n_segs) hi = n_segs;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (f.segs[mid].batch0 <= b) lo = mid; else hi = mid;
                    }
                    segidx = lo;
                    seg = f.segs[lo];
                    seg_end = lo + 1 < n_segs ? f.segs[lo + 1].batch0 : ~0ull;
                    have = true;
                }
                const uint64_t jb = b - seg.batch0;
                d.t0 = jb * per_item;
                const uint64_t left = seg.T - d.t0;
                d.n = (uint32_t)(left < per_item ? left : per_item);
                d.mesh = seg.mesh;
                d.pair0 = seg.pair0;
                d.npairs = 1u;
                d.wbase = seg.word0 + jb * G - rd.w0;
            }
            S.desc[s] = d;
        }
        d.b = __shfl_sync(0xffffffffu, d.b, 0);
        const bool end = d.b >= rd.b1;
        if (!end) {
            d.t0 = __shfl_sync(0xffffffffu, d.t0, 0);
            d.n = __shfl_sync(0xffffffffu, d.n, 0);
            d.mesh = __shfl_sync(0xffffffffu, d.mesh, 0);
            d.pair0 = __shfl_sync(0xffffffffu, d.pair0, 0);
            // the mesh record and the pair constants: from the previous slot
            // when the item continues the same segment (no global round
            // trips), else from the frame tables, one word a lane
            constexpr int kMW = sizeof(MeshDev) / 4, kFW = sizeof(FastPair) / 4;
            static_assert(kMW <= 32 && kFW <= 32, "one word a lane");
            if (j > 0 && d.mesh == cur_mesh && d.pair0 == cur_pair) {
                const int ps = (j - 1) % kNI;
                if (lane < kMW) reinterpret_cast<uint32_t *>(&S.mesh[s])[lane] =
                    reinterpret_cast<const uint32_t *>(&S.mesh[ps])[lane];
                if (lane < kFW) reinterpret_cast<uint32_t *>(&S.fp[s])[lane] =
                    reinterpret_cast<const uint32_t *>(&S.fp[ps])[lane];
            } else {
                if (lane < kMW) reinterpret_cast<uint32_t *>(&S.mesh[s])[lane] =
                    __ldg(reinterpret_cast<const uint32_t *>(f.meshes + d.mesh) + lane);
                const PairDev &pr = f.pairs[d.pair0];
                const ViewDev &vw = f.views[pr.view];
                // FastPair words: rx ry rw (fn 0..11), k (fk 0..3), lim (wsafe, win, W - 1, H - 1), sl (fs 0..2, 0)
                float w = 0.0f;
                if (lane < 12) w = pr.fn[lane];
                else if (lane < 16) w = pr.fk[lane - 12];
                else if (lane == 16) w = pr.wsafe;
                else if (lane == 17) w = pr.win;
                else if (lane == 18) w = (float)(vw.W - 1);
                else if (lane == 19) w = (float)(vw.H - 1);
                else if (lane < 23) w = pr.fs[lane - 20];
                else if (lane == 23) w = pr.nlo;
                if (lane < kFW) reinterpret_cast<float *>(&S.fp[s])[lane] = w;
                cur_mesh = d.mesh;
                cur_pair = d.pair0;
            }
            __syncwarp();
            const MeshDev &mesh = S.mesh[s];
            const uint32_t bytes = 12u * d.n;
            const uint32_t *src = mesh.idx + 3 * d.t0;
            const bool tma = (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (bytes & 15) == 0;
            if (!tma)
                for (uint32_t w = lane; w < bytes / 4; w += 32) S.idx[s][w] = __ldg(src + w);
            __syncwarp();
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&S.ifull[s], tma ? bytes : 0u);
                if (tma) bulk_copy_g2s(S.idx[s], src, bytes, &S.ifull[s]);
            } else {
                mbar_arrive(&S.ifull[s]);
            }
        }
        // the windows of the previous item, whose indices have had a grab's
        // time to land
        if (j >= 1) {
            const MeshDev &pm = S.mesh[(j - 1) % kNI];
            if (!win_stage(f, S, j - 1, prev_n, pm)) {
                if (lane == 0) atomicOr(f.err, kErrTimeout);
                return;
            }
        }
        if (end) {                                     // tell the consumers to stop
            const int vs = j % kNV;
            if (j >= (uint32_t)kNV && !mbar_wait(&S.vempty[vs], ((j / kNV) - 1) & 1u)) {
                if (lane == 0) atomicOr(f.err, kErrTimeout);
                return;
            }
            if (lane == 0) mbar_arrive_expect_tx(&S.vfull[vs], 0u);
            else mbar_arrive(&S.vfull[vs]);
            return;
        }
        prev_n = d.n;
    }
}

// Persistent single-pair stage-1 cull of round r with vertex windows (see the
// top of this file).  The survivor bitmap words are those of k_stage1: the
// warp's ballot over triangles (k + u) * 256 + 32 warp + lane of the item is
// word (k + u) * 8 + warp.
__global__ void __launch_bounds__(s1::kThreads, s1w::kBlocks) k_stage1_win(const __grid_constant__ FrameDev f,
                                                                           uint32_t r) {
    using namespace s1w;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const RoundDev rd = f.rounds[r];
    const int n_segs = (int)f.hdr->n_segs;
    const uint32_t tpt = f.tpt;
    const uint64_t per_item = (uint64_t)kConsumers * tpt;
    const uint32_t G = kConsumerWarps * tpt;

    if (tid == 0) {
        for (int s = 0; s < kNI; ++s) {
            mbar_init(&S.ifull[s], 32);                // the producer warp's lanes (lane 0 with the copy's bytes)
            mbar_init(&S.iempty[s], kConsumerWarps);
        }
        for (int s = 0; s < kNV; ++s) {
            mbar_init(&S.vfull[s], 32);                // the producer warp's lanes
            mbar_init(&S.vempty[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumerWarps) {
        win_producer(f, S, rd, r, n_segs, per_item, G);
        return;
    }

    for (uint32_t j = 0;; ++j) {
        const int s = j % kNI, vs = j % kNV;
        // the windows' arrival also means the indices arrived: the producer
        // waited for them before choosing the windows
        bool ok = mbar_wait(&S.vfull[vs], (j / kNV) & 1u);
        const s1::Desc d = S.desc[s];
        const bool end = d.b >= rd.b1;
        ok = ok && (end || mbar_wait(&S.ifull[s], (j / kNI) & 1u));
        const MeshDev &mesh = S.mesh[s];
        const uint64_t V = mesh.V;
        const float *gpos = mesh.pos;
        const FastPair &fp = S.fp[s];
        const float4 rx = fp.rx, ry = fp.ry, rw = fp.rw, k4 = fp.k, lim = fp.lim;
        const WinDesc wd = S.wd[vs];
        float *win = S.win[vs];
        // phase 1: every window vertex once, read into registers before the
        // barrier and written back (8 bytes each, over the raw data) after it
        constexpr int kPer = (kWinCap + kConsumers - 1) / kConsumers;
        const uint32_t nwin = ok && !end ? wd.n0 + wd.n1 : 0u;
        uint2 vr[kPer];
#pragma unroll
        for (int c = 0; c < kPer; ++c) {
            const uint32_t i = tid + c * kConsumers;
            if (i < nwin) vr[c] = win_range(rx, ry, rw, k4, lim, win[3 * i], win[3 * i + 1], win[3 * i + 2]);
        }
        // every consumer thread reaches this barrier once per item, timed out
        // or not, and all of them leave together if any wait gave up
        if (!consumers_all(ok)) {
            if (tid == 0) atomicOr(f.err, kErrTimeout);
            return;
        }
        if (end) break;
        uint2 *xf = reinterpret_cast<uint2 *>(win);
#pragma unroll
        for (int c = 0; c < kPer; ++c) {
            const uint32_t i = tid + c * kConsumers;
            if (i < nwin) xf[i] = vr[c];
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
        // phase 2: one thread per triangle
        const uint32_t *idx = S.idx[s];
        for (uint32_t k = 0; k < tpt; ++k) {           // uniform trip count: the warp stays converged
            const uint32_t lt = k * kConsumers + tid;
            bool valid = lt < d.n;
            uint32_t iv[3] = {0u, 0u, 0u};
            if (valid) {
                iv[0] = idx[3 * lt]; iv[1] = idx[3 * lt + 1]; iv[2] = idx[3 * lt + 2];
                if (max(iv[0], max(iv[1], iv[2])) >= V) {
                    if (f.check) atomicOr(f.err, kErrIndex);
                    valid = false;
                }
            }
            uint32_t l[3];
            bool miss = false;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint32_t l0 = iv[c] - wd.b0, l1 = iv[c] - wd.b1;
                l[c] = l0 < wd.n0 ? l0 : wd.n0 + l1;
                miss |= l[c] >= wd.n0 + wd.n1;
            }
            miss &= valid;
            uint2 e[3];
            if (!__any_sync(0xffffffffu, miss)) {
#pragma unroll
                for (int c = 0; c < 3; ++c) e[c] = xf[valid ? l[c] : 0u];
            } else {
                // some vertex of the warp lies outside the windows: those are
                // transformed from global memory with the same arithmetic
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (valid && l[c] < wd.n0 + wd.n1) {
                        e[c] = xf[l[c]];
                    } else if (valid) {
                        const float *p = gpos + 3 * (uint64_t)iv[c];
                        e[c] = win_range(rx, ry, rw, k4, lim, __ldg(p), __ldg(p + 1), __ldg(p + 2));
                    } else {
                        e[c] = make_uint2(0u, 0u);
                    }
                }
            }
            const bool live = valid && !win_culled(e[0], e[1], e[2]);
            if (f.stats && valid && !live) stat_add(f, kStatIn, 1), stat_add(f, kStatTiny, 1);
            const unsigned bm = __ballot_sync(0xffffffffu, live);
            if (lane == 0) f.bits[d.wbase + k * kConsumerWarps + warp] = bm;
        }
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&S.iempty[s]);
            mbar_arrive(&S.vempty[vs]);
        }
    }
}
