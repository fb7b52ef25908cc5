// compress.cu -- the geometry encoding of Section 4.6, done on the device when
// a mesh is uploaded compressed: indices bit-packed relative to their
// minimum, positions as 16-bit fixed point over the mesh bounds.  The
// decoding lives in device.cuh (mesh_index, mesh_vertex) and in the
// compressed variant of the stage-1 cull kernel.
#include "internal.h"

namespace curast {

// Minimum and maximum of n words: out[0] (start ~0) and out[1] (start 0).
__global__ void __launch_bounds__(256) k_minmax_u32(const uint32_t *v, uint64_t n, unsigned *out) {
    unsigned lo = ~0u, hi = 0u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned x = __ldg(v + i);
        lo = min(lo, x);
        hi = max(hi, x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, lo);
        atomicMax(out + 1, hi);
    }
}

// Word w of the packed stream holds bits [32 w, 32 w + 32); index k sits at
// bits [k bits, k bits + bits), little-endian.  One thread per word: no
// two threads write the same word.
__global__ void __launch_bounds__(256) k_pack_indices(const uint32_t *idx, uint64_t n, uint32_t imin, uint32_t bits,
                                                      uint32_t *words, uint64_t nwords) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride) {
        uint32_t out = 0;
        if (bits) {
            const uint64_t b0 = 32 * w, b1 = b0 + 32;
            for (uint64_t k = b0 / bits; k < n && k * bits < b1; ++k) {
                const uint64_t v = (uint64_t)(__ldg(idx + k) - imin);
                const int64_t off = (int64_t)(k * bits) - (int64_t)b0;     // -31 .. 31
                out |= off >= 0 ? (uint32_t)(v << off) : (uint32_t)(v >> -off);
            }
        }
        words[w] = out;
    }
}

// q = rint(65535 (p - lo) / size) per axis in double, clamped to [0, 65535];
// 0 on a flat axis.
__global__ void __launch_bounds__(256) k_quantize_positions(const float *pos, uint64_t V, double lo0, double lo1,
                                                            double lo2, double s0, double s1, double s2, uint16_t *q) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const double lo[3] = {lo0, lo1, lo2}, size[3] = {s0, s1, s2};
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * V; i += stride) {
        const int a = (int)(i % 3);
        double v = 0.0;
        if (size[a] > 0.0) v = rint(__dmul_rn(65535.0, __ddiv_rn(__dsub_rn((double)__ldg(pos + i), lo[a]), size[a])));
        if (!(v >= 0.0)) v = 0.0;
        if (v > 65535.0) v = 65535.0;
        q[i] = (uint16_t)v;
    }
}

// Grid flags of a compressed mesh, bit k of word w for the 128-triangle
// group G = 32 w + k: set when the group lies wholly inside the mesh and each
// of its 32 runs of four triangles, 4 l .. 4 l + 3, lists the strip of a
// row-major grid, (s0 s1 s2) (s2 s1 s3) (s2 s3 s4) (s4 s3 s5) with s2 = s0 + 1,
// s4 = s0 + 2, s3 = s1 + 1, s5 = s1 + 2, every index below V.  The cull then
// decodes s0 and s1 alone and knows the other ten index fields.  One warp a
// word.
__global__ void __launch_bounds__(256) k_grid_flags(const uint32_t *idx, uint64_t T, uint64_t V, uint32_t *flags,
                                                    uint64_t nwords) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nwords; w += warps) {
        uint32_t word = 0;
        for (int k = 0; k < 32; ++k) {
            const uint64_t grp = 32 * w + (uint64_t)k;
            bool ok = (grp + 1) * 128 <= T;
            if (ok) {
                const uint32_t *p = idx + 3 * (grp * 128 + 4 * (uint64_t)lane);
                uint32_t x[12];
                for (int c = 0; c < 12; ++c) x[c] = __ldg(p + c);
                const uint64_t s0 = x[0], s1 = x[1];
                ok = s0 + 2 < V && s1 + 2 < V && x[2] == s0 + 1 && x[3] == s0 + 1 && x[4] == s1 &&
                     x[5] == s1 + 1 && x[6] == s0 + 1 && x[7] == s1 + 1 && x[8] == s0 + 2 && x[9] == s0 + 2 &&
                     x[10] == s1 + 1 && x[11] == s1 + 2;
            }
            if (__all_sync(0xffffffffu, ok)) word |= 1u << k;
        }
        if (lane == 0) flags[w] = word;
    }
}

cudaError_t launch_grid_flags(const uint32_t *idx, uint64_t T, uint64_t V, uint32_t *flags, uint64_t nwords,
                              cudaStream_t s) {
    if (nwords == 0) return cudaSuccess;
    k_grid_flags<<<1024, 256, 0, s>>>(idx, T, V, flags, nwords);
    return cudaGetLastError();
}

cudaError_t launch_minmax_u32(const uint32_t *v, uint64_t n, unsigned *out2, cudaStream_t s) {
    k_minmax_u32<<<1024, 256, 0, s>>>(v, n, out2);
    return cudaGetLastError();
}

cudaError_t launch_pack_indices(const uint32_t *idx, uint64_t n, uint32_t imin, uint32_t bits, uint32_t *words,
                                uint64_t nwords, cudaStream_t s) {
    k_pack_indices<<<2048, 256, 0, s>>>(idx, n, imin, bits, words, nwords);
    return cudaGetLastError();
}

cudaError_t launch_quantize_positions(const float *pos, uint64_t V, const double lo[3], const double size[3],
                                      uint16_t *q, cudaStream_t s) {
    k_quantize_positions<<<2048, 256, 0, s>>>(pos, V, lo[0], lo[1], lo[2], size[0], size[1], size[2], q);
    return cudaGetLastError();
}

}  // namespace curast
