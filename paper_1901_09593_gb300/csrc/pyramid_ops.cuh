// pyramid_ops.cuh -- per-thread pyramid operations (Sec. III, Fig. 1; reading: 5-tap
// binomial [1 4 6 4 1]/16 per axis, clamp-to-edge, 2x decimation, (sum + 128) >> 8), shared
// by the standalone pyramid kernels (pyramid.cu) and the batched persistent kernel.
// Each call writes 4 consecutive bytes of an apron buffer row: output (Y, X0..X0+3) with
// Y in [-APY, H+APY) and X0 + APX a multiple of 4 below W + 2*APX.
#pragma once

#include "msbm_device.cuh"

namespace msbm {

// Apron value at (Y, X) = image pixel (clamp(Y), clamp(X)) of the caller's image.
__device__ __forceinline__ void copy_quad(const uint8_t *__restrict__ src, size_t spitch, int W, int H,
                                          uint8_t *dst, int dpitch, int X0, int Y) {
    int y = min(max(Y, 0), H - 1);
    const uint8_t *row = src + (size_t)y * spitch;
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int x = min(max(X0 + i, 0), W - 1);
        v |= static_cast<uint32_t>(__ldg(row + x)) << (8 * i);
    }
    // X0 + APX is a multiple of 4 and the buffer row start is 128-byte aligned.
    *reinterpret_cast<uint32_t *>(dst + (ptrdiff_t)Y * dpitch + X0) = v;
}

// Apron value at (Y, X) of level k = the reduce of level k-1 at (clamp(Y), clamp(X)).  The
// 5 x 5 support 2y-2 .. 2y+2, 2x-2 .. 2x+2 lies inside the finer level's apron, so it is
// read without clamping.
__device__ __forceinline__ void reduce_quad(const uint8_t *__restrict__ src, int spitch, uint8_t *dst,
                                            int dpitch, int Wd, int Hd, int X0, int Y) {
    int y = min(max(Y, 0), Hd - 1);
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int x = min(max(X0 + i, 0), Wd - 1);
        int acc = 0;
        const uint8_t *base = src + (ptrdiff_t)(2 * y - 2) * spitch + (2 * x - 2);
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int cb = (b == 0 || b == 4) ? 1 : (b == 2 ? 6 : 4);
            int col = __ldg(base + b) + 4 * __ldg(base + spitch + b) + 6 * __ldg(base + 2 * spitch + b) +
                      4 * __ldg(base + 3 * spitch + b) + __ldg(base + 4 * spitch + b);
            acc += cb * col;
        }
        v |= static_cast<uint32_t>((acc + 128) >> 8) << (8 * i);
    }
    *reinterpret_cast<uint32_t *>(dst + (ptrdiff_t)Y * dpitch + X0) = v;
}

}  // namespace msbm
