// pyramid_ops.cuh -- the level-0 apron copy of one-level passes in the batched persistent
// kernel (batch.cu): each call writes 4 consecutive bytes of an apron buffer row, output
// (Y, X0..X0+3) with Y in [-APY, H+APY) and X0 + APX a multiple of 4 below W + 2*APX.
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

}  // namespace msbm
