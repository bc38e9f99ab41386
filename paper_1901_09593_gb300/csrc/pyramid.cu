// pyramid.cu -- Gaussian pyramid of the stereo pair (Sec. III, Fig. 1).
//
// Reading of the unstated filter: 5-tap binomial [1 4 6 4 1]/16 on each axis,
// clamp-to-edge, 2x decimation to ceil(W/2) x ceil(H/2), integer result
// (sum + 128) >> 8.  Levels stay uint8 so every ZNCC window sum is an exact integer.
//
// Both kernels write whole apron buffers: the value stored at (Y, X), for Y in
// [-APY, H+APY) and X in [-APX, W+APX), is the level pixel at (clamp(Y), clamp(X)), so the
// matching kernels read clamp-to-edge windows without index clamping.
// Bound: HBM/L2 traffic (1 B read per source pixel, 1 B written per output pixel); the
// levels of a frame are small enough to stay resident in L2.
#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "pyramid_fused.cuh"

namespace msbm {

// Level 0: copy the caller's image (any pitch) into the apron buffer with replication.
// One thread per 16 consecutive output bytes of one apron row; blockIdx.z selects left (0)
// / right (1).  Interior runs whose source is 8-byte aligned are moved with two 8-byte
// loads and one 16-byte store; runs touching the apron or misaligned fall back to bytes.
__global__ void apron_copy_kernel(const uint8_t *__restrict__ srcL, const uint8_t *__restrict__ srcR,
                                  size_t spitch, int W, int H, uint8_t *dstL, uint8_t *dstR,
                                  int dpitch) {
    const uint8_t *src = blockIdx.z ? srcR : srcL;
    uint8_t *dst = blockIdx.z ? dstR : dstL;   // points at image (0, 0)
    const int X0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16 - APX;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y - APY;
    if (Y >= H + APY || X0 >= W + APX) return;
    const int y = min(max(Y, 0), H - 1);
    const uint8_t *row = src + (size_t)y * spitch;
    uint4 out;
    if (X0 >= 0 && X0 + 16 <= W && ((reinterpret_cast<uintptr_t>(row + X0) & 7) == 0)) {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(row + X0));
        const uint2 b = __ldg(reinterpret_cast<const uint2 *>(row + X0 + 8));
        out = make_uint4(a.x, a.y, b.x, b.y);
    } else {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t v = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int x = min(max(X0 + 4 * q + i, 0), W - 1);
                v |= static_cast<uint32_t>(__ldg(row + x)) << (8 * i);
            }
            w[q] = v;
        }
        out = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // X0 + APX is a multiple of 16 and rows are 128-byte aligned; the 16 bytes may run past
    // W + APX into the row's padding (the pitch is a multiple of 128 >= W + 2*APX).
    *reinterpret_cast<uint4 *>(dst + (ptrdiff_t)Y * dpitch + X0) = out;
}

cudaError_t launch_apron_copy(const uint8_t *L, const uint8_t *R, size_t spitch, const LevelBuf &lv,
                              cudaStream_t st) {
    dim3 blk(32, 8);
    const int cols16 = (lv.W + 2 * APX + 15) / 16;
    dim3 grd((cols16 + blk.x - 1) / blk.x, (lv.H + 2 * APY + blk.y - 1) / blk.y, 2);
    apron_copy_kernel<<<grd, blk, 0, st>>>(L, R, spitch, lv.W, lv.H, lv.img(0), lv.img(1), lv.pitch);
    return cudaGetLastError();
}

// ---- fused pyramid: levels s+1 .. s+F (F <= PF_MAXF) in one launch (pyramid_fused.cuh) ----
// One CTA of PF_NT threads per tile and image (measured with 16 x 4 tiles: 256 threads
// beat 512 on the 2880 x 1984 pair and match it on the 1400 x 1000 pair; 128 threads are
// 3.4 us slower on the 1400 x 1000 pass).
constexpr int PF_NT = 256;

template <int F>
__global__ void __launch_bounds__(PF_NT) pyr_fused_kernel(const __grid_constant__ PyrFuseArgs a) {
    __shared__ __align__(16) uint8_t sm[PF_SMEM];
    pdl_launch_dependents();
    pyr_fused_tile<F, PF_NT>(a, a.src[blockIdx.z], a.spitch, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x,
                             gridDim.y, sm);
}

cudaError_t launch_pyr_fused(const PyrFuseArgs &a, cudaStream_t st) {
    if (a.F < 1 || a.F > PF_MAXF) return cudaErrorInvalidValue;
    dim3 grd((a.W[a.F] + PF_TX - 1) / PF_TX, (a.H[a.F] + PF_TY - 1) / PF_TY, 2);
    switch (a.F) {
        case 1: pyr_fused_kernel<1><<<grd, PF_NT, 0, st>>>(a); break;
        case 2: pyr_fused_kernel<2><<<grd, PF_NT, 0, st>>>(a); break;
        default: pyr_fused_kernel<3><<<grd, PF_NT, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// Dense copy of a level's interior (for inspection and tests).
__global__ void level_extract_kernel(const uint8_t *__restrict__ src, int spitch, int W, int H,
                                     uint8_t *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < W && y < H) dst[(size_t)y * W + x] = src[(ptrdiff_t)y * spitch + x];
}

cudaError_t launch_level_extract(const LevelBuf &lv, int which, uint8_t *out, cudaStream_t st) {
    dim3 blk(32, 8), grd((lv.W + 31) / 32, (lv.H + 7) / 8);
    level_extract_kernel<<<grd, blk, 0, st>>>(lv.img(which), lv.pitch, lv.W, lv.H, out);
    return cudaGetLastError();
}

}  // namespace msbm
