// pyramid.cu -- Gaussian pyramid of the stereo pair (Sec. III, Fig. 1).
//
// Reading of the unstated filter: 5-tap binomial [1 4 6 4 1]/16 on each axis,
// clamp-to-edge, 2x decimation to ceil(W/2) x ceil(H/2), integer result
// (sum + 128) >> 8.  Levels stay uint8 so every ZNCC window sum is an exact integer.
//
// Both kernels write whole apron buffers: the value stored at (Y, X), for Y in
// [-APY, H+APY) and X in [-APX, W+APX), is the level pixel at (clamp(Y), clamp(X)).  The
// reduce step therefore reads its 5x5 support straight from the finer apron buffer with
// no index clamping (2y+a and 2x+b stay within two pixels of the image, inside the apron).
// Bound: HBM/L2 traffic (1 B read per source pixel, 1 B written per output pixel); the
// levels of a frame are small enough to stay resident in L2.
#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "pyramid_ops.cuh"

namespace msbm {

// Level 0: copy the caller's image (any pitch) into the apron buffer with replication.
// One thread per 4 consecutive output bytes; blockIdx.z selects left (0) / right (1).
__global__ void apron_copy_kernel(const uint8_t *__restrict__ srcL, const uint8_t *__restrict__ srcR,
                                  size_t spitch, int W, int H, uint8_t *dstL, uint8_t *dstR,
                                  int dpitch) {
    const uint8_t *src = blockIdx.z ? srcR : srcL;
    uint8_t *dst = blockIdx.z ? dstR : dstL;   // points at image (0, 0)
    int X0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4 - APX;
    int Y = blockIdx.y * blockDim.y + threadIdx.y - APY;
    if (Y >= H + APY || X0 >= W + APX) return;
    copy_quad(src, spitch, W, H, dst, dpitch, X0, Y);
}

// Level k from level k-1.  One thread per 4 consecutive output bytes.
__global__ void pyr_reduce_kernel(const uint8_t *__restrict__ srcL, const uint8_t *__restrict__ srcR,
                                  int spitch, uint8_t *dstL, uint8_t *dstR, int dpitch, int Wd,
                                  int Hd) {
    const uint8_t *src = blockIdx.z ? srcR : srcL;   // image (0, 0) of level k-1
    uint8_t *dst = blockIdx.z ? dstR : dstL;
    int X0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4 - APX;
    int Y = blockIdx.y * blockDim.y + threadIdx.y - APY;
    if (Y >= Hd + APY || X0 >= Wd + APX) return;
    reduce_quad(src, spitch, dst, dpitch, Wd, Hd, X0, Y);
}

static dim3 apron_grid(int W, int H, dim3 blk) {
    int cols4 = (W + 2 * APX + 3) / 4;
    return dim3((cols4 + blk.x - 1) / blk.x, (H + 2 * APY + blk.y - 1) / blk.y, 2);
}

cudaError_t launch_apron_copy(const uint8_t *L, const uint8_t *R, size_t spitch, const LevelBuf &lv,
                              cudaStream_t st) {
    dim3 blk(32, 8);
    apron_copy_kernel<<<apron_grid(lv.W, lv.H, blk), blk, 0, st>>>(L, R, spitch, lv.W, lv.H, lv.img(0),
                                                                 lv.img(1), lv.pitch);
    return cudaGetLastError();
}

cudaError_t launch_pyr_reduce(const LevelBuf &src, const LevelBuf &dst, cudaStream_t st) {
    dim3 blk(32, 8);
    pyr_reduce_kernel<<<apron_grid(dst.W, dst.H, blk), blk, 0, st>>>(src.img(0), src.img(1), src.pitch,
                                                                    dst.img(0), dst.img(1), dst.pitch,
                                                                    dst.W, dst.H);
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
