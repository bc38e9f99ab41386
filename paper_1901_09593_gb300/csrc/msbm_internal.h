// msbm_internal.h -- host-side structures and kernel launchers of libmsbm (not part of
// the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "msbm.h"
#include "msbm_device.cuh"

namespace msbm {

// Launch k<<<g, b, smem, st>>>(args...); with pdl, as a programmatic dependent of the
// stream's previous kernel (k must call pdl_wait() before reading what that kernel writes).
template <typename... P, typename... A>
cudaError_t launch_k(void (*k)(P...), dim3 g, dim3 b, size_t smem, cudaStream_t st, bool pdl, A &&...args) {
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// One pyramid level of both images: two apron buffers (see msbm_device.cuh) plus the
// tensor maps the ZNCC kernels stage tiles with.
struct LevelBuf {
    int W = 0, H = 0, Dk = 0;
    int nh = 0;                  // window half-width matched at this level
    int pitch = 0;               // bytes per buffer row (multiple of 128)
    int rows = 0;                // H + 2*APY
    uint8_t *base[2] = {nullptr, nullptr};  // buffer starts: image pixel (-APY, -APX)
    int16_t *d = nullptr;        // this level's disparity map (levels >= 1)
    float *c = nullptr;          // this level's cost map (levels >= 1)
    int16_t *dtmp = nullptr;     // pre-median disparity map (SELECTIVE_MEDIAN)
    uint8_t *mask = nullptr;     // fallback mask (BETA_FALLBACK)
    unsigned *cells = nullptr;   // fallback cells {count, next, cy * ceil(W/2) + cx ...} (BETA_FALLBACK)
    int2 *rstat = nullptr;       // right-window statistics plane {S, bits(rsqrt(V)) or 0}: H rows
    int rspitch = 0;             // of rspitch entries (a multiple of 16), one per pixel
    int rty = 8;                 // rows of the staged restricted tile (MSBM_FLAG_TEST_TIMEOUT)
    // TMA maps over the apron buffers.  Full-range tile (8 + 2n rows high):
    //   tmFL   : left,  32*SX + 32 bytes wide, SX per level
    //   tmR256 : right, 256 bytes wide
    // Restricted tile (rty + 2n rows high):
    //   tmRL   : left,  64 bytes wide
    //   tmRR128, tmRR256 : right, 128 / 256 bytes wide
    //   tmS128, tmS256 : right statistics plane, 128 / 256 entries wide, rty rows
    CUtensorMap tmFL, tmR256, tmRL, tmRR128, tmRR256, tmS128, tmS256;
    int full_sx = 4;             // full-range tile width 32*full_sx at this level
    int full_zblock = 0;         // full-range z-block (0 = the tile's maximum)
    bool coarse = false;         // plain full-range search by the small-level kernel
    uint8_t *img(int which) const {
        return base[which] + (size_t)APY * pitch + APX;
    }
};

// Per-tile arguments of the full-range ZNCC tile (zncc_full_tile.cuh).
struct FullTileArgs {
    int W, H, Dk;
    int zblock;          // candidates staged per pass (multiple of 32; 0 = the tile's maximum)
    int16_t *d_out;
    float *c_out;
    unsigned long long *evals;
    int *err;
    int force_timeout;
};

struct FullArgs {
    CUtensorMap tmL;     // box {32*SX + 32, 8 + 2n} over the left apron buffer
    CUtensorMap tmR;     // box {256, 8 + 2n} over the right apron buffer
    FullTileArgs t;
};

// Per-tile arguments of the restricted ZNCC tile (zncc_restricted_tile.cuh).
struct RestrTileArgs {
    const uint8_t *skip; // NULL, or pixels the fallback search overwrites (not counted here)
    const uint8_t *Limg; // level image origins (apron buffers), for the wide-span path
    const uint8_t *Rimg;
    int pitch;
    int W, H, Dk, r;
    const int16_t *prior;
    int Wp, Hp;
    int16_t *d_out;
    float *c_out;
    unsigned long long *evals;
    int *err;
    int force_timeout;
    const int2 *rstat;   // the level's right statistics plane (the cell kernel reads it)
    int rspitch;
};

// Arguments of the standalone restricted kernels: the cell kernel (zncc_cell_tile.cuh)
// reads t only; the staged vertical-pair tile (zncc_restricted_tile.cuh, ty = LevelBuf::rty
// rows) also the tensor maps.
struct RestrArgs {
    CUtensorMap tmL;     // box {64, ty + 2n} over the left apron buffer
    CUtensorMap tmR128;  // box {128, ty + 2n} over the right apron buffer
    CUtensorMap tmR256;  // box {256, ty + 2n} over the right apron buffer
    CUtensorMap tmS;     // box {128, ty} over the right statistics plane
    CUtensorMap tmS256;  // box {256, ty} over the right statistics plane
    RestrTileArgs t;
};

cudaError_t launch_apron_copy(const uint8_t *L, const uint8_t *R, size_t spitch, const LevelBuf &lv,
                              cudaStream_t st);

// Fused pyramid launch: levels s+1 .. s+F from level s (index 0 below is level s).
constexpr int PF_MAXF = 3;
struct PyrFuseArgs {
    const uint8_t *src[2];      // level s image origins: the caller's images (s = 0) or apron buffers
    size_t spitch;
    int F;                      // reductions fused, 1 .. PF_MAXF
    int write_src;              // 1: also write level s's apron buffers (s = 0)
    int W[PF_MAXF + 1], H[PF_MAXF + 1];
    uint8_t *dst[PF_MAXF + 1][2];   // apron buffer image origins of levels s .. s+F
    int dpitch[PF_MAXF + 1];
};
cudaError_t launch_pyr_fused(const PyrFuseArgs &a, cudaStream_t st);
cudaError_t launch_level_extract(const LevelBuf &lv, int which, uint8_t *out, cudaStream_t st);
cudaError_t launch_zncc_full(const FullArgs &a, int nh, int sx, cudaStream_t st, bool pdl = false);
// Full-range search of the pixels in l.mask only (beta fallback), over the cell list l.cells
// that the gate built; needs l.rstat computed.
cudaError_t launch_zncc_sparse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st);
// Small-level full-range search (one thread per pixel); fits: the full-range tiles of a
// W x H level would not fill the GPU.
bool zncc_coarse_fits(int W, int H, int sms);
cudaError_t launch_zncc_coarse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st, bool pdl = false);
// beta gate of a W x H level from the coarser Wc x Hc cost; cells (NULL: not built): the
// list of 2 x 2 cells with a masked pixel, laid out as LevelBuf::cells.
cudaError_t launch_beta_gate(const float *Cc, int Wc, int Hc, int W, int H, float beta, uint8_t *mask,
                             unsigned *cells, cudaStream_t st);
cudaError_t launch_alpha_refine(const LevelBuf &l, int nh, float alpha, int16_t *d, float *C,
                                unsigned long long *evals, cudaStream_t st);
cudaError_t launch_selective_median(const int16_t *d_in, const float *C, int W, int H, float alpha, int16_t *d_out,
                                    cudaStream_t st);
cudaError_t zncc_full_prepare(int nh, int sx);
// Right-window statistics planes (rstat) of n consecutive levels (lv[0 .. n-1]) in one launch.
cudaError_t launch_level_stats(const LevelBuf *lv, int n, int nh, cudaStream_t st);
cudaError_t zncc_restricted_prepare(int nh);
cudaError_t launch_zncc_restricted(const RestrArgs &a, int nh, cudaStream_t st, bool pdl = false);

}  // namespace msbm
