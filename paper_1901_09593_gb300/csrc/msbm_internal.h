// msbm_internal.h -- host-side structures and kernel launchers of libmsbm (not part of
// the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "msbm.h"
#include "msbm_device.cuh"

namespace msbm {

// One pyramid level of both images: two apron buffers (see msbm_device.cuh) plus the
// tensor maps the ZNCC kernels stage tiles with.
struct LevelBuf {
    int W = 0, H = 0, Dk = 0;
    int pitch = 0;               // bytes per buffer row (multiple of 128)
    int rows = 0;                // H + 2*APY
    uint8_t *base[2] = {nullptr, nullptr};  // buffer starts: image pixel (-APY, -APX)
    int16_t *d = nullptr;        // this level's disparity map (levels >= 1)
    float *c = nullptr;          // this level's cost map (levels >= 1)
    // TMA maps over the apron buffers.  Boxes are ROWS = 8 + 2n rows high:
    //   tm64[i]  : 64 bytes wide  (restricted-kernel left tile and narrow right spans)
    //   tm256[i] : 256 bytes wide (wide right spans, full-range right spans)
    //   tmFL[i]  : 32*SX + 32 bytes wide (full-range left tile), SX chosen per level
    CUtensorMap tm64[2];
    CUtensorMap tm256[2];
    CUtensorMap tmFL[2];
    int full_sx = 4;             // full-range tile width 32*full_sx at this level
    int full_zblock = 0;         // full-range z-block (0 = the tile's maximum)
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
};

struct RestrArgs {
    CUtensorMap tmL;     // box {64, 8 + 2n}
    CUtensorMap tmR64;   // box {64, 8 + 2n}
    CUtensorMap tmR256;  // box {256, 8 + 2n}
    RestrTileArgs t;
};

cudaError_t launch_apron_copy(const uint8_t *L, const uint8_t *R, size_t spitch, const LevelBuf &lv,
                              cudaStream_t st);
cudaError_t launch_pyr_reduce(const LevelBuf &src, const LevelBuf &dst, cudaStream_t st);
cudaError_t launch_level_extract(const LevelBuf &lv, int which, uint8_t *out, cudaStream_t st);
cudaError_t launch_zncc_full(const FullArgs &a, int nh, int sx, cudaStream_t st);
cudaError_t zncc_full_prepare(int nh, int sx);
cudaError_t launch_zncc_restricted(const RestrArgs &a, int nh, cudaStream_t st);
size_t zncc_full_smem_bytes(int nh, int sx);

}  // namespace msbm
