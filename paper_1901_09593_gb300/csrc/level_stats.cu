// level_stats.cu -- the right-window statistics plane of a pyramid level, read by the
// restricted ZNCC search (Sec. III-C; the per-window terms of Eq. 2): for every pixel (y, x)
// of the right image, S = sum of the (2n+1)^2 window (clamp-to-edge) and
// rsqrt(N * sum I^2 - S^2), or 0 for a flat window.  Every right window a restricted
// candidate reads is one entry, computed once instead of once per candidate that reads it.
//
// One launch covers several levels, their 64 x 32 tiles (level_stats_tile.cuh) numbered
// consecutively.  Bound: a few integer operations and 8 bytes written per pixel.
#include <math.h>
#include <string.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "level_stats_tile.cuh"

namespace msbm {

namespace {

constexpr int ST_MAXL = 24;      // planes (levels) per launch

struct StatsArgs {
    int n;                          // levels in this launch
    int first[ST_MAXL + 1];         // first tile of each level; first[n] = total tiles
    int tiles_x[ST_MAXL];
    const uint8_t *R[ST_MAXL];      // image origins (apron buffers)
    int pitch[ST_MAXL], W[ST_MAXL], H[ST_MAXL], opitch[ST_MAXL];
    int2 *out[ST_MAXL];
};

template <int NH>
__global__ void __launch_bounds__(256) level_stats_kernel(const __grid_constant__ StatsArgs a) {
    __shared__ __align__(16) uint8_t sm[StatsCfg<NH>::BYTES];
    int lv = 0;
    while (lv + 1 < a.n && static_cast<int>(blockIdx.x) >= a.first[lv + 1]) ++lv;
    const int tile = blockIdx.x - a.first[lv];
    const int by = tile / a.tiles_x[lv], bx = tile - by * a.tiles_x[lv];
    stats_tile<NH>(a.R[lv], a.pitch[lv], a.W[lv], a.H[lv], a.out[lv], a.opitch[lv], bx, by, sm);
}

template <int NH>
cudaError_t stats_launch(const StatsArgs &a, cudaStream_t st) {
    level_stats_kernel<NH><<<a.first[a.n], 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_level_stats(const LevelBuf *lv, int n, int nh, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    if (n > ST_MAXL) return cudaErrorInvalidValue;
    StatsArgs a;
    memset(&a, 0, sizeof(a));
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const LevelBuf &l = lv[i];
        if (!l.rstat) return cudaErrorInvalidValue;
        a.tiles_x[m] = (l.W + ST_TX - 1) / ST_TX;
        a.first[m + 1] = a.first[m] + a.tiles_x[m] * ((l.H + ST_TY - 1) / ST_TY);
        a.R[m] = l.img(1);
        a.pitch[m] = l.pitch;
        a.W[m] = l.W;
        a.H[m] = l.H;
        a.out[m] = l.rstat;
        a.opitch[m] = l.rspitch;
        ++m;
    }
    a.n = m;
    switch (nh) {
        case 1: return stats_launch<1>(a, st);
        case 2: return stats_launch<2>(a, st);
        case 3: return stats_launch<3>(a, st);
        case 4: return stats_launch<4>(a, st);
        case 5: return stats_launch<5>(a, st);
        case 6: return stats_launch<6>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
