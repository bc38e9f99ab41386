// level_stats.cu -- the window statistics plane of a pyramid level's right image, read by the
// restricted ZNCC search (Sec. III-C, Eq. 1-4 terms of the right window): for every pixel
// (y, x), S = sum of the (2n+1)^2 window (clamp-to-edge) and rsqrt(N * sum I^2 - S^2), or
// 0 for a flat window.  Every right window a restricted candidate reads is one entry, so the
// matching kernel does no window statistics of its own.
//
// Per CTA a 64 x 32 tile of one level (one launch covers several levels, their tiles numbered
// consecutively): the image rows are staged in shared memory (coordinates clamped to the
// image), vertical window sums slide down 8-row groups of each column, horizontal sums slide
// along 8-column segments of each row, and the tile leaves in coalesced stores.  All sums are
// exact integers.  Bound: a few integer operations and 8 bytes written per pixel.
#include <math.h>
#include <string.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {

namespace {

constexpr int ST_TX = 64, ST_TY = 32;

constexpr int ST_MAXL = 16;

struct StatsArgs {
    int n;                          // levels in this launch
    int first[ST_MAXL + 1];         // first tile of each level; first[n] = total tiles
    int tiles_x[ST_MAXL];
    const uint8_t *R[ST_MAXL];      // right image origins (apron buffers)
    int pitch[ST_MAXL], W[ST_MAXL], H[ST_MAXL], opitch[ST_MAXL];
    int2 *out[ST_MAXL];
};

template <int NH>
__global__ void __launch_bounds__(256) right_stats_kernel(const __grid_constant__ StatsArgs a) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN;
    int lv = 0;
    while (lv + 1 < a.n && static_cast<int>(blockIdx.x) >= a.first[lv + 1]) ++lv;
    const int tile = blockIdx.x - a.first[lv];
    const uint8_t *__restrict__ R = a.R[lv];
    const int pitch = a.pitch[lv], W = a.W[lv], H = a.H[lv], opitch = a.opitch[lv];
    int2 *__restrict__ out = a.out[lv];
    constexpr int SC = ST_TX + 2 * NH, SR = ST_TY + 2 * NH;   // staged columns, rows
    constexpr int VP = SC + 1;                                 // packed-sum row stride (words)
    __shared__ uint8_t sb[SR][SC];
    __shared__ uint32_t vp[ST_TY][VP];                         // q | s << 20 of each column window
    __shared__ int2 so[ST_TY][ST_TX];
    const int by = tile / a.tiles_x[lv], bx = tile - by * a.tiles_x[lv];
    const int x0 = bx * ST_TX, y0 = by * ST_TY, tid = threadIdx.x;
    {
        constexpr int T = (SR * SC + 255) / 256;
        uint8_t v[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t, r = i / SC, c = i - r * SC;
            const int yy = min(max(y0 - NH + r, 0), H - 1), xx = min(max(x0 - NH + c, 0), W - 1);
            v[t] = i < SR * SC ? __ldg(R + (ptrdiff_t)yy * pitch + xx) : 0;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            if (i < SR * SC) sb[i / SC][i % SC] = v[t];
        }
    }
    __syncthreads();
    // vertical: column c, rows 8g .. 8g+7
    for (int i = tid; i < SC * (ST_TY / 8); i += 256) {
        const int g = i / SC, c = i - g * SC;
        uint32_t s = 0, q = 0;
#pragma unroll
        for (int t = 0; t < WIN; ++t) {
            const uint32_t v = sb[8 * g + t][c];
            s += v;
            q += v * v;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            vp[8 * g + r][c] = q | (s << 20);      // s < 4096, q < 2^20 for windows up to 13 x 13
            if (r < 7) {
                const uint32_t a = sb[8 * g + r + WIN][c], b = sb[8 * g + r][c];
                s += a - b;
                q += a * a - b * b;
            }
        }
    }
    __syncthreads();
    // horizontal: row r, columns 8g .. 8g+7 (256 items)
    {
        const int r = tid >> 3, g = tid & 7;
        const uint32_t *row = &vp[r][8 * g];
        int s = 0, q = 0;
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
            s += static_cast<int>(row[j] >> 20);
            q += static_cast<int>(row[j] & 0xFFFFFu);
        }
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int V = N * q - s * s;
            so[r][8 * g + x] = make_int2(s, V > 0 ? __float_as_int(rsqrtf(static_cast<float>(V))) : 0);
            if (x < 7) {
                s += static_cast<int>(row[x + WIN] >> 20) - static_cast<int>(row[x] >> 20);
                q += static_cast<int>(row[x + WIN] & 0xFFFFFu) - static_cast<int>(row[x] & 0xFFFFFu);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < ST_TX * ST_TY / 256; ++t) {
        const int i = tid + 256 * t, r = i / ST_TX, c = i % ST_TX;
        if (y0 + r < H && x0 + c < W) out[(size_t)(y0 + r) * opitch + x0 + c] = so[r][c];
    }
}

template <int NH>
cudaError_t stats_launch(const StatsArgs &a, cudaStream_t st) {
    right_stats_kernel<NH><<<a.first[a.n], 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_right_stats(const LevelBuf *lv, int n, int nh, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    if (n > ST_MAXL) return cudaErrorInvalidValue;
    StatsArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    for (int i = 0; i < n; ++i) {
        const LevelBuf &l = lv[i];
        if (!l.rstat) return cudaErrorInvalidValue;
        a.tiles_x[i] = (l.W + ST_TX - 1) / ST_TX;
        a.first[i + 1] = a.first[i] + a.tiles_x[i] * ((l.H + ST_TY - 1) / ST_TY);
        a.R[i] = l.img(1);
        a.pitch[i] = l.pitch;
        a.W[i] = l.W;
        a.H[i] = l.H;
        a.out[i] = l.rstat;
        a.opitch[i] = l.rspitch;
    }
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
