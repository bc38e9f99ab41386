// level_stats_tile.cuh -- one 64 x 32 tile of a right-window statistics plane, shared by
// the standalone launch (level_stats.cu) and the batched persistent kernel (batch.cu): for
// every pixel (y, x), S = sum of the (2n+1)^2 window (clamp-to-edge) and rsqrt(N * sum I^2 -
// S^2), or 0 for a flat window (Sec. III-A, Eq. 1-4 terms of the right window).  The image
// rows are staged in shared memory with word loads from the level's apron buffer (whose
// replicated border makes the clamp-to-edge windows of every image pixel plain reads; words
// past the apron feed only pixels outside the image and stay zero), vertical window sums
// slide down 8-row groups of each column, horizontal sums slide along 8-column segments of
// each row, and the tile leaves in coalesced stores.  All sums are exact integers.
#pragma once

#include <math.h>

#include "msbm_device.cuh"

namespace msbm {

constexpr int ST_TX = 64, ST_TY = 32;

template <int NH>
struct StatsCfg {
    static constexpr int SC = ST_TX + 2 * NH, SR = ST_TY + 2 * NH;   // window columns, staged rows
    static constexpr int XO = 4 * ((NH + 3) / 4);                     // staged columns start XO early
    static constexpr int SB = ST_TX + 2 * XO;                         // staged row bytes (word multiple)
    static constexpr int VP = SC + 1;                                 // packed-sum row stride (words)
    static constexpr size_t OFF_VP = (SR * SB + 15) / 16 * 16;
    static constexpr size_t OFF_SO = OFF_VP + (size_t)ST_TY * VP * 4;
    static constexpr int SOP = ST_TX + 1;                            // output row stride (entries)
    static constexpr size_t BYTES = (OFF_SO + (size_t)ST_TY * SOP * 8 + 15) / 16 * 16;
};

// Tile (bx, by) of the plane out (opitch entries per row) of the W x H image R (pitch bytes):
// R is the image origin of an apron buffer (APY rows and APX columns of replicated border,
// 4-byte aligned rows).  sm: StatsCfg<NH>::BYTES bytes, 16-aligned.  blockDim.x == NT.
template <int NH, int NT = 256>
__device__ void stats_tile(const uint8_t *__restrict__ R, int pitch, int W, int H, int2 *__restrict__ out,
                           int opitch, int bx, int by, uint8_t *sm) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN;
    using C = StatsCfg<NH>;
    constexpr int SC = C::SC, SR = C::SR, VP = C::VP, XO = C::XO, SB = C::SB;
    static_assert(NH <= APY && XO <= APX, "windows inside the apron");
    static_assert(NT % 32 == 0 && 256 % NT == 0, "thread count");
    uint32_t (*vp)[VP] = reinterpret_cast<uint32_t (*)[VP]>(sm + C::OFF_VP);   // q | s << 20 per column window
    int2 (*so)[C::SOP] = reinterpret_cast<int2 (*)[C::SOP]>(sm + C::OFF_SO);
    const int x0 = bx * ST_TX, y0 = by * ST_TY, tid = threadIdx.x;
    {
        constexpr int NWR = SB / 4, NWT = SR * NWR, T = (NWT + NT - 1) / NT;
        uint32_t v[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t, r = i / NWR, w = i - r * NWR;
            const int Y = y0 - NH + r, X = x0 - XO + 4 * w;
            v[t] = (i < NWT && Y < H + APY && X + 3 < W + APX)
                       ? __ldg(reinterpret_cast<const uint32_t *>(R + (ptrdiff_t)Y * pitch + X))
                       : 0u;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t;
            if (i < NWT) reinterpret_cast<uint32_t *>(sm)[i] = v[t];
        }
    }
    // window column c of the old layout (image column x0 - NH + c) is staged byte c + XO - NH
    const uint8_t *sb = sm + (XO - NH);
    __syncthreads();
    // vertical: column c, rows 8g .. 8g+7
    for (int i = tid; i < SC * (ST_TY / 8); i += NT) {
        const int g = i / SC, c = i - g * SC;
        uint32_t s = 0, q = 0;
#pragma unroll
        for (int t = 0; t < WIN; ++t) {
            const uint32_t v = sb[(8 * g + t) * SB + c];
            s += v;
            q += v * v;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            vp[8 * g + r][c] = q | (s << 20);      // s < 4096, q < 2^20 for windows up to 13 x 13
            if (r < 7) {
                const uint32_t a = sb[(8 * g + r + WIN) * SB + c], b = sb[(8 * g + r) * SB + c];
                s += a - b;
                q += a * a - b * b;
            }
        }
    }
    __syncthreads();
    // horizontal: row r, columns 8g .. 8g+7 (256 items; the odd packed-sum row stride and the
    // padded output stride keep a warp's 32 rows on distinct banks)
    for (int g = tid >> 5; g < 8; g += NT / 32) {
        const int r = tid & 31;                    // a warp: one segment of 32 rows
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
    for (int t = 0; t < ST_TX * ST_TY / NT; ++t) {
        const int i = tid + NT * t, r = i / ST_TX, c = i % ST_TX;
        if (y0 + r < H && x0 + c < W) out[(size_t)(y0 + r) * opitch + x0 + c] = so[r][c];
    }
}

}  // namespace msbm
