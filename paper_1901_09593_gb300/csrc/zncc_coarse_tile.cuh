// zncc_coarse_tile.cuh -- one tile of the small-level full-range ZNCC winner-take-all
// (Sec. III-A, Eq. 1-4: every admissible candidate 0 <= z <= min(D_k - 1, x) of every pixel),
// shared by the standalone launch (zncc_coarse.cu) and the batched persistent kernel
// (batch.cu).  A tile is 32 x TY pixels; ZS = 8 / TY threads share a pixel and take every
// ZS-th group of 4 candidates (zncc_region.cuh), so that a small level still spreads over
// many CTAs with short per-thread chains.  The CTA stages the tile's left rows once and, per
// 32-candidate chunk, the right rows and their window statistics.  Each thread keeps its
// best in ascending z with a strict compare; the ZS partial winners of a pixel (adjacent
// lanes) merge as (ordered score, ~z) keys, so exact ties keep the smallest z.
#pragma once

#include <math.h>

#include "msbm_device.cuh"
#include "zncc_region.cuh"

namespace msbm {

constexpr int CO_TX = 32, CO_TY = 8;

template <int NH, int TY = CO_TY>
struct CoarseCfg {
    static constexpr int SLW = CO_TX + 2 * NH, SLH = TY + 2 * NH;      // staged left region
    static constexpr int SLP = (SLW + 3) / 4 * 4 + 4;                   // its row stride: whole words + 1
    static constexpr int SU = CO_TX + region::ZC - 1;                   // right window columns per chunk
    static constexpr int SRW = SU + 2 * NH;                             // staged right columns per chunk
    static constexpr int SRWW = (SRW + 3) / 4 + 2;                      // words per staged right row
    static constexpr size_t al(size_t v) { return (v + 15) / 16 * 16; }
    static constexpr size_t OFF_SR = 16;                                // [0,16): evaluation sum
    static constexpr size_t OFF_SL = OFF_SR + al((size_t)SLH * SRWW * 4);
    static constexpr size_t OFF_VS = OFF_SL + al((size_t)SLH * SLP);
    static constexpr size_t OFF_VQ = OFF_VS + al((size_t)TY * SRW * 4);
    static constexpr size_t OFF_ST = OFF_VQ + al((size_t)TY * SRW * 4);
    static constexpr size_t BYTES = OFF_ST + al((size_t)TY * SU * 8);
};

// Tile (bx, by) of 32 x TY pixels of a W x H level (apron buffers L, R with `pitch`).  sm:
// CoarseCfg<NH, TY>::BYTES bytes, 16-aligned.  blockDim.x == NT == 32 * TY * ZS.  evals (may
// be NULL) gains the tile's evaluations.
template <int NH, int TY = CO_TY, int NT = 256>
__device__ void coarse_tile(const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int Dk, int16_t *d_out,
                            float *c_out, unsigned long long *evals, int bx, int by, uint8_t *sm) {
    using region::ZC;
    using C = CoarseCfg<NH, TY>;
    constexpr int ZS = NT / (CO_TX * TY);          // threads per pixel
    static_assert(ZS * CO_TX * TY == NT && (ZS & (ZS - 1)) == 0, "tile shape");
    constexpr int WIN = 2 * NH + 1, NW = (WIN + 3) / 4;
    constexpr int SLW = C::SLW, SLP = C::SLP, SLH = C::SLH, SU = C::SU, SRW = C::SRW, SRWW = C::SRWW;
    unsigned long long &evsum = *reinterpret_cast<unsigned long long *>(sm);
    uint32_t *sR = reinterpret_cast<uint32_t *>(sm + C::OFF_SR);
    uint8_t *sL = sm + C::OFF_SL;
    int *vs = reinterpret_cast<int *>(sm + C::OFF_VS);
    int *vq = reinterpret_cast<int *>(sm + C::OFF_VQ);
    int2 *stR = reinterpret_cast<int2 *>(sm + C::OFF_ST);
    const int tid = threadIdx.x, zs = tid % ZS, pix = tid / ZS, pr = pix / CO_TX, pc = pix % CO_TX;
    const int x0 = bx * CO_TX, y0 = by * TY;
    const int x = x0 + pc, y = y0 + pr;
    if (tid == 0) evsum = 0ull;
    // the left rows and the first chunk's right rows in one round trip
    region::stage_rows2<SLH, SLW, SLP, SLH, SRW, SRWW * 4, NT>(sL, L, y0 - NH, x0 - NH, reinterpret_cast<uint8_t *>(sR),
                                                           R, y0 - NH, x0 - (ZC - 1) - NH, pitch, W, H);
    __syncthreads();
    uint32_t Lw[WIN][NW];
    const int2 la = region::pack_left_w<NH, SLP>(sL, pr, pc, Lw);
    const int zmax = min(Dk - 1, x);
    const int zmax_tile = min(Dk - 1, min(x0 + CO_TX, W) - 1);
    // the thread walks its candidates in ascending z and keeps the first maximum (strict
    // compare): the best score with the smallest z among exact ties
    float bs = -INFINITY;
    int bz = 0;
    for (int z0 = 0; z0 <= zmax_tile; z0 += ZC) {
        if (z0 > 0) {
            __syncthreads();      // the previous chunk's rows and statistics are consumed
            region::stage_rows<SLH, SRW, SRWW * 4, NT>(reinterpret_cast<uint8_t *>(sR), R, pitch, W, H, y0 - NH,
                                                    x0 - (z0 + ZC - 1) - NH);
            __syncthreads();
        }
        region::window_stats<NH, TY, SU, SRWW * 4, NT>(reinterpret_cast<const uint8_t *>(sR), vs, vq, stR);
#pragma unroll 1
        for (int g = zs; g < ZC / 4 && z0 + 4 * g <= zmax; g += ZS) {
            const int um = pc + ZC - 4 - 4 * g;       // staged column of candidate z0 + 4g + 3
            uint32_t sab[4];
            region::sab4<NH, SRWW>(sR, pr, um, Lw, sab);
#pragma unroll
            for (int o = 3; o >= 0; --o) {               // ascending z
                const int z = z0 + 4 * g + 3 - o;
                const float r = region::rho_of<NH>(sab[o], la, stR[pr * SU + um + o]);
                if (z <= zmax && r > bs) {
                    bs = r;
                    bz = z;
                }
            }
        }
    }
    if constexpr (ZS > 1) {
        // merge the pixel's ZS partial winners (adjacent lanes): best score, then smallest z
        unsigned long long key = wta_key(bs, bz);
#pragma unroll
        for (int m = 1; m < ZS; m <<= 1) {
            const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, key, m);
            key = o > key ? o : key;
        }
        bs = float_from_order_key(static_cast<uint32_t>(key >> 32));
        bz = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(key));
    }
    const bool in = x < W && y < H && zs == 0;
    if (in) {
        const size_t p = (size_t)y * W + x;
        d_out[p] = static_cast<int16_t>(bz);
        if (c_out) c_out[p] = fminf(1.f, fmaxf(-1.f, bs));
    }
    if (evals) {
        const unsigned cnt = __reduce_add_sync(0xFFFFFFFFu, in ? static_cast<unsigned>(zmax + 1) : 0u);
        if ((tid & 31) == 0) atomicAdd(&evsum, static_cast<unsigned long long>(cnt));
        __syncthreads();
        if (tid == 0) atomicAdd(evals, evsum);
    }
}

}  // namespace msbm
