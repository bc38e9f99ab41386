// zncc_restricted_px_tile.cuh -- the restricted ZNCC winner-take-all tile with one thread per
// pixel (32 x 8 pixels per CTA), used by the standalone restricted kernel.  The batched kernel
// uses the 2 x 2-block tile of zncc_restricted_tile.cuh, which amortises its per-tile work
// over four times the pixels but leaves small and mid-size levels with too few CTAs.
// The refinement search at a finer pyramid level (Sec. III-C, Eq. 8-9,
// first branch): each pixel evaluates only dhat - r .. dhat + r around the nearest-
// neighbour upsample dhat = 2 * d^{k+1}(y/2, x/2) of the coarser disparity (the paper's
// "3 comparisons per pixel" is r = 1), clipped to 0 .. min(D_k - 1, x).
//
// Design (per CTA: 32 x 8 pixels, one thread per pixel):
//  * Each thread reads its prior; the CTA reduces the union [zlo, zhi] of its pixels'
//    candidate spans.  The left tile and the right span [x0 - zhi - n, x1 - zlo + n] are
//    staged into shared memory by TMA (one 64-byte box for the left tile, one 64- or
//    256-byte box for the right span, one mbarrier, bounded wait).  A span wider than
//    256 bytes (a tile straddling a large disparity jump) reads the right image straight
//    from global memory instead.
//  * Right-window statistics for the span are built once per CTA with separable sums.
//  * Each thread packs its left window (2n+1 rows of ceil((2n+1)/4) words, zero-padded)
//    into registers and gets Sa, Saa with dp4a.  For each window row it loads the right
//    bytes covering a group of G consecutive candidates once, aligns them with funnel
//    shifts, and accumulates sum a*b for every candidate of the group with dp4a.  All sums
//    are exact int32 (windows up to 13 x 13); c = N*Sab - Sa*Sb is exact; the only
//    rounding is rho = float(c) * rsqrt(Va) * rsqrt(Vb).
//  * WTA on a 64-bit (ordered rho, ~z) key, so exact ties keep the smallest z.
// Bound: the integer dot-product pipe (about 2*ceil((2n+1)/4)*(2n+1) dp4a + shifts per
// evaluation); HBM traffic is a few bytes per pixel.
#pragma once

#include <limits.h>
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {
namespace tiles {


constexpr int PX_TX = 32;
constexpr int PX_TY = 8;

template <int NH>
struct RCfgPx {
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int N = WIN * WIN;
    static constexpr int NW = (WIN + 3) / 4;     // words per packed window row
    static constexpr int ROWS = PX_TY + 2 * NH;
    static constexpr uint32_t LASTMASK =
        (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    // shared memory carve (bytes): [0,128) barrier, flag, span scalars, evaluation sum
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t OFF_SL = 128;
    static constexpr size_t OFF_SR = OFF_SL + al((size_t)ROWS * 64);
    static constexpr size_t OFF_TMP = OFF_SR + al((size_t)(ROWS + 1) * 256);
    static constexpr size_t OFF_STR = OFF_TMP + (size_t)PX_TY * 256 * 8;
    static constexpr size_t BYTES = OFF_STR + (size_t)PX_TY * 256 * 8;
};

__device__ __forceinline__ uint32_t fsr_px(uint32_t lo, uint32_t hi, int bytes) {
    return __funnelshift_r(lo, hi, 8 * bytes);
}

// Restricted WTA of one 32 x 8 tile (bx, by) by the calling CTA (blockDim.x = 256, one
// thread per pixel).  `smem` holds RCfg::BYTES bytes, 128-aligned; its first 8 bytes are an
// mbarrier the caller has initialised (count 1) and `parity` is its next phase parity,
// advanced here.  Returns false if a bounded wait gave up (the error word is then set).
template <int NH, int G>
__device__ bool restr_tile_px(const RestrTileArgs &a, const CUtensorMap *tmL, const CUtensorMap *tmR64,
                           const CUtensorMap *tmR256, int bx, int by, uint8_t *smem, uint32_t &parity) {
    using C = RCfgPx<NH>;
    constexpr int ROWS = C::ROWS, WIN = C::WIN, NW = C::NW;
    // right bytes per row for one candidate group (after alignment) and words to load
    constexpr int GB = G - 1 + WIN;
    constexpr int NWA = (GB + 3) / 4 + 1;     // aligned words after the shift
    constexpr int NWL = NWA + 1;              // raw words loaded
    uint64_t &bar = *reinterpret_cast<uint64_t *>(smem);
    int &flag = *reinterpret_cast<int *>(smem + 8);
    int &zlo_s = *reinterpret_cast<int *>(smem + 12);
    int &zhi_s = *reinterpret_cast<int *>(smem + 16);
    int &mode_s = *reinterpret_cast<int *>(smem + 20);
    int &xs_s = *reinterpret_cast<int *>(smem + 24);
    unsigned long long &evsum = *reinterpret_cast<unsigned long long *>(smem + 32);
    uint8_t (*sL)[64] = reinterpret_cast<uint8_t (*)[64]>(smem + C::OFF_SL);
    // right span: ROWS rows of 64 (narrow box) or 256 (wide box) bytes, plus one spare
    // row so that a candidate group's over-read past the last row stays in the array
    uint8_t *sR = smem + C::OFF_SR;
    int2 (*tmpV)[256] = reinterpret_cast<int2 (*)[256]>(smem + C::OFF_TMP);
    int2 (*stR)[256] = reinterpret_cast<int2 (*)[256]>(smem + C::OFF_STR);   // {Sb, bits(rsqrt(Vb))}

    const int tid = threadIdx.x, tx = tid & (PX_TX - 1), ty = tid / PX_TX;
    const int x0 = bx * PX_TX, y0 = by * PX_TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < a.W && y < a.H;
    const int Dk = a.Dk;

    int lo = INT_MAX, hi = -1;
    if (active) {
        int zmx = min(Dk - 1, x);
        int py = min(y >> 1, a.Hp - 1), px = min(x >> 1, a.Wp - 1);
        int dh = 2 * static_cast<int>(a.prior[(size_t)py * a.Wp + px]);
        dh = min(max(dh, 0), zmx);
        lo = max(0, dh - a.r);
        hi = min(zmx, dh + a.r);
    }
    if (tid == 0) {
        zlo_s = INT_MAX; zhi_s = -1; evsum = 0ull;
    }
    __syncthreads();
    {
        int wlo = __reduce_min_sync(0xFFFFFFFFu, lo);
        int whi = __reduce_max_sync(0xFFFFFFFFu, hi);
        unsigned cnt = (active && !(a.skip && a.skip[(size_t)y * a.W + x])) ? static_cast<unsigned>(hi - lo + 1) : 0u;
        unsigned wcnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (tx == 0) {
            atomicMin(&zlo_s, wlo);
            atomicMax(&zhi_s, whi);
            atomicAdd(&evsum, static_cast<unsigned long long>(wcnt));
        }
    }
    __syncthreads();
    const int zlo = zlo_s, zhi = zhi_s;
    const int xlast = min(x0 + PX_TX, a.W) - 1;
    const int rs = x0 - zhi - NH;              // first right column any window reads
    const int re = xlast - zlo + NH;           // last
    if (tid == 0) {
        int xs = (rs + APX) & ~15;
        int width = re + APX + 1 - xs;
        int mode = width <= 64 ? 1 : (width <= 256 ? 2 : 0);
        mode_s = mode;
        xs_s = xs;
        uint32_t bytes = ROWS * 64 + (mode == 1 ? ROWS * 64 : (mode == 2 ? ROWS * 256 : 0));
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, bytes);
        tma_load_2d(&sL[0][0], tmL, &bar, x0 - 16 + APX, y0 - NH + APY);
        if (mode == 1) tma_load_2d(sR, tmR64, &bar, xs, y0 - NH + APY);
        if (mode == 2) tma_load_2d(sR, tmR256, &bar, xs, y0 - NH + APY);
    }
    if (!tma_batch_wait(&bar, parity, &flag, a.force_timeout != 0, a.err)) return false;
    parity ^= 1;
    const int mode = mode_s, xs = xs_s;
    const int soff = APX - xs;                 // staging column of image column X: X + soff
    const int rst = mode == 1 ? 64 : 256;      // staging row stride

    // ---- right statistics over the span (staged modes)
    const int SW = re - rs + 1 - 2 * NH;       // statistics columns: image rs + n + v
    if (mode != 0) {
        for (int c = tid; c < SW + 2 * NH; c += PX_TX * PX_TY) {
            const int col = rs + c + soff;
            int s = 0, q = 0;
#pragma unroll
            for (int t = 0; t < WIN; ++t) { int v = sR[t * rst + col]; s += v; q += v * v; }
            tmpV[0][c] = make_int2(s, q);
#pragma unroll 1
            for (int ry = 1; ry < PX_TY; ++ry) {
                int vn = sR[(ry + 2 * NH) * rst + col], vo = sR[(ry - 1) * rst + col];
                s += vn - vo;
                q += vn * vn - vo * vo;
                tmpV[ry][c] = make_int2(s, q);
            }
        }
        __syncthreads();
        for (int i = tid; i < PX_TY * SW; i += PX_TX * PX_TY) {
            int ry = i / SW, v = i - ry * SW;
            int s = 0, q = 0;
#pragma unroll
            for (int j = 0; j < WIN; ++j) { int2 t = tmpV[ry][v + j]; s += t.x; q += t.y; }
            int V = C::N * q - s * s;
            float r = V > 0 ? rsqrtf(static_cast<float>(V)) : 0.f;
            stR[ry][v] = make_int2(s, __float_as_int(r));
        }
        __syncthreads();
    }
    if (!active) return true;

    // ---- left window, packed: row t holds columns x-n .. x+n in NW words
    uint32_t Lw[WIN][NW];
    uint32_t Sa = 0, Saa = 0;
    {
        const int sc = tx + 16 - NH;           // staging column of x - n
        const int w0 = sc >> 2, sh = sc & 3;
#pragma unroll
        for (int t = 0; t < WIN; ++t) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(&sL[ty + t][0]);
            uint32_t raw[NW + 1];
#pragma unroll
            for (int k = 0; k <= NW; ++k) raw[k] = row[w0 + k];
#pragma unroll
            for (int k = 0; k < NW; ++k) Lw[t][k] = fsr_px(raw[k], raw[k + 1], sh);
            Lw[t][NW - 1] &= C::LASTMASK;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                Sa = dp4a_u8(Lw[t][k], 0x01010101u, Sa);
                Saa = dp4a_u8(Lw[t][k], Lw[t][k], Saa);
            }
        }
    }
    const int Va = C::N * static_cast<int>(Saa) - static_cast<int>(Sa) * static_cast<int>(Sa);
    const float rA = Va > 0 ? rsqrtf(static_cast<float>(Va)) : 0.f;

    unsigned long long bestk = 0ull;
    if (mode != 0) {
        // groups of G candidates, walking down from hi: group covers z = zg - j, j < G
        for (int zg = hi; zg >= lo; zg -= G) {
            uint32_t acc[G];
#pragma unroll
            for (int j = 0; j < G; ++j) acc[j] = 0;
            // staging column of the first byte of candidate j's window: sc0 + j
            const int sc0 = x - zg - NH + soff;
            const int w0 = sc0 >> 2, sh = sc0 & 3;
#pragma unroll
            for (int t = 0; t < WIN; ++t) {
                const uint32_t *row = reinterpret_cast<const uint32_t *>(sR + (ty + t) * rst);
                uint32_t raw[NWL], al[NWA];
#pragma unroll
                for (int k = 0; k < NWL; ++k) raw[k] = row[w0 + k];
#pragma unroll
                for (int k = 0; k < NWA; ++k) al[k] = fsr_px(raw[k], raw[k + 1], sh);
#pragma unroll
                for (int j = 0; j < G; ++j) {
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        uint32_t b = (j & 3) ? fsr_px(al[(j >> 2) + k], al[(j >> 2) + k + 1], j & 3)
                                             : al[(j >> 2) + k];
                        acc[j] = dp4a_u8(Lw[t][k], b, acc[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int z = zg - j;
                if (z < lo) break;
                const int2 st = stR[ty][x - z - (rs + NH)];
                const int c = C::N * static_cast<int>(acc[j]) - static_cast<int>(Sa) * st.x;
                const float rho = static_cast<float>(c) * rA * __int_as_float(st.y);
                unsigned long long k = wta_key(rho, z);
                bestk = k > bestk ? k : bestk;
            }
        }
    } else {
        // wide span: read the right image from global memory (apron buffer, no clamping)
        for (int z = lo; z <= hi; ++z) {
            uint32_t Sab = 0, Sb = 0, Sbb = 0;
#pragma unroll
            for (int t = 0; t < WIN; ++t) {
                const uint8_t *rrow = a.Rimg + (ptrdiff_t)(y - NH + t) * a.pitch + (x - z - NH);
                uint32_t raw[NW];
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    uint32_t w = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (4 * k + b < WIN) w |= static_cast<uint32_t>(__ldg(rrow + 4 * k + b)) << (8 * b);
                    raw[k] = w;
                }
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    Sab = dp4a_u8(Lw[t][k], raw[k], Sab);
                    Sb = dp4a_u8(raw[k], 0x01010101u, Sb);
                    Sbb = dp4a_u8(raw[k], raw[k], Sbb);
                }
            }
            const int Vb = C::N * static_cast<int>(Sbb) - static_cast<int>(Sb) * static_cast<int>(Sb);
            const float rB = Vb > 0 ? rsqrtf(static_cast<float>(Vb)) : 0.f;
            const int c = C::N * static_cast<int>(Sab) - static_cast<int>(Sa) * static_cast<int>(Sb);
            const float rho = static_cast<float>(c) * rA * rB;
            unsigned long long k = wta_key(rho, z);
            bestk = k > bestk ? k : bestk;
        }
    }
    const int z = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(bestk & 0xFFFFFFFFull));
    float rho = float_from_order_key(static_cast<uint32_t>(bestk >> 32));
    rho = fminf(1.f, fmaxf(-1.f, rho));
    a.d_out[(size_t)y * a.W + x] = static_cast<int16_t>(z);
    if (a.c_out) a.c_out[(size_t)y * a.W + x] = rho;
    if (tid == 0 && a.evals) atomicAdd(a.evals, evsum);
    return true;
}

}  // namespace tiles
}  // namespace msbm
