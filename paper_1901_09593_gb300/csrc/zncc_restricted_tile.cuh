// zncc_restricted_tile.cuh -- the restricted ZNCC winner-take-all tile (Sec. III-C,
// Eq. 8-9, first branch), shared by the standalone kernel (zncc_restricted.cu) and the
// batched persistent kernel (batch.cu).  Each pixel evaluates dhat - r .. dhat + r around
// the nearest-neighbour upsample dhat = 2 * d^{k+1}(y/2, x/2) of the coarser disparity (the
// paper's "3 comparisons per pixel" is r = 1), clipped to 0 .. min(D_k - 1, x); dhat is
// first clamped into that range (a no-op for priors produced by the coarser level).
//
// Design (per CTA: a (NCOL*QX) x TY pixel tile, TY = 16 or 8, of QX x TY/2 threads; each thread owns an
// NCOL x 2 block of pixels, NCOL = 2 (2 x 2 blocks) or 1 (vertical pairs)):
//  * The pixels of a block aligned to even coordinates share one prior cell, hence one
//    candidate span (up to the per-pixel clip at x, handled by masking).
//  * The CTA reduces the union [zlo, zhi] of its spans; the left tile (a (TX+32)-byte box) and the
//    right span [x0 - zhi - n, x1 - zlo + n] (128- or 256-byte box) are staged into shared
//    memory by TMA with one mbarrier and a bounded wait.  A span wider than 256 bytes (a
//    tile straddling a large disparity jump) reads the right image from global memory.
//  * Right-window statistics of the span are built once per CTA by all threads (vertical
//    sums, then horizontal sums; exact integers), or, in plane mode, staged by TMA with the
//    image rows from the level's precomputed statistics plane.
//  * Each thread packs the 2n+2 left rows of its columns as dp4a words.  For each staged
//    right row and each group of G consecutive candidates it loads the right bytes once,
//    aligns them with funnel shifts, extracts the G+NCOL-1 distinct window offsets its
//    columns need, and accumulates sum a*b with dp4a.  The two pixels of a column share
//    the products of their 2n common rows.  All sums are exact int32 (windows up to
//    13 x 13); c = N*Sab - Sa*Sb is exact; the only rounding is
//    rho = float(c) * rsqrt(Vb) * rsqrt(Va).
//  * WTA in ascending z with a strict compare, so exact ties keep the smallest z.
// Bound: the integer dot-product pipe; HBM traffic is a few bytes per pixel.
#pragma once

#include <limits.h>
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {
namespace tiles {

constexpr int RT_TY = 16;      // default tile height (pixels)

template <int NH, int QX = 32, int NCOL = 2, bool PLANE = false, int TY = RT_TY>
struct RCfg {
    static_assert(TY == 8 || TY == 16, "tile height");
    static constexpr int TX = NCOL * QX;         // tile width (pixels)
    static constexpr int THREADS = QX * (TY / 2);
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int N = WIN * WIN;
    static constexpr int NW = (WIN + 3) / 4;     // words per packed window row
    static constexpr int ROWS = TY + 2 * NH;     // staged rows
    static constexpr int LBOX = TX + 32;         // left box: image columns x0-16 .. x0+TX+16
    static constexpr uint32_t LASTMASK =
        (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    // shared memory carve (bytes): [0,128) barrier, flag, span scalars, evaluation sum
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t OFF_SL = 128;
    static constexpr size_t PAD_R = 128;         // readable slack before the right span
    static constexpr size_t OFF_SR = OFF_SL + al((size_t)ROWS * LBOX) + PAD_R;
    static constexpr size_t OFF_TMP = OFF_SR + al((size_t)(ROWS + 1) * 256);
    static constexpr size_t OFF_STR = OFF_TMP + (size_t)TY * 256 * 4;
    // plane mode stages the span's entries of the level's statistics plane at OFF_TMP instead
    static constexpr size_t OFF_SS = OFF_TMP;
    static constexpr size_t BYTES = PLANE ? OFF_SS + (size_t)TY * 256 * 8 : OFF_STR + (size_t)TY * 256 * 8;
};

__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, int bytes) {
    return __funnelshift_r(lo, hi, 8 * bytes);
}

// Restricted WTA of one (NCOL*QX) x TY tile (bx, by) by the calling CTA (blockDim.x = QX*TY/2).
// `smem` holds RCfg::BYTES bytes, 128-aligned; its first 8 bytes are an mbarrier the caller
// has initialised (count 1) and `parity` is its next phase parity, advanced here.  tmL is a
// (NCOL*QX + 32)-byte-wide box over the left apron buffer, tmR128/tmR256 128/256-byte boxes
// over the right one.  PLANE: the right-window statistics are staged by TMA from the level's
// statistics plane (tmS128 / tmS256: 128 / 256 x 16 boxes of 8-byte entries) instead of being
// built in the CTA.  Returns false if a bounded wait gave up (the error word is then set).
template <int NH, int G, int QX = 32, int NCOL = 2, bool PLANE = false, int TY = RT_TY>
__device__ bool restr_tile(const RestrTileArgs &a, const CUtensorMap *tmL, const CUtensorMap *tmR128,
                           const CUtensorMap *tmR256, const CUtensorMap *tmS128, const CUtensorMap *tmS256,
                           int bx, int by, uint8_t *smem, uint32_t &parity) {
    using C = RCfg<NH, QX, NCOL, PLANE, TY>;
    constexpr int RT_TX = C::TX, RT_THREADS = C::THREADS;
    constexpr int ROWS = C::ROWS, WIN = C::WIN, NW = C::NW;
    // right bytes one row of a candidate group needs for both columns: G + WIN, plus up to
    // 3 of misalignment; NWA aligned words hold them with one word to spare for extraction
    constexpr int NO = G + NCOL - 1;          // distinct window offsets of a candidate group
    constexpr int NWA = (NO - 1 + WIN + 3) / 4 + 1;
    constexpr int NWL = NWA + 1;              // raw words loaded per row
    uint64_t &bar = *reinterpret_cast<uint64_t *>(smem);
    int &flag = *reinterpret_cast<int *>(smem + 8);
    int &zlo_s = *reinterpret_cast<int *>(smem + 12);
    int &zhi_s = *reinterpret_cast<int *>(smem + 16);
    int &mode_s = *reinterpret_cast<int *>(smem + 20);
    int &xs_s = *reinterpret_cast<int *>(smem + 24);
    unsigned long long &evsum = *reinterpret_cast<unsigned long long *>(smem + 32);
    uint8_t *sL = smem + C::OFF_SL;                       // [ROWS][LBOX]
    uint8_t *sR = smem + C::OFF_SR;                       // [ROWS + 1][64|128|256] + slack before
    uint32_t *tmpV = reinterpret_cast<uint32_t *>(smem + C::OFF_TMP);   // [TY][256] packed (Q | S << 20)
    int2 *stR = reinterpret_cast<int2 *>(smem + C::OFF_STR);           // [TY][256] {Sb, bits(rsqrt(Vb))}
    const int2 *stS = reinterpret_cast<const int2 *>(smem + C::OFF_SS);  // plane mode: [TY][128|256]

    const int tid = threadIdx.x, qx = tid % QX, qy = tid / QX;
    const int x0 = bx * RT_TX, y0 = by * TY;
    const int xa = x0 + NCOL * qx, ya = y0 + 2 * qy;    // top-left pixel of this thread's block
    const int Dk = a.Dk;
    bool colv[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) colv[c] = xa + c < a.W;
    const bool rowv[2] = {ya < a.H, ya + 1 < a.H};
    const bool any = colv[0] && rowv[0];

    // candidate spans of the two columns (rows share them)
    int lo_c[NCOL], hi_c[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
        lo_c[c] = INT_MAX;
        hi_c[c] = -1;
    }
    if (any) {
        const int py = min(ya >> 1, a.Hp - 1), px = min(xa >> 1, a.Wp - 1);
        const int p2 = 2 * static_cast<int>(a.prior[(size_t)py * a.Wp + px]);
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            if (!colv[c]) continue;
            const int zmx = min(Dk - 1, xa + c);
            const int dh = min(max(p2, 0), zmx);
            lo_c[c] = max(0, dh - a.r);
            hi_c[c] = min(zmx, dh + a.r);
        }
    }
    int lo_u = lo_c[0], hi_u = hi_c[0];
#pragma unroll
    for (int c = 1; c < NCOL; ++c) {
        lo_u = min(lo_u, lo_c[c]);
        hi_u = max(hi_u, hi_c[c]);
    }
    if (tid == 0) {
        zlo_s = INT_MAX; zhi_s = -1; evsum = 0ull;
    }
    __syncthreads();
    {
        const int wlo = __reduce_min_sync(0xFFFFFFFFu, lo_u);
        const int whi = __reduce_max_sync(0xFFFFFFFFu, hi_u);
        unsigned cnt = 0;
#pragma unroll
        for (int c = 0; c < NCOL; ++c)
#pragma unroll
            for (int r2 = 0; r2 < 2; ++r2)
                if (colv[c] && rowv[r2] && !(a.skip && a.skip[(size_t)(ya + r2) * a.W + xa + c]))
                    cnt += static_cast<unsigned>(hi_c[c] - lo_c[c] + 1);
        const unsigned wcnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if ((tid & 31) == 0) {
            atomicMin(&zlo_s, wlo);
            atomicMax(&zhi_s, whi);
            atomicAdd(&evsum, static_cast<unsigned long long>(wcnt));
        }
    }
    __syncthreads();
    const int zlo = zlo_s, zhi = zhi_s;
    const int xlast = min(x0 + RT_TX, a.W) - 1;
    const int rs = x0 - zhi - NH;              // first right column any window reads
    const int re = xlast - zlo + NH;           // last
    const int sxs = (x0 - zhi) & ~1;           // plane mode: first staged plane column (even)
    if (tid == 0) {
        const int xs = (rs + APX) & ~15;
        const int width = re + APX + 1 - xs;
        const int mode = width <= 128 ? 1 : (width <= 256 ? 2 : 0);
        mode_s = mode;
        xs_s = xs;
        uint32_t bytes = ROWS * C::LBOX + (mode == 1 ? ROWS * 128 : (mode == 2 ? ROWS * 256 : 0));
        if (PLANE) bytes += mode == 1 ? TY * 128 * 8 : (mode == 2 ? TY * 256 * 8 : 0);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, bytes);
        tma_load_2d(sL, tmL, &bar, x0 - 16 + APX, y0 - NH + APY);
        if (mode == 1) tma_load_2d(sR, tmR128, &bar, xs, y0 - NH + APY);
        if (mode == 2) tma_load_2d(sR, tmR256, &bar, xs, y0 - NH + APY);
        if (PLANE && mode == 1) tma_load_2d(const_cast<int2 *>(stS), tmS128, &bar, sxs, y0);
        if (PLANE && mode == 2) tma_load_2d(const_cast<int2 *>(stS), tmS256, &bar, sxs, y0);
    }
    if (!tma_batch_wait(&bar, parity, &flag, a.force_timeout != 0, a.err)) return false;
    parity ^= 1;
    const int mode = mode_s, xs = xs_s;
    const int soff = APX - xs;                 // staging column of image column X: X + soff
    const int rst = mode == 1 ? 128 : 256;     // staging row stride (bytes; plane entries)

    // ---- right statistics over the span (staged modes, no plane), all threads
    const int SW = re - rs + 1 - 2 * NH;       // statistics columns: image rs + n + v
    if (!PLANE && mode != 0) {
        // vertical window sums of every (output row, span column), spread over all threads
        const int cols = SW + 2 * NH;
        for (int i = tid; i < TY * cols; i += RT_THREADS) {
            const int ry = i / cols, c = i - ry * cols;
            const uint8_t *p = sR + ry * rst + rs + c + soff;
            uint32_t s = 0, q = 0;
#pragma unroll
            for (int t = 0; t < WIN; ++t) {
                const uint32_t v = p[t * rst];
                s += v;
                q += v * v;
            }
            tmpV[ry * 256 + c] = q | (s << 20);    // s < 4096, q < 2^20 for windows <= 13
        }
        __syncthreads();
        // horizontal sums, then rsqrt of the window variance
        for (int i = tid; i < TY * SW; i += RT_THREADS) {
            const int ry = i / SW, v = i - ry * SW;
            int s = 0, q = 0;
#pragma unroll
            for (int j = 0; j < WIN; ++j) {
                const uint32_t t = tmpV[ry * 256 + v + j];
                s += static_cast<int>(t >> 20);
                q += static_cast<int>(t & 0xFFFFFu);
            }
            const int V = C::N * q - s * s;
            const float r = V > 0 ? rsqrtf(static_cast<float>(V)) : 0.f;
            stR[ry * 256 + v] = make_int2(s, __float_as_int(r));
        }
        __syncthreads();
    }
    if (!any) return true;

    // ---- left windows: rows ya-n .. ya+1+n (2n+2) of columns xa and xa+1, packed
    uint32_t Lw[NCOL][WIN + 1][NW];
    int Sa[NCOL][2], rAi[NCOL][2];
    float rA[NCOL][2];
    {
        const int sc = NCOL * qx + 16 - NH;    // staging column of xa - n
        const int w0 = sc >> 2, sh = sc & 3;
#pragma unroll
        for (int t = 0; t <= WIN; ++t) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(sL + (2 * qy + t) * C::LBOX);
            uint32_t raw[NW + 2];
#pragma unroll
            for (int k = 0; k < NW + 2; ++k) raw[k] = row[w0 + k];
            uint32_t alw[NW + 1];
#pragma unroll
            for (int k = 0; k <= NW; ++k) alw[k] = fsr(raw[k], raw[k + 1], sh);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                Lw[0][t][k] = alw[k];
                if constexpr (NCOL == 2) Lw[NCOL - 1][t][k] = fsr(alw[k], alw[k + 1], 1);
            }
#pragma unroll
            for (int c = 0; c < NCOL; ++c) Lw[c][t][NW - 1] &= C::LASTMASK;
        }
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            uint32_t s_mid = 0, q_mid = 0, s0 = 0, q0 = 0, s1 = 0, q1 = 0;
#pragma unroll
            for (int t = 1; t < WIN; ++t)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    s_mid = dp4a_u8(Lw[c][t][k], 0x01010101u, s_mid);
                    q_mid = dp4a_u8(Lw[c][t][k], Lw[c][t][k], q_mid);
                }
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                s0 = dp4a_u8(Lw[c][0][k], 0x01010101u, s0);
                q0 = dp4a_u8(Lw[c][0][k], Lw[c][0][k], q0);
                s1 = dp4a_u8(Lw[c][WIN][k], 0x01010101u, s1);
                q1 = dp4a_u8(Lw[c][WIN][k], Lw[c][WIN][k], q1);
            }
            const int sa0 = static_cast<int>(s_mid + s0), sa1 = static_cast<int>(s_mid + s1);
            const int va0 = C::N * static_cast<int>(q_mid + q0) - sa0 * sa0;
            const int va1 = C::N * static_cast<int>(q_mid + q1) - sa1 * sa1;
            Sa[c][0] = sa0;
            Sa[c][1] = sa1;
            rA[c][0] = va0 > 0 ? rsqrtf(static_cast<float>(va0)) : 0.f;
            rA[c][1] = va1 > 0 ? rsqrtf(static_cast<float>(va1)) : 0.f;
            rAi[c][0] = va0 > 0;
            rAi[c][1] = va1 > 0;
        }
    }

    float best[NCOL][2];
    int bz[NCOL][2];
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
            best[c][r2] = -INFINITY;
            bz[c][r2] = lo_c[c];
        }

    if (mode != 0) {
        for (int zg = lo_u; zg <= hi_u; zg += G) {
            // accumulators: rows 1..2n shared by both pixel rows, row 0 and row 2n+1 apart
            uint32_t mid[NCOL][G], top[NCOL][G], bot[NCOL][G];
#pragma unroll
            for (int c = 0; c < NCOL; ++c)
#pragma unroll
                for (int j = 0; j < G; ++j) mid[c][j] = top[c][j] = bot[c][j] = 0;
            // window of column c, candidate zg + j starts at staging column b0 + (G-1-j) + c
            const int b0 = xa - (zg + G - 1) - NH + soff;      // >= -(G-1): inside the slack
            const int w0 = b0 >> 2, sh = b0 & 3;                // arithmetic shift: floor
#pragma unroll
            for (int t = 0; t <= WIN; ++t) {
                const uint32_t *row = reinterpret_cast<const uint32_t *>(sR + (2 * qy + t) * rst);
                uint32_t raw[NWL], alw[NWA];
#pragma unroll
                for (int k = 0; k < NWL; ++k) raw[k] = row[w0 + k];
#pragma unroll
                for (int k = 0; k < NWA; ++k) alw[k] = fsr(raw[k], raw[k + 1], sh);
                // the NO distinct window offsets o = 0 .. G + NCOL - 2
                uint32_t Wo[NO][NW];
#pragma unroll
                for (int o = 0; o < NO; ++o)
#pragma unroll
                    for (int k = 0; k < NW; ++k)
                        Wo[o][k] = (o & 3) ? fsr(alw[(o >> 2) + k], alw[(o >> 2) + k + 1], o & 3)
                                           : alw[(o >> 2) + k];
#pragma unroll
                for (int c = 0; c < NCOL; ++c)
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const int o = G - 1 - j + c;
#pragma unroll
                        for (int k = 0; k < NW; ++k) {
                            if (t == 0)
                                top[c][j] = dp4a_u8(Lw[c][t][k], Wo[o][k], top[c][j]);
                            else if (t == WIN)
                                bot[c][j] = dp4a_u8(Lw[c][t][k], Wo[o][k], bot[c][j]);
                            else
                                mid[c][j] = dp4a_u8(Lw[c][t][k], Wo[o][k], mid[c][j]);
                        }
                    }
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int z = zg + j;
                if (z > hi_u) break;
#pragma unroll
                for (int c = 0; c < NCOL; ++c) {
                    if (!colv[c] || z < lo_c[c] || z > hi_c[c]) continue;
                    const int col = xa + c - z - (rs + NH);   // statistics column of x - z
#pragma unroll
                    for (int r2 = 0; r2 < 2; ++r2) {
                        if (!rowv[r2]) continue;
                        const int2 st = PLANE ? stS[(2 * qy + r2) * rst + (xa + c - z - sxs)]
                                              : stR[(2 * qy + r2) * 256 + col];
                        const int sab = static_cast<int>(mid[c][j] + (r2 ? bot[c][j] : top[c][j]));
                        const int cc = C::N * sab - Sa[c][r2] * st.x;
                        const float rho = static_cast<float>(cc) * __int_as_float(st.y);
                        if (rho > best[c][r2]) {
                            best[c][r2] = rho;
                            bz[c][r2] = z;
                        }
                    }
                }
            }
        }
    } else {
        // wide span: read the right image from global memory (apron buffer, no clamping)
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            if (!colv[c]) continue;
#pragma unroll
            for (int r2 = 0; r2 < 2; ++r2) {
                if (!rowv[r2]) continue;
                const int x = xa + c, y = ya + r2;
                for (int z = lo_c[c]; z <= hi_c[c]; ++z) {
                    uint32_t Sab = 0, Sb = 0, Sbb = 0;
#pragma unroll
                    for (int t = 0; t < WIN; ++t) {
                        const uint8_t *rrow = a.Rimg + (ptrdiff_t)(y - NH + t) * a.pitch + (x - z - NH);
#pragma unroll
                        for (int k = 0; k < NW; ++k) {
                            uint32_t w = 0;
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                if (4 * k + b < WIN) w |= static_cast<uint32_t>(__ldg(rrow + 4 * k + b)) << (8 * b);
                            Sab = dp4a_u8(Lw[c][t + r2][k], w, Sab);
                            Sb = dp4a_u8(w, 0x01010101u, Sb);
                            Sbb = dp4a_u8(w, w, Sbb);
                        }
                    }
                    const int Vb = C::N * static_cast<int>(Sbb) - static_cast<int>(Sb) * static_cast<int>(Sb);
                    const float rB = Vb > 0 ? rsqrtf(static_cast<float>(Vb)) : 0.f;
                    const int cc = C::N * static_cast<int>(Sab) - Sa[c][r2] * static_cast<int>(Sb);
                    const float rho = static_cast<float>(cc) * rB;
                    if (rho > best[c][r2]) {
                        best[c][r2] = rho;
                        bz[c][r2] = z;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
            if (!colv[c] || !rowv[r2]) continue;
            // rsqrt(Va) scales every candidate of the pixel alike: applied once here.  A flat
            // left window has c = 0 for every candidate, so the smallest z wins with rho = 0.
            float rho = rAi[c][r2] ? best[c][r2] * rA[c][r2] : 0.f;
            rho = fminf(1.f, fmaxf(-1.f, rho));
            const size_t o = (size_t)(ya + r2) * a.W + xa + c;
            a.d_out[o] = static_cast<int16_t>(bz[c][r2]);
            if (a.c_out) a.c_out[o] = rho;
        }
    if (tid == 0 && a.evals) atomicAdd(a.evals, evsum);
    return true;
}

}  // namespace tiles
}  // namespace msbm
