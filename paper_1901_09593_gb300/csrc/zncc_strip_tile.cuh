// zncc_strip_tile.cuh -- the restricted ZNCC winner-take-all tile of the standalone pass
// (Sec. III-C, Eq. 8-9, first branch).  Each pixel evaluates dhat - r .. dhat + r around the
// nearest-neighbour upsample dhat = 2 * d^{k+1}(y/2, x/2) of the coarser disparity (the
// paper's "3 comparisons per pixel" is r = 1), clipped to 0 .. min(D_k - 1, x); dhat is
// first clamped into that range (a no-op for priors produced by the coarser level).
//
// Design (a 32 x TY pixel tile, TY = 8 or 16, of 32 x TY/4 threads; each thread owns a
// vertical strip of four pixels of one column, which spans two prior cells):
//  * The CTA reduces the union [zlo, zhi] of its spans; the left tile (a 64-byte box), the
//    right span [x0 - zhi - n, x1 - zlo + n] (a 128-byte box), the span's entries of the
//    level's right statistics plane (128 x TY) and the tile's entries of the left statistics
//    plane (32 x TY) are staged by TMA on one mbarrier with a bounded wait.  A union too wide
//    for 128 bytes (a tile across a large disparity jump) is staged in several passes, each
//    covering the smallest pending candidate groups of the tile.
//  * Each thread's candidates are its two prior cells' spans in groups of G, ascending, a
//    candidate two spans share being evaluated once.
//  * The four pixels' windows cover 2n + 4 rows.  For each of those rows the thread aligns
//    its left window row once (word loads and funnel shifts) and the right bytes of a group
//    of G consecutive candidates once, extracts the G window offsets, and accumulates
//    sum a*b with dp4a into running chains: the 2n - 2 rows all four windows share, the
//    three rows above (chained from them) and the three below, so that each pixel's window
//    sum costs two dp4a per window row over the strip plus two additions per candidate.
//    All sums are exact int32 (windows up to 13 x 13); c = N*Sab - Sa*Sb is exact; the only
//    rounding is rho = float(c) * rsqrt(Vb) * rsqrt(Va).
//  * A warp whose threads all see one full-width span for both prior cells (the common
//    case) evaluates its single group without per-candidate span tests.
//  * WTA in ascending z with a strict compare, so exact ties keep the smallest z.
// Bound: instruction issue (dp4a, funnel shifts, shared loads); HBM traffic is a few bytes
// per pixel.
#pragma once

#include <limits.h>
#include <math.h>

#include <type_traits>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {
namespace tiles {

template <int NH, int TY>
struct SCfg {
    static_assert(TY == 8 || TY == 16, "tile height");
    static constexpr int TX = 32;                // tile width (pixels)
    static constexpr int THREADS = 32 * (TY / 4);
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int N = WIN * WIN;
    static constexpr int NW = (WIN + 3) / 4;     // words per packed window row
    static constexpr int ROWS = TY + 2 * NH;     // staged rows
    static constexpr int SROWS = 4 + 2 * NH;     // rows one strip's windows cover
    static constexpr int LBOX = 64;              // left box: image columns x0-16 .. x0+48
    static constexpr uint32_t LASTMASK =
        (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    // shared memory carve (bytes): [0,128) barrier, flag, span scalars, evaluation sum
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t OFF_SL = 128;
    static constexpr size_t PAD_R = 128;         // readable slack before the right span
    static constexpr size_t OFF_SR = OFF_SL + al((size_t)ROWS * LBOX) + PAD_R;
    static constexpr size_t OFF_SS = OFF_SR + al((size_t)(ROWS + 2) * 128);   // right plane [TY][128]
    static constexpr size_t OFF_SLS = OFF_SS + (size_t)TY * 128 * 8;          // left plane [TY][32]
    static constexpr size_t BYTES = OFF_SLS + (size_t)TY * 32 * 8;
};

__device__ __forceinline__ uint32_t sfsr(uint32_t lo, uint32_t hi, int bytes) {
    return __funnelshift_r(lo, hi, 8 * bytes);
}

// One group of G candidates zg .. zg+G-1 for the thread's four pixels (rows 4*qy + p of the
// staged tile, p = 0..3).  sRrow0: the thread's first staged right row; rst: right row
// stride; b0: staging column of the window of candidate zg+G-1 (may be slightly negative:
// the slack before the span).  Calls fin(p, X) with pixel p's window sums of a*b for the G
// candidates (X[j] for candidate zg + j) as soon as they are final, pixel 0 first, so that
// only one pixel's sums are live at a time.
template <int NH, int G, int TY, typename Fin>
__device__ __forceinline__ void strip_sums(const uint8_t *sLrow0, int w0L, int shL, const uint8_t *sRrow0,
                                           int rst, int b0, Fin &&fin) {
    using C = SCfg<NH, TY>;
    constexpr int WIN = C::WIN, NW = C::NW, SROWS = C::SROWS;
    constexpr int NWA = (G - 1 + WIN + 3) / 4 + 1;    // aligned words covering the group
    constexpr int NWL = NWA + 1;                       // raw words loaded per row
    const int w0 = b0 >> 2, sh = b0 & 3;               // arithmetic shift: floor
    // chains: M = rows 3 .. 2n (shared by all four windows); T = M + rows 2, 1 (top of
    // pixels 1, 2); B = M + rows 2n+1, 2n+2 (bottom of pixels 1, 2)
    uint32_t M[G], T2[G], T12[G], B1[G], X[G];
#pragma unroll
    for (int j = 0; j < G; ++j) M[j] = 0;
    // row order: shared rows first, then 2, 1, 0 (chained from M), then 2n+1 .. 2n+3
#pragma unroll
    for (int i = 0; i < SROWS; ++i) {
        // strip row tt: 3 .. 2n, then 2, 1, 0, then 2n+1, 2n+2, 2n+3
        const int tt = i < 2 * NH - 2 ? 3 + i : (i < 2 * NH + 1 ? 2 - (i - (2 * NH - 2)) : i);
        // left window row tt of the strip, aligned
        uint32_t Lw[NW];
        {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(sLrow0 + tt * C::LBOX);
            uint32_t raw[NW + 1];
#pragma unroll
            for (int k = 0; k <= NW; ++k) raw[k] = row[w0L + k];
#pragma unroll
            for (int k = 0; k < NW; ++k) Lw[k] = sfsr(raw[k], raw[k + 1], shL);
            Lw[NW - 1] &= C::LASTMASK;
        }
        // right bytes of the group, aligned, and the window of each candidate
        const uint32_t *rrow = reinterpret_cast<const uint32_t *>(sRrow0 + tt * rst);
        uint32_t raw[NWL], alw[NWA];
#pragma unroll
        for (int k = 0; k < NWL; ++k) raw[k] = rrow[w0 + k];
#pragma unroll
        for (int k = 0; k < NWA; ++k) alw[k] = sfsr(raw[k], raw[k + 1], sh);
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const int o = G - 1 - j;                   // window offset of candidate zg + j
            uint32_t acc;
            if (tt >= 3 && tt <= 2 * NH) acc = M[j];
            else if (tt == 2) acc = M[j];
            else if (tt == 1) acc = T2[j];
            else if (tt == 0) acc = T12[j];
            else if (tt == 2 * NH + 1) acc = M[j];
            else acc = B1[j];                          // rows 2n+2, 2n+3 continue the B chain
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t w = (o & 3) ? sfsr(alw[(o >> 2) + k], alw[(o >> 2) + k + 1], o & 3)
                                           : alw[(o >> 2) + k];
                acc = dp4a_u8(Lw[k], w, acc);
            }
            if (tt >= 3 && tt <= 2 * NH) M[j] = acc;
            else if (tt == 2) T2[j] = acc;                  // M + r2        (pixel 2's top)
            else if (tt == 1) T12[j] = acc;                 // M + r1 + r2   (pixel 1's top)
            else if (tt == 0) X[j] = acc;                   // pixel 0: rows 0 .. 2n
            else if (tt == 2 * NH + 1) {                    // M + r(2n+1)
                X[j] = T12[j] + acc - M[j];                 // pixel 1: rows 1 .. 2n+1
                B1[j] = acc;
            } else if (tt == 2 * NH + 2) {                  // M + r(2n+1) + r(2n+2)
                X[j] = T2[j] + acc - M[j];                  // pixel 2: rows 2 .. 2n+2
                B1[j] = acc;
            } else {
                X[j] = acc;                                 // pixel 3: rows 3 .. 2n+3
            }
        }
        if (tt == 0) fin(std::integral_constant<int, 0>{}, X);
        if (tt == 2 * NH + 1) fin(std::integral_constant<int, 1>{}, X);
        if (tt == 2 * NH + 2) fin(std::integral_constant<int, 2>{}, X);
        if (tt == 2 * NH + 3) fin(std::integral_constant<int, 3>{}, X);
    }
}

// Restricted WTA of one 32 x TY tile (bx, by) by the calling CTA (blockDim.x = 32 * TY / 4).
// `smem` holds SCfg::BYTES bytes, 128-aligned; its first 8 bytes are an mbarrier the caller
// has initialised (count 1) and `parity` is its next phase parity, advanced here.  Returns
// false if a bounded wait gave up (the error word is then set).
template <int NH, int G, int TY>
__device__ bool strip_tile(const RestrTileArgs &a, const CUtensorMap *tmL, const CUtensorMap *tmR128,
                           const CUtensorMap *tmS, const CUtensorMap *tmSL, int bx, int by, uint8_t *smem,
                           uint32_t &parity) {
    using C = SCfg<NH, TY>;
    // candidates one pass can stage: 32 + ZR + 2n columns plus up to 15 of alignment in 128
    constexpr int ZR = 128 - C::TX - 2 * NH - 15;
    static_assert(ZR >= G - 1, "a group must fit one pass");
    uint64_t &bar = *reinterpret_cast<uint64_t *>(smem);
    int &flag = *reinterpret_cast<int *>(smem + 8);
    int *za_s = reinterpret_cast<int *>(smem + 16);       // [2]: next pass start (alternating)
    int &xs_s = *reinterpret_cast<int *>(smem + 24);
    int *wlo_s = reinterpret_cast<int *>(smem + 32);      // [TY/4] per-warp span union
    int *whi_s = reinterpret_cast<int *>(smem + 48);
    unsigned *wcnt_s = reinterpret_cast<unsigned *>(smem + 64);   // [TY/4] per-warp evaluations
    const uint8_t *sL = smem + C::OFF_SL;                               // [ROWS][64]
    const uint8_t *sR = smem + C::OFF_SR;                               // [ROWS + 1][128]
    const int2 *stS = reinterpret_cast<const int2 *>(smem + C::OFF_SS);   // [TY][128] right plane
    const int2 *stL = reinterpret_cast<const int2 *>(smem + C::OFF_SLS);  // [TY][32] left plane

    const int tid = threadIdx.x, qx = tid & 31, qy = tid >> 5;
    const int x0 = bx * C::TX, y0 = by * TY;
    const int xa = x0 + qx, ya = y0 + 4 * qy;           // the strip: column xa, rows ya .. ya+3
    const int Dk = a.Dk;
    const bool colv = xa < a.W;
    bool rowv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) rowv[p] = colv && ya + p < a.H;
    const bool any = rowv[0];

    // candidate spans of the two prior cells (rows ya/2 and ya/2 + 1)
    int lo_c[2] = {INT_MAX, INT_MAX}, hi_c[2] = {-1, -1};
    if (any) {
        const int px = min(xa >> 1, a.Wp - 1);
        const int zmx = min(Dk - 1, xa);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!rowv[2 * h]) continue;
            const int py = min((ya >> 1) + h, a.Hp - 1);
            const int p2 = 2 * static_cast<int>(a.prior[(size_t)py * a.Wp + px]);
            const int dh = min(max(p2, 0), zmx);
            lo_c[h] = max(0, dh - a.r);
            hi_c[h] = min(zmx, dh + a.r);
        }
    }
    const int lo_u = min(lo_c[0], lo_c[1]), hi_u = max(hi_c[0], hi_c[1]);
    // the thread's groups, ascending: the lower cell's span from its start in steps of G, then
    // the rest of the other cell's span (candidates a group already covered are not repeated)
    const bool swap = lo_c[1] < lo_c[0];
    const int l1 = swap ? lo_c[1] : lo_c[0], h1 = swap ? hi_c[1] : hi_c[0];
    const int l2 = swap ? lo_c[0] : lo_c[1], h2 = swap ? hi_c[0] : hi_c[1];
    int next = any ? l1 : INT_MAX, cell = 0;
    // a warp takes the check-free path when every strip in it has one full-width span
    const bool uni_t = !any || (hi_c[0] - lo_c[0] + 1 == G && (!rowv[2] || (lo_c[1] == lo_c[0] && hi_c[1] == hi_c[0])));
    const bool uni_w = __all_sync(0xFFFFFFFFu, uni_t);
    {
        // the tile's span union and evaluation count: one slot per warp, one barrier
        const int wlo = __reduce_min_sync(0xFFFFFFFFu, lo_u);
        const int whi = __reduce_max_sync(0xFFFFFFFFu, hi_u);
        unsigned cnt = 0;
#pragma unroll
        for (int p = 0; p < 4; ++p)
            if (rowv[p] && !(a.skip && a.skip[(size_t)(ya + p) * a.W + xa]))
                cnt += static_cast<unsigned>(hi_c[p >> 1] - lo_c[p >> 1] + 1);
        const unsigned wcnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if ((tid & 31) == 0) {
            wlo_s[qy] = wlo;
            whi_s[qy] = whi;
            wcnt_s[qy] = wcnt;
        }
        if (tid == 0) za_s[0] = za_s[1] = INT_MAX;   // pass-start slots, first used after a barrier
    }
    __syncthreads();
    int zlo = wlo_s[0], zhi = whi_s[0];
#pragma unroll
    for (int w = 1; w < TY / 4; ++w) {
        zlo = min(zlo, wlo_s[w]);
        zhi = max(zhi, whi_s[w]);
    }
    const int xlast = min(x0 + C::TX, a.W) - 1;
    // one pass when the tile's whole candidate union fits the 128-byte staging box
    const bool single = ((xlast - zlo + NH) + APX + 1 - ((x0 - zhi - NH + APX) & ~15)) <= 128;
    const bool uni = single && uni_w;

    // left windows of the four pixels: {Sa, rsqrt(Va)} are read from the staged left plane
    // where they are used
    float best[4];
    int bz[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        best[p] = -INFINITY;
        bz[p] = lo_c[p >> 1];
    }
    const int sc = qx + 16 - NH;               // left staging column of xa - n
    const int w0L = sc >> 2, shL = sc & 3;
    const uint8_t *sLrow0 = sL + (4 * qy) * C::LBOX;
    const uint8_t *sRrow0 = sR + (4 * qy) * 128;

    int za = zlo;
    for (int pass = 0;; ++pass) {
        const int zb = single ? zhi : za + ZR;  // candidates staged in this pass: za .. zb
        const int sxs = (x0 - zb) & ~1;        // first staged right-plane column (even)
        if (tid == 0) {
            const int xs = (x0 - zb - NH + APX) & ~15;
            xs_s = xs;
            uint32_t bytes = C::ROWS * 128 + TY * 128 * 8;
            if (pass == 0) bytes += C::ROWS * C::LBOX + TY * 32 * 8;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar, bytes);
            if (pass == 0) {
                tma_load_2d(smem + C::OFF_SL, tmL, &bar, x0 - 16 + APX, y0 - NH + APY);
                tma_load_2d(smem + C::OFF_SLS, tmSL, &bar, x0, y0);
            }
            tma_load_2d(smem + C::OFF_SR, tmR128, &bar, xs, y0 - NH + APY);
            tma_load_2d(smem + C::OFF_SS, tmS, &bar, sxs, y0);
        }
        if (!tma_batch_wait(&bar, parity, &flag, a.force_timeout != 0, a.err)) return false;
        parity ^= 1;
        const int soff = APX - xs_s;           // staging column of image column X: X + soff

        // one group of G candidates zg .. zg+G-1 for the four pixels
        auto eval_group = [&](const int zg, auto check_tag) {
            constexpr bool check = decltype(check_tag)::value;
            const int b0 = xa - (zg + G - 1) - NH + soff;   // >= -(G-1): inside the slack
            strip_sums<NH, G, TY>(sLrow0, w0L, shL, sRrow0, 128, b0, [&](auto pc, const uint32_t (&X)[G]) {
                constexpr int p = decltype(pc)::value;
                const int sa = stL[(4 * qy + p) * 32 + qx].x;
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int z = zg + j;
                    // (a branch here measured faster than a predicated, branch-free mask:
                    // 2880 x 1984 pass 235 vs 263 us)
                    if (check && (z < lo_c[p >> 1] || z > hi_c[p >> 1])) continue;
                    const int2 st = stS[(4 * qy + p) * 128 + (xa - z - sxs)];
                    const int cc = C::N * static_cast<int>(X[j]) - sa * st.x;
                    const float rho = static_cast<float>(cc) * __int_as_float(st.y);
                    if (rho > best[p]) {
                        best[p] = rho;
                        bz[p] = z;
                    }
                }
            });
        };
        if (uni) {
            // (threads outside the image have no span: INT_MAX would overflow the offsets)
            if (any) eval_group(lo_c[0], std::false_type{});
            break;
        }
        // groups that fit this pass (all of them in a single pass), in ascending order
        while (next != INT_MAX && (single || next + G - 1 <= zb)) {
            eval_group(next, std::true_type{});
            const int z = next + G;
            if (cell == 0 && z <= h1) {
                next = z;
            } else if (cell == 0 && l2 != INT_MAX && max(l2, z) <= h2) {
                cell = 1;
                next = max(l2, z);
            } else if (cell == 1 && z <= h2) {
                next = z;
            } else {
                next = INT_MAX;
            }
        }
        if (single) break;
        // the next pass starts at the smallest pending group; the barrier also keeps the
        // staged span until every thread is done with it
        const int wmin = __reduce_min_sync(0xFFFFFFFFu, next);
        if ((tid & 31) == 0) atomicMin(&za_s[pass & 1], wmin);
        __syncthreads();
        za = za_s[pass & 1];
        if (tid == 0) za_s[(pass + 1) & 1] = INT_MAX;
        if (za == INT_MAX) break;
    }
    if (!any) return true;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        if (!rowv[p]) continue;
        // rsqrt(Va) scales every candidate of the pixel alike: applied once here.  A flat
        // left window (rA = 0) has c = 0 for every candidate, so the smallest z wins with 0.
        float rho = best[p] * __int_as_float(stL[(4 * qy + p) * 32 + qx].y);
        rho = fminf(1.f, fmaxf(-1.f, rho));
        const size_t o = (size_t)(ya + p) * a.W + xa;
        a.d_out[o] = static_cast<int16_t>(bz[p]);
        if (a.c_out) a.c_out[o] = rho;
    }
    if (tid == 0 && a.evals) {
        unsigned long long ev = 0;
#pragma unroll
        for (int w = 0; w < TY / 4; ++w) ev += wcnt_s[w];
        atomicAdd(a.evals, ev);
    }
    return true;
}

}  // namespace tiles
}  // namespace msbm
