// zncc_cell_tile.cuh -- the restricted ZNCC winner-take-all search (Sec. III-C, Eq. 8-9,
// first branch) with one thread per prior cell: the 2 x 2 pixels (2cx .. 2cx+1, 2cy .. 2cy+1)
// whose nearest-neighbour upsampled prior is the same coarser disparity d^{k+1}(cy, cx).
// Candidates as in the staged tiles: dhat = 2 d^{k+1} clamped into 0 .. min(D_k - 1, x),
// then dhat - r .. dhat + r clipped to the same range (the paper's "3 comparisons per pixel"
// is r = 1).
//
// Nothing is staged: every operand is read where it lies (the two level images in their
// apron buffers, the level's right statistics plane) through the L1 cache, so the thread
// waits on no other thread: no barriers, no shared memory, no device waits, and no span
// reduction or staging mode however far apart the cells of a neighbourhood search.
//  * The four pixels of a cell share every loaded word.  Per candidate group (G consecutive
//    z) and window row, the right image row is loaded once as aligned words, funnel-shifted
//    into the G + 1 distinct window offsets the two columns' candidates need and multiplied
//    with both columns' left words by dp4a; the two pixel rows share the products of their
//    2n common window rows (2n + 2 rows for 2 pixel rows).
//  * Left-window sums come from the same loaded rows; right-window sums and rsqrt of their
//    variances from the plane.  All sums are exact int32 (windows up to 13 x 13) and
//    c = N * Sab - Sa * Sb is exact; the only rounding is
//    rho = float(c) * rsqrt(Vb) * rsqrt(Va): the arithmetic of the staged tiles, which
//    therefore give identical maps.
//  * WTA in ascending z with a strict compare: exact ties keep the smallest z.
// Reads stay inside the apron buffers: columns from x - z - n - 3 (>= -16) to at most 16
// past the last image column, rows from y - n to y + 1 + n.
#pragma once

#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {
namespace tiles {

__device__ __forceinline__ uint32_t cell_fsr(uint32_t lo, uint32_t hi, int bytes) {
    return __funnelshift_r(lo, hi, 8 * bytes);
}

// The aligned word holding byte p, and p's byte position in it.
__device__ __forceinline__ const uint32_t *cell_words(const uint8_t *p, int &sh) {
    const uintptr_t u = reinterpret_cast<uintptr_t>(p);
    sh = static_cast<int>(u & 3u);
    return reinterpret_cast<const uint32_t *>(u & ~static_cast<uintptr_t>(3));
}

// Restricted WTA of cell (cx, cy) (2cx < W, 2cy < H): writes its pixels' disparities and
// costs, returns its evaluation count (pixels in a.skip excluded).  G candidates per group
// (2r + 1 up to 7; wider radii run several groups).
template <int NH, int G>
__device__ __forceinline__ unsigned cell_search(const RestrTileArgs &a, int cx, int cy) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN, NW = (WIN + 3) / 4;
    constexpr uint32_t LASTMASK = (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    constexpr int NO = G + 1;                          // distinct window offsets of a group
    constexpr int NWA = (NO - 1 + WIN + 3) / 4 + 1;    // aligned right words per row
    constexpr int NWL = NWA + 1;                       // raw right words loaded per row
    const int xa = 2 * cx, ya = 2 * cy;
    const bool colv1 = xa + 1 < a.W, rowv1 = ya + 1 < a.H;
    const int p2 = 2 * static_cast<int>(a.prior[(size_t)cy * a.Wp + cx]);
    int lo_c[2], hi_c[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int zmx = min(a.Dk - 1, xa + c);
        const int dh = min(max(p2, 0), zmx);
        lo_c[c] = max(0, dh - a.r);
        hi_c[c] = min(zmx, dh + a.r);
    }
    if (!colv1) {
        lo_c[1] = INT_MAX;
        hi_c[1] = -1;
    }
    const int lo_u = min(lo_c[0], lo_c[1]), hi_u = max(hi_c[0], hi_c[1]);
    unsigned cnt = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
            if ((c == 0 || colv1) && (r2 == 0 || rowv1) &&
                !(a.skip && a.skip[(size_t)(ya + r2) * a.W + xa + c]))
                cnt += static_cast<unsigned>(hi_c[c] - lo_c[c] + 1);

    const int wpr = a.pitch >> 2;                      // words per buffer row
    int lsh;
    const uint32_t *Lw = cell_words(a.Limg + (ptrdiff_t)(ya - NH) * a.pitch + (xa - NH), lsh);
    const uint8_t *Rrow = a.Rimg + (ptrdiff_t)(ya - NH) * a.pitch;

    float best[2][2];
    int bz[2][2], Sa[2][2];
    float rA[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
            best[c][r2] = -INFINITY;
            bz[c][r2] = lo_c[c];
            Sa[c][r2] = 0;
            rA[c][r2] = 0.f;
        }

    for (int zg = lo_u; zg <= hi_u; zg += G) {
        // window of column c, candidate zg + j starts at byte b0 + (G - 1 - j) + c
        int rsh;
        const uint32_t *Rw = cell_words(Rrow + (xa - (zg + G - 1) - NH), rsh);
        // right statistics of the group's G + 1 window columns X = xa + 1 - zg - m, loaded
        // ahead of the rows; column c, candidate zg + j reads m = 1 - c + j.  Entries no
        // candidate reads (X outside the image, the row below a bottom pixel outside it) are
        // not loaded (reading them from a padded plane instead measured slower: the
        // 1400 x 1000 pass 49.7 -> 53.8 us).
        int2 stv[2][G + 1];
        const int2 *sp = a.rstat + (size_t)ya * a.rspitch + (xa + 1 - zg);
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
            for (int m = 0; m <= G; ++m) {
                const int X = xa + 1 - zg - m;
                stv[r2][m] = (X >= 0 && X < a.W && (r2 == 0 || rowv1)) ? __ldg(sp + r2 * a.rspitch - m)
                                                                      : make_int2(0, 0);
            }
        // T: window row 0 (top pixel only), then rows 0 .. 2n (top pixel's sum);
        // M: rows 1 .. 2n (both pixels), then rows 1 .. 2n + 1 (bottom pixel's sum)
        uint32_t T[2][G], M[2][G];
        uint32_t s_t[2], q_t[2], s_m[2], q_m[2], s_b[2], q_b[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            s_t[c] = q_t[c] = s_m[c] = q_m[c] = s_b[c] = q_b[c] = 0;
#pragma unroll
            for (int j = 0; j < G; ++j) T[c][j] = M[c][j] = 0;
        }
#pragma unroll
        for (int t = 0; t <= WIN; ++t) {
            // left words of both columns
            uint32_t lr[NW + 2], la[NW + 1], Lc[2][NW];
#pragma unroll
            for (int k = 0; k < NW + 2; ++k) lr[k] = __ldg(Lw + t * wpr + k);
#pragma unroll
            for (int k = 0; k <= NW; ++k) la[k] = cell_fsr(lr[k], lr[k + 1], lsh);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                Lc[0][k] = la[k];
                Lc[1][k] = cell_fsr(la[k], la[k + 1], 1);
            }
            Lc[0][NW - 1] &= LASTMASK;
            Lc[1][NW - 1] &= LASTMASK;
            // left-window sums
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    if (t == 0) {
                        s_t[c] = dp4a_u8(Lc[c][k], 0x01010101u, s_t[c]);
                        q_t[c] = dp4a_u8(Lc[c][k], Lc[c][k], q_t[c]);
                    } else if (t == WIN) {
                        s_b[c] = dp4a_u8(Lc[c][k], 0x01010101u, s_b[c]);
                        q_b[c] = dp4a_u8(Lc[c][k], Lc[c][k], q_b[c]);
                    } else {
                        s_m[c] = dp4a_u8(Lc[c][k], 0x01010101u, s_m[c]);
                        q_m[c] = dp4a_u8(Lc[c][k], Lc[c][k], q_m[c]);
                    }
                }
            // right words of the group, aligned, and the NO window offsets
            uint32_t raw[NWL], alw[NWA], Wo[NO][NW];
#pragma unroll
            for (int k = 0; k < NWL; ++k) raw[k] = __ldg(Rw + t * wpr + k);
#pragma unroll
            for (int k = 0; k < NWA; ++k) alw[k] = cell_fsr(raw[k], raw[k + 1], rsh);
#pragma unroll
            for (int o = 0; o < NO; ++o)
#pragma unroll
                for (int k = 0; k < NW; ++k)
                    Wo[o][k] = (o & 3) ? cell_fsr(alw[(o >> 2) + k], alw[(o >> 2) + k + 1], o & 3)
                                       : alw[(o >> 2) + k];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int o = G - 1 - j + c;
                    if (t == WIN) T[c][j] += M[c][j];
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        if (t == 0)
                            T[c][j] = dp4a_u8(Lc[c][k], Wo[o][k], T[c][j]);
                        else
                            M[c][j] = dp4a_u8(Lc[c][k], Wo[o][k], M[c][j]);
                    }
                }
        }
        // left-window statistics of the four pixels (the same in every group)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int r2 = 0; r2 < 2; ++r2) {
                const int s = static_cast<int>(s_m[c] + (r2 ? s_b[c] : s_t[c]));
                const int v = N * static_cast<int>(q_m[c] + (r2 ? q_b[c] : q_t[c])) - s * s;
                Sa[c][r2] = s;
                rA[c][r2] = v > 0 ? rsqrtf(static_cast<float>(v)) : 0.f;
            }
        // WTA over the group; a cell whose four pixels take all G candidates (no clipping at
        // the image's left edge or at D_k, both pixel rows and columns inside the image)
        // skips the per-candidate range checks
        auto wta = [&](auto checked) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int z = zg + j;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (decltype(checked)::value && (z < lo_c[c] || z > hi_c[c])) continue;
#pragma unroll
                    for (int r2 = 0; r2 < 2; ++r2) {
                        if (decltype(checked)::value && r2 && !rowv1) continue;
                        const int2 st = stv[r2][1 - c + j];
                        const int sab = static_cast<int>(r2 ? M[c][j] : T[c][j]);
                        const int cc = N * sab - Sa[c][r2] * st.x;
                        const float rho = static_cast<float>(cc) * __int_as_float(st.y);
                        if (rho > best[c][r2]) {
                            best[c][r2] = rho;
                            bz[c][r2] = z;
                        }
                    }
                }
            }
        };
        const bool full = rowv1 && lo_c[0] == zg && lo_c[1] == zg && hi_c[0] == zg + G - 1 &&
                          hi_c[1] == zg + G - 1;
        if (full)
            wta(std::false_type{});
        else
            wta(std::true_type{});
    }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
            if ((c && !colv1) || (r2 && !rowv1)) continue;
            // rsqrt(Va) scales every candidate of the pixel alike: applied once here.  A flat
            // left window has c = 0 for every candidate, so the smallest z wins with rho = 0.
            float rho = rA[c][r2] > 0.f ? best[c][r2] * rA[c][r2] : 0.f;
            rho = fminf(1.f, fmaxf(-1.f, rho));
            const size_t o = (size_t)(ya + r2) * a.W + xa + c;
            a.d_out[o] = static_cast<int16_t>(bz[c][r2]);
            if (a.c_out) a.c_out[o] = rho;
        }
    return cnt;
}

}  // namespace tiles
}  // namespace msbm
