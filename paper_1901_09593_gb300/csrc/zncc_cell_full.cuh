// zncc_cell_full.cuh -- the full-range ZNCC winner-take-all search of one 2 x 2 cell (Eq. 8-9,
// second branch), for the beta fallback's masked pixels: the cell form of the restricted
// search (zncc_cell_tile.cuh) over every admissible candidate 0 .. min(D_k - 1, x) in groups
// of G, split into parts that several lanes search and merge.
//
// Operands are read where they lie (the level's apron buffers and right statistics plane,
// through L1).  Reads stay inside the apron buffers: rows y - n .. y + 1 + n; columns from
// x - (z + G - 1) - n rounded down to a word (>= -16, as z <= x + 1 and G + n <= 13) to 16
// past the last image column for the right image, and, for the left words at n = 6, 17 past
// it (the first byte of the next buffer row at worst; it is masked off).
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "msbm_device.cuh"
#include "zncc_cell_tile.cuh"

namespace msbm {
namespace tiles {

// Best candidate of each pixel of a beta-fallback cell over part of its full range.
struct CellBest {
    float best[2][2];   // max over the part of c * rsqrt(Vb) (rsqrt(Va) not applied), -inf if none
    int bz[2][2];       // its smallest z
    float rA[2][2];     // rsqrt(Va), 0 for a flat left window
    bool m[2][2];       // masked pixels of the cell
    int hi[2];          // last admissible candidate of each column (-1: column outside)
};

// Candidate groups of cell (cx, cy) in the full-range search: groups of G from z = 0.
template <int G>
__device__ __forceinline__ int cell_full_groups(int W, int Dk, int cx) {
    const int xa = 2 * cx, hi_u = min(Dk - 1, xa + 1 < W ? xa + 1 : xa);
    return (hi_u + G) / G;
}

// Full-range WTA (Eq. 8-9, second branch: every admissible z in 0 .. min(D_k - 1, x)) of the
// masked pixels of cell (cx, cy), for the beta fallback, over candidate groups g0 .. g1 - 1
// (z = G g0 .. G g1 - 1; the caller merges the parts of a cell).  The cell's four pixels
// share each right row's loads and alignment shifts and the products of their common window
// rows, as in cell_search; their left windows (words and sums) are built once, before the
// candidate groups.  Same arithmetic as cell_search.
template <int NH, int G>
__device__ __forceinline__ CellBest cell_full_part(const uint8_t *Limg, const uint8_t *Rimg, int pitch, int W,
                                                   int H, int Dk, const uint8_t *mask, const int2 *rstat,
                                                   int rspitch, int cx, int cy, int g0, int g1) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN, NW = (WIN + 3) / 4;
    constexpr uint32_t LASTMASK = (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    constexpr int NO = G + 1, NWA = (NO - 1 + WIN + 3) / 4 + 1, NWL = NWA + 1;
    const int xa = 2 * cx, ya = 2 * cy;
    const bool colv1 = xa + 1 < W, rowv1 = ya + 1 < H;
    CellBest o;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2) {
            o.m[c][r2] = (c == 0 || colv1) && (r2 == 0 || rowv1) && mask[(size_t)(ya + r2) * W + xa + c] != 0;
            o.best[c][r2] = -INFINITY;
            o.bz[c][r2] = 0;
        }
    int *hi_c = o.hi;
    hi_c[0] = min(Dk - 1, xa);
    hi_c[1] = colv1 ? min(Dk - 1, xa + 1) : -1;
    float (&best)[2][2] = o.best;
    int (&bz)[2][2] = o.bz;
    float (&rA)[2][2] = o.rA;
    const int wpr = pitch >> 2;
    int lsh;
    const uint32_t *Lw = cell_words(Limg + (ptrdiff_t)(ya - NH) * pitch + (xa - NH), lsh);
    const uint8_t *Rrow = Rimg + (ptrdiff_t)(ya - NH) * pitch;
    // left words of both columns over all 2n + 2 rows, and the four pixels' left statistics
    uint32_t Lc[WIN + 1][2][NW];
    int Sa[2][2];
    {
        uint32_t s_t[2] = {0u, 0u}, q_t[2] = {0u, 0u}, s_m[2] = {0u, 0u}, q_m[2] = {0u, 0u}, s_b[2] = {0u, 0u},
                 q_b[2] = {0u, 0u};
#pragma unroll
        for (int t = 0; t <= WIN; ++t) {
            uint32_t lr[NW + 2], la[NW + 1];
#pragma unroll
            for (int k = 0; k < NW + 2; ++k) lr[k] = __ldg(Lw + t * wpr + k);
#pragma unroll
            for (int k = 0; k <= NW; ++k) la[k] = cell_fsr(lr[k], lr[k + 1], lsh);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                Lc[t][0][k] = la[k];
                Lc[t][1][k] = cell_fsr(la[k], la[k + 1], 1);
            }
            Lc[t][0][NW - 1] &= LASTMASK;
            Lc[t][1][NW - 1] &= LASTMASK;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const uint32_t w = Lc[t][c][k];
                    if (t == 0) {
                        s_t[c] = dp4a_u8(w, 0x01010101u, s_t[c]);
                        q_t[c] = dp4a_u8(w, w, q_t[c]);
                    } else if (t == WIN) {
                        s_b[c] = dp4a_u8(w, 0x01010101u, s_b[c]);
                        q_b[c] = dp4a_u8(w, w, q_b[c]);
                    } else {
                        s_m[c] = dp4a_u8(w, 0x01010101u, s_m[c]);
                        q_m[c] = dp4a_u8(w, w, q_m[c]);
                    }
                }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int r2 = 0; r2 < 2; ++r2) {
                const int sv = static_cast<int>(s_m[c] + (r2 ? s_b[c] : s_t[c]));
                const int v = N * static_cast<int>(q_m[c] + (r2 ? q_b[c] : q_t[c])) - sv * sv;
                Sa[c][r2] = sv;
                rA[c][r2] = v > 0 ? rsqrtf(static_cast<float>(v)) : 0.f;
            }
    }
    for (int zg = G * g0; zg < G * g1; zg += G) {
        int rsh;
        const uint32_t *Rw = cell_words(Rrow + (xa - (zg + G - 1) - NH), rsh);
        // right statistics of the group's G + 1 window columns X = xa + 1 - zg - mm (column c,
        // candidate zg + j reads mm = 1 - c + j); columns outside the image are never selected
        int2 stv[2][NO];
        const int2 *sp = rstat + (size_t)ya * rspitch + (xa + 1 - zg);
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
            for (int mm = 0; mm < NO; ++mm) {
                const int X = xa + 1 - zg - mm;
                stv[r2][mm] = (X >= 0 && X < W && (r2 == 0 || rowv1)) ? __ldg(sp + r2 * rspitch - mm)
                                                                     : make_int2(0, 0);
            }
        uint32_t T[2][G], M[2][G];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int j = 0; j < G; ++j) T[c][j] = M[c][j] = 0;
#pragma unroll
        for (int t = 0; t <= WIN; ++t) {
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
                            T[c][j] = dp4a_u8(Lc[t][c][k], Wo[o][k], T[c][j]);
                        else
                            M[c][j] = dp4a_u8(Lc[t][c][k], Wo[o][k], M[c][j]);
                    }
                }
        }
        auto wta = [&](auto checked) {
#pragma unroll
            for (int j = 0; j < G; ++j) {
                const int z = zg + j;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (decltype(checked)::value && z > hi_c[c]) continue;
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
        // the whole group admissible for all four pixels: no per-candidate checks
        if (rowv1 && colv1 && zg + G - 1 <= min(hi_c[0], hi_c[1]))
            wta(std::false_type{});
        else
            wta(std::true_type{});
    }
    return o;
}

}  // namespace tiles
}  // namespace msbm
