// zncc_region.cuh -- building blocks of the small-region ZNCC kernels (the coarsest level's
// full-range search, zncc_coarse.cu, and alpha refinement, gated.cu): a CTA stages the image
// rows of a pixel region and, per chunk of 32 candidates, the right rows those candidates
// read; it forms the right-window statistics of the chunk, and each thread evaluates its
// pixel's ZNCC (Sec. III-A, Eq. 1-4) for 4 consecutive candidates at a time: the left window
// is packed once as dp4a words, the right row words are loaded once per 4 candidates and the
// 4 windows extracted with funnel shifts.  All window sums are exact integers; the score is
// rho = float(N Sab - Sa Sb) * rsqrt(Va) * rsqrt(Vb), 0 for a flat window.
#pragma once

#include <math.h>

#include "msbm_device.cuh"

namespace msbm {
namespace region {

constexpr int ZC = 32;     // candidates per chunk

// Rows y0 .. y0 + ROWS - 1 and columns x0 .. x0 + NCOLS - 1 of an image (clamp-to-edge) into
// shared bytes with row stride STRIDE (zero from column NCOLS on).  Every thread's loads are
// issued before its first store.  blockDim.x == NT.
template <int ROWS, int NCOLS, int STRIDE, int NT = 256>
__device__ __forceinline__ void stage_rows(uint8_t *dst, const uint8_t *img, int pitch, int W, int H, int y0,
                                           int x0) {
    constexpr int NB = ROWS * STRIDE, T = (NB + NT - 1) / NT;
    uint8_t v[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int i = threadIdx.x + NT * t, r = i / STRIDE, c = i - r * STRIDE;
        const int yy = min(max(y0 + r, 0), H - 1), xx = min(max(x0 + c, 0), W - 1);
        v[t] = (i < NB && c < NCOLS) ? __ldg(img + (ptrdiff_t)yy * pitch + xx) : 0;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int i = threadIdx.x + NT * t;
        if (i < NB) dst[i] = v[t];
    }
}

// Two stage_rows calls in one round trip: every load of both regions is issued before the
// first store.  blockDim.x == NT.
template <int ROWS_A, int NCOLS_A, int STRIDE_A, int ROWS_B, int NCOLS_B, int STRIDE_B, int NT = 256>
__device__ __forceinline__ void stage_rows2(uint8_t *dstA, const uint8_t *imgA, int yA, int xA, uint8_t *dstB,
                                            const uint8_t *imgB, int yB, int xB, int pitch, int W, int H) {
    constexpr int NA = ROWS_A * STRIDE_A, TA = (NA + NT - 1) / NT;
    constexpr int NB = ROWS_B * STRIDE_B, TB = (NB + NT - 1) / NT;
    uint8_t va[TA], vb[TB];
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        const int i = threadIdx.x + NT * t, r = i / STRIDE_A, c = i - r * STRIDE_A;
        const int yy = min(max(yA + r, 0), H - 1), xx = min(max(xA + c, 0), W - 1);
        va[t] = (i < NA && c < NCOLS_A) ? __ldg(imgA + (ptrdiff_t)yy * pitch + xx) : 0;
    }
#pragma unroll
    for (int t = 0; t < TB; ++t) {
        const int i = threadIdx.x + NT * t, r = i / STRIDE_B, c = i - r * STRIDE_B;
        const int yy = min(max(yB + r, 0), H - 1), xx = min(max(xB + c, 0), W - 1);
        vb[t] = (i < NB && c < NCOLS_B) ? __ldg(imgB + (ptrdiff_t)yy * pitch + xx) : 0;
    }
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        const int i = threadIdx.x + NT * t;
        if (i < NA) dstA[i] = va[t];
    }
#pragma unroll
    for (int t = 0; t < TB; ++t) {
        const int i = threadIdx.x + NT * t;
        if (i < NB) dstB[i] = vb[t];
    }
}

// Window statistics of staged rows s (row stride STRIDE bytes): for r < OR, u < OU,
// st[r * OU + u] = {S, bits(rsqrt(N Q - S^2)) or 0} of rows r .. r+2n, columns u .. u+2n.
// vs, vq: OR x (OU + 2n) scratch.  Ends with a barrier.  blockDim.x == NT.
template <int NH, int OR, int OU, int STRIDE, int NT = 256>
__device__ __forceinline__ void window_stats(const uint8_t *s, int *vs, int *vq, int2 *st) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN, VC = OU + 2 * NH;
    for (int i = threadIdx.x; i < OR * VC; i += NT) {
        const int r = i / VC, c = i - r * VC;
        int a = 0, q = 0;
#pragma unroll
        for (int t = 0; t < WIN; ++t) {
            const int v = s[(r + t) * STRIDE + c];
            a += v;
            q += v * v;
        }
        vs[i] = a;
        vq[i] = q;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < OR * OU; i += NT) {
        const int r = i / OU, u = i - r * OU;
        int a = 0, q = 0;
#pragma unroll
        for (int b = 0; b < WIN; ++b) {
            a += vs[r * VC + u + b];
            q += vq[r * VC + u + b];
        }
        const int V = N * q - a * a;
        st[i] = make_int2(a, V > 0 ? __float_as_int(rsqrtf(static_cast<float>(V))) : 0);
    }
    __syncthreads();
}

// The left window whose top-left byte is staged at s[r * STRIDE + c], packed as dp4a words
// (bytes past the window zero), and its {Sa, bits(rsqrt(Va)) or 0}.
template <int NH, int STRIDE>
__device__ __forceinline__ int2 pack_left(const uint8_t *s, int r, int c, uint32_t (&Lw)[2 * NH + 1][(2 * NH + 4) / 4]) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN, NW = (WIN + 3) / 4;
    uint32_t a = 0, q = 0;
#pragma unroll
    for (int i = 0; i < WIN; ++i)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            uint32_t w = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * k + b < WIN) w |= static_cast<uint32_t>(s[(r + i) * STRIDE + c + 4 * k + b]) << (8 * b);
            Lw[i][k] = w;
            a = dp4a_u8(w, 0x01010101u, a);
            q = dp4a_u8(w, w, q);
        }
    const int V = N * static_cast<int>(q) - static_cast<int>(a) * static_cast<int>(a);
    return make_int2(static_cast<int>(a), V > 0 ? __float_as_int(rsqrtf(static_cast<float>(V))) : 0);
}

// pack_left on rows staged with a word-multiple stride that leaves at least one readable
// word past each window: whole-word loads and funnel shifts instead of byte loads.
template <int NH, int STRIDE>
__device__ __forceinline__ int2 pack_left_w(const uint8_t *s, int r, int c,
                                            uint32_t (&Lw)[2 * NH + 1][(2 * NH + 4) / 4]) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN, NW = (WIN + 3) / 4;
    constexpr uint32_t LAST = (WIN % 4 == 0) ? 0xFFFFFFFFu : ((1u << (8 * (WIN % 4))) - 1u);
    static_assert(STRIDE % 4 == 0, "word stride");
    const int w0 = c >> 2, sh = 8 * (c & 3);
    uint32_t a = 0, q = 0;
#pragma unroll
    for (int i = 0; i < WIN; ++i) {
        const uint32_t *row = reinterpret_cast<const uint32_t *>(s + (r + i) * STRIDE) + w0;
        uint32_t raw[NW + 1];
#pragma unroll
        for (int k = 0; k <= NW; ++k) raw[k] = row[k];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            uint32_t w = __funnelshift_r(raw[k], raw[k + 1], sh);
            if (k == NW - 1) w &= LAST;
            Lw[i][k] = w;
            a = dp4a_u8(w, 0x01010101u, a);
            q = dp4a_u8(w, w, q);
        }
    }
    const int V = N * static_cast<int>(q) - static_cast<int>(a) * static_cast<int>(a);
    return make_int2(static_cast<int>(a), V > 0 ? __float_as_int(rsqrtf(static_cast<float>(V))) : 0);
}

// Sab of the packed left window with the 4 right windows whose top-left bytes are staged at
// columns um + o (o = 0..3), row r, of word-staged rows sR (WSTRIDE words per row; each row
// readable 2 words past its last window byte).
template <int NH, int WSTRIDE>
__device__ __forceinline__ void sab4(const uint32_t *sR, int r, int um,
                                     const uint32_t (&Lw)[2 * NH + 1][(2 * NH + 4) / 4], uint32_t (&sab)[4]) {
    constexpr int WIN = 2 * NH + 1, NW = (WIN + 3) / 4;
    const int w0 = um >> 2, sh = 8 * (um & 3);
#pragma unroll
    for (int o = 0; o < 4; ++o) sab[o] = 0u;
#pragma unroll
    for (int i = 0; i < WIN; ++i) {
        const uint32_t *row = sR + (r + i) * WSTRIDE + w0;
        uint32_t raw[NW + 2], alw[NW + 1];
#pragma unroll
        for (int k = 0; k < NW + 2; ++k) raw[k] = row[k];
#pragma unroll
        for (int k = 0; k <= NW; ++k) alw[k] = __funnelshift_r(raw[k], raw[k + 1], sh);
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t w = o ? __funnelshift_r(alw[k], alw[k + 1], 8 * o) : alw[k];
                sab[o] = dp4a_u8(Lw[i][k], w, sab[o]);
            }
    }
}

// rho of one candidate from the exact sums (0 when either window is flat).
template <int NH>
__device__ __forceinline__ float rho_of(uint32_t sab, int2 la, int2 rb) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN;
    if (la.y == 0 || rb.y == 0) return 0.f;
    return static_cast<float>(N * static_cast<int>(sab) - la.x * rb.x) * __int_as_float(la.y) * __int_as_float(rb.y);
}

}  // namespace region
}  // namespace msbm
