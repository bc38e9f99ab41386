// pyramid_fused.cuh -- one tile of the fused Gaussian pyramid (Sec. III, Fig. 1): levels
// s+1 .. s+F built from level s by one CTA, shared by the standalone launch (pyramid.cu) and
// the batched persistent kernel (batch.cu).  Filter reading: 5-tap binomial [1 4 6 4 1]/16
// per axis, clamp-to-edge, 2x decimation to ceil(W/2) x ceil(H/2), (sum + 128) >> 8.
#pragma once

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {

// One CTA per (PF_TX x PF_TY tile of the coarsest fused level c = s + F, image).  Level j of
// the CTA's pyramid (j = 0 is level s) covers the fixed region of RW(j) x RH(j) pixels whose
// first image column is lox_j = 2 lox_{j+1} - 2 (rows likewise): the 5 x 5 support of every
// pixel of region j+1, and the CTA's own part of level j (2^(F-j) times its tile).  Regions
// keep their full size at image borders, and every shared level holds at each position the
// value of the clamped image position (level s by clamped loads, finer levels by an edge
// replication pass on border CTAs), so the filter needs no clamping:
//  * level s is read once, word-wise (bytes only where a word crosses the image border or
//    the caller's rows are not word-aligned), into rows that start 2 bytes before the region;
//  * a horizontal [1 4 6 4 1] pass makes 4 outputs per thread from 3 words (funnel shifts
//    and dp4a: weights 1, 4, 6, 4 plus the fifth byte), packed as 16-bit sums;
//  * a vertical pass adds 5 rows of those sums, two columns per 32-bit word (each 16-bit
//    half stays below 2^16), rounds with (v + 128) >> 8 and packs 4 output bytes;
//  * every written level's own part, plus the apron on border CTAs, leaves in 16-byte
//    chunks.
// Every loop runs over a compile-time item count with compile-time divisors.  The integer
// sums are those of the 5 x 5 binomial support, hence exact.  Neighbouring CTAs recompute
// the overlapping halos instead of exchanging them.
// 16 x 4 tiles of the coarsest fused level: twice the CTAs of 16 x 8 tiles for 7 % more
// halo work, which shortens the launch (measured on the 1400 x 1000 and 2880 x 1984 pairs)
constexpr int PF_TX = 16, PF_TY = 4;
// every written level's own part leaves in 16-byte chunks starting at multiples of 16
// columns: the coarsest tile width must be a multiple of 16
static_assert(PF_TX % 16 == 0, "fused pyramid tile width");

template <int F>
struct PyrGeom {
    __host__ __device__ static constexpr int RW(int j) { return j >= F ? PF_TX : 2 * RW(j + 1) + 3; }
    __host__ __device__ static constexpr int RH(int j) { return j >= F ? PF_TY : 2 * RH(j + 1) + 3; }
    __host__ __device__ static constexpr int NQ(int j) { return (RW(j) + 3) / 4; }      // output quads of level j
    // shared row stride of level j (bytes): the next horizontal pass reads words 2q .. 2q+2
    // (2q .. 2q+3 for level s, whose rows start 2 bytes early); the vertical pass writes 4 NQ(j)
    __host__ __device__ static constexpr int STR(int j) {
        return j >= F ? 4 * NQ(j)
                      : (j == 0 ? 8 * NQ(1) + 8
                                : (8 * NQ(j + 1) + 4 > 4 * NQ(j) ? 8 * NQ(j + 1) + 4 : 4 * NQ(j)));
    }
    __host__ __device__ static constexpr int al16(int v) { return (v + 15) / 16 * 16; }
    __host__ __device__ static constexpr int OFF(int j) { return j == 0 ? 0 : OFF(j - 1) + al16(STR(j - 1) * RH(j - 1)); }
    static constexpr int OFF_T = OFF(F + 1);                          // horizontal-pass sums
    static constexpr int BYTES = OFF_T + 8 * NQ(1) * RH(0);
};

// shared bytes of a CTA (F = 3 needs the most: levels 53 x 160, 25 x 76, 11 x 36, 4 x 16 plus
// 53 x 19 sum quads)
constexpr int PF_SMEM = (PyrGeom<3>::BYTES + 1023) / 1024 * 1024;
static_assert(PyrGeom<2>::BYTES <= PF_SMEM && PyrGeom<1>::BYTES <= PF_SMEM, "fused pyramid shared memory");

// Levels J .. F of the CTA's pyramid from level J - 1 in shared memory (compile-time J).
template <int F, int J, int NT>
__device__ __forceinline__ void pyr_levels(const PyrFuseArgs &a, const int (&lox)[F + 1], const int (&loy)[F + 1],
                                           uint8_t *sm) {
    using G = PyrGeom<F>;
    constexpr int j = J;
    const int tid = threadIdx.x;
    // the horizontal pass reads level j-1 region columns 8q .. 8q+11 (8q+2 .. 8q+13 staged for
    // level s): all inside the stride, and inside the columns the vertical pass of level j-1
    // computed (4 NQ(j-1)) for j >= 2
    static_assert(j == 1 ? 8 * G::NQ(1) + 8 <= G::STR(0)
                         : (8 * G::NQ(j) + 4 <= G::STR(j - 1) && 8 * G::NQ(j) + 3 <= 4 * G::NQ(j - 1)),
                  "horizontal pass reads");
    static_assert(2 * (G::RH(j) - 1) + 4 <= G::RH(j - 1) - 1, "vertical pass rows");
    constexpr int OFFP = G::OFF(j - 1), OFFJ = G::OFF(j);
    const uint8_t *Pp = sm + OFFP;
    uint8_t *P = sm + OFFJ;
    uint2 *t2 = reinterpret_cast<uint2 *>(sm + G::OFF_T);
    constexpr int NQj = G::NQ(j), SP = G::STR(j - 1), RHp = G::RH(j - 1), RHj = G::RH(j), SJ = G::STR(j);
    // horizontal: RH(j-1) rows x NQ(j) quads -> 16-bit sums of 4 outputs per item
    {
        constexpr int N = RHp * NQj;
        for (int i = tid; i < N; i += NT) {
            const int r = i / NQj, q = i - r * NQj;
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(Pp + r * SP) + 2 * q;
            uint32_t a0, a1, a2;
            if constexpr (j == 1) {   // level s rows start 2 bytes before the region
                const uint32_t r0 = wr[0], r1 = wr[1], r2 = wr[2], r3 = wr[3];
                a0 = __funnelshift_r(r0, r1, 16);
                a1 = __funnelshift_r(r1, r2, 16);
                a2 = __funnelshift_r(r2, r3, 16);
            } else {
                a0 = wr[0];
                a1 = wr[1];
                a2 = wr[2];
            }
            constexpr uint32_t K = 0x04060401u;              // weights 1, 4, 6, 4 of taps 0..3
            const uint32_t v0 = dp4a_u8(a0, K, a1 & 0xFFu);
            const uint32_t v1 = dp4a_u8(__funnelshift_r(a0, a1, 16), K, (a1 >> 16) & 0xFFu);
            const uint32_t v2 = dp4a_u8(a1, K, a2 & 0xFFu);
            const uint32_t v3 = dp4a_u8(__funnelshift_r(a1, a2, 16), K, (a2 >> 16) & 0xFFu);
            t2[i] = make_uint2(__byte_perm(v0, v1, 0x5410), __byte_perm(v2, v3, 0x5410));
        }
    }
    __syncthreads();
    // vertical: RH(j) rows x NQ(j) quads -> 4 output bytes per item
    {
        constexpr int N = RHj * NQj;
        for (int i = tid; i < N; i += NT) {
            const int r = i / NQj, q = i - r * NQj;
            const uint2 *c = t2 + (2 * r) * NQj + q;
            const uint2 w0 = c[0], w1 = c[NQj], w2 = c[2 * NQj], w3 = c[3 * NQj], w4 = c[4 * NQj];
            uint32_t lo = w0.x + 4u * w1.x + 6u * w2.x + 4u * w3.x + w4.x;   // two 16-bit sums
            uint32_t hi = w0.y + 4u * w1.y + 6u * w2.y + 4u * w3.y + w4.y;
            lo = ((lo + 0x00800080u) >> 8) & 0x00FF00FFu;
            hi = ((hi + 0x00800080u) >> 8) & 0x00FF00FFu;
            reinterpret_cast<uint32_t *>(P + r * SJ)[q] = __byte_perm(lo, hi, 0x6420);
        }
    }
    __syncthreads();
    // border CTAs: positions outside the image take the clamped position's value
    {
        const int Wj = a.W[j], Hj = a.H[j];
        const int xl = -lox[j], xr = Wj - 1 - lox[j];        // in-image region columns
        const int yl = -loy[j], yr = Hj - 1 - loy[j];
        constexpr int NC = 4 * NQj;
        if (xl > 0 || xr < NC - 1 || yl > 0 || yr < RHj - 1) {
            if (xl > 0 || xr < NC - 1) {
                for (int i = tid; i < RHj * NC; i += NT) {
                    const int r = i / NC, c = i - r * NC;
                    if (c < xl) P[r * SJ + c] = P[r * SJ + xl];
                    else if (c > xr) P[r * SJ + c] = P[r * SJ + xr];
                }
                __syncthreads();
            }
            if (yl > 0 || yr < RHj - 1) {
                for (int i = tid; i < RHj * NQj; i += NT) {
                    const int r = i / NQj, q = i - r * NQj;
                    const int rs = min(max(r, yl), yr);
                    if (rs != r)
                        reinterpret_cast<uint32_t *>(P + r * SJ)[q] =
                            reinterpret_cast<const uint32_t *>(P + rs * SJ)[q];
                }
                __syncthreads();
            }
        }
    }
    if constexpr (J < F) pyr_levels<F, J + 1, NT>(a, lox, loy, sm);
}

// Own part (+ apron on border CTAs) of level J and the finer written levels, 16-byte chunks
// over the fixed grid of (tile / 16 + 2) chunk columns x (tile + 2 APY) rows around the own
// part (compile-time J).
template <int F, int J, int NT>
__device__ __forceinline__ void pyr_store(const PyrFuseArgs &a, const int (&lox)[F + 1], const int (&loy)[F + 1],
                                          int bx, int by, int img, int nbx, int nby, const uint8_t *sm) {
    using G = PyrGeom<F>;
    constexpr int j = J;
    constexpr int tx = PF_TX << (F - j), ty = PF_TY << (F - j);
    constexpr int CX = tx / 16 + 2, RY = ty + 2 * APY, N = CX * RY, SJ = G::STR(j), OFFJ = G::OFF(j);
    if (j > 0 || a.write_src) {
        const bool first_x = bx == 0, last_x = bx == nbx - 1;
        const bool first_y = by == 0, last_y = by == nby - 1;
        const int Wj = a.W[j], Hj = a.H[j];
        const int X0j = bx * tx, Y0j = by * ty;
        const int xs = first_x ? -APX : X0j, xe = last_x ? Wj + APX : X0j + tx;
        const int ys = first_y ? -APY : Y0j, ye = last_y ? Hj + APY : Y0j + ty;
        const uint8_t *P = sm + OFFJ;
        const int cb = j == 0 ? 2 - lox[0] : -lox[j];           // shared column of image column X: X + cb
        uint8_t *dst = a.dst[j][img];
        const ptrdiff_t dp = a.dpitch[j];
        for (int i = threadIdx.x; i < N; i += NT) {
            const int ry = i / CX, cx = i - ry * CX;
            const int X0 = X0j - 16 + 16 * cx, Y = Y0j - APY + ry;
            if (X0 < xs || X0 >= xe || Y < ys || Y >= ye) continue;
            const uint8_t *row = P + (min(max(Y, 0), Hj - 1) - loy[j]) * SJ;
            uint4 out;
            if (X0 >= 0 && X0 + 15 < Wj) {
                const int sc = X0 + cb;                                 // a multiple of 2
                const uint32_t *w = reinterpret_cast<const uint32_t *>(row + (sc & ~3));
                if (sc & 3) {
                    const uint32_t r0 = w[0], r1 = w[1], r2 = w[2], r3 = w[3], r4 = w[4];
                    out = make_uint4(__funnelshift_r(r0, r1, 16), __funnelshift_r(r1, r2, 16),
                                     __funnelshift_r(r2, r3, 16), __funnelshift_r(r3, r4, 16));
                } else {
                    out = make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else {
                uint32_t w[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t v = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        v |= static_cast<uint32_t>(row[min(max(X0 + 4 * k + b, 0), Wj - 1) + cb]) << (8 * b);
                    w[k] = v;
                }
                out = make_uint4(w[0], w[1], w[2], w[3]);
            }
            *reinterpret_cast<uint4 *>(dst + (ptrdiff_t)Y * dp + X0) = out;
        }
    }
    if constexpr (J < F) pyr_store<F, J + 1, NT>(a, lox, loy, bx, by, img, nbx, nby, sm);
}

// One tile (bx, by) of image `img` (0 left, 1 right) of a launch with nbx x nby tiles; the
// source level is src (pitch spitch; overrides a.src).  sm: PF_SMEM bytes, 16-aligned.
// blockDim.x == NT.
template <int F, int NT = 256>
__device__ void pyr_fused_tile(const PyrFuseArgs &a, const uint8_t *src, size_t spitch, int bx, int by, int img,
                               int nbx, int nby, uint8_t *sm) {
    using G = PyrGeom<F>;
    const int tid = threadIdx.x;
    int lox[F + 1], loy[F + 1];
    lox[F] = bx * PF_TX;
    loy[F] = by * PF_TY;
#pragma unroll
    for (int j = F - 1; j >= 0; --j) {
        lox[j] = 2 * lox[j + 1] - 2;
        loy[j] = 2 * loy[j + 1] - 2;
    }

    // ---- level s: rows loy0 .. loy0 + RH(0) - 1, bytes from image column lox0 - 2, clamped
    {
        constexpr int NW = G::STR(0) / 4, N = NW * G::RH(0), T = (N + NT - 1) / NT;
        const int W0 = a.W[0], H0 = a.H[0], xb = lox[0] - 2;
        const bool wordok = ((reinterpret_cast<uintptr_t>(src) | spitch) & 3) == 0;
        uint32_t v[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t, r = i / NW, w = i - r * NW;
            const int X = xb + 4 * w;
            const uint8_t *row = src + (size_t)min(max(loy[0] + r, 0), H0 - 1) * spitch;
            uint32_t u = 0;
            if (i < N) {
                if (wordok && X >= 0 && X + 3 < W0) {
                    u = __ldg(reinterpret_cast<const uint32_t *>(row + X));
                } else {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        u |= static_cast<uint32_t>(__ldg(row + min(max(X + b, 0), W0 - 1))) << (8 * b);
                }
            }
            v[t] = u;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t;
            if (i < N) reinterpret_cast<uint32_t *>(sm)[i] = v[t];
        }
    }
    __syncthreads();

    pyr_levels<F, 1, NT>(a, lox, loy, sm);

    pyr_store<F, 0, NT>(a, lox, loy, bx, by, img, nbx, nby, sm);
}

}  // namespace msbm
