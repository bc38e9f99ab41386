// pyramid_fused.cuh -- one tile of the fused Gaussian pyramid (Sec. III, Fig. 1): levels
// s+1 .. s+F built from level s by one CTA, shared by the standalone launch (pyramid.cu) and
// the batched persistent kernel (batch.cu).  Filter reading: 5-tap binomial [1 4 6 4 1]/16
// per axis, clamp-to-edge, 2x decimation to ceil(W/2) x ceil(H/2), (sum + 128) >> 8.
#pragma once

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {

// One CTA per (PF_TX x PF_TY tile of the coarsest fused level c = s + F, image).  Level j of
// the CTA's pyramid covers the in-image index range N_j: N_c is the CTA's own tile and
// N_j = [2 lo(N_{j+1}) - 2, 2 hi(N_{j+1}) + 2] clipped to the image, which holds the 5 x 5
// support (clamped) of every pixel of N_{j+1} and the CTA's own part of level j (2^(c-j)
// times its tile).  Shared level j holds columns org_j = lo(N_j) rounded down to a multiple
// of 4 onward (rows a multiple of 4 bytes), so every pass moves whole words:
//  * level s is read once with 4-byte loads (bytes where the caller's rows are unaligned);
//  * a horizontal [1 4 6 4 1] pass makes 4 outputs per thread from 3 aligned words with
//    funnel shifts and dp4a (weights 1,4,6,4 plus the fifth byte), into 16-bit sums;
//  * a vertical pass adds 5 rows of those sums two columns per 32-bit word (each 16-bit
//    half stays below 2^16), rounds with (v + 128) >> 8 and packs 4 output bytes;
//  * every written level's own part, plus the apron on border CTAs, leaves in 16-byte
//    chunks (word loads inside the image, clamped byte loads in the apron).
// Near the image border (or the region edge) the horizontal pass falls back to clamped
// bytes.  The integer sums are those of the 5 x 5 binomial support, hence exact.  Neighbouring
// CTAs recompute the overlapping halos instead of exchanging them.
constexpr int PF_TX = 16, PF_TY = 8;
// shared bytes for F = 3 at most 29864: level regions of up to 152x85, 76x41, 40x19, 20x8
// bytes plus the widest horizontal-pass buffer (85 rows x 76 16-bit sums)
constexpr int PF_SMEM = 30 * 1024;

// (i, step) -> (row, column) walk of a rows x n grid without a division per step.  The two
// quotients at construction use IEEE single-precision division, exact here: for
// 0 <= a, b < 2^16 the correctly rounded a / b truncates to floor(a / b).
__device__ __forceinline__ int small_div(int a, int b) {
    return __float2int_rz(__fdiv_rn(static_cast<float>(a), static_cast<float>(b)));
}

struct GridWalk {
    int r, c, dr, dc, n;
    __device__ GridWalk(int i0, int step, int n_) : n(n_) {
        r = small_div(i0, n);
        c = i0 - r * n;
        dr = small_div(step, n);
        dc = step - dr * n;
    }
    __device__ void next() {
        r += dr;
        c += dc;
        if (c >= n) {
            c -= n;
            ++r;
        }
    }
};

// One tile (bx, by) of image `img` (0 left, 1 right) of a launch with nbx x nby tiles; the
// source level is src (pitch spitch; overrides a.src).  sm: PF_SMEM bytes, 16-aligned.
// blockDim.x == 256.
template <int F>
__device__ void pyr_fused_tile(const PyrFuseArgs &a, const uint8_t *src, size_t spitch, int bx, int by, int img,
                               int nbx, int nby, uint8_t *sm) {
    const int tid = threadIdx.x;
    int lox[F + 1], hix[F + 1], loy[F + 1], hiy[F + 1];
    lox[F] = bx * PF_TX;
    hix[F] = min(lox[F] + PF_TX, a.W[F]) - 1;
    loy[F] = by * PF_TY;
    hiy[F] = min(loy[F] + PF_TY, a.H[F]) - 1;
#pragma unroll
    for (int j = F - 1; j >= 0; --j) {
        lox[j] = max(0, 2 * lox[j + 1] - 2);
        hix[j] = min(a.W[j] - 1, 2 * hix[j + 1] + 2);
        loy[j] = max(0, 2 * loy[j + 1] - 2);
        hiy[j] = min(a.H[j] - 1, 2 * hiy[j + 1] + 2);
    }
    // shared level j: ny[j] rows of str[j] bytes, first column org[j]
    int ny[F + 1], org[F + 1], str[F + 1], off[F + 2];
    off[0] = 0;
#pragma unroll
    for (int j = 0; j <= F; ++j) {
        ny[j] = hiy[j] - loy[j] + 1;
        org[j] = lox[j] & ~3;
        str[j] = (hix[j] + 1 - org[j] + 3) / 4 * 4;
        off[j + 1] = off[j] + (str[j] * ny[j] + 15) / 16 * 16;
    }
    uint8_t *tmpb = sm + off[F + 1];

    // level s into shared memory (all loads issued before any store)
    {
        constexpr int NY0 = (PF_TY << F) + 3 * ((1 << F) - 1), NX0 = (PF_TX << F) + 3 * ((1 << F) - 1);
        constexpr int NWD = (NX0 + 6) / 4, T = (NY0 * NWD + 255) / 256;
        const bool wordok = ((reinterpret_cast<uintptr_t>(src) | spitch) & 3) == 0;
        const int nw = str[0] / 4, n = nw * ny[0], W0 = a.W[0];
        uint32_t v[T];
        GridWalk g(tid, 256, nw);
#pragma unroll
        for (int t = 0; t < T; ++t, g.next()) {
            v[t] = 0;
            if (tid + 256 * t < n) {
                const int X = org[0] + 4 * g.c;
                const uint8_t *row = src + (size_t)(loy[0] + g.r) * spitch;
                if (wordok && X + 3 < W0) {
                    v[t] = __ldg(reinterpret_cast<const uint32_t *>(row + X));
                } else {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (X + b < W0) v[t] |= static_cast<uint32_t>(__ldg(row + X + b)) << (8 * b);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            if (i < n) reinterpret_cast<uint32_t *>(sm)[i] = v[t];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 1; j <= F; ++j) {
        const uint8_t *Pp = sm + off[j - 1];
        const int op = org[j - 1], sp = str[j - 1], Wp = a.W[j - 1], Hp = a.H[j - 1];
        const int nq = str[j] / 4;                        // column quads of level j
        const int fhi = min(op + sp, Wp) - 1;             // last column the fast path may read
        // horizontal: ny[j-1] rows x nq quads -> 16-bit sums, 4 per thread.  Whether a quad's
        // 11 input bytes lie inside the staged row and the image depends on its column only:
        // quads mlo .. mhi take the word path, the few others (region edges, image borders)
        // the clamped byte path, in a loop of their own so that no warp runs both.
        {
            const int mlo = max(0, (op + 2 - 2 * org[j] + 7) >> 3);          // 2x - 2 >= op
            const int mhi = min(nq - 1, (fhi - 8 - 2 * org[j]) >> 3);         // 2x + 8 <= fhi
            const int nf = max(0, mhi - mlo + 1);
            uint2 *t2 = reinterpret_cast<uint2 *>(tmpb);
            if (nf > 0) {
                const int n = ny[j - 1] * nf;
                GridWalk g(tid, 256, nf);
                for (int i = tid; i < n; i += 256, g.next()) {
                    const int m = mlo + g.c, x = org[j] + 4 * m;     // first output column
                    const int s0 = 2 * x - 2 - op;                   // even
                    const uint32_t *wr = reinterpret_cast<const uint32_t *>(Pp + g.r * sp) + (s0 >> 2);
                    const int sh = (s0 & 3) * 8;                     // 0 or 16
                    const uint32_t r0 = wr[0], r1 = wr[1], r2 = wr[2];
                    const uint32_t r3 = sh ? wr[3] : 0u;
                    const uint32_t a0 = __funnelshift_r(r0, r1, sh), a1 = __funnelshift_r(r1, r2, sh),
                                   a2 = __funnelshift_r(r2, r3, sh);
                    constexpr uint32_t K = 0x04060401u;              // weights 1, 4, 6, 4 of taps 0..3
                    const uint32_t v0 = dp4a_u8(a0, K, a1 & 0xFFu);
                    const uint32_t v1 = dp4a_u8(__funnelshift_r(a0, a1, 16), K, (a1 >> 16) & 0xFFu);
                    const uint32_t v2 = dp4a_u8(a1, K, a2 & 0xFFu);
                    const uint32_t v3 = dp4a_u8(__funnelshift_r(a1, a2, 16), K, (a2 >> 16) & 0xFFu);
                    t2[g.r * nq + m] = make_uint2(v0 | (v1 << 16), v2 | (v3 << 16));
                }
            }
            if (nf < nq) {
                const int ns = nq - nf, n = ny[j - 1] * ns;
                GridWalk g(tid, 256, ns);
                for (int i = tid; i < n; i += 256, g.next()) {
                    const int m = g.c < mlo ? g.c : g.c + nf, x = org[j] + 4 * m;
                    const uint8_t *row = Pp + g.r * sp;              // column X at row[X - op]
                    uint32_t v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int xx = min(max(x + q, lox[j]), hix[j]);   // columns outside N_j: unused
                        const int x2 = 2 * xx - 2 - op;
                        const int c0 = max(x2, -op), c1 = max(x2 + 1, -op);
                        const int c2 = min(x2 + 2, Wp - 1 - op), c3 = min(x2 + 3, Wp - 1 - op),
                                  c4 = min(x2 + 4, Wp - 1 - op);
                        v[q] = row[c0] + 4u * row[c1] + 6u * row[c2] + 4u * row[c3] + row[c4];
                    }
                    t2[g.r * nq + m] = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
                }
            }
        }
        __syncthreads();
        // vertical: ny[j] rows x nq quads -> 4 output bytes per thread
        {
            uint8_t *P = sm + off[j];
            const int n = ny[j] * nq, ylo = -loy[j - 1], yhi = Hp - 1 - loy[j - 1];
            const uint2 *t2 = reinterpret_cast<const uint2 *>(tmpb);
            GridWalk g(tid, 256, nq);
            for (int i = tid; i < n; i += 256, g.next()) {
                const int y2 = 2 * (loy[j] + g.r) - 2 - loy[j - 1];
                const uint2 w0 = t2[max(y2, ylo) * nq + g.c], w1 = t2[max(y2 + 1, ylo) * nq + g.c];
                const uint2 w2 = t2[min(y2 + 2, yhi) * nq + g.c], w3 = t2[min(y2 + 3, yhi) * nq + g.c];
                const uint2 w4 = t2[min(y2 + 4, yhi) * nq + g.c];
                uint32_t lo = w0.x + 4u * w1.x + 6u * w2.x + 4u * w3.x + w4.x;   // two 16-bit sums
                uint32_t hi = w0.y + 4u * w1.y + 6u * w2.y + 4u * w3.y + w4.y;
                lo = ((lo + 0x00800080u) >> 8) & 0x00FF00FFu;
                hi = ((hi + 0x00800080u) >> 8) & 0x00FF00FFu;
                reinterpret_cast<uint32_t *>(P)[g.r * nq + g.c] = __byte_perm(lo, hi, 0x6420);
            }
        }
        __syncthreads();
    }
    // own parts (+ aprons on border CTAs) of every written level, 16-byte chunks
    const bool first_x = bx == 0, last_x = bx == nbx - 1;
    const bool first_y = by == 0, last_y = by == nby - 1;
#pragma unroll
    for (int j = 0; j <= F; ++j) {
        if (j == 0 && !a.write_src) continue;
        const int tx = PF_TX << (F - j), ty = PF_TY << (F - j);
        const int Wj = a.W[j], Hj = a.H[j];
        const int xs = first_x ? -APX : bx * tx, xe = last_x ? Wj + APX : (bx + 1) * tx;
        const int ys = first_y ? -APY : by * ty, ye = last_y ? Hj + APY : (by + 1) * ty;
        const int ncx = (xe - xs + 15) / 16, n = ncx * (ye - ys);
        const uint8_t *P = sm + off[j];
        uint8_t *dst = a.dst[j][img];
        GridWalk g(tid, 256, ncx);
        for (int i = tid; i < n; i += 256, g.next()) {
            const int X0 = xs + 16 * g.c, Y = ys + g.r;
            const uint8_t *row = P + (min(max(Y, 0), Hj - 1) - loy[j]) * str[j] - org[j];
            uint4 out;
            if (X0 >= 0 && X0 + 15 < Wj) {
                const uint32_t *w = reinterpret_cast<const uint32_t *>(row + X0);   // X0 - org[j] = 0 mod 4
                out = make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                uint32_t w[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t v = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        v |= static_cast<uint32_t>(row[min(max(X0 + 4 * k + b, 0), Wj - 1)]) << (8 * b);
                    w[k] = v;
                }
                out = make_uint4(w[0], w[1], w[2], w[3]);
            }
            *reinterpret_cast<uint4 *>(dst + (ptrdiff_t)Y * a.dpitch[j] + X0) = out;
        }
    }
}

}  // namespace msbm
