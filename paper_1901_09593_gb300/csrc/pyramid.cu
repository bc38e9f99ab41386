// pyramid.cu -- Gaussian pyramid of the stereo pair (Sec. III, Fig. 1).
//
// Reading of the unstated filter: 5-tap binomial [1 4 6 4 1]/16 on each axis,
// clamp-to-edge, 2x decimation to ceil(W/2) x ceil(H/2), integer result
// (sum + 128) >> 8.  Levels stay uint8 so every ZNCC window sum is an exact integer.
//
// Both kernels write whole apron buffers: the value stored at (Y, X), for Y in
// [-APY, H+APY) and X in [-APX, W+APX), is the level pixel at (clamp(Y), clamp(X)).  The
// reduce step therefore reads its 5x5 support straight from the finer apron buffer with
// no index clamping (2y+a and 2x+b stay within two pixels of the image, inside the apron).
// Bound: HBM/L2 traffic (1 B read per source pixel, 1 B written per output pixel); the
// levels of a frame are small enough to stay resident in L2.
#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "pyramid_ops.cuh"

namespace msbm {

// Level 0: copy the caller's image (any pitch) into the apron buffer with replication.
// One thread per 16 consecutive output bytes of one apron row; blockIdx.z selects left (0)
// / right (1).  Interior runs whose source is 8-byte aligned are moved with two 8-byte
// loads and one 16-byte store; runs touching the apron or misaligned fall back to bytes.
__global__ void apron_copy_kernel(const uint8_t *__restrict__ srcL, const uint8_t *__restrict__ srcR,
                                  size_t spitch, int W, int H, uint8_t *dstL, uint8_t *dstR,
                                  int dpitch) {
    const uint8_t *src = blockIdx.z ? srcR : srcL;
    uint8_t *dst = blockIdx.z ? dstR : dstL;   // points at image (0, 0)
    const int X0 = (blockIdx.x * blockDim.x + threadIdx.x) * 16 - APX;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y - APY;
    if (Y >= H + APY || X0 >= W + APX) return;
    const int y = min(max(Y, 0), H - 1);
    const uint8_t *row = src + (size_t)y * spitch;
    uint4 out;
    if (X0 >= 0 && X0 + 16 <= W && ((reinterpret_cast<uintptr_t>(row + X0) & 7) == 0)) {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(row + X0));
        const uint2 b = __ldg(reinterpret_cast<const uint2 *>(row + X0 + 8));
        out = make_uint4(a.x, a.y, b.x, b.y);
    } else {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t v = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int x = min(max(X0 + 4 * q + i, 0), W - 1);
                v |= static_cast<uint32_t>(__ldg(row + x)) << (8 * i);
            }
            w[q] = v;
        }
        out = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // X0 + APX is a multiple of 16 and rows are 128-byte aligned; the 16 bytes may run past
    // W + APX into the row's padding (the pitch is a multiple of 128 >= W + 2*APX).
    *reinterpret_cast<uint4 *>(dst + (ptrdiff_t)Y * dpitch + X0) = out;
}

// Level k from level k-1.  One thread per 4 consecutive output bytes (the 5x5 support is
// read through the L1 cache; at these level sizes this beats a shared-memory staging pass).
__global__ void pyr_reduce_kernel(const uint8_t *__restrict__ srcL, const uint8_t *__restrict__ srcR,
                                  int spitch, uint8_t *dstL, uint8_t *dstR, int dpitch, int Wd,
                                  int Hd) {
    const uint8_t *src = blockIdx.z ? srcR : srcL;   // image (0, 0) of level k-1
    uint8_t *dst = blockIdx.z ? dstR : dstL;
    int X0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4 - APX;
    int Y = blockIdx.y * blockDim.y + threadIdx.y - APY;
    if (Y >= Hd + APY || X0 >= Wd + APX) return;
    reduce_quad(src, spitch, dst, dpitch, Wd, Hd, X0, Y);
}

cudaError_t launch_apron_copy(const uint8_t *L, const uint8_t *R, size_t spitch, const LevelBuf &lv,
                              cudaStream_t st) {
    dim3 blk(32, 8);
    const int cols16 = (lv.W + 2 * APX + 15) / 16;
    dim3 grd((cols16 + blk.x - 1) / blk.x, (lv.H + 2 * APY + blk.y - 1) / blk.y, 2);
    apron_copy_kernel<<<grd, blk, 0, st>>>(L, R, spitch, lv.W, lv.H, lv.img(0), lv.img(1), lv.pitch);
    return cudaGetLastError();
}

cudaError_t launch_pyr_reduce(const LevelBuf &src, const LevelBuf &dst, cudaStream_t st) {
    dim3 blk(32, 8);
    const int cols4 = (dst.W + 2 * APX + 3) / 4;
    dim3 grd((cols4 + blk.x - 1) / blk.x, (dst.H + 2 * APY + blk.y - 1) / blk.y, 2);
    pyr_reduce_kernel<<<grd, blk, 0, st>>>(src.img(0), src.img(1), src.pitch, dst.img(0), dst.img(1), dst.pitch,
                                           dst.W, dst.H);
    return cudaGetLastError();
}

// ---- fused pyramid: levels s+1 .. s+F (F <= PF_MAXF) in one launch ----------------------
//
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
// bytes.  The integer sums equal pyr_reduce_kernel's, hence the same bytes.  Neighbouring
// CTAs recompute the overlapping halos instead of exchanging them.
constexpr int PF_TX = 16, PF_TY = 8;
// shared bytes for F = 3 at most 29864: level regions of up to 152x85, 76x41, 40x19, 20x8
// bytes plus the widest horizontal-pass buffer (85 rows x 76 16-bit sums)
constexpr int PF_SMEM = 30 * 1024;

// (i, step) -> (row, column) walk of a rows x n grid without a division per step
struct GridWalk {
    int r, c, dr, dc, n;
    __device__ GridWalk(int i0, int step, int n_) : n(n_) {
        r = i0 / n;
        c = i0 - r * n;
        dr = step / n;
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

template <int F>
__global__ void __launch_bounds__(256) pyr_fused_kernel(const __grid_constant__ PyrFuseArgs a) {
    __shared__ __align__(16) uint8_t sm[PF_SMEM];
    const int img = blockIdx.z, tid = threadIdx.x;
    int lox[F + 1], hix[F + 1], loy[F + 1], hiy[F + 1];
    lox[F] = blockIdx.x * PF_TX;
    hix[F] = min(lox[F] + PF_TX, a.W[F]) - 1;
    loy[F] = blockIdx.y * PF_TY;
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
        const uint8_t *src = a.src[img];
        const bool wordok = ((reinterpret_cast<uintptr_t>(src) | a.spitch) & 3) == 0;
        const int nw = str[0] / 4, n = nw * ny[0], W0 = a.W[0];
        uint32_t v[T];
        GridWalk g(tid, 256, nw);
#pragma unroll
        for (int t = 0; t < T; ++t, g.next()) {
            v[t] = 0;
            if (tid + 256 * t < n) {
                const int X = org[0] + 4 * g.c;
                const uint8_t *row = src + (size_t)(loy[0] + g.r) * a.spitch;
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
        // horizontal: ny[j-1] rows x nq quads -> 16-bit sums, 4 per thread
        {
            const int n = ny[j - 1] * nq;
            GridWalk g(tid, 256, nq);
            for (int i = tid; i < n; i += 256, g.next()) {
                const int x = org[j] + 4 * g.c;           // first output column
                const uint8_t *row = Pp + g.r * sp;       // column X at row[X - op]
                uint32_t o01, o23;
                if (2 * x - 2 >= op && 2 * x + 8 <= fhi) {
                    const int s0 = 2 * x - 2 - op;        // even
                    const uint32_t *wr = reinterpret_cast<const uint32_t *>(row) + (s0 >> 2);
                    const int sh = (s0 & 3) * 8;          // 0 or 16
                    const uint32_t r0 = wr[0], r1 = wr[1], r2 = wr[2];
                    const uint32_t r3 = sh ? wr[3] : 0u;
                    const uint32_t a0 = __funnelshift_r(r0, r1, sh), a1 = __funnelshift_r(r1, r2, sh),
                                   a2 = __funnelshift_r(r2, r3, sh);
                    constexpr uint32_t K = 0x04060401u;   // weights 1, 4, 6, 4 of taps 0..3
                    const uint32_t v0 = dp4a_u8(a0, K, a1 & 0xFFu);
                    const uint32_t v1 = dp4a_u8(__funnelshift_r(a0, a1, 16), K, (a1 >> 16) & 0xFFu);
                    const uint32_t v2 = dp4a_u8(a1, K, a2 & 0xFFu);
                    const uint32_t v3 = dp4a_u8(__funnelshift_r(a1, a2, 16), K, (a2 >> 16) & 0xFFu);
                    o01 = v0 | (v1 << 16);
                    o23 = v2 | (v3 << 16);
                } else {
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
                    o01 = v[0] | (v[1] << 16);
                    o23 = v[2] | (v[3] << 16);
                }
                reinterpret_cast<uint2 *>(tmpb)[g.r * nq + g.c] = make_uint2(o01, o23);
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
    const bool first_x = blockIdx.x == 0, last_x = blockIdx.x == gridDim.x - 1;
    const bool first_y = blockIdx.y == 0, last_y = blockIdx.y == gridDim.y - 1;
#pragma unroll
    for (int j = 0; j <= F; ++j) {
        if (j == 0 && !a.write_src) continue;
        const int tx = PF_TX << (F - j), ty = PF_TY << (F - j);
        const int Wj = a.W[j], Hj = a.H[j];
        const int bx = static_cast<int>(blockIdx.x), by = static_cast<int>(blockIdx.y);
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

cudaError_t launch_pyr_fused(const PyrFuseArgs &a, cudaStream_t st) {
    if (a.F < 1 || a.F > PF_MAXF) return cudaErrorInvalidValue;
    dim3 grd((a.W[a.F] + PF_TX - 1) / PF_TX, (a.H[a.F] + PF_TY - 1) / PF_TY, 2);
    switch (a.F) {
        case 1: pyr_fused_kernel<1><<<grd, 256, 0, st>>>(a); break;
        case 2: pyr_fused_kernel<2><<<grd, 256, 0, st>>>(a); break;
        default: pyr_fused_kernel<3><<<grd, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// Dense copy of a level's interior (for inspection and tests).
__global__ void level_extract_kernel(const uint8_t *__restrict__ src, int spitch, int W, int H,
                                     uint8_t *dst) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < W && y < H) dst[(size_t)y * W + x] = src[(ptrdiff_t)y * spitch + x];
}

cudaError_t launch_level_extract(const LevelBuf &lv, int which, uint8_t *out, cudaStream_t st) {
    dim3 blk(32, 8), grd((lv.W + 31) / 32, (lv.H + 7) / 8);
    level_extract_kernel<<<grd, blk, 0, st>>>(lv.img(which), lv.pitch, lv.W, lv.H, out);
    return cudaGetLastError();
}

}  // namespace msbm
