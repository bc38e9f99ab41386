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
// times its tile).  Level s is read once into shared memory; each finer-to-coarser step is a
// horizontal then a vertical [1 4 6 4 1] pass with the support index clamped to the level
// (the same integer sums as pyr_reduce_kernel, hence the same bytes); every level's own part
// plus, on border CTAs, the apron is then written in 16-byte chunks.  Neighbouring CTAs
// recompute the overlapping halos instead of exchanging them.
constexpr int PF_TX = 16, PF_TY = 8;
// shared bytes for F = 3: level regions 152x85 (word-aligned rows) + 73x41 + 35x19 + 16x8
// (16-byte rounded) plus the widest horizontal-pass buffer 85 x 73 x 2: 29146
constexpr int PF_SMEM = 30 * 1024;

template <int F>
__global__ void __launch_bounds__(256) pyr_fused_kernel(const __grid_constant__ PyrFuseArgs a) {
    __shared__ __align__(16) uint8_t sm[PF_SMEM];
    const int img = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int lox[F + 1], hix[F + 1], loy[F + 1], hiy[F + 1], off[F + 2];
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
    // shared level j: row stride str[j], first column org[j] (level s: word-aligned origin)
    int nx[F + 1], ny[F + 1], org[F + 1], str[F + 1];
    off[0] = 0;
#pragma unroll
    for (int j = 0; j <= F; ++j) {
        nx[j] = hix[j] - lox[j] + 1;
        ny[j] = hiy[j] - loy[j] + 1;
        org[j] = j == 0 ? (lox[0] & ~3) : lox[j];
        str[j] = j == 0 ? (hix[0] + 1 - org[0] + 3) / 4 * 4 : nx[j];
        off[j + 1] = off[j] + (str[j] * ny[j] + 15) / 16 * 16;
    }
    uint16_t *tmp = reinterpret_cast<uint16_t *>(sm + off[F + 1]);

    // level s into shared memory as words (all loads issued before any store): 4-byte loads
    // where the source rows are 4-byte aligned and the word lies inside the row, else bytes
    {
        constexpr int NY0 = (PF_TY << F) + 3 * ((1 << F) - 1), NX0 = (PF_TX << F) + 3 * ((1 << F) - 1);
        constexpr int NWD = (NX0 + 6) / 4, T = (NY0 * NWD + 255) / 256;
        const uint8_t *src = a.src[img];
        const bool wordok = ((reinterpret_cast<uintptr_t>(src) | a.spitch) & 3) == 0;
        const int nw = str[0] / 4, n = nw * ny[0], W0 = a.W[0];
        uint32_t v[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + 256 * t;
            v[t] = 0;
            if (i < n) {
                const int r = i / nw, X = org[0] + 4 * (i - r * nw);
                const uint8_t *row = src + (size_t)(loy[0] + r) * a.spitch;
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
    // levels s+1 .. c
#pragma unroll
    for (int j = 1; j <= F; ++j) {
        const uint8_t *Pp = sm + off[j - 1];
        uint8_t *P = sm + off[j];
        const int Wp = a.W[j - 1], Hp = a.H[j - 1];
        for (int r = warp; r < ny[j - 1]; r += 8)
            for (int q = lane; q < nx[j]; q += 32) {
                const int x2 = 2 * (lox[j] + q) - 2;
                const uint8_t *row = Pp + r * str[j - 1] - org[j - 1];
                const int v = row[max(x2, 0)] + 4 * row[max(x2 + 1, 0)] + 6 * row[min(x2 + 2, Wp - 1)] +
                              4 * row[min(x2 + 3, Wp - 1)] + row[min(x2 + 4, Wp - 1)];
                tmp[r * nx[j] + q] = static_cast<uint16_t>(v);
            }
        __syncthreads();
        for (int r = warp; r < ny[j]; r += 8) {
            const int y2 = 2 * (loy[j] + r) - 2 - loy[j - 1];
            const int ylo = -loy[j - 1], yhi = Hp - 1 - loy[j - 1];
            const uint16_t *t0 = tmp + max(y2, ylo) * nx[j];
            const uint16_t *t1 = tmp + max(y2 + 1, ylo) * nx[j];
            const uint16_t *t2 = tmp + min(y2 + 2, yhi) * nx[j];
            const uint16_t *t3 = tmp + min(y2 + 3, yhi) * nx[j];
            const uint16_t *t4 = tmp + min(y2 + 4, yhi) * nx[j];
            for (int q = lane; q < nx[j]; q += 32) {
                const int v = t0[q] + 4 * t1[q] + 6 * t2[q] + 4 * t3[q] + t4[q];
                P[r * nx[j] + q] = static_cast<uint8_t>((v + 128) >> 8);
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
        const int xs = first_x ? -APX : blockIdx.x * tx, xe = last_x ? Wj + APX : (blockIdx.x + 1) * tx;
        const int ys = first_y ? -APY : blockIdx.y * ty, ye = last_y ? Hj + APY : (blockIdx.y + 1) * ty;
        const int ncx = (xe - xs + 15) / 16, n = ncx * (ye - ys);
        const uint8_t *P = sm + off[j];
        uint8_t *dst = a.dst[j][img];
        for (int i = tid; i < n; i += 256) {
            const int r = i / ncx, X0 = xs + 16 * (i - r * ncx), Y = ys + r;
            const uint8_t *row = P + (min(max(Y, 0), Hj - 1) - loy[j]) * str[j] - org[j];
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t v = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    v |= static_cast<uint32_t>(row[min(max(X0 + 4 * k + b, 0), Wj - 1)]) << (8 * b);
                w[k] = v;
            }
            *reinterpret_cast<uint4 *>(dst + (ptrdiff_t)Y * a.dpitch[j] + X0) = make_uint4(w[0], w[1], w[2], w[3]);
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
