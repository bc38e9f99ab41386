// gated.cu -- the gated steps of the full method (Sec. III-B, the second branch of
// Eq. 8-9, Sec. III-D), each a small kernel around the matching kernels:
//  * beta gate (Sec. III-C): the cost prior C_hat^k = BI(C^{k+1}) -- bicubic (Catmull-Rom)
//    upsampling with fine pixel (y, x) at coarse coordinates (y/2, x/2), clamp-to-edge --
//    and the fallback mask C_hat <= beta, plus one flag per full-range tile that holds a
//    fallback pixel (the gated full-range pass then runs only those tiles and writes only
//    the fallback pixels);
//  * alpha refinement (Eq. 5-7) at the coarsest level: for a pixel with C' <= alpha, the
//    average of the ZNCC over its 3 x 3 neighbourhood (neighbours inside the image) for
//    every admissible candidate, and its argmax / max;
//  * selective median (Eq. 10): for a pixel with C <= alpha, the lower median of the 5 x 5
//    neighbours whose cost exceeds alpha (unchanged when none does).
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {

namespace {

// Catmull-Rom weights of the samples at offsets -1, 0, 1, 2 for the fractional position
// of fine index i (0 or 1/2).
__device__ __forceinline__ void cr_weights(int i, float w[4], int &base) {
    base = i >> 1;
    if (i & 1) {
        w[0] = -1.f / 16.f; w[1] = 9.f / 16.f; w[2] = 9.f / 16.f; w[3] = -1.f / 16.f;
    } else {
        w[0] = 0.f; w[1] = 1.f; w[2] = 0.f; w[3] = 0.f;
    }
}

__global__ void beta_gate_kernel(const float *__restrict__ Cc, int Wc, int Hc, int W, int H, float beta,
                                 uint8_t *mask, int *tile_flags, int tile_w, int tile_h, int tiles_x) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    bool fb = false;
    if (x < W && y < H) {
        float wy[4], wx[4];
        int by, bx;
        cr_weights(y, wy, by);
        cr_weights(x, wx, bx);
        float s = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int yy = min(max(by - 1 + a, 0), Hc - 1);
            float r = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) r = fmaf(wx[b], __ldg(Cc + (size_t)yy * Wc + min(max(bx - 1 + b, 0), Wc - 1)), r);
            s = fmaf(wy[a], r, s);
        }
        fb = !(s > beta);
        mask[(size_t)y * W + x] = fb ? 1 : 0;
        if (fb) atomicOr(tile_flags + (y / tile_h) * tiles_x + x / tile_w, 1);
    }
}

// Exact-integer ZNCC of the left window at (y, x) and the right window at (y, x - z), read
// from apron buffers (no clamping needed); rho from c * rsqrt(Va) * rsqrt(Vb).
template <int NH>
__device__ __forceinline__ float zncc_direct(const uint8_t *L, const uint8_t *R, int pitch, int y, int x, int z) {
    constexpr int WIN = 2 * NH + 1, N = WIN * WIN;
    int sa = 0, sb = 0, saa = 0, sbb = 0, sab = 0;
#pragma unroll
    for (int i = -NH; i <= NH; ++i) {
        const uint8_t *lr = L + (ptrdiff_t)(y + i) * pitch + x;
        const uint8_t *rr = R + (ptrdiff_t)(y + i) * pitch + x - z;
#pragma unroll
        for (int j = -NH; j <= NH; ++j) {
            const int a = __ldg(lr + j), b = __ldg(rr + j);
            sa += a; sb += b; saa += a * a; sbb += b * b; sab += a * b;
        }
    }
    const int va = N * saa - sa * sa, vb = N * sbb - sb * sb;
    if (va <= 0 || vb <= 0) return 0.f;
    return static_cast<float>(N * sab - sa * sb) * rsqrtf(static_cast<float>(va)) * rsqrtf(static_cast<float>(vb));
}

// One warp per pixel; the warp skips pixels whose cost exceeds alpha.
template <int NH>
__global__ void alpha_refine_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int Dk,
                                    float alpha, int16_t *d, float *C, unsigned long long *evals) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= W * H) return;
    const int y = p / W, x = p - y * W;
    if (C[p] > alpha) return;
    const int zmax = min(Dk - 1, x);
    const int y0 = max(y - 1, 0), y1 = min(y + 1, H - 1), x0 = max(x - 1, 0), x1 = min(x + 1, W - 1);
    const float inv = 1.f / static_cast<float>((y1 - y0 + 1) * (x1 - x0 + 1));
    unsigned long long best = 0ull;
    for (int z = lane; z <= zmax; z += 32) {
        float s = 0.f;
        for (int m = y0; m <= y1; ++m)
            for (int q = x0; q <= x1; ++q) s += zncc_direct<NH>(L, R, pitch, m, q, z);
        const unsigned long long k = wta_key(s * inv, z);
        best = k > best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = k > best ? k : best;
    }
    if (lane == 0) {
        d[p] = static_cast<int16_t>(0xFFFFFFFFu - static_cast<uint32_t>(best & 0xFFFFFFFFull));
        C[p] = float_from_order_key(static_cast<uint32_t>(best >> 32));
        if (evals)
            atomicAdd(evals, static_cast<unsigned long long>((y1 - y0 + 1) * (x1 - x0 + 1)) * (zmax + 1));
    }
}

__global__ void selective_median_kernel(const int16_t *__restrict__ d_in, const float *__restrict__ C, int W,
                                        int H, float alpha, int16_t *d_out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t o = (size_t)y * W + x;
    int16_t out = d_in[o];
    if (!(C[o] > alpha)) {
        int v[25], cnt = 0;
        for (int m = max(y - 2, 0); m <= min(y + 2, H - 1); ++m)
            for (int q = max(x - 2, 0); q <= min(x + 2, W - 1); ++q) {
                const size_t p = (size_t)m * W + q;
                if (__ldg(C + p) > alpha) v[cnt++] = __ldg(d_in + p);
            }
        if (cnt > 0) {
            for (int i = 1; i < cnt; ++i) {           // insertion sort of at most 24 values
                const int t = v[i];
                int j = i - 1;
                while (j >= 0 && v[j] > t) {
                    v[j + 1] = v[j];
                    --j;
                }
                v[j + 1] = t;
            }
            out = static_cast<int16_t>(v[(cnt - 1) / 2]);
        }
    }
    d_out[o] = out;
}

}  // namespace

cudaError_t launch_beta_gate(const float *Cc, int Wc, int Hc, int W, int H, float beta, uint8_t *mask,
                             int *tile_flags, int tile_w, int tile_h, cudaStream_t st) {
    const int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    cudaError_t e = cudaMemsetAsync(tile_flags, 0, sizeof(int) * tiles_x * tiles_y, st);
    if (e != cudaSuccess) return e;
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
    beta_gate_kernel<<<grd, blk, 0, st>>>(Cc, Wc, Hc, W, H, beta, mask, tile_flags, tile_w, tile_h, tiles_x);
    return cudaGetLastError();
}

template <int NH>
static cudaError_t alpha_launch(const LevelBuf &l, float alpha, int16_t *d, float *C, unsigned long long *evals,
                                cudaStream_t st) {
    const int warps = 8;
    dim3 blk(32 * warps), grd((l.W * l.H + warps - 1) / warps);
    alpha_refine_kernel<NH><<<grd, blk, 0, st>>>(l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, alpha, d, C, evals);
    return cudaGetLastError();
}

cudaError_t launch_alpha_refine(const LevelBuf &l, int nh, float alpha, int16_t *d, float *C,
                                unsigned long long *evals, cudaStream_t st) {
    switch (nh) {
        case 1: return alpha_launch<1>(l, alpha, d, C, evals, st);
        case 2: return alpha_launch<2>(l, alpha, d, C, evals, st);
        case 3: return alpha_launch<3>(l, alpha, d, C, evals, st);
        case 4: return alpha_launch<4>(l, alpha, d, C, evals, st);
        case 5: return alpha_launch<5>(l, alpha, d, C, evals, st);
        case 6: return alpha_launch<6>(l, alpha, d, C, evals, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_selective_median(const int16_t *d_in, const float *C, int W, int H, float alpha, int16_t *d_out,
                                    cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
    selective_median_kernel<<<grd, blk, 0, st>>>(d_in, C, W, H, alpha, d_out);
    return cudaGetLastError();
}

}  // namespace msbm
