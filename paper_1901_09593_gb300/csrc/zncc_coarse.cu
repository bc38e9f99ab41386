// zncc_coarse.cu -- full-range ZNCC winner-take-all (Sec. III-A, Eq. 1-4) for small levels
// (normally the coarsest pyramid level): every admissible candidate 0 <= z <= min(D_k - 1, x)
// of every pixel.  The full-range tile kernel (zncc_full.cu) is built for throughput on large
// searches; on a level of a few ten thousand pixels its 32 x 8 tiles leave most SMs idle and
// each CTA runs a long serial chain.  Here one thread owns one pixel of a 32 x 8 tile and
// walks the candidates 4 at a time (zncc_region.cuh): the CTA stages the tile's left rows
// once and, per 32-candidate chunk, the right rows and their window statistics.  WTA on the
// 64-bit (ordered rho, ~z) key: exact ties keep the smallest z.
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_region.cuh"

namespace msbm {

namespace {

constexpr int CO_TX = 32, CO_TY = 8;

template <int NH>
__global__ void __launch_bounds__(256) zncc_coarse_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W,
                                                          int H, int Dk, int16_t *d_out, float *c_out,
                                                          unsigned long long *evals) {
    using region::ZC;
    constexpr int WIN = 2 * NH + 1, NW = (WIN + 3) / 4;
    constexpr int SLW = CO_TX + 2 * NH, SLH = CO_TY + 2 * NH;   // staged left region
    constexpr int SU = CO_TX + ZC - 1;                          // right window columns per chunk
    constexpr int SRW = SU + 2 * NH;                            // staged right columns per chunk
    constexpr int SRWW = (SRW + 3) / 4 + 2;                     // words per staged right row
    __shared__ uint8_t sL[SLH * SLW];
    __shared__ uint32_t sR[SLH * SRWW];
    __shared__ int vs[CO_TY * SRW], vq[CO_TY * SRW];
    __shared__ int2 stR[CO_TY * SU];
    __shared__ unsigned long long evsum;
    const int tid = threadIdx.x, pr = tid / CO_TX, pc = tid % CO_TX;
    const int x0 = blockIdx.x * CO_TX, y0 = blockIdx.y * CO_TY;
    const int x = x0 + pc, y = y0 + pr;
    if (tid == 0) evsum = 0ull;
    region::stage_rows<SLH, SLW, SLW>(sL, L, pitch, W, H, y0 - NH, x0 - NH);
    __syncthreads();
    uint32_t Lw[WIN][NW];
    const int2 la = region::pack_left<NH, SLW>(sL, pr, pc, Lw);
    const int zmax = min(Dk - 1, x);
    const int zmax_tile = min(Dk - 1, min(x0 + CO_TX, W) - 1);
    unsigned long long best = 0ull;
    for (int z0 = 0; z0 <= zmax_tile; z0 += ZC) {
        __syncthreads();      // the previous chunk's rows and statistics are consumed
        region::stage_rows<SLH, SRW, SRWW * 4>(reinterpret_cast<uint8_t *>(sR), R, pitch, W, H, y0 - NH,
                                                x0 - (z0 + ZC - 1) - NH);
        __syncthreads();
        region::window_stats<NH, CO_TY, SU, SRWW * 4>(reinterpret_cast<const uint8_t *>(sR), vs, vq, stR);
#pragma unroll 1
        for (int g = 0; g < ZC / 4 && z0 + 4 * g <= zmax; ++g) {
            const int um = pc + ZC - 4 - 4 * g;       // staged column of candidate z0 + 4g + 3
            uint32_t sab[4];
            region::sab4<NH, SRWW>(sR, pr, um, Lw, sab);
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int z = z0 + 4 * g + 3 - o;
                if (z > zmax) continue;
                const unsigned long long k = wta_key(region::rho_of<NH>(sab[o], la, stR[pr * SU + um + o]), z);
                best = k > best ? k : best;
            }
        }
    }
    const bool in = x < W && y < H;
    if (in) {
        const size_t p = (size_t)y * W + x;
        d_out[p] = static_cast<int16_t>(0xFFFFFFFFu - static_cast<uint32_t>(best & 0xFFFFFFFFull));
        if (c_out) c_out[p] = fminf(1.f, fmaxf(-1.f, float_from_order_key(static_cast<uint32_t>(best >> 32))));
    }
    if (evals) {
        const unsigned cnt = __reduce_add_sync(0xFFFFFFFFu, in ? static_cast<unsigned>(zmax + 1) : 0u);
        if ((tid & 31) == 0) atomicAdd(&evsum, static_cast<unsigned long long>(cnt));
        __syncthreads();
        if (tid == 0) atomicAdd(evals, evsum);
    }
}

template <int NH>
cudaError_t coarse_launch(const LevelBuf &l, int16_t *d, float *c, unsigned long long *evals, cudaStream_t st) {
    dim3 grd((l.W + CO_TX - 1) / CO_TX, (l.H + CO_TY - 1) / CO_TY);
    zncc_coarse_kernel<NH><<<grd, 256, 0, st>>>(l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, d, c, evals);
    return cudaGetLastError();
}

}  // namespace

bool zncc_coarse_fits(int W, int H, int sms) {
    // the full-range tile kernel's 32 x 8 tiles cannot fill the GPU twice over
    return (long)((W + 31) / 32) * ((H + 7) / 8) < 2L * sms;
}

cudaError_t launch_zncc_coarse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st) {
    switch (nh) {
        case 1: return coarse_launch<1>(l, d, c, evals, st);
        case 2: return coarse_launch<2>(l, d, c, evals, st);
        case 3: return coarse_launch<3>(l, d, c, evals, st);
        case 4: return coarse_launch<4>(l, d, c, evals, st);
        case 5: return coarse_launch<5>(l, d, c, evals, st);
        case 6: return coarse_launch<6>(l, d, c, evals, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
