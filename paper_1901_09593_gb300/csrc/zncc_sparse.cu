// zncc_sparse.cu -- the beta fallback's full-range search (Sec. III-C, Eq. 8-9 second branch)
// for the masked pixels of a level only: every admissible candidate 0 <= z <= min(D_k - 1, x)
// of each pixel whose bicubic cost prior failed the gate.
//
// One CTA per 64-pixel segment of one row.  The CTA compacts the segment's masked pixels
// with warp ballots (a segment without any exits at once), stages the left rows of the
// segment and, per 256-candidate chunk, the right rows the chunk reads, and gives each
// masked pixel to one warp: the lanes take groups of 4 consecutive candidates, extract the 4
// right windows from 3 aligned words per row with funnel shifts and accumulate sum a*b with
// dp4a (zncc_region.cuh); the right-window statistics come from the level's plane, staged
// per chunk.  The warp
// reduces its 64-bit (ordered rho, ~z) keys: exact ties keep the smallest z.  Work is
// proportional to the masked pixels, not to the tiles that hold one.
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_region.cuh"

namespace msbm {

namespace {

constexpr int SP_S = 64;         // pixels per segment
constexpr int SP_THREADS = 128;  // 4 warps
constexpr int SP_ZCH = 256;      // candidates per chunk

template <int NH>
struct SparseCfg {
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int SLW = SP_S + 2 * NH;                  // staged left columns
    static constexpr int SRW = SP_S + SP_ZCH - 1 + 2 * NH;     // staged right columns per chunk
    static constexpr int SRWW = (SRW + 3) / 4 + 2;             // words per staged right row
};

template <int NH>
__global__ void __launch_bounds__(SP_THREADS) zncc_sparse_kernel(const uint8_t *L, const uint8_t *R, int pitch,
                                                                 int W, int H, int Dk, const uint8_t *mask,
                                                                 const int2 *rstat, int rspitch, int16_t *d_out,
                                                                 float *c_out, unsigned long long *evals) {
    using C = SparseCfg<NH>;
    constexpr int WIN = C::WIN, NW = (WIN + 3) / 4, SLW = C::SLW, SRW = C::SRW, SRWW = C::SRWW;
    __shared__ uint8_t sL[WIN * SLW];
    __shared__ uint32_t sR[WIN * SRWW];
    __shared__ int2 sS[SP_S + SP_ZCH - 1];         // plane entries of the chunk's right windows
    __shared__ int list[SP_S];
    __shared__ unsigned long long best[SP_S];
    __shared__ uint32_t sLw[SP_S][WIN][NW];        // each masked pixel's packed left window
    __shared__ int2 sLa[SP_S];                     // and its {Sa, bits(rsqrt(Va)) or 0}
    __shared__ int nlist;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * SP_S, y = blockIdx.y;
    if (tid == 0) nlist = 0;
    __syncthreads();
    if (tid < SP_S) {
        const int x = x0 + tid;
        const bool m = x < W && mask[(size_t)y * W + x] != 0;
        const unsigned b = __ballot_sync(0xFFFFFFFFu, m);
        int base = 0;
        if (lane == 0 && b) base = atomicAdd(&nlist, __popc(b));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (m) {
            const int slot = base + __popc(b & ((1u << lane) - 1u));
            list[slot] = tid;
            best[slot] = 0ull;
        }
    }
    __syncthreads();
    const int n = nlist;
    if (n == 0) return;
    region::stage_rows<WIN, SLW, SLW, SP_THREADS>(sL, L, pitch, W, H, y - NH, x0 - NH);
    __syncthreads();
    // one thread packs each masked pixel's left window once for all lanes and chunks
    for (int e = tid; e < n; e += SP_THREADS) {
        uint32_t Lw[WIN][NW];
        sLa[e] = region::pack_left<NH, SLW>(sL, 0, list[e], Lw);
#pragma unroll
        for (int i = 0; i < WIN; ++i)
#pragma unroll
            for (int k = 0; k < NW; ++k) sLw[e][i][k] = Lw[i][k];
    }
    // the segment's largest admissible candidate
    const int zmax_seg = min(Dk - 1, min(x0 + SP_S, W) - 1);
    for (int z0 = 0; z0 <= zmax_seg; z0 += SP_ZCH) {
        __syncthreads();      // the previous chunk's rows are consumed
        region::stage_rows<WIN, SRW, SRWW * 4, SP_THREADS>(reinterpret_cast<uint8_t *>(sR), R, pitch, W, H, y - NH,
                                                x0 - (z0 + SP_ZCH - 1) - NH);
        {
            // entry u: right window at column x0 - (z0 + ZCH - 1) + u (columns < 0 or >= W are
            // never read by an admissible candidate)
            const int c0 = x0 - (z0 + SP_ZCH - 1);
            constexpr int NS = SP_S + SP_ZCH - 1, T = (NS + SP_THREADS - 1) / SP_THREADS;
            int2 v[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int u = tid + SP_THREADS * t, col = c0 + u;
                v[t] = (u < NS && col >= 0 && col < W) ? __ldg(rstat + (size_t)y * rspitch + col) : make_int2(0, 0);
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int u = tid + SP_THREADS * t;
                if (u < NS) sS[u] = v[t];
            }
        }
        __syncthreads();
        // lanes per pixel: enough for the chunk's candidate groups (a small D_k leaves a full
        // warp mostly idle, so 2 or 4 pixels then share a warp)
        const int ng = (min(SP_ZCH, zmax_seg - z0 + 1) + 3) / 4;
        const int lpe = ng > 16 ? 32 : (ng > 8 ? 16 : 8);
        const int sub = lane / lpe, sl = lane - sub * lpe, per = 32 / lpe;
        for (int base = warp * per; base < n; base += (SP_THREADS / 32) * per) {
            const int e = base + sub;
            unsigned long long k = 0ull;
            if (e < n) {
                const int px = list[e], x = x0 + px;
                const int zmax = min(Dk - 1, x);
                if (z0 <= zmax) {
                    uint32_t Lw[WIN][NW];
#pragma unroll
                    for (int i = 0; i < WIN; ++i)
#pragma unroll
                        for (int kk = 0; kk < NW; ++kk) Lw[i][kk] = sLw[e][i][kk];
                    const int2 la = sLa[e];
                    // groups of 4 candidates z0 + 4g .. z0 + 4g + 3; the lane keeps its best
                    // (score, z) with a strict compare in ascending z, so ties keep the smallest
                    float bs = -INFINITY;
                    int bz = -1;
                    for (int g = sl; 4 * g < SP_ZCH && z0 + 4 * g <= zmax; g += lpe) {
                        const int um = px + SP_ZCH - 4 - 4 * g;      // staged column of candidate z0 + 4g + 3
                        uint32_t sab[4];
                        region::sab4<NH, SRWW>(sR, 0, um, Lw, sab);
#pragma unroll
                        for (int o = 3; o >= 0; --o) {               // ascending z
                            const int z = z0 + 4 * g + 3 - o;
                            const float r = region::rho_of<NH>(sab[o], la, sS[um + o]);
                            if (z <= zmax && r > bs) {
                                bs = r;
                                bz = z;
                            }
                        }
                    }
                    if (bz >= 0) k = wta_key(bs, bz);
                }
            }
            for (int sh = lpe / 2; sh > 0; sh >>= 1) {
                const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, k, sh);
                k = t > k ? t : k;
            }
            if (e < n && sl == 0 && k > best[e]) best[e] = k;
        }
    }
    __syncthreads();
    unsigned long long cnt = 0;
    for (int e = tid; e < n; e += SP_THREADS) {
        const int x = x0 + list[e];
        const size_t p = (size_t)y * W + x;
        const unsigned long long k = best[e];
        d_out[p] = static_cast<int16_t>(0xFFFFFFFFu - static_cast<uint32_t>(k & 0xFFFFFFFFull));
        if (c_out) c_out[p] = fminf(1.f, fmaxf(-1.f, float_from_order_key(static_cast<uint32_t>(k >> 32))));
        cnt += static_cast<unsigned long long>(min(Dk - 1, x) + 1);
    }
    if (evals) {
        cnt = __reduce_add_sync(0xFFFFFFFFu, static_cast<unsigned>(cnt));
        if (lane == 0 && cnt) atomicAdd(evals, cnt);
    }
}

template <int NH>
cudaError_t sparse_launch(const LevelBuf &l, int16_t *d, float *c, unsigned long long *evals, cudaStream_t st) {
    dim3 grd((l.W + SP_S - 1) / SP_S, l.H);
    zncc_sparse_kernel<NH><<<grd, SP_THREADS, 0, st>>>(l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, l.mask, l.rstat,
                                                       l.rspitch, d, c, evals);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_zncc_sparse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st) {
    if (!l.mask || !l.rstat) return cudaErrorInvalidValue;
    switch (nh) {
        case 1: return sparse_launch<1>(l, d, c, evals, st);
        case 2: return sparse_launch<2>(l, d, c, evals, st);
        case 3: return sparse_launch<3>(l, d, c, evals, st);
        case 4: return sparse_launch<4>(l, d, c, evals, st);
        case 5: return sparse_launch<5>(l, d, c, evals, st);
        case 6: return sparse_launch<6>(l, d, c, evals, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
