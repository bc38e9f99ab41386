// gated.cu -- the gated steps of the full method (Sec. III-B, the second branch of
// Eq. 8-9, Sec. III-D), each a small kernel around the matching kernels:
//  * beta gate (Sec. III-C): the cost prior C_hat^k = BI(C^{k+1}) -- bicubic (Catmull-Rom)
//    upsampling with fine pixel (y, x) at coarse coordinates (y/2, x/2), clamp-to-edge --
//    and the fallback mask C_hat <= beta, with the list of 2 x 2 cells that hold a fallback
//    pixel (the fallback pixels' full-range search, zncc_sparse.cu, walks that list);
//  * alpha refinement (Eq. 5-7) at the coarsest level: for a pixel with C' <= alpha, the
//    average of the ZNCC over its 3 x 3 neighbourhood (neighbours inside the image) for
//    every admissible candidate z <= min(D_k - 1, x), and its argmax / max;
//  * selective median (Eq. 10): for a pixel with C <= alpha, the lower median of the 5 x 5
//    neighbours whose cost exceeds alpha (unchanged when none does).
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_region.cuh"

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

// The gate for the 2 x 2 cell (cx, cy) of one thread, 32 cells of a row per warp.  With
// cells, the cells holding a masked pixel are also appended to the list cells[2 ..] (one
// atomic per warp, lane order within it), cells[0] counting them; the caller zeroes
// cells[0 .. 1] before the launch.
__global__ void beta_gate_kernel(const float *__restrict__ Cc, int Wc, int Hc, int W, int H, float beta,
                                 uint8_t *mask, unsigned *cells) {
    const int cx = blockIdx.x * 32 + threadIdx.x, cy = blockIdx.y * blockDim.y + threadIdx.y;
    bool any = false;
#pragma unroll
    for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int x = 2 * cx + c, y = 2 * cy + r2;
            if (x >= W || y >= H) continue;
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
                for (int b = 0; b < 4; ++b)
                    r = fmaf(wx[b], __ldg(Cc + (size_t)yy * Wc + min(max(bx - 1 + b, 0), Wc - 1)), r);
                s = fmaf(wy[a], r, s);
            }
            const bool m = !(s > beta);
            mask[(size_t)y * W + x] = m ? 1 : 0;
            any |= m;
        }
    if (!cells) return;
    const unsigned b = __ballot_sync(0xFFFFFFFFu, any);
    if (!b) return;
    const int lane = threadIdx.x;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(cells, static_cast<unsigned>(__popc(b)));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (any) cells[2 + base + __popc(b & ((1u << lane) - 1u))] = static_cast<unsigned>(cy) * ((W + 1) / 2) + cx;
}

// Alpha refinement on a 16 x 8 tile.  E(q, z), the ZNCC of every pixel q of the tile's
// 18 x 10 neighbourhood region at every candidate z, is computed once per 32-candidate chunk
// into shared memory (zncc_region.cuh; 0 for region pixels outside the image), then two
// threads per refined pixel (cost <= alpha) sum E over its 3 x 3 neighbours (rows, then
// columns: the in-image neighbours, since the others add 0) for 16 candidates each, scale by
// 1 / (in-image neighbours) and keep the WTA of the means on a 64-bit (ordered mean, ~z)
// key: ties keep the smallest z.
constexpr int AR_TW = 16, AR_TH = 8, AR_RW = AR_TW + 2, AR_RH = AR_TH + 2;
constexpr int AR_NP = AR_RW * AR_RH;     // region pixels (180)

template <int NH>
__global__ void __launch_bounds__(256) alpha_refine_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W,
                                                           int H, int Dk, float alpha, int16_t *d, float *C,
                                                           unsigned long long *evals) {
    using region::ZC;
    constexpr int WIN = 2 * NH + 1, NW = (WIN + 3) / 4;
    constexpr int SLW = AR_RW + 2 * NH, SLH = AR_RH + 2 * NH;   // staged left region
    constexpr int SU = AR_RW + ZC - 1;                          // right window columns per chunk
    constexpr int SRW = SU + 2 * NH;                            // staged right columns per chunk
    constexpr int SRWW = (SRW + 3) / 4 + 2;                     // words per staged right row
    __shared__ uint8_t sL[SLH * SLW];
    __shared__ uint32_t sR[SLH * SRWW];
    __shared__ int vs[AR_RH * SRW], vq[AR_RH * SRW];
    __shared__ int2 stR[AR_RH * SU];
    __shared__ float E[AR_NP][ZC + 1];
    __shared__ unsigned long long best[AR_TW * AR_TH];
    __shared__ int qual[AR_TW * AR_TH];
    __shared__ int any;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * AR_TW, y0 = blockIdx.y * AR_TH;
    const int rx0 = x0 - 1, ry0 = y0 - 1;        // region origin (may lie outside the image)
    if (tid == 0) any = 0;
    __syncthreads();
    if (tid < AR_TW * AR_TH) {
        const int x = x0 + tid % AR_TW, y = y0 + tid / AR_TW;
        const int q = x < W && y < H && !(C[(size_t)y * W + x] > alpha);
        qual[tid] = q;
        best[tid] = 0ull;
        if (q) any = 1;
    }
    region::stage_rows<SLH, SLW, SLW>(sL, L, pitch, W, H, ry0 - NH, rx0 - NH);
    __syncthreads();
    if (!any) return;
    // this thread's region pixel: packed left window and its statistics
    const int pr = tid / AR_RW, pc = tid - pr * AR_RW;
    const bool pin = tid < AR_NP && ry0 + pr >= 0 && ry0 + pr < H && rx0 + pc >= 0 && rx0 + pc < W;
    uint32_t Lw[WIN][NW];
    int2 la = make_int2(0, 0);
    if (tid < AR_NP) la = region::pack_left<NH, SLW>(sL, pr, pc, Lw);
    // the refined pixel and candidate half of this thread in the averaging step
    const int ow = tid & (AR_TW * AR_TH - 1), oh = tid >> 7;
    const int xw = x0 + ow % AR_TW, yw = y0 + ow / AR_TW;
    const int e0 = (ow / AR_TW) * AR_RW + ow % AR_TW;     // region index of (yw - 1, xw - 1)
    const int zmax_w = min(Dk - 1, xw);
    const float inv = 1.f / static_cast<float>((min(yw + 1, H - 1) - max(yw - 1, 0) + 1) *
                                               (min(xw + 1, W - 1) - max(xw - 1, 0) + 1));
    const int zmax_tile = min(Dk - 1, min(x0 + AR_TW, W) - 1);
    for (int z0 = 0; z0 <= zmax_tile; z0 += ZC) {
        __syncthreads();      // the previous chunk's E and staging are consumed
        region::stage_rows<SLH, SRW, SRWW * 4>(reinterpret_cast<uint8_t *>(sR), R, pitch, W, H, ry0 - NH,
                                                rx0 - (z0 + ZC - 1) - NH);
        __syncthreads();
        region::window_stats<NH, AR_RH, SU, SRWW * 4>(reinterpret_cast<const uint8_t *>(sR), vs, vq, stR);
        if (tid < AR_NP) {
#pragma unroll 1
            for (int g = 0; g < ZC / 4; ++g) {
                const int um = pc + ZC - 4 - 4 * g;       // staged column of candidate z0 + 4g + 3
                uint32_t sab[4];
                region::sab4<NH, SRWW>(sR, pr, um, Lw, sab);
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    E[tid][4 * g + 3 - o] = pin ? region::rho_of<NH>(sab[o], la, stR[pr * SU + um + o]) : 0.f;
            }
        }
        __syncthreads();
        if (qual[ow]) {
            unsigned long long k = 0ull;
#pragma unroll 4
            for (int zz = 16 * oh; zz < 16 * oh + 16; ++zz) {
                const int z = z0 + zz;
                if (z > zmax_w) break;
                float s = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) s += E[e0 + a * AR_RW + b][zz];
                const unsigned long long kk = wta_key(s * inv, z);
                k = kk > k ? kk : k;
            }
            if (k) atomicMax(&best[ow], k);
        }
    }
    __syncthreads();
    if (tid < AR_TW * AR_TH && qual[tid]) {
        const size_t p = (size_t)yw * W + xw;
        const unsigned long long k = best[tid];
        d[p] = static_cast<int16_t>(0xFFFFFFFFu - static_cast<uint32_t>(k & 0xFFFFFFFFull));
        C[p] = float_from_order_key(static_cast<uint32_t>(k >> 32));
        if (evals) {
            const int ya = max(yw - 1, 0), yb = min(yw + 1, H - 1), xa = max(xw - 1, 0), xb = min(xw + 1, W - 1);
            atomicAdd(evals, static_cast<unsigned long long>((yb - ya + 1) * (xb - xa + 1)) * (zmax_w + 1));
        }
    }
}

// Comparator list of Batcher's merge-exchange sort (Knuth, TAOCP vol. 3, Sec. 5.2.2,
// Algorithm M) for n inputs, built at compile time.
template <int n>
struct MergeExchange {
    static constexpr int count() {
        int t = 0;
        while ((1 << t) < n) ++t;
        int m = 0;
        for (int p = 1 << (t - 1); p > 0; p >>= 1)
            for (int q = 1 << (t - 1), r = 0, d = p; d > 0; d = q - p, q >>= 1, r = p)
                for (int i = 0; i + d < n; ++i)
                    if ((i & p) == r) ++m;
        return m;
    }
    static constexpr int M = count();
    int a[M], b[M];
    constexpr MergeExchange() : a(), b() {
        int t = 0;
        while ((1 << t) < n) ++t;
        int m = 0;
        for (int p = 1 << (t - 1); p > 0; p >>= 1)
            for (int q = 1 << (t - 1), r = 0, d = p; d > 0; d = q - p, q >>= 1, r = p)
                for (int i = 0; i + d < n; ++i)
                    if ((i & p) == r) {
                        a[m] = i;
                        b[m] = i + d;
                        ++m;
                    }
    }
};

// Lane-wise unsigned 16-bit minimum / maximum of two packed pairs.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// tiles of 32 x MED_TY pixels, 256 threads of MED_TY / 8 pixels each (rows 8 apart)
constexpr int MED_TX = 32, MED_R = 2;
constexpr int MED_SMALL_TILES_PER_SM = 2;
constexpr int MED_SW = MED_TX + 2 * MED_R;
constexpr int MED_NONE = 0x7FFF;     // a neighbour that does not vote (outside, or cost <= alpha)

// Eq. 10 on a 32 x MED_TY tile (256 threads, MED_TY / 8 pixels each): the 5 x 5 neighbourhood
// (inside the image) is staged in shared memory as voting disparities (cost > alpha) or
// MED_NONE, costs and disparities loaded together (one round trip).  A voting pixel keeps
// its disparity; the tile's pixels with cost <= alpha and at least one voter are collected in
// a list (warp-aggregated shared atomics), and the CTA's threads sort them: each job sorts
// the pixel's 24 neighbours (the pixel does not vote itself) with a merge-exchange network,
// so the voters come first in ascending order, and takes the lower median of the voters.  A
// pixel with cost <= alpha and no voter keeps its disparity.
template <int MED_TY>
__global__ void __launch_bounds__(256)
selective_median_kernel(const int16_t *__restrict__ d_in, const float *__restrict__ C, int W, int H, float alpha,
                        int16_t *d_out) {
    constexpr int NT = 256, NB = (2 * MED_R + 1) * (2 * MED_R + 1) - 1, RS = 8, MED_RPT = MED_TY / RS;
    constexpr int MED_SH = MED_TY + 2 * MED_R;
    static_assert(MED_TX * RS == NT && MED_TY % RS == 0 && MED_SW <= 64, "median tile");
    __shared__ int16_t sv[MED_SH][MED_SW];
    __shared__ uint16_t job[MED_TX * MED_TY];   // tile pixels to sort
    __shared__ unsigned long long vmask[MED_SH];
    __shared__ int njob_s;
    const int x0 = blockIdx.x * MED_TX, y0 = blockIdx.y * MED_TY;
    const int tid = threadIdx.x, lane = tid & 31, tx = tid % MED_TX, ty = tid / MED_TX;
    if (tid == 0) njob_s = 0;
    {
        constexpr int NS = MED_SH * MED_SW, T = (NS + NT - 1) / NT;
        float cv[T];
        int dv[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t, yy = y0 - MED_R + i / MED_SW, xx = x0 - MED_R + i % MED_SW;
            cv[t] = 0.f;
            dv[t] = MED_NONE;
            if (i < NS && yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const size_t p = (size_t)yy * W + xx;
                cv[t] = __ldg(C + p);
                dv[t] = __ldg(d_in + p);
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int i = tid + NT * t;
            if (i < NS) sv[i / MED_SW][i % MED_SW] = static_cast<int16_t>(cv[t] > alpha ? dv[t] : MED_NONE);
        }
    }
    __syncthreads();
    // voter bitmask of every staged row (bit c: column c votes), one ballot pair per row
    for (int r = tid >> 5; r < MED_SH; r += NT / 32) {
        const unsigned lo = __ballot_sync(0xFFFFFFFFu, sv[r][lane] != MED_NONE);
        const unsigned hi = __ballot_sync(0xFFFFFFFFu, lane + 32 < MED_SW && sv[r][min(lane + 32, MED_SW - 1)] != MED_NONE);
        if (lane == 0) vmask[r] = static_cast<unsigned long long>(lo) | (static_cast<unsigned long long>(hi) << 32);
    }
    __syncthreads();
    const int x = x0 + tx;
#pragma unroll
    for (int j = 0; j < MED_RPT; ++j) {
        const int ry = ty + RS * j, y = y0 + ry;
        const bool in = x < W && y < H;
        const int centre = sv[ry + MED_R][tx + MED_R];
        bool need = false;
        if (in && centre == MED_NONE) {
            // some voter among the 24 neighbours (the centre itself does not vote)
            unsigned long long any = 0;
#pragma unroll
            for (int m = 0; m <= 2 * MED_R; ++m) any |= vmask[ry + m] >> tx;
            need = (any & ((1ull << (2 * MED_R + 1)) - 1ull)) != 0;
        }
        if (in && !need) {
            const size_t o = (size_t)y * W + x;
            d_out[o] = centre != MED_NONE ? static_cast<int16_t>(centre) : d_in[o];
        }
        // collect the pixels to sort: one shared atomic per warp and row
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, need);
        int first = 0;
        if (lane == 0 && bal) first = atomicAdd(&njob_s, __popc(bal));
        first = __shfl_sync(0xFFFFFFFFu, first, 0);
        if (need) job[first + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint16_t>(ry * MED_TX + tx);
    }
    __syncthreads();
    // the jobs in pairs, one pair a thread: the two pixels' neighbourhoods share each 32-bit
    // word of the network (pixel 2k in the low half, 2k + 1 in the high half; an odd count's
    // last pixel is paired with itself and written once), so one min.u16x2 / max.u16x2 pair
    // performs a comparator for both.  Voting disparities are 0 .. D_k - 1 < MED_NONE, so
    // unsigned 16-bit order is their order and the non-voters sort last.
    const int njob = njob_s, npair = (njob + 1) / 2;
    for (int k = tid; k < npair; k += NT) {
        const int ta = job[2 * k], tb = 2 * k + 1 < njob ? job[2 * k + 1] : ta;
        const int ax = ta % MED_TX, ay = ta / MED_TX, bx = tb % MED_TX, by = tb / MED_TX;
        uint32_t v[NB];
#pragma unroll
        for (int m = 0, i = 0; m <= 2 * MED_R; ++m)
#pragma unroll
            for (int q = 0; q <= 2 * MED_R; ++q) {
                if (m == MED_R && q == MED_R) continue;
                v[i] = static_cast<uint32_t>(static_cast<uint16_t>(sv[ay + m][ax + q])) |
                       (static_cast<uint32_t>(static_cast<uint16_t>(sv[by + m][bx + q])) << 16);
                ++i;
            }
        // voters of each window: the staged rows' vote bits (the centre does not vote)
        int ca = 0, cb = 0;
#pragma unroll
        for (int m = 0; m <= 2 * MED_R; ++m) {
            ca += __popcll((vmask[ay + m] >> ax) & ((1ull << (2 * MED_R + 1)) - 1ull));
            cb += __popcll((vmask[by + m] >> bx) & ((1ull << (2 * MED_R + 1)) - 1ull));
        }
        constexpr MergeExchange<NB> net;
#pragma unroll
        for (int c = 0; c < net.M; ++c) {
            const uint32_t lo = min_u16x2(v[net.a[c]], v[net.b[c]]), hi = max_u16x2(v[net.a[c]], v[net.b[c]]);
            v[net.a[c]] = lo;
            v[net.b[c]] = hi;
        }
        const int wa = (ca - 1) / 2, wb = (cb - 1) / 2;    // at most NB / 2 - 1
        uint32_t oa = v[0], ob = v[0];
#pragma unroll
        for (int i = 1; i < NB / 2; ++i) {
            if (i == wa) oa = v[i];
            if (i == wb) ob = v[i];
        }
        d_out[(size_t)(y0 + ay) * W + x0 + ax] = static_cast<int16_t>(oa & 0xFFFFu);
        if (2 * k + 1 < njob) d_out[(size_t)(y0 + by) * W + x0 + bx] = static_cast<int16_t>(ob >> 16);
    }
}

}  // namespace

cudaError_t launch_beta_gate(const float *Cc, int Wc, int Hc, int W, int H, float beta, uint8_t *mask,
                             unsigned *cells, cudaStream_t st) {
    const int ncx = (W + 1) / 2, ncy = (H + 1) / 2;
    if (cells) {
        const cudaError_t e = cudaMemsetAsync(cells, 0, 2 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
    }
    dim3 blk(32, 4), grd((ncx + 31) / 32, (ncy + 3) / 4);
    beta_gate_kernel<<<grd, blk, 0, st>>>(Cc, Wc, Hc, W, H, beta, mask, cells);
    return cudaGetLastError();
}

template <int NH>
static cudaError_t alpha_launch(const LevelBuf &l, float alpha, int16_t *d, float *C, unsigned long long *evals,
                                cudaStream_t st) {
    dim3 grd((l.W + AR_TW - 1) / AR_TW, (l.H + AR_TH - 1) / AR_TH);
    alpha_refine_kernel<NH><<<grd, 256, 0, st>>>(l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, alpha, d, C, evals);
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
    // 32 x 32 tiles amortise the staged halo and the barriers over four times the pixels of
    // 32 x 8 tiles; a level too small to give every SM two such tiles takes 32 x 8 (measured
    // on the 1400 x 1000 selective-median pass: 68.1 -> 66.1 us, level 2 taking 32 x 8;
    // 32 x 8 or 32 x 16 at every level: 70.1 / 68.1 us)
    const long tiles32 = (long)((W + MED_TX - 1) / MED_TX) * ((H + 31) / 32);
    static int sms = 0;   // SMs of the device (queried once per process)
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sms = v;
    }
    if (tiles32 < MED_SMALL_TILES_PER_SM * sms) {
        dim3 grd((W + MED_TX - 1) / MED_TX, (H + 7) / 8);
        selective_median_kernel<8><<<grd, 256, 0, st>>>(d_in, C, W, H, alpha, d_out);
    } else {
        dim3 grd((W + MED_TX - 1) / MED_TX, (H + 31) / 32);
        selective_median_kernel<32><<<grd, 256, 0, st>>>(d_in, C, W, H, alpha, d_out);
    }
    return cudaGetLastError();
}

}  // namespace msbm
