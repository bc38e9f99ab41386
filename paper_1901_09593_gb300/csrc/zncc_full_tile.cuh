// zncc_full_tile.cuh -- the full-range ZNCC winner-take-all tile, shared by the standalone
// kernel (zncc_full.cu) and the batched persistent kernel (batch.cu).
// Full-range ZNCC winner-take-all (Sec. III-A, Eq. 1-4): every admissible
// candidate 0 <= z <= min(D_k - 1, x) of every pixel.  Used at the coarsest pyramid level
// and, with K = 1, as flat block matching.
//
// Design (per CTA: a tile of TX = 32*SX columns x TY = 8 rows, 4 warps):
//  * The left tile and, per z-block, the right span are staged HBM/L2 -> shared memory by
//    TMA (cp.async.bulk.tensor, one mbarrier, bounded wait) and widened once to float.
//  * Window statistics of both images (S = sum I, rsqrt(N*sum I^2 - S^2)) are computed
//    in the CTA from the staged tiles with separable sliding sums (exact integers).
//  * The cross term Sab(x, z) = sum a*b is a 2-D box filter of the products
//    L(y, x') * R(y, x' - z) for each z.  Each lane owns SX adjacent columns and ZC
//    consecutive candidates and walks down the TY rows: per row it slides (2n + SX)
//    column sums per candidate (one add, one subtract) and then slides the horizontal
//    window across its SX columns.  Every partial sum is an integer below 2^24, so FP32
//    holds it exactly.
//  * c = N*Sab - Sa*Sb is formed without rounding loss: Sa = Sa_hi + Sa_lo with Sa_hi a
//    multiple of 256 makes Sa_hi*Sb exact in FP32, and two FMAs finish the sum with one
//    rounding relative to c.  The per-candidate score is c * rsqrt(Vb); the left-side
//    factor rsqrt(Va) is applied once per pixel at the end.
//  * WTA: each lane keeps the best of its ZC candidates per pixel and merges it into the
//    CTA's per-pixel best with a 64-bit atomicMax on (ordered score, ~z) in shared memory,
//    which keeps exact ties on the smallest z.
// Bound: the FP32/ALU pipe (about 15 instructions per evaluation); HBM traffic is a few
// bytes per pixel, independent of D.
#pragma once

#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {
namespace tiles {


constexpr int FT_TY = 8;
constexpr int FT_NWARP = 4;   // warps of the standalone kernel (z-block granularity)

template <int NH, int SX, int ZC>
struct FullCfg {
    static constexpr int TY = FT_TY;
    static constexpr int TX = 32 * SX;
    static constexpr int ROWS = TY + 2 * NH;
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int N = WIN * WIN;
    static constexpr int LBOX = TX + 32;                       // left TMA box width
    static constexpr int ZB = ((256 - TX - 32) / 32) * 32;     // z-block (right box = 256 B)
    static constexpr int LW = TX + 2 * NH;                     // widened left columns
    static constexpr int LFP = ((LW + 3) / 4) * 4 + 4;
    static constexpr int RW = TX + ZB + 2 * NH - 1;            // widened right columns
    static constexpr int RFP = ((RW + 3) / 4) * 4 + 8;
    static constexpr int SW = TX + ZB - 1;                     // right statistics columns
    static constexpr int SFP = ((SW + 3) / 4) * 4 + 4;
    static constexpr int NC = SX + 2 * NH;                     // column sums per lane
    static constexpr int NR = NC + ZC - 1;                     // right values per row
    static_assert(ZB >= 32 && ZB % (FT_NWARP * ZC) == 0, "z-block");
    static_assert(15 + RW <= 256, "right span must fit one 256-byte box");
    // shared memory carve (bytes, each region 128-aligned)
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t OFF_SL = 128;                       // [0,128): barrier + flag
    static constexpr size_t OFF_SR = OFF_SL + al((size_t)ROWS * LBOX);
    static constexpr size_t OFF_LF = OFF_SR + al((size_t)ROWS * 256);
    static constexpr size_t OFF_RF = OFF_LF + al((size_t)ROWS * LFP * 4);
    static constexpr size_t OFF_STL = OFF_RF + al((size_t)ROWS * RFP * 4);
    static constexpr size_t OFF_STR = OFF_STL + al((size_t)3 * TY * TX * 4);
    static constexpr size_t OFF_TMP = OFF_STR + al((size_t)TY * SFP * 8);
    static constexpr size_t OFF_BEST = OFF_TMP + al((size_t)TY * RFP * 4);
    static constexpr size_t BYTES = OFF_BEST + al((size_t)TY * TX * 8);
};

// Load N consecutive floats starting at an address aligned to A floats.
template <int N, int A>
__device__ __forceinline__ void load_run(const float *p, float (&out)[N]) {
    if constexpr (A == 4) {
        constexpr int V = (N + 3) / 4;
        float tmp[V * 4];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            float4 q = reinterpret_cast<const float4 *>(p)[i];
            tmp[4 * i] = q.x; tmp[4 * i + 1] = q.y; tmp[4 * i + 2] = q.z; tmp[4 * i + 3] = q.w;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = tmp[i];
    } else if constexpr (A == 2) {
        constexpr int V = (N + 1) / 2;
        float tmp[V * 2];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            float2 q = reinterpret_cast<const float2 *>(p)[i];
            tmp[2 * i] = q.x; tmp[2 * i + 1] = q.y;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = tmp[i];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = p[i];
    }
}

template <int N, int A>
__device__ __forceinline__ void load_run2(const float2 *p, float2 (&out)[N]) {
    if constexpr (A >= 2) {
        constexpr int V = (N + 1) / 2;
        float2 tmp[V * 2];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            float4 q = reinterpret_cast<const float4 *>(p)[i];
            tmp[2 * i] = make_float2(q.x, q.y);
            tmp[2 * i + 1] = make_float2(q.z, q.w);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = tmp[i];
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = p[i];
    }
}

// One lane's walk down the TY rows for one chunk of ZC candidates.
template <int NH, int SX, int ZC, bool CHECK>
__device__ __forceinline__ void full_chunk(const float *Lf, const float *Rf, const float *stL,
                                           const float2 *stR, unsigned long long *best, int lane,
                                           int rbase, int xl, int zc, int Dk) {
    using C = FullCfg<NH, SX, ZC>;
    constexpr int NC = C::NC, NR = C::NR, TX = C::TX;
    constexpr int A = SX >= 4 ? 4 : SX;
    const int lbase = SX * lane;
    const float Nf = static_cast<float>(C::N);
    float colP[NC][ZC];
    {
        float lr[NC], rr[NR];
#pragma unroll
        for (int t = 0; t <= 2 * NH; ++t) {
            load_run<NC, A>(Lf + t * C::LFP + lbase, lr);
            load_run<NR, A>(Rf + t * C::RFP + rbase, rr);
#pragma unroll
            for (int u = 0; u < NC; ++u)
#pragma unroll
                for (int v = 0; v < ZC; ++v)
                    colP[u][v] = (t == 0) ? lr[u] * rr[u - v + ZC - 1]
                                          : fmaf(lr[u], rr[u - v + ZC - 1], colP[u][v]);
        }
    }
#pragma unroll 1
    for (int ry = 0; ry < C::TY; ++ry) {
        if (ry > 0) {
            float ln[NC], lo[NC], rn[NR], ro[NR];
            load_run<NC, A>(Lf + (ry + 2 * NH) * C::LFP + lbase, ln);
            load_run<NC, A>(Lf + (ry - 1) * C::LFP + lbase, lo);
            load_run<NR, A>(Rf + (ry + 2 * NH) * C::RFP + rbase, rn);
            load_run<NR, A>(Rf + (ry - 1) * C::RFP + rbase, ro);
#pragma unroll
            for (int u = 0; u < NC; ++u)
#pragma unroll
                for (int v = 0; v < ZC; ++v) {
                    // add first, then subtract: every intermediate stays an integer < 2^24
                    float t = fmaf(ln[u], rn[u - v + ZC - 1], colP[u][v]);
                    colP[u][v] = fmaf(-lo[u], ro[u - v + ZC - 1], t);
                }
        }
        float sah[SX], sal[SX];
        load_run<SX, A>(stL + 0 * C::TY * TX + ry * TX + lbase, sah);
        load_run<SX, A>(stL + 1 * C::TY * TX + ry * TX + lbase, sal);
        float2 sr[SX + ZC - 1];
        load_run2<SX + ZC - 1, A>(stR + ry * C::SFP + rbase, sr);
        float bs[SX];
        int bz[SX];
#pragma unroll
        for (int s = 0; s < SX; ++s) { bs[s] = -INFINITY; bz[s] = 0; }
#pragma unroll
        for (int v = 0; v < ZC; ++v) {
            float S = colP[0][v];
#pragma unroll
            for (int u = 1; u <= 2 * NH; ++u) S += colP[u][v];
#pragma unroll
            for (int s = 0; s < SX; ++s) {
                if (s > 0) S = (S + colP[s + 2 * NH][v]) - colP[s - 1][v];
                const float2 q = sr[s - v + ZC - 1];
                const float c = fmaf(-sal[s], q.x, fmaf(Nf, S, -(sah[s] * q.x)));
                const float sc = c * q.y;
                const int z = zc + v;
                bool ok = sc > bs[s];
                if (CHECK) ok = ok && (z <= xl + s) && (z < Dk);
                if (ok) { bs[s] = sc; bz[s] = z; }
            }
        }
#pragma unroll
        for (int s = 0; s < SX; ++s)
            if (bs[s] != -INFINITY) atomicMax(best + ry * TX + lbase + s, wta_key(bs[s], bz[s]));
    }
}

// Window statistics from a widened tile: vertical sliding sums into tmp (one word per
// column sum: q | s << 20, s < 4096 and q < 2^20 for columns of up to 13 bytes), then
// horizontal sums.  Output column v uses tile columns v .. v + 2n.  Writes (S, rsqrt(V)) or,
// for the left tile, the split (S_hi, S_lo) and rsqrt(V) into three planes.  All sums are
// exact integers.
template <int NH, bool LEFT>
__device__ __forceinline__ void tile_stats(const float *img, int pitch, int cols_in, uint32_t *tmp,
                                           int tmp_pitch, int cols_out, float2 *outR, int outR_pitch,
                                           float *outL, int TXo) {
    constexpr int TY = FT_TY, WIN = 2 * NH + 1, N = WIN * WIN;
    for (int c = threadIdx.x; c < cols_in; c += blockDim.x) {
        int s = 0, q = 0;
#pragma unroll
        for (int t = 0; t < WIN; ++t) {
            const int v = static_cast<int>(img[t * pitch + c]);
            s += v; q += v * v;
        }
        tmp[c] = static_cast<uint32_t>(q) | (static_cast<uint32_t>(s) << 20);
#pragma unroll 1
        for (int ry = 1; ry < TY; ++ry) {
            const int vn = static_cast<int>(img[(ry + 2 * NH) * pitch + c]);
            const int vo = static_cast<int>(img[(ry - 1) * pitch + c]);
            s += vn - vo;
            q += vn * vn - vo * vo;
            tmp[ry * tmp_pitch + c] = static_cast<uint32_t>(q) | (static_cast<uint32_t>(s) << 20);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TY * cols_out; i += blockDim.x) {
        int ry = i / cols_out, v = i - ry * cols_out;
        int si = 0, qi = 0;
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
            const uint32_t t = tmp[ry * tmp_pitch + v + j];
            si += static_cast<int>(t >> 20);
            qi += static_cast<int>(t & 0xFFFFFu);
        }
        const float s = static_cast<float>(si);
        int V = N * qi - si * si;                      // exact: |N*Q| < 2^31 for n <= 6
        float r = V > 0 ? rsqrtf(static_cast<float>(V)) : 0.f;
        if (LEFT) {
            outL[0 * TY * TXo + ry * TXo + v] = static_cast<float>(si & ~255);
            outL[1 * TY * TXo + ry * TXo + v] = static_cast<float>(si & 255);
            outL[2 * TY * TXo + ry * TXo + v] = r;
        } else {
            outR[ry * outR_pitch + v] = make_float2(s, r);
        }
    }
}

// Full-range WTA of one TX x TY tile (bx, by) by the calling CTA (blockDim.x = 32 * nwarps,
// any nwarps).  `smem` holds FullCfg::BYTES bytes, 128-aligned; its first 8 bytes are an
// mbarrier the caller has initialised (count 1) and `parity` is its next phase parity,
// advanced here.  Returns false if a bounded wait gave up (the error word is then set).
template <int NH, int SX, int ZC>
__device__ bool full_tile(const FullTileArgs &a, const CUtensorMap *tmL, const CUtensorMap *tmR, int bx, int by,
                          uint8_t *smem, uint32_t &parity) {
    using C = FullCfg<NH, SX, ZC>;
    constexpr int TX = C::TX, TY = C::TY, ROWS = C::ROWS;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *flag = reinterpret_cast<int *>(smem + 8);
    uint8_t *sL = smem + C::OFF_SL;
    uint8_t *sR = smem + C::OFF_SR;
    float *Lf = reinterpret_cast<float *>(smem + C::OFF_LF);
    float *Rf = reinterpret_cast<float *>(smem + C::OFF_RF);
    float *stL = reinterpret_cast<float *>(smem + C::OFF_STL);
    float2 *stR = reinterpret_cast<float2 *>(smem + C::OFF_STR);
    uint32_t *tmp = reinterpret_cast<uint32_t *>(smem + C::OFF_TMP);
    unsigned long long *best = reinterpret_cast<unsigned long long *>(smem + C::OFF_BEST);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int x0 = bx * TX, y0 = by * TY;
    const int Dk = a.Dk;
    const int ZBmax = (a.zblock > 0 && a.zblock <= C::ZB) ? (a.zblock & ~31) : C::ZB;
    const bool force_to = a.force_timeout != 0;

    // ---- left tile: image columns [x0 - 16, x0 + TX + 16), rows [y0 - n, y0 + TY + n)
    if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, ROWS * C::LBOX);
        tma_load_2d(sL, tmL, bar, x0 - 16 + APX, y0 - NH + APY);
    }
    if (!tma_batch_wait(bar, parity, flag, force_to, a.err)) return false;
    parity ^= 1;
    for (int i = tid; i < ROWS * C::LW; i += blockDim.x) {
        int t = i / C::LW, u = i - t * C::LW;            // Lf col u <-> image col x0 - n + u
        Lf[t * C::LFP + u] = static_cast<float>(sL[t * C::LBOX + u + 16 - NH]);
    }
    for (int i = tid; i < TY * TX; i += blockDim.x) best[i] = 0ull;
    __syncthreads();
    tile_stats<NH, true>(Lf, C::LFP, C::LW, tmp, C::RFP, TX, nullptr, 0, stL, TX);
    __syncthreads();

    const int xlim = min(x0 + TX, a.W);                 // z <= x < xlim
    const int zend = min(Dk, xlim);
    for (int zb = 0; zb < zend; zb += ZBmax) {
        const int ZBr = min(ZBmax, ((zend - zb + 31) / 32) * 32);
        const int origR = x0 - NH - zb - ZBr + 1;        // image col of Rf column 0
        const int xs = (origR + APX) & ~15;             // TMA x (buffer coords), 16-aligned
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, ROWS * 256);
            tma_load_2d(sR, tmR, bar, xs, y0 - NH + APY);
        }
        if (!tma_batch_wait(bar, parity, flag, force_to, a.err)) return false;
        parity ^= 1;
        const int rw = TX + ZBr + 2 * NH - 1, off = origR + APX - xs;
        for (int i = tid; i < ROWS * rw; i += blockDim.x) {
            int t = i / rw, u = i - t * rw;
            Rf[t * C::RFP + u] = static_cast<float>(sR[t * 256 + u + off]);
        }
        __syncthreads();
        tile_stats<NH, false>(Rf, C::RFP, rw, tmp, C::RFP, TX + ZBr - 1, stR, C::SFP, nullptr, 0);
        __syncthreads();

        const int nchunk = ZBr / ZC;
        const int xl = x0 + SX * lane;
        for (int m = warp; m < nchunk; m += nwarp) {
            const int zc = zb + m * ZC;
            if (zc >= Dk || zc > xl + SX - 1) continue;  // nothing admissible for this lane
            const int rbase = SX * lane + ZBr - ZC - m * ZC;
            const bool chk = (zc + ZC - 1 > xl) || (zc + ZC > Dk);
            if (chk)
                full_chunk<NH, SX, ZC, true>(Lf, Rf, stL, stR, best, lane, rbase, xl, zc, Dk);
            else
                full_chunk<NH, SX, ZC, false>(Lf, Rf, stL, stR, best, lane, rbase, xl, zc, Dk);
        }
        __syncthreads();
    }

    // ---- finalize: rho = score * rsqrt(Va), clamp, write
    unsigned long long cnt = 0;
    for (int i = tid; i < TY * TX; i += blockDim.x) {
        int ry = i / TX, px = i - ry * TX;
        int x = x0 + px, y = y0 + ry;
        if (x >= a.W || y >= a.H) continue;
        unsigned long long k = best[i];
        int z = static_cast<int>(0xFFFFFFFFu - static_cast<uint32_t>(k & 0xFFFFFFFFull));
        float sc = float_from_order_key(static_cast<uint32_t>(k >> 32));
        float rho = sc * stL[2 * TY * TX + i];
        rho = fminf(1.f, fmaxf(-1.f, rho));
        a.d_out[(size_t)y * a.W + x] = static_cast<int16_t>(z);
        if (a.c_out) a.c_out[(size_t)y * a.W + x] = rho;
        cnt += min(Dk - 1, x) + 1;
    }
    if (a.evals && cnt) atomicAdd(a.evals, cnt);
    return true;
}

}  // namespace tiles
}  // namespace msbm
