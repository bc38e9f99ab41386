// zncc_sparse.cu -- the beta fallback's full-range search (Sec. III-C, Eq. 8-9 second branch)
// for the masked pixels of a level only: every admissible candidate 0 <= z <= min(D_k - 1, x)
// of each pixel whose bicubic cost prior failed the gate.
//
// The gate (gated.cu) lists the 2 x 2 cells that hold a masked pixel.  A persistent grid
// (the CTAs the SMs hold at once) walks that list: each warp takes the next 32 / P entries
// with one atomic, P lanes per cell each searching a part of its candidate groups
// (tiles::cell_full_part: the four pixels share each right row's loads and the products of
// their common window rows; candidates in groups of 8, exact integer sums by dp4a, the
// right-window statistics from the level's plane), merged by shuffles.  Groups of 8: the
// same alignment shifts per row as 7 (offsets 1-3 and 5-7 of a group's 9 windows), and
// power-of-two disparity ranges split evenly over the lanes.  Work is
// proportional to the masked cells, the warps stay full whatever the mask's layout, and
// splitting a cell's range over P lanes makes the units of work small enough that the last
// ones do not leave most of the GPU idle.
#include <math.h>

#include <algorithm>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_cell_full.cuh"

namespace msbm {

namespace {

constexpr int SPC_THREADS = 128;
constexpr int SPC_PART_GROUPS = 4;  // fewest candidate groups a lane searches when lanes share a cell

// candidates per group G and resident CTAs per SM (3: 168 registers a thread) of window
// half-width NH: fewer candidates at the widest windows, whose left words take more
// registers; no spills at any NH
template <int NH>
struct SpcCfg {
    static constexpr int G = NH <= 4 ? 8 : (NH == 5 ? 4 : 2);
    static constexpr int MB = 3;
};

// P (1, 2 or 4) lanes share a cell, lane l searching part l % P of its candidate groups;
// the parts merge by shuffles (larger score, then smaller z: the sequential scan's winner) and
// the part-0 lane writes the cell's masked pixels.
template <int NH>
__global__ void __launch_bounds__(SPC_THREADS, SpcCfg<NH>::MB)
    zncc_sparse_cell_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int Dk, const uint8_t *mask,
                            const int2 *rstat, int rspitch, unsigned *cells, int P, int16_t *d_out, float *c_out,
                            unsigned long long *evals) {
    constexpr int G = SpcCfg<NH>::G;
    const unsigned n = cells[0];
    const int ncx = (W + 1) / 2, lane = threadIdx.x & 31, part = lane & (P - 1);
    const unsigned per_warp = 32u / static_cast<unsigned>(P);
    unsigned long long cnt = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(cells + 1, per_warp);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const unsigned i = base + static_cast<unsigned>(lane) / static_cast<unsigned>(P);
        tiles::CellBest b;
        int cx = 0, cy = 0;
        if (i < n) {
            const unsigned e = cells[2 + i];
            cy = static_cast<int>(e / static_cast<unsigned>(ncx));
            cx = static_cast<int>(e - static_cast<unsigned>(cy) * ncx);
            const int ng = tiles::cell_full_groups<G>(W, Dk, cx);
            b = tiles::cell_full_part<NH, G>(L, R, pitch, W, H, Dk, mask, rstat, rspitch, cx, cy, part * ng / P,
                                             (part + 1) * ng / P);
        } else {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int r2 = 0; r2 < 2; ++r2) {
                    b.best[c][r2] = -INFINITY;
                    b.bz[c][r2] = 0;
                }
        }
        for (int sh = 1; sh < P; sh <<= 1)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int r2 = 0; r2 < 2; ++r2) {
                    const float ob = __shfl_xor_sync(0xFFFFFFFFu, b.best[c][r2], sh);
                    const int oz = __shfl_xor_sync(0xFFFFFFFFu, b.bz[c][r2], sh);
                    if (ob > b.best[c][r2] || (ob == b.best[c][r2] && oz < b.bz[c][r2])) {
                        b.best[c][r2] = ob;
                        b.bz[c][r2] = oz;
                    }
                }
        if (i < n && part == 0) {
            const int xa = 2 * cx, ya = 2 * cy;
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int r2 = 0; r2 < 2; ++r2) {
                    if (!b.m[c][r2]) continue;
                    // rsqrt(Va) scales every candidate of the pixel alike: applied once here.  A
                    // flat left window has c = 0 for every candidate: the smallest z wins with 0.
                    float rho = b.rA[c][r2] > 0.f ? b.best[c][r2] * b.rA[c][r2] : 0.f;
                    rho = fminf(1.f, fmaxf(-1.f, rho));
                    const size_t o = (size_t)(ya + r2) * W + xa + c;
                    d_out[o] = static_cast<int16_t>(b.bz[c][r2]);
                    if (c_out) c_out[o] = rho;
                    cnt += static_cast<unsigned long long>(b.hi[c] + 1);
                }
        }
    }
    for (int sh = 16; sh > 0; sh >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, sh);
    if (lane == 0 && evals && cnt) atomicAdd(evals, cnt);
}

template <int NH>
cudaError_t sparse_launch(const LevelBuf &l, int16_t *d, float *c, unsigned long long *evals, cudaStream_t st) {
    // the CTAs resident at once (queried once per process), and no more than a list of
    // every cell would give one cell a thread
    static int resident = 0;
    if (resident == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, zncc_sparse_cell_kernel<NH>, SPC_THREADS, 0);
        if (e != cudaSuccess) return e;
        resident = std::max(sms * per, 1);
    }
    // lanes per cell: the most (up to 4) that still give each at least SPC_PART_GROUPS groups
    const int ng = (std::min(l.Dk, l.W) + SpcCfg<NH>::G - 1) / SpcCfg<NH>::G;
    int P = 1;
    while (P < 4 && ng / (2 * P) >= SPC_PART_GROUPS) P *= 2;
    const long cells = (long)((l.W + 1) / 2) * ((l.H + 1) / 2);
    const long ctas = std::max<long>(1, std::min<long>(resident, (cells * P + SPC_THREADS - 1) / SPC_THREADS));
    zncc_sparse_cell_kernel<NH><<<static_cast<unsigned>(ctas), SPC_THREADS, 0, st>>>(
        l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, l.mask, l.rstat, l.rspitch, l.cells, P, d, c, evals);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_zncc_sparse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st) {
    if (!l.mask || !l.rstat || !l.cells) return cudaErrorInvalidValue;
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
