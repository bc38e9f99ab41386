// zncc_sparse.cu -- the beta fallback's full-range search (Sec. III-C, Eq. 8-9 second branch)
// for the masked pixels of a level only: every admissible candidate 0 <= z <= min(D_k - 1, x)
// of each pixel whose bicubic cost prior failed the gate.
//
// The gate (gated.cu) lists the 2 x 2 cells that hold a masked pixel.  A persistent grid
// (the CTAs the SMs hold at once) walks that list: each warp takes the next 32 entries with
// one atomic, one thread per cell, and runs the cell's full-range search
// (tiles::cell_search_full: the four pixels share each right row's loads and the products
// of their common window rows; candidates in groups of 7, exact integer sums by dp4a, the
// right-window statistics from the level's plane).  Work is proportional to the masked
// cells, and the warps stay full whatever the mask's layout.
#include <math.h>

#include <algorithm>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_cell_tile.cuh"

namespace msbm {

namespace {

constexpr int SPC_THREADS = 128;
constexpr int SPC_MIN_CTAS = 3;   // 168 registers a thread

// candidates per group (fewer at the widest window, whose left words take more registers)
template <int NH>
struct SpcG {
    static constexpr int value = NH <= 5 ? 7 : 4;
};

template <int NH>
__global__ void __launch_bounds__(SPC_THREADS, SPC_MIN_CTAS)
    zncc_sparse_cell_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int Dk, const uint8_t *mask,
                            const int2 *rstat, int rspitch, unsigned *cells, int16_t *d_out, float *c_out,
                            unsigned long long *evals) {
    const unsigned n = cells[0];
    const int ncx = (W + 1) / 2, lane = threadIdx.x & 31;
    unsigned long long cnt = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(cells + 1, 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const unsigned i = base + lane;
        if (i < n) {
            const unsigned e = cells[2 + i];
            const int cy = static_cast<int>(e / static_cast<unsigned>(ncx));
            const int cx = static_cast<int>(e - static_cast<unsigned>(cy) * ncx);
            cnt += tiles::cell_search_full<NH, SpcG<NH>::value>(L, R, pitch, W, H, Dk, mask, rstat, rspitch, d_out,
                                                                c_out, cx, cy);
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
    const long cells = (long)((l.W + 1) / 2) * ((l.H + 1) / 2);
    const long ctas = std::max<long>(1, std::min<long>(resident, (cells + SPC_THREADS - 1) / SPC_THREADS));
    zncc_sparse_cell_kernel<NH><<<static_cast<unsigned>(ctas), SPC_THREADS, 0, st>>>(
        l.img(0), l.img(1), l.pitch, l.W, l.H, l.Dk, l.mask, l.rstat, l.rspitch, l.cells, d, c, evals);
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
