// zncc_restricted.cu -- standalone launches of the restricted ZNCC winner-take-all search
// (Sec. III-C, Eq. 8-9, first branch).  Two designs, chosen per level by its size and window:
//  * large levels, windows of 9 x 9 and more: the strip tile (zncc_strip_tile.cuh), one CTA of 128 threads per 32 x 16
//    tile, each thread a vertical strip of four pixels that share the products of their
//    common window rows; left- and right-window statistics from the level's planes;
//  * otherwise: the cell kernel (zncc_cell_tile.cuh), one thread per prior cell (2 x 2
//    pixels), operands read through L1 with no staging, barriers or waits.  It replaced the
//    TMA-staged vertical-pair tile (zncc_restricted_tile.cuh, 32 x 8 pixels per CTA), whose
//    per-CTA latency chain (prior load, span reduction, TMA wait) left its warps stalled at
//    barriers: level 0 of the 1400 x 1000 pair (7 x 7, r = 2) 26.6 -> 20.5 us, the pass
//    56.2 -> 49.6 us.  The staged tile still runs under MSBM_FLAG_TEST_TIMEOUT, whose
//    bounded TMA wait it exercises.
#include "zncc_cell_tile.cuh"
#include "zncc_restricted_tile.cuh"
#include "zncc_strip_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

// ---- strip tile (32 x 16)
constexpr int ST_TY = 16;
// Minimum CTAs per SM the register allocation must allow: seven (72 registers; with each
// pixel's epilogue run as soon as its window sums are final, <n = 4, G = 7> spills 4 bytes).
// Level 0 of the 2880 x 1984 pair (9 x 9, r = 3): 104.5 us at seven, 106.5 at eight (64
// registers), 108.5 at six.
constexpr int strip_min_ctas(int nh) { return nh <= 4 ? 7 : 3; }

template <int NH, int G>
__global__ void __launch_bounds__(SCfg<NH, ST_TY>::THREADS, strip_min_ctas(NH))
    zncc_strip_kernel(const __grid_constant__ RestrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    strip_tile<NH, G, ST_TY>(a.t, &a.tmL, &a.tmR128, &a.tmS, &a.tmSL, blockIdx.x, blockIdx.y, smem, parity);
}

// ---- vertical-pair tile (32 x 8)
constexpr int VP_TY = 8;
// Up to 9 x 9 windows run eight CTAs per SM (64 registers); larger ones four.
constexpr int pair_min_ctas(int nh) { return nh <= 4 ? 8 : 4; }

template <int NH, int G>
__global__ void __launch_bounds__(32 * VP_TY / 2, pair_min_ctas(NH))
    zncc_restricted_kernel(const __grid_constant__ RestrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    restr_tile<NH, G, 32, 1, true, VP_TY>(a.t, &a.tmL, &a.tmR128, &a.tmR256, &a.tmS, &a.tmS256, blockIdx.x,
                                          blockIdx.y, smem, parity);
}

// ---- cell kernel: one thread per prior cell, 32 x 4 cells (64 x 8 pixels) per CTA.  Five
// CTAs per SM (96 registers): level 0 of the 1400 x 1000 pair 20.5 us, against 21.5 at four
// (128 registers) and 22.5 at six (80 registers, more spills); 256-thread CTAs were slower.
constexpr int CELL_THREADS = 128;
constexpr int CELL_MIN_CTAS = 5;

template <int NH, int G>
__global__ void __launch_bounds__(CELL_THREADS, CELL_MIN_CTAS) zncc_cell_kernel(const RestrTileArgs a) {
    __shared__ unsigned long long evsum;
    if (threadIdx.x == 0) evsum = 0ull;
    __syncthreads();
    const int cx = blockIdx.x * 32 + (threadIdx.x & 31);
    const int cy = blockIdx.y * (CELL_THREADS / 32) + (threadIdx.x >> 5);
    unsigned cnt = 0;
    if (2 * cx < a.W && 2 * cy < a.H) cnt = cell_search<NH, G>(a, cx, cy);
    const unsigned wc = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((threadIdx.x & 31) == 0 && wc) atomicAdd(&evsum, static_cast<unsigned long long>(wc));
    __syncthreads();
    if (threadIdx.x == 0 && a.evals && evsum) atomicAdd(a.evals, evsum);
}

template <int NH, int G>
cudaError_t prepare_t() {
    // dynamic shared memory opt-in, and the largest shared-memory carveout so that shared
    // memory does not cap the resident CTAs below what the registers allow
    cudaError_t e = cudaFuncSetAttribute(zncc_strip_kernel<NH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(SCfg<NH, ST_TY>::BYTES));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(zncc_strip_kernel<NH, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(zncc_restricted_kernel<NH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(RCfg<NH, 32, 1, true, VP_TY>::BYTES));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(zncc_restricted_kernel<NH, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int NH, int G>
cudaError_t launch_restr_t(const RestrArgs &a, int ty, cudaStream_t st) {
    if (ty == VP_TY && !a.t.force_timeout) {
        // the cell kernel has no device waits; the test flag keeps the staged tile, whose
        // bounded TMA wait it exercises
        dim3 grd((a.t.Wp + 31) / 32, (a.t.Hp + CELL_THREADS / 32 - 1) / (CELL_THREADS / 32));
        zncc_cell_kernel<NH, G><<<grd, CELL_THREADS, 0, st>>>(a.t);
    } else if (ty == ST_TY) {
        using C = SCfg<NH, ST_TY>;
        static_assert(C::BYTES <= 227 * 1024, "strip tile shape");
        dim3 grd((a.t.W + C::TX - 1) / C::TX, (a.t.H + ST_TY - 1) / ST_TY);
        zncc_strip_kernel<NH, G><<<grd, C::THREADS, C::BYTES, st>>>(a);
    } else {
        using C = RCfg<NH, 32, 1, true, VP_TY>;
        static_assert(C::TX == 32 && C::BYTES <= 227 * 1024, "restricted tile shape");
        dim3 grd((a.t.W + C::TX - 1) / C::TX, (a.t.H + VP_TY - 1) / VP_TY);
        zncc_restricted_kernel<NH, G><<<grd, C::THREADS, C::BYTES, st>>>(a);
    }
    return cudaGetLastError();
}

// G, the candidates a thread evaluates per group, is 2r + 1 (at most 7; wider radii run
// several groups)
template <int NH>
cudaError_t prepare_nh() {
    cudaError_t e = prepare_t<NH, 1>();
    if (e == cudaSuccess) e = prepare_t<NH, 3>();
    if (e == cudaSuccess) e = prepare_t<NH, 5>();
    if (e == cudaSuccess) e = prepare_t<NH, 7>();
    return e;
}

template <int NH>
cudaError_t launch_restr_nh(const RestrArgs &a, int ty, cudaStream_t st) {
    switch (a.t.r) {
        case 0: return launch_restr_t<NH, 1>(a, ty, st);
        case 1: return launch_restr_t<NH, 3>(a, ty, st);
        case 2: return launch_restr_t<NH, 5>(a, ty, st);
        default: return launch_restr_t<NH, 7>(a, ty, st);
    }
}

}  // namespace

int restr_tile_rows(int W, int H, int nh, int sms) {
    // The strip tile for windows of 9 x 9 and more where its 32 x 16 grid gives every SM at
    // least eight CTAs.  Measured (level 0 / whole pass): 2880 x 1984, 9 x 9, r = 3:
    // 104.5 / 224 us against 151.6 / 258 us for the vertical-pair tile; 1400 x 1000, 7 x 7,
    // r = 2: the same level-0 time for both tiles, the pass 59.9 us with the strip tile (its
    // left-window plane) against 55.8 us.
    const long ctas = (long)((W + 31) / 32) * ((H + 15) / 16);
    return (nh >= 4 && ctas >= 8L * sms) ? ST_TY : VP_TY;
}

cudaError_t zncc_restricted_prepare(int nh) {
    switch (nh) {
        case 1: return prepare_nh<1>();
        case 2: return prepare_nh<2>();
        case 3: return prepare_nh<3>();
        case 4: return prepare_nh<4>();
        case 5: return prepare_nh<5>();
        case 6: return prepare_nh<6>();
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zncc_restricted(const RestrArgs &a, int nh, int ty, cudaStream_t st) {
    if (ty != ST_TY && ty != VP_TY) return cudaErrorInvalidValue;
    switch (nh) {
        case 1: return launch_restr_nh<1>(a, ty, st);
        case 2: return launch_restr_nh<2>(a, ty, st);
        case 3: return launch_restr_nh<3>(a, ty, st);
        case 4: return launch_restr_nh<4>(a, ty, st);
        case 5: return launch_restr_nh<5>(a, ty, st);
        case 6: return launch_restr_nh<6>(a, ty, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
