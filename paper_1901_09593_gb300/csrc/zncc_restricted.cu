// zncc_restricted.cu -- standalone launches of the restricted ZNCC winner-take-all search
// (Sec. III-C, Eq. 8-9, first branch).
//  * The cell kernel (zncc_cell_tile.cuh): one thread per prior cell (2 x 2 pixels),
//    operands read through L1 with no staging, barriers or waits.  It replaced two
//    TMA-staged tiles whose per-CTA latency chain (prior load, span reduction, TMA wait)
//    left their warps stalled at barriers: level 0 of the 1400 x 1000 pair (7 x 7, r = 2)
//    26.6 -> 20.5 us (the pass 56.2 -> 48.1 us) against the vertical-pair tile, and the
//    2880 x 1984 pass (9 x 9, r = 3) 228 -> 167 us against the strip tile (32 x 16 pixels,
//    four-pixel vertical strips) at its two finest levels and the pair tile below.
//  * The vertical-pair tile (zncc_restricted_tile.cuh, 32 x 8 pixels per CTA of 128
//    threads) runs under MSBM_FLAG_TEST_TIMEOUT only: its bounded TMA wait is the path
//    that flag exercises.
#include "zncc_cell_tile.cuh"
#include "zncc_restricted_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

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

// ---- cell kernel: one thread per prior cell, 32 x 4 cells (64 x 8 pixels) per CTA, four
// CTAs per SM (128 registers).  Measured passes: 1400 x 1000 (7 x 7) 48.1 us against 49.7
// at five CTAs per SM (96 registers, spills); 2880 x 1984 (9 x 9) 169 us against 179 at
// five and (before the unchecked path for unclipped cells) 218 at six; 256-thread CTAs were
// slower.
constexpr int CELL_THREADS = 128;
constexpr int CELL_MIN_CTAS = 4;
// A level of windows up to 7 x 7 whose grid fits in one wave at five CTAs per SM (96
// registers) but not at four takes the five-CTA build: level 1 of the 1400 x 1000 pair (693
// CTAs) instead of running a second wave of 85 CTAs (pass 49.7 -> 47.9 us).  Larger windows
// spill at 96 registers (level 2 of the 2880 x 1984 pair, 9 x 9: 12.3 -> 14.3 us), so keep four.
constexpr int CELL_MIN_CTAS_ONE_WAVE = 5;

template <int NH, int G, int MINB>
__global__ void __launch_bounds__(CELL_THREADS, MINB) zncc_cell_kernel(const RestrTileArgs a) {
    __shared__ unsigned long long evsum;
    pdl_launch_dependents();
    if (threadIdx.x == 0) evsum = 0ull;
    __syncthreads();
    pdl_wait();
    const int cx = blockIdx.x * 32 + (threadIdx.x & 31);
    const int cy = blockIdx.y * (CELL_THREADS / 32) + (threadIdx.x >> 5);
    unsigned cnt = 0;
    if (2 * cx < a.W && 2 * cy < a.H) cnt = cell_search<NH, G>(a, cx, cy);
    const unsigned wc = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((threadIdx.x & 31) == 0 && wc) atomicAdd(&evsum, static_cast<unsigned long long>(wc));
    __syncthreads();
    if (threadIdx.x == 0 && a.evals && evsum) atomicAdd(a.evals, evsum);
}

// SMs of the current device (queried once per process)
int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            return 1;
    }
    return n;
}

template <int NH, int G>
cudaError_t prepare_t() {
    // dynamic shared memory opt-in of the staged tile, and the largest shared-memory
    // carveout so that shared memory does not cap its resident CTAs below what the registers
    // allow
    cudaError_t e = cudaFuncSetAttribute(zncc_restricted_kernel<NH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(RCfg<NH, 32, 1, true, VP_TY>::BYTES));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(zncc_restricted_kernel<NH, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int NH, int G>
cudaError_t launch_restr_t(const RestrArgs &a, cudaStream_t st, bool pdl) {
    if (!a.t.force_timeout) {
        dim3 grd((a.t.Wp + 31) / 32, (a.t.Hp + CELL_THREADS / 32 - 1) / (CELL_THREADS / 32));
        const long ctas = (long)grd.x * grd.y, sms = sm_count();
        if (NH <= 3 && ctas > CELL_MIN_CTAS * sms && ctas <= CELL_MIN_CTAS_ONE_WAVE * sms)
            return launch_k(zncc_cell_kernel<NH, G, CELL_MIN_CTAS_ONE_WAVE>, grd, dim3(CELL_THREADS), 0, st, pdl,
                            a.t);
        return launch_k(zncc_cell_kernel<NH, G, CELL_MIN_CTAS>, grd, dim3(CELL_THREADS), 0, st, pdl, a.t);
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
cudaError_t launch_restr_nh(const RestrArgs &a, cudaStream_t st, bool pdl) {
    switch (a.t.r) {
        case 0: return launch_restr_t<NH, 1>(a, st, pdl);
        case 1: return launch_restr_t<NH, 3>(a, st, pdl);
        case 2: return launch_restr_t<NH, 5>(a, st, pdl);
        default: return launch_restr_t<NH, 7>(a, st, pdl);
    }
}

}  // namespace

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

cudaError_t launch_zncc_restricted(const RestrArgs &a, int nh, cudaStream_t st, bool pdl) {
    switch (nh) {
        case 1: return launch_restr_nh<1>(a, st, pdl);
        case 2: return launch_restr_nh<2>(a, st, pdl);
        case 3: return launch_restr_nh<3>(a, st, pdl);
        case 4: return launch_restr_nh<4>(a, st, pdl);
        case 5: return launch_restr_nh<5>(a, st, pdl);
        case 6: return launch_restr_nh<6>(a, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
