// zncc_restricted.cu -- standalone launch of the restricted ZNCC winner-take-all tile
// (Sec. III-C, Eq. 8-9, first branch; design in zncc_restricted_tile.cuh): one CTA of
// 128 threads per 32 x 8 tile, each thread a vertical pair of pixels that share a prior
// cell and the products of their 2n common window rows; right-window statistics from the
// level's plane (level_stats.cu).
#include "zncc_restricted_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

constexpr int SA_QX = 32;    // threads per tile row; tile width SA_QX pixels
constexpr int SA_NCOL = 1;

// Minimum CTAs per SM the register allocation must allow.  Up to 9 x 9 windows run four
// CTAs per SM (64 registers): for r = 3 at 7 x 7 that costs 20 spilled bytes instead of 78
// registers (3 CTAs per SM), at 9 x 9 196 bytes instead of 99 registers (2 CTAs per SM), and
// level 0 of the 2880 x 1984 pair (9 x 9, r = 3) went 190 -> 150 us (three CTAs per SM at 80
// registers: 156 us).  Without a minimum the compiler may also take more registers for smaller
// groups.  Larger windows keep two CTAs per SM.
constexpr int restr_min_ctas(int nh) { return nh <= 4 ? 4 : 2; }

// Tile height: 32 x 8 tiles of 128 threads, eight CTAs per SM, hide each CTA's latency chain
// (prior load, span reduction, TMA wait) behind more independent CTAs than 32 x 16 tiles of
// 256 threads at four per SM (measured: 1400 x 1000 pass 58.3 -> 54.5 us, level 0 28.7 ->
// 26.6 us; 2880 x 1984 pass 265 -> 248 us), at 1.27x the staged halo rows per pixel.
constexpr int SA_TY = 8;

template <int NH, int G>
__global__ void __launch_bounds__(SA_QX * SA_TY / 2, restr_min_ctas(NH) * 16 / SA_TY)
    zncc_restricted_kernel(const __grid_constant__ RestrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    restr_tile<NH, G, SA_QX, SA_NCOL, true, SA_TY>(a.t, &a.tmL, &a.tmR128, &a.tmR256, &a.tmS128, &a.tmS256,
                                                   blockIdx.x, blockIdx.y, smem, parity);
}

template <int NH, int G>
cudaError_t prepare_t() {
    using C = RCfg<NH, SA_QX, SA_NCOL, true, SA_TY>;
    return cudaFuncSetAttribute(zncc_restricted_kernel<NH, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::BYTES));
}

template <int NH, int G>
cudaError_t launch_restr_t(const RestrArgs &a, cudaStream_t st) {
    using C = RCfg<NH, SA_QX, SA_NCOL, true, SA_TY>;
    static_assert(C::TX == 32 && C::BYTES <= 227 * 1024, "restricted tile shape");
    dim3 grd((a.t.W + C::TX - 1) / C::TX, (a.t.H + SA_TY - 1) / SA_TY);
    zncc_restricted_kernel<NH, G><<<grd, C::THREADS, C::BYTES, st>>>(a);
    return cudaGetLastError();
}

// G, the candidates a thread evaluates per staged right word group, is 2r + 1 (at most 7)
template <int NH>
cudaError_t prepare_nh() {
    cudaError_t e = prepare_t<NH, 1>();
    if (e == cudaSuccess) e = prepare_t<NH, 3>();
    if (e == cudaSuccess) e = prepare_t<NH, 5>();
    if (e == cudaSuccess) e = prepare_t<NH, 7>();
    return e;
}

template <int NH>
cudaError_t launch_restr_nh(const RestrArgs &a, cudaStream_t st) {
    switch (a.t.r) {
        case 0: return launch_restr_t<NH, 1>(a, st);
        case 1: return launch_restr_t<NH, 3>(a, st);
        case 2: return launch_restr_t<NH, 5>(a, st);
        default: return launch_restr_t<NH, 7>(a, st);
    }
}

}  // namespace

int restr_tile_rows() { return SA_TY; }

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

cudaError_t launch_zncc_restricted(const RestrArgs &a, int nh, cudaStream_t st) {
    switch (nh) {
        case 1: return launch_restr_nh<1>(a, st);
        case 2: return launch_restr_nh<2>(a, st);
        case 3: return launch_restr_nh<3>(a, st);
        case 4: return launch_restr_nh<4>(a, st);
        case 5: return launch_restr_nh<5>(a, st);
        case 6: return launch_restr_nh<6>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
