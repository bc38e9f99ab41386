// zncc_restricted.cu -- standalone launch of the restricted ZNCC winner-take-all tile
// (Sec. III-C, Eq. 8-9, first branch; design in zncc_strip_tile.cuh): one CTA per 32 x TY
// tile, each thread a vertical strip of four pixels that share the products of their
// common window rows; left- and right-window statistics from the level's planes
// (level_stats.cu).
#include "zncc_strip_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

// Minimum CTAs per SM the register allocation must allow (128-thread CTAs at TY = 16).
constexpr int strip_min_ctas(int nh, int ty) { return (nh <= 4 ? 6 : 3) * (16 / ty); }

template <int NH, int G, int TY>
__global__ void __launch_bounds__(SCfg<NH, TY>::THREADS, strip_min_ctas(NH, TY))
    zncc_restricted_kernel(const __grid_constant__ RestrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    strip_tile<NH, G, TY>(a.t, &a.tmL, &a.tmR128, &a.tmR256, &a.tmS, &a.tmSL, blockIdx.x, blockIdx.y, smem, parity);
}

template <int NH, int G, int TY>
cudaError_t prepare_t() {
    using C = SCfg<NH, TY>;
    return cudaFuncSetAttribute(zncc_restricted_kernel<NH, G, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(C::BYTES));
}

template <int NH, int G, int TY>
cudaError_t launch_restr_t(const RestrArgs &a, cudaStream_t st) {
    using C = SCfg<NH, TY>;
    static_assert(C::BYTES <= 227 * 1024, "restricted tile shape");
    dim3 grd((a.t.W + C::TX - 1) / C::TX, (a.t.H + TY - 1) / TY);
    zncc_restricted_kernel<NH, G, TY><<<grd, C::THREADS, C::BYTES, st>>>(a);
    return cudaGetLastError();
}

// G, the candidates a thread evaluates per group, is 2r + 1 (at most 7; wider radii run
// several groups)
template <int NH, int TY>
cudaError_t prepare_nt() {
    cudaError_t e = prepare_t<NH, 1, TY>();
    if (e == cudaSuccess) e = prepare_t<NH, 3, TY>();
    if (e == cudaSuccess) e = prepare_t<NH, 5, TY>();
    if (e == cudaSuccess) e = prepare_t<NH, 7, TY>();
    return e;
}

template <int NH>
cudaError_t prepare_nh() {
    cudaError_t e = prepare_nt<NH, 8>();
    if (e == cudaSuccess) e = prepare_nt<NH, 16>();
    return e;
}

template <int NH, int TY>
cudaError_t launch_restr_nt(const RestrArgs &a, cudaStream_t st) {
    switch (a.t.r) {
        case 0: return launch_restr_t<NH, 1, TY>(a, st);
        case 1: return launch_restr_t<NH, 3, TY>(a, st);
        case 2: return launch_restr_t<NH, 5, TY>(a, st);
        default: return launch_restr_t<NH, 7, TY>(a, st);
    }
}

template <int NH>
cudaError_t launch_restr_nh(const RestrArgs &a, int ty, cudaStream_t st) {
    return ty == 8 ? launch_restr_nt<NH, 8>(a, st) : launch_restr_nt<NH, 16>(a, st);
}

}  // namespace

int restr_tile_rows(int W, int H, int sms) {
    // 32 x 16 tiles unless they would give fewer than four CTAs per SM
    const long ctas = (long)((W + 31) / 32) * ((H + 15) / 16);
    return ctas >= 4L * sms ? 16 : 8;
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
    if (ty != 8 && ty != 16) return cudaErrorInvalidValue;
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
