// zncc_restricted.cu -- standalone launch of the restricted ZNCC winner-take-all tile
// (Sec. III-C, Eq. 8-9, first branch; design in zncc_restricted_px_tile.cuh): one CTA of
// 256 threads, one per pixel, per 32 x 8 tile.
#include "zncc_restricted_px_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

template <int NH, int G>
__global__ void __launch_bounds__(256) zncc_restricted_kernel(const __grid_constant__ RestrArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t parity = 0;
    restr_tile_px<NH, G>(a.t, &a.tmL, &a.tmR64, &a.tmR256, blockIdx.x, blockIdx.y, smem, parity);
}

template <int NH, int G>
cudaError_t launch_restr_t(const RestrArgs &a, cudaStream_t st) {
    using C = RCfgPx<NH>;
    static_assert(C::BYTES <= 48 * 1024, "restricted tile fits the default shared memory");
    dim3 grd((a.t.W + PX_TX - 1) / PX_TX, (a.t.H + PX_TY - 1) / PX_TY);
    zncc_restricted_kernel<NH, G><<<grd, PX_TX * PX_TY, C::BYTES, st>>>(a);
    return cudaGetLastError();
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
