// zncc_full.cu -- standalone launch of the full-range ZNCC winner-take-all tile
// (Sec. III-A, Eq. 1-4; design in zncc_full_tile.cuh): one CTA of 4 warps per tile.
#include "zncc_full_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

// Three CTAs per SM: the 7 x 7, 128-column tile takes 168 registers and 68.5 KB of shared
// memory (its window-statistics temporaries packed one word per column sum).
template <int NH, int SX, int ZC>
__global__ void __launch_bounds__(128, 3) zncc_full_kernel(const __grid_constant__ FullArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_launch_dependents();
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();
    uint32_t parity = 0;
    full_tile<NH, SX, ZC>(a.t, &a.tmL, &a.tmR, blockIdx.x, blockIdx.y, smem, parity);
}

template <int NH, int SX>
cudaError_t launch_full_t(const FullArgs *a, cudaStream_t st, bool pdl) {
    constexpr int ZC = NH <= 4 ? 8 : 4;
    using C = FullCfg<NH, SX, ZC>;
    auto kern = zncc_full_kernel<NH, SX, ZC>;
    if (!a) {  // preparation: the dynamic shared memory this instantiation needs, and the
               // largest carveout so that shared memory does not cap the resident CTAs
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C::BYTES));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return e;
    }
    dim3 grd((a->t.W + C::TX - 1) / C::TX, (a->t.H + C::TY - 1) / C::TY);
    return launch_k(kern, grd, dim3(128), C::BYTES, st, pdl, *a);
}

template <int NH>
cudaError_t launch_full_nh(const FullArgs *a, int sx, cudaStream_t st, bool pdl) {
    switch (sx) {
        case 1: return launch_full_t<NH, 1>(a, st, pdl);
        case 2: return launch_full_t<NH, 2>(a, st, pdl);
        default: return launch_full_t<NH, 4>(a, st, pdl);
    }
}

cudaError_t full_dispatch(const FullArgs *a, int nh, int sx, cudaStream_t st, bool pdl) {
    switch (nh) {
        case 1: return launch_full_nh<1>(a, sx, st, pdl);
        case 2: return launch_full_nh<2>(a, sx, st, pdl);
        case 3: return launch_full_nh<3>(a, sx, st, pdl);
        case 4: return launch_full_nh<4>(a, sx, st, pdl);
        case 5: return launch_full_nh<5>(a, sx, st, pdl);
        case 6: return launch_full_nh<6>(a, sx, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace


cudaError_t launch_zncc_full(const FullArgs &a, int nh, int sx, cudaStream_t st, bool pdl) {
    return full_dispatch(&a, nh, sx, st, pdl);
}

cudaError_t zncc_full_prepare(int nh, int sx) { return full_dispatch(nullptr, nh, sx, nullptr, false); }

}  // namespace msbm
