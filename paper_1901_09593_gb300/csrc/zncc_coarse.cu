// zncc_coarse.cu -- standalone launch of the small-level full-range ZNCC winner-take-all
// (Sec. III-A, Eq. 1-4; design in zncc_coarse_tile.cuh), normally at the coarsest pyramid
// level.  The full-range tile kernel (zncc_full.cu) is built for throughput on large searches;
// on a level of a few ten thousand pixels its 32 x 8 tiles leave most SMs idle and each CTA
// runs a long serial chain, while here 32 x 2 pixel tiles with four threads per pixel (each
// taking every fourth group of 4 candidates) spread the level over many short CTAs.
#include <math.h>

#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "zncc_coarse_tile.cuh"

namespace msbm {

namespace {

constexpr int SA_NT = 256;       // threads per CTA (128 measured the same)
constexpr int SA_TY = SA_NT / 128;  // tile rows: 2, four threads per pixel (measured: beats 4 and 8 rows)

template <int NH>
__global__ void __launch_bounds__(SA_NT) zncc_coarse_kernel(const uint8_t *L, const uint8_t *R, int pitch, int W,
                                                          int H, int Dk, int16_t *d_out, float *c_out,
                                                          unsigned long long *evals) {
    __shared__ __align__(16) uint8_t sm[CoarseCfg<NH, SA_TY>::BYTES];
    pdl_launch_dependents();
    pdl_wait();
    coarse_tile<NH, SA_TY, SA_NT>(L, R, pitch, W, H, Dk, d_out, c_out, evals, blockIdx.x, blockIdx.y, sm);
}

template <int NH>
cudaError_t coarse_launch(const LevelBuf &l, int16_t *d, float *c, unsigned long long *evals, cudaStream_t st,
                          bool pdl) {
    dim3 grd((l.W + CO_TX - 1) / CO_TX, (l.H + SA_TY - 1) / SA_TY);
    return launch_k(zncc_coarse_kernel<NH>, grd, dim3(SA_NT), 0, st, pdl, (const uint8_t *)l.img(0),
                    (const uint8_t *)l.img(1), l.pitch, l.W, l.H, l.Dk, d, c, evals);
}

}  // namespace

bool zncc_coarse_fits(int W, int H, int sms) {
    // the full-range tile kernel's 32 x 8 tiles cannot fill the GPU twice over
    return (long)((W + 31) / 32) * ((H + 7) / 8) < 2L * sms;
}

cudaError_t launch_zncc_coarse(const LevelBuf &l, int nh, int16_t *d, float *c, unsigned long long *evals,
                               cudaStream_t st, bool pdl) {
    switch (nh) {
        case 1: return coarse_launch<1>(l, d, c, evals, st, pdl);
        case 2: return coarse_launch<2>(l, d, c, evals, st, pdl);
        case 3: return coarse_launch<3>(l, d, c, evals, st, pdl);
        case 4: return coarse_launch<4>(l, d, c, evals, st, pdl);
        case 5: return coarse_launch<5>(l, d, c, evals, st, pdl);
        case 6: return coarse_launch<6>(l, d, c, evals, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace msbm
