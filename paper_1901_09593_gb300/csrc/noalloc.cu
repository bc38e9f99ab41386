// noalloc.cu -- flat full-range ZNCC block matching that allocates no device memory.
//
// Who needs this: callers that cannot call cudaMalloc.  cudaMalloc (and cudaFree) can
// synchronise the whole device, which a real-time loop sharing the GPU with other streams
// cannot afford mid-frame, and some host frameworks own every byte of device memory
// through their own pool and forbid allocations made behind their back.  Such callers
// pass only their inputs and outputs; the scratch this path needs (the two replicated-
// apron image buffers the full-range kernel stages its TMA tiles from, plus one status
// word) lives in the file-scope device array below, which is part of this module's image:
// every GPU that loads the module holds it until the process exits.
//
// The computation is the existing K = 1 path: the apron copy kernel and the full-range
// ZNCC winner-take-all kernel, launched on the caller's stream with the scratch address
// instead of context-owned buffers.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "msbm.h"
#include "msbm_internal.h"

using namespace msbm;

namespace {

// Scratch: [0, 256) status word, then the left and right apron buffers.
static __device__ __align__(256) uint8_t g_noalloc_scratch[MSBM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
int g_num_sms[kMaxDevices] = {0};   // per device, once its architecture has been checked
typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_entry() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

bool encode_map(CUtensorMap *m, uint8_t *base, int pitch, int rows, int box_w, int box_h) {
    EncodeFn fn = encode_entry();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-device checks, once: the architecture and the SM count (neither changes while the
// process lives).
msbm_status check_device(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_num_sms[dev]) return MSBM_OK;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return MSBM_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3) || !encode_entry()) return MSBM_ERR_UNSUPPORTED;
    g_num_sms[dev] = prop.multiProcessorCount;
    return MSBM_OK;
}

// The scratch array's device address in the current context.  Host code only sees a
// stand-in for the symbol; the address is looked up again on every call (the lookup
// allocates nothing once the module is loaded), so a context created anew after
// cudaDeviceReset, where the module may load at another address, gets its own address.
msbm_status scratch_address(uint8_t **out) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MSBM_ERR_CUDA;
    *out = static_cast<uint8_t *>(ptr);
    return MSBM_OK;
}

int pick_sx(int W, int H, int sms) {
    for (int sx = 4; sx > 1; sx /= 2) {
        long ctas = (long)((W + 32 * sx - 1) / (32 * sx)) * ((H + 7) / 8);
        if (ctas >= 2L * sms) return sx;
    }
    return 1;
}

}  // namespace

extern "C" msbm_status msbm_flat_disparity_noalloc(const uint8_t *d_left, const uint8_t *d_right,
                                                   size_t pitch_bytes, int32_t width, int32_t height,
                                                   int32_t max_disp, int32_t window, int16_t *d_out,
                                                   float *cost_out, int32_t *d_status, void *cuda_stream) {
    if (!d_left || !d_right || !d_out) return MSBM_ERR_INVALID_ARG;
    if (width < 1 || width > 16384 || height < 1 || height > 16384) return MSBM_ERR_INVALID_ARG;
    if (max_disp < 1 || max_disp > 4096) return MSBM_ERR_INVALID_ARG;
    if (window < 3 || window > 13 || (window & 1) == 0) return MSBM_ERR_INVALID_ARG;
    if (pitch_bytes < (size_t)width) return MSBM_ERR_INVALID_ARG;

    const int pitch = (width + 2 * APX + 127) / 128 * 128;
    const int rows = height + 2 * APY;
    const size_t img_bytes = ((size_t)pitch * rows + 255) / 256 * 256;
    if (256 + 2 * img_bytes > (size_t)MSBM_NOALLOC_SCRATCH_BYTES) return MSBM_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MSBM_ERR_CUDA;
    msbm_status s = check_device(dev);
    if (s != MSBM_OK) return s;
    uint8_t *scratch = nullptr;
    s = scratch_address(&scratch);
    if (s != MSBM_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    LevelBuf lv;
    lv.W = width;
    lv.H = height;
    lv.Dk = max_disp;
    lv.pitch = pitch;
    lv.rows = rows;
    lv.base[0] = scratch + 256;
    lv.base[1] = scratch + 256 + img_bytes;
    const int nh = window / 2, rowsF = 8 + 2 * nh;
    const int sx = pick_sx(width, height, g_num_sms[dev]);
    // the kernel's dynamic shared memory opt-in, in the current context (a host-side call
    // that allocates nothing)
    if (zncc_full_prepare(nh, sx) != cudaSuccess) return MSBM_ERR_CUDA;
    FullArgs a;
    memset(&a, 0, sizeof(a));
    if (!encode_map(&a.tmL, lv.base[0], pitch, rows, 32 * sx + 32, rowsF) ||
        !encode_map(&a.tmR, lv.base[1], pitch, rows, 256, rowsF))
        return MSBM_ERR_UNSUPPORTED;
    a.t.W = width;
    a.t.H = height;
    a.t.Dk = max_disp;
    a.t.zblock = 0;
    a.t.d_out = d_out;
    a.t.c_out = cost_out;
    a.t.evals = nullptr;
    // the failure word starts at zero on every call
    a.t.err = d_status ? d_status : reinterpret_cast<int *>(scratch);
    a.t.force_timeout = 0;
    cudaError_t e = cudaMemsetAsync(a.t.err, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_apron_copy(d_left, d_right, pitch_bytes, lv, st);
    if (e == cudaSuccess) e = launch_zncc_full(a, nh, sx, st);
    return e == cudaSuccess ? MSBM_OK : MSBM_ERR_CUDA;
}
