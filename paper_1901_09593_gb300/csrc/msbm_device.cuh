// msbm_device.cuh -- device-side building blocks shared by the libmsbm kernels:
// level-buffer geometry, mbarrier + TMA (cp.async.bulk.tensor) wrappers with bounded
// waits, and the order-preserving key used by the winner-take-all reductions.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace msbm {

// Every pyramid level is stored with a replicated apron around the image so that
// clamp-to-edge window reads are plain reads and TMA tile origins stay 16-byte aligned.
constexpr int APX = 16;  // apron columns left and right
constexpr int APY = 8;   // apron rows above and below
constexpr int MAX_NH = 6;  // largest window half-width (13 x 13)

// Device error codes written to the context's error word (mirror msbm_status values).
constexpr int DEV_ERR_TIMEOUT = 5;

// Limit, in clock64 cycles, of a bounded mbarrier wait (about 1 s at 2 GHz).
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Poll until the phase with `parity` completes or `limit` cycles pass.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// x (innermost, bytes for uint8 maps) must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}

// Stage-completion protocol for one TMA batch: thread 0 polls the barrier with a bound;
// the outcome is broadcast through `flag`.  On success every thread re-observes the
// completed phase (an immediate acquire) before reading the tile.  On failure thread 0
// records the timeout, keeps waiting (bounded) so that no copy is left in flight when the
// CTA exits, and every thread sees `false`.
__device__ __forceinline__ bool tma_batch_wait(uint64_t *bar, uint32_t parity, int *flag,
                                               bool force_timeout, int *err) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        bool ok = force_timeout ? false : mbar_wait_bounded(bar, parity, WAIT_LIMIT_CYCLES);
        if (!ok) {
            atomicCAS(err, 0, DEV_ERR_TIMEOUT);
            mbar_wait_bounded(bar, parity, WAIT_LIMIT_CYCLES);  // drain
        }
        *flag = ok ? 1 : 0;
    }
    __syncthreads();
    bool ok = *flag != 0;
    if (ok) mbar_try_wait(bar, parity);
    return ok;
}

// Programmatic dependent launch (griddepcontrol): a kernel launched with the programmatic
// stream serialization attribute may be scheduled while its stream predecessor is still
// running, once every CTA of the predecessor has called pdl_launch_dependents (or exited);
// pdl_wait returns when the predecessor has completed and its writes are visible.  A kernel
// launched that way calls pdl_wait before it touches anything the predecessor writes.  For
// a kernel launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Unsigned 4-way byte dot product with accumulate (one dp4a instruction).
__device__ __forceinline__ uint32_t dp4a_u8(uint32_t a, uint32_t b, uint32_t c) {
    return __dp4a(a, b, c);
}

// Order-preserving map float -> uint32 (larger float -> larger key).  It orders -0 below
// +0; the ZNCC kernels only produce a zero score as +0 (the covariance term is an exact
// +0 whenever either window is flat, and +0 times a finite scale stays +0).
__device__ __forceinline__ uint32_t float_order_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float float_from_order_key(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// 64-bit WTA key: score in the high word, (0xFFFFFFFF - z) in the low word, so that the
// maximum key is the best score with the smallest z among exact ties.
__device__ __forceinline__ unsigned long long wta_key(float score, int z) {
    return (static_cast<unsigned long long>(float_order_key(score)) << 32) |
           static_cast<unsigned long long>(0xFFFFFFFFu - static_cast<uint32_t>(z));
}

}  // namespace msbm
