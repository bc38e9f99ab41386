// batch.cu -- many stereo pairs of uneven sizes and disparity ranges through all pyramid
// levels in one persistent launch (the hierarchical pass of Sec. III, Fig. 1, per pair).
//
// Work queue.  Each pair's pass is a chain of 2K stages:
//   stage 0          level-0 copy into the pair's apron buffers      (row bands)
//   stage 1 .. K-1   pyramid reduce producing level k                 (row bands)
//   stage K          full-range search at level K-1 (Eq. 3-4)         (TX x 8 tiles)
//   stage K+1+j      restricted search at level K-2-j (Eq. 8-9)       (64 x 16 tiles)
// Stage s of a pair needs every tile of stage s-1 of the same pair.  The host lays the
// (pair, stage) segments out stage-major (stage 0 of every pair, then stage 1, ...), which is
// a topological order, and the CTAs of one persistent grid take items from the flattened
// list with one atomic counter.  An item whose predecessor stage is unfinished waits on the
// pair's completion counter with a bounded spin (clock64 limit); because items are taken in
// topological order, every item waited on was taken earlier by a running CTA, so the queue
// cannot deadlock whatever the grid size.  On a timeout the kernel records MSBM_ERR_TIMEOUT
// and all CTAs stop taking work.
//
// Tiles are the same device functions as the standalone kernels (zncc_full_tile.cuh,
// zncc_restricted_tile.cuh, pyramid_ops.cuh); the full-range tile width (sx) and z-block per
// pair come from the caller (the autotuner).  The grid is sized from the occupancy of the
// kernel (co-resident CTAs).  The launch (counter resets + kernel) is captured in a CUDA
// graph; per-run caller pointers live in a small device table copied before each replay.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "msbm.h"
#include "msbm_device.cuh"
#include "msbm_internal.h"
#include "pyramid_ops.cuh"
#include "zncc_full_tile.cuh"
#include "zncc_restricted_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

constexpr int BT_MAXK = 12;
constexpr int BT_THREADS = 256;
constexpr int BT_BAND = 16;          // apron rows per copy/reduce item
constexpr int BT_MAX_NH = 4;         // windows up to 9 x 9
constexpr int BT_ZC = 4;             // candidates per lane chunk in batched full-range tiles
constexpr int BT_RTX = RCfg<1, 32>::TX;   // restricted tile width (64 pixels, 256 threads)
constexpr long long BT_WAIT_LIMIT = 4000000000LL;   // ~2 s at 2 GHz
constexpr long long BT_TEST_WAIT_LIMIT = 2000000LL; // ~1 ms (MSBM_FLAG_TEST_TIMEOUT)

struct BLevel {
    int W, H, Dk, pitch;
    uint8_t *L, *R;          // image origins in the apron buffers
    int16_t *d;              // maps of levels >= 1
    float *c;
    int sx, zblock;          // full-range tiling (coarsest level only)
    int tiles_x;             // tiles across for this level's matching stage
};

struct BPair {
    int W, H, D, K, nh, r;
    BLevel lv[BT_MAXK];
};

struct BMaps {               // TMA descriptors of one (pair, level), 64-byte aligned
    CUtensorMap mRL, mR128, mR256, mF256, mFL;
};

struct BIO {                 // per-run caller pointers of one pair
    const uint8_t *L, *R;
    size_t pitch;
    int16_t *d;
    float *c;
};

struct BSeg {
    long long start;         // first flattened item index
    int pair, stage, ntiles, need;   // need = tiles of the pair's previous stage
};

struct BatchArgs {
    const BPair *pairs;
    const BMaps *maps;       // [pair * BT_MAXK + level]
    const BIO *io;
    const BSeg *segs;
    int nseg;
    long long total;
    int *head;               // queue counter
    int *done;               // [pair * 2 * BT_MAXK + stage] finished tiles
    unsigned long long *evals;
    int *err;
    int withhold;            // test hook: never publish completion of stage 0
    long long wait_limit;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int NH>
__device__ bool run_match(const BatchArgs &a, const BPair &P, const BMaps *mp, const BIO &io, int stage,
                          int tile, uint8_t *smem, uint32_t &parity) {
    const int K = P.K;
    if (stage == K) {                                    // coarsest full search
        const int k = K - 1;
        const BLevel &l = P.lv[k];
        FullTileArgs t = {};   // no gating in the batch: mask / tile flags stay NULL
        t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.zblock = l.zblock;
        t.d_out = k == 0 ? io.d : l.d;
        t.c_out = k == 0 ? io.c : l.c;
        t.evals = a.evals; t.err = a.err; t.force_timeout = 0;
        const int bx = tile % l.tiles_x, by = tile / l.tiles_x;
        if (l.sx == 1) return full_tile<NH, 1, BT_ZC>(t, &mp[k].mFL, &mp[k].mF256, bx, by, smem, parity);
        return full_tile<NH, 2, BT_ZC>(t, &mp[k].mFL, &mp[k].mF256, bx, by, smem, parity);
    }
    const int k = K - 2 - (stage - K - 1);              // restricted level
    const BLevel &l = P.lv[k];
    RestrTileArgs t = {};
    t.Limg = l.L; t.Rimg = l.R; t.pitch = l.pitch;
    t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.r = P.r;
    t.prior = P.lv[k + 1].d; t.Wp = P.lv[k + 1].W; t.Hp = P.lv[k + 1].H;
    t.d_out = k == 0 ? io.d : l.d;
    t.c_out = k == 0 ? io.c : l.c;
    t.evals = a.evals; t.err = a.err; t.force_timeout = 0;
    const int bx = tile % l.tiles_x, by = tile / l.tiles_x;
    switch (P.r) {
        case 0: return restr_tile<NH, 1>(t, &mp[k].mRL, &mp[k].mR128, &mp[k].mR256, nullptr, nullptr, bx, by, smem, parity);
        case 1: return restr_tile<NH, 3>(t, &mp[k].mRL, &mp[k].mR128, &mp[k].mR256, nullptr, nullptr, bx, by, smem, parity);
        case 2: return restr_tile<NH, 5>(t, &mp[k].mRL, &mp[k].mR128, &mp[k].mR256, nullptr, nullptr, bx, by, smem, parity);
        default: return restr_tile<NH, 7>(t, &mp[k].mRL, &mp[k].mR128, &mp[k].mR256, nullptr, nullptr, bx, by, smem, parity);
    }
}

__global__ void __launch_bounds__(BT_THREADS, 2) batch_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ long long item_s;
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();   // the previous item is finished with shared memory
        if (tid == 0) {
            long long it = a.total;
            if (*reinterpret_cast<volatile int *>(a.err) == 0) it = atomicAdd(a.head, 1);
            item_s = it;
        }
        __syncthreads();
        const long long it = item_s;
        if (it >= a.total) break;
        // segment of this item: the last segment whose start is <= it
        int lo = 0, hi = a.nseg - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].start <= it) lo = mid; else hi = mid - 1;
        }
        const BSeg sg = a.segs[lo];
        const int tile = static_cast<int>(it - sg.start);
        if (tid == 0) {
            int ok = 1;
            if (sg.stage > 0) {
                const int *cnt = a.done + sg.pair * 2 * BT_MAXK + sg.stage - 1;
                const long long t0 = clock64();
                while (ld_acquire(cnt) < sg.need) {
                    if (clock64() - t0 > a.wait_limit) {
                        atomicCAS(a.err, 0, DEV_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                fence_proxy_async_global();   // other CTAs' stores -> this CTA's TMA reads
            }
            ok_s = ok;
        }
        __syncthreads();
        if (!ok_s) break;
        __threadfence();
        const BPair &P = a.pairs[sg.pair];
        const BIO io = a.io[sg.pair];
        bool ok = true;
        if (sg.stage < P.K) {
            // copy (stage 0) or reduce (stage k): BT_BAND apron rows of level `stage`
            const BLevel &d = P.lv[sg.stage];
            const int quads = (d.W + 2 * APX + 3) / 4;
            const int y0 = tile * BT_BAND - APY;
            const int nrow = min(BT_BAND, d.H + APY - y0);
            for (int i = tid; i < 2 * nrow * quads; i += BT_THREADS) {
                const int img = i / (nrow * quads), j = i - img * nrow * quads;
                const int Y = y0 + j / quads, X0 = (j % quads) * 4 - APX;
                uint8_t *dst = img ? d.R : d.L;
                if (sg.stage == 0)
                    copy_quad(img ? io.R : io.L, io.pitch, d.W, d.H, dst, d.pitch, X0, Y);
                else {
                    const BLevel &s = P.lv[sg.stage - 1];
                    reduce_quad(img ? s.R : s.L, s.pitch, dst, d.pitch, d.W, d.H, X0, Y);
                }
            }
        } else {
            const BMaps *mp = a.maps + sg.pair * BT_MAXK;
            switch (P.nh) {
                case 1: ok = run_match<1>(a, P, mp, io, sg.stage, tile, smem, parity); break;
                case 2: ok = run_match<2>(a, P, mp, io, sg.stage, tile, smem, parity); break;
                case 3: ok = run_match<3>(a, P, mp, io, sg.stage, tile, smem, parity); break;
                default: ok = run_match<4>(a, P, mp, io, sg.stage, tile, smem, parity); break;
            }
        }
        (void)ok;   // a failed wait has set the error word; the loop head then stops
        __syncthreads();   // every thread's stores of this item are issued
        if (tid == 0) {
            __threadfence();
            if (!(a.withhold && sg.stage == 0)) atomicAdd(a.done + sg.pair * 2 * BT_MAXK + sg.stage, 1);
        }
    }
}

size_t batch_smem_bytes() {
    size_t m = 0;
    m = std::max(m, FullCfg<BT_MAX_NH, 2, BT_ZC>::BYTES);
    m = std::max(m, FullCfg<BT_MAX_NH, 1, BT_ZC>::BYTES);
    m = std::max(m, RCfg<BT_MAX_NH>::BYTES);
    for (size_t b : {FullCfg<1, 2, BT_ZC>::BYTES, FullCfg<2, 2, BT_ZC>::BYTES, FullCfg<3, 2, BT_ZC>::BYTES,
                     RCfg<1>::BYTES, RCfg<2>::BYTES, RCfg<3>::BYTES})
        m = std::max(m, b);
    return m;
}

typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                             CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                             CUtensorMapFloatOOBfill);

EncodeFn encode_fn_b() {
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

bool encode_b(CUtensorMap *m, uint8_t *base, int pitch, int rows, int bw, int bh) {
    EncodeFn fn = encode_fn_b();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline msbm_status cst(cudaError_t e) {
    return e == cudaSuccess ? MSBM_OK : (e == cudaErrorMemoryAllocation ? MSBM_ERR_OOM : MSBM_ERR_CUDA);
}

}  // namespace
}  // namespace msbm

using namespace msbm;

struct msbm_batch {
    int n = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    std::vector<BPair> pairs;
    std::vector<BIO> io_host;
    std::vector<void *> allocs;
    BPair *d_pairs = nullptr;
    BMaps *d_maps = nullptr;
    BIO *d_io = nullptr;
    BSeg *d_segs = nullptr;
    int *d_head = nullptr, *d_done = nullptr, *d_err = nullptr;
    unsigned long long *d_evals = nullptr;
    int nseg = 0;
    long long total = 0;
    int grid = 0;
    size_t smem = 0;
    bool withhold = false;
    bool io_uploaded = false;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(msbm_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void *p : b->allocs) cudaFree(p);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" {

msbm_status msbm_batch_create(const msbm_params *pairs, int32_t n_pairs, const int32_t *full_sx,
                              const int32_t *full_zblock, void *cuda_stream, msbm_batch **out) {
    if (!out) return MSBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!pairs || n_pairs < 1 || n_pairs > 4096) return MSBM_ERR_INVALID_ARG;
    for (int i = 0; i < n_pairs; ++i) {
        const msbm_params &p = pairs[i];
        if (p.width < 1 || p.width > 16384 || p.height < 1 || p.height > 16384) return MSBM_ERR_INVALID_ARG;
        if (p.max_disp < 1 || p.max_disp > 4096 || p.levels < 1 || p.levels > BT_MAXK) return MSBM_ERR_INVALID_ARG;
        if (p.window < 3 || p.window > 2 * BT_MAX_NH + 1 || (p.window & 1) == 0) return MSBM_ERR_INVALID_ARG;
        if (p.radius < 0 || p.radius > 16) return MSBM_ERR_INVALID_ARG;
        if (p.flags & ~(MSBM_FLAG_NO_GRAPH | MSBM_FLAG_TEST_TIMEOUT)) return MSBM_ERR_INVALID_ARG;
        if (full_sx && full_sx[i] != 1 && full_sx[i] != 2) return MSBM_ERR_INVALID_ARG;
        if (full_zblock && (full_zblock[i] < 0 || full_zblock[i] % 32 != 0)) return MSBM_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return MSBM_ERR_UNSUPPORTED;
    if (!(prop.major == 10 && prop.minor == 3) || !encode_fn_b()) return MSBM_ERR_UNSUPPORTED;

    msbm_batch *b = new (std::nothrow) msbm_batch();
    if (!b) return MSBM_ERR_OOM;
    b->n = n_pairs;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->withhold = (pairs[0].flags & MSBM_FLAG_TEST_TIMEOUT) != 0;
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    auto dalloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) b->allocs.push_back(*p);
    };
    std::vector<BMaps> maps((size_t)n_pairs * BT_MAXK);
    memset(maps.data(), 0, maps.size() * sizeof(BMaps));
    b->pairs.resize(n_pairs);
    bool enc_ok = true;
    for (int i = 0; i < n_pairs && e == cudaSuccess; ++i) {
        const msbm_params &p = pairs[i];
        BPair &P = b->pairs[i];
        memset(&P, 0, sizeof(P));
        P.W = p.width; P.H = p.height; P.D = p.max_disp; P.K = p.levels; P.nh = p.window / 2; P.r = p.radius;
        int W = p.width, H = p.height;
        const int rowsF = 8 + 2 * P.nh, rowsR = RT_TY + 2 * P.nh;
        for (int k = 0; k < P.K && e == cudaSuccess; ++k) {
            BLevel &l = P.lv[k];
            l.W = W; l.H = H;
            l.Dk = (int)(((long)p.max_disp + (1L << k) - 1) >> k);
            l.pitch = (W + 2 * APX + 127) / 128 * 128;
            const int rows = H + 2 * APY;
            const size_t bytes = (size_t)l.pitch * rows;
            uint8_t *buf = nullptr;
            dalloc(reinterpret_cast<void **>(&buf), 2 * bytes);
            if (e != cudaSuccess) break;
            e = cudaMemset(buf, 0, 2 * bytes);
            l.L = buf + (size_t)APY * l.pitch + APX;
            l.R = buf + bytes + (size_t)APY * l.pitch + APX;
            if (k > 0) {
                dalloc(reinterpret_cast<void **>(&l.d), (size_t)W * H * sizeof(int16_t));
                dalloc(reinterpret_cast<void **>(&l.c), (size_t)W * H * sizeof(float));
            }
            l.sx = full_sx ? full_sx[i] : (W >= 512 ? 2 : 1);
            l.zblock = full_zblock ? full_zblock[i] : 0;
            l.tiles_x = (k == P.K - 1) ? (W + 32 * l.sx - 1) / (32 * l.sx) : (W + BT_RTX - 1) / BT_RTX;
            BMaps &m = maps[(size_t)i * BT_MAXK + k];
            enc_ok = enc_ok && encode_b(&m.mRL, buf, l.pitch, rows, BT_RTX + 32, rowsR) &&
                     encode_b(&m.mR128, buf + bytes, l.pitch, rows, 128, rowsR) &&
                     encode_b(&m.mR256, buf + bytes, l.pitch, rows, 256, rowsR) &&
                     encode_b(&m.mF256, buf + bytes, l.pitch, rows, 256, rowsF) &&
                     encode_b(&m.mFL, buf, l.pitch, rows, 32 * l.sx + 32, rowsF);
            W = (W + 1) / 2;
            H = (H + 1) / 2;
        }
    }
    if (e != cudaSuccess || !enc_ok) {
        msbm_status s = e != cudaSuccess ? cst(e) : MSBM_ERR_UNSUPPORTED;
        batch_free(b);
        return s;
    }
    // stage-major segment list; within a stage, larger stages first
    std::vector<BSeg> segs;
    int max_stages = 0;
    for (auto &P : b->pairs) max_stages = std::max(max_stages, 2 * P.K);
    auto ntiles = [](const BPair &P, int s) {
        if (s < P.K) return (P.lv[s].H + 2 * APY + BT_BAND - 1) / BT_BAND;
        const int k = s == P.K ? P.K - 1 : P.K - 2 - (s - P.K - 1);
        const int th = s == P.K ? 8 : RT_TY;   // full-range tiles are 8 rows, restricted 16
        return P.lv[k].tiles_x * ((P.lv[k].H + th - 1) / th);
    };
    long long pos = 0;
    for (int s = 0; s < max_stages; ++s) {
        std::vector<int> idx;
        for (int i = 0; i < n_pairs; ++i)
            if (s < 2 * b->pairs[i].K) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            return ntiles(b->pairs[x], s) > ntiles(b->pairs[y], s);
        });
        for (int i : idx) {
            BSeg g;
            g.start = pos;
            g.pair = i;
            g.stage = s;
            g.ntiles = ntiles(b->pairs[i], s);
            g.need = s > 0 ? ntiles(b->pairs[i], s - 1) : 0;
            pos += g.ntiles;
            segs.push_back(g);
        }
    }
    b->nseg = (int)segs.size();
    b->total = pos;
    dalloc(reinterpret_cast<void **>(&b->d_pairs), sizeof(BPair) * n_pairs);
    dalloc(reinterpret_cast<void **>(&b->d_maps), sizeof(BMaps) * maps.size());
    dalloc(reinterpret_cast<void **>(&b->d_io), sizeof(BIO) * n_pairs);
    dalloc(reinterpret_cast<void **>(&b->d_segs), sizeof(BSeg) * segs.size());
    dalloc(reinterpret_cast<void **>(&b->d_head), sizeof(int));
    dalloc(reinterpret_cast<void **>(&b->d_done), sizeof(int) * n_pairs * 2 * BT_MAXK);
    dalloc(reinterpret_cast<void **>(&b->d_err), sizeof(int));
    dalloc(reinterpret_cast<void **>(&b->d_evals), sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pairs, b->pairs.data(), sizeof(BPair) * n_pairs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_maps, maps.data(), sizeof(BMaps) * maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_segs, segs.data(), sizeof(BSeg) * segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_evals, 0, sizeof(unsigned long long));
    b->smem = batch_smem_bytes();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, BT_THREADS, b->smem);
    if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
    if (e != cudaSuccess) {
        msbm_status s = cst(e);
        batch_free(b);
        return s;
    }
    b->grid = occ * prop.multiProcessorCount;
    b->io_host.assign(n_pairs, BIO{nullptr, nullptr, 0, nullptr, nullptr});
    *out = b;
    return MSBM_OK;
}

static msbm_status batch_enqueue(msbm_batch *b, cudaStream_t st) {
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.pairs = b->d_pairs; a.maps = b->d_maps; a.io = b->d_io; a.segs = b->d_segs;
    a.nseg = b->nseg; a.total = b->total; a.head = b->d_head; a.done = b->d_done;
    a.evals = b->d_evals; a.err = b->d_err;
    a.withhold = b->withhold ? 1 : 0;
    a.wait_limit = b->withhold ? BT_TEST_WAIT_LIMIT : BT_WAIT_LIMIT;
    cudaError_t e = cudaMemsetAsync(b->d_head, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * b->n * 2 * BT_MAXK, st);
    if (e == cudaSuccess) {
        batch_kernel<<<b->grid, BT_THREADS, b->smem, st>>>(a);
        e = cudaGetLastError();
    }
    return cst(e);
}

msbm_status msbm_batch_run(msbm_batch *b, const uint8_t *const *d_lefts, const uint8_t *const *d_rights,
                           const size_t *pitches, int16_t *const *d_outs, float *const *cost_outs) {
    if (!b || !d_lefts || !d_rights || !pitches || !d_outs) return MSBM_ERR_INVALID_ARG;
    bool changed = !b->io_uploaded;
    for (int i = 0; i < b->n; ++i) {
        if (!d_lefts[i] || !d_rights[i] || !d_outs[i] || pitches[i] < (size_t)b->pairs[i].W)
            return MSBM_ERR_INVALID_ARG;
        BIO v{d_lefts[i], d_rights[i], pitches[i], d_outs[i], cost_outs ? cost_outs[i] : nullptr};
        BIO &h = b->io_host[i];
        if (memcmp(&v, &h, sizeof(BIO)) != 0) {
            h = v;
            changed = true;
        }
    }
    cudaError_t e = cudaSuccess;
    if (changed) {
        e = cudaMemcpyAsync(b->d_io, b->io_host.data(), sizeof(BIO) * b->n, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return cst(e);
        e = cudaStreamSynchronize(b->stream);   // the host table may change before the next run
        if (e != cudaSuccess) return cst(e);
        b->io_uploaded = true;
    }
    if (!b->exec) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return cst(e);
        msbm_status s = batch_enqueue(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
        if (s != MSBM_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return s != MSBM_OK ? s : cst(e);
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cst(e);
        }
    }
    return cst(cudaGraphLaunch(b->exec, b->stream));
}

msbm_status msbm_batch_sync(msbm_batch *b) {
    if (!b) return MSBM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MSBM_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MSBM_ERR_CUDA;
    if (err) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return static_cast<msbm_status>(err);
    }
    return MSBM_OK;
}

msbm_status msbm_batch_eval_count(msbm_batch *b, int64_t *count, int32_t reset) {
    if (!b || !count) return MSBM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return MSBM_ERR_CUDA;
    unsigned long long v = 0;
    if (cudaMemcpy(&v, b->d_evals, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return MSBM_ERR_CUDA;
    *count = static_cast<int64_t>(v);
    if (reset && cudaMemset(b->d_evals, 0, sizeof(v)) != cudaSuccess) return MSBM_ERR_CUDA;
    return MSBM_OK;
}

msbm_status msbm_batch_info(const msbm_batch *b, int64_t *n_items, int32_t *grid, int32_t *n_segments) {
    if (!b) return MSBM_ERR_INVALID_ARG;
    if (n_items) *n_items = b->total;
    if (grid) *grid = b->grid;
    if (n_segments) *n_segments = b->nseg;
    return MSBM_OK;
}

msbm_status msbm_batch_destroy(msbm_batch *b) {
    if (!b) return MSBM_OK;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    return MSBM_OK;
}

}  // extern "C"
