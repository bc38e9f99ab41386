// batch.cu -- many stereo pairs of uneven sizes and disparity ranges through all pyramid
// levels in one persistent launch (the hierarchical pass of Sec. III, Fig. 1, per pair).
//
// Work queue.  Each pair's pass is a chain of stages (the host's per-pair stage table):
//   pyramid          fused groups of up to 3 reduce levels (pyramid_fused.cuh), 16 x 4 tiles
//                    of the group's coarsest level per image; a plain band copy when K = 1
//   coarsest level   full-range search at level K-1 (Eq. 3-4): the small-level tile
//                    (zncc_coarse_tile.cuh) for D_k <= 64, else the full-range tile
//   statistics       right-window statistics planes of levels 0 .. K-2 (level_stats_tile.cuh)
//   restricted       level K-2 .. 0 (Eq. 8-9), 32 x 8 tiles of vertical pixel pairs reading
//                    the level's statistics plane (zncc_restricted_tile.cuh, plane mode)
// Stage s of a pair needs every tile of stage s-1 of the same pair.  The host lays the
// (pair, stage) segments out stage-major (stage 0 of every pair, then stage 1, ...), which is
// a topological order, and the CTAs of one persistent grid take items from the flattened
// list with one atomic counter.  An item whose predecessor stage is unfinished waits on the
// pair's completion counter with a bounded spin (clock64 limit); because items are taken in
// topological order, every item waited on was taken earlier by a running CTA, so the queue
// cannot deadlock whatever the grid size.  On a timeout the kernel records MSBM_ERR_TIMEOUT
// and all CTAs stop taking work.
//
// Tiles are the same device functions as the standalone kernels; the full-range tile width
// (sx) and z-block per pair come from the caller (the autotuner).  The grid is sized from the
// occupancy of the kernel (co-resident CTAs).  The launch (counter resets + kernel) is
// captured in a CUDA graph; per-run caller pointers live in a small device table copied
// before each replay.
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
#include "level_stats_tile.cuh"
#include "pyramid_fused.cuh"
#include "pyramid_ops.cuh"
#include "zncc_cell_tile.cuh"
#include "zncc_coarse_tile.cuh"
#include "zncc_full_tile.cuh"
#include "zncc_restricted_tile.cuh"

namespace msbm {

namespace {

using namespace tiles;

constexpr int BT_MAXK = 12;
constexpr int BT_MAXG = (BT_MAXK + PF_MAXF - 2) / PF_MAXF;   // fused pyramid groups
constexpr int BT_MAXS = BT_MAXG + 2 + BT_MAXK;              // stages per pair
constexpr int BT_THREADS = 128;
// Two builds of the kernel: with the full-range tile (128 registers; its ~57 KB footprint
// allows 3 CTAs per SM) for batches whose coarsest levels exceed BT_COARSE_DK candidates, and
// without it (64 registers; up to 8 CTAs per SM, 7 by the statistics tile's shared memory)
// otherwise.  128-thread CTAs (restricted items on 32 x 8 tiles) give each SM about twice the
// independent CTAs of 256-thread ones.
constexpr int BT_CTAS_FULL = 4, BT_CTAS_LEAN = 8;
constexpr int BT_BAND = 16;          // apron rows per copy item (K = 1)
constexpr int BT_MAX_NH = 4;         // windows up to 9 x 9
constexpr int BT_ZC = 4;             // candidates per lane chunk in batched full-range tiles
constexpr int BT_COARSE_DK = 64;     // coarsest levels with D_k up to this use the small-level tile
constexpr int BT_NCOL = 1;           // restricted tile: vertical pixel pairs
constexpr int BT_RTY = 8;            // restricted tile rows (32 x 8 tiles, 128 threads)
constexpr int BT_CO_TY = 4;          // small-level full-range tile rows (one thread per pixel)
constexpr int BT_RTX = RCfg<1, 32, BT_NCOL, true, BT_RTY>::TX;   // restricted tile width
constexpr int BT_AUX = 128;          // shared bytes before the scratch of non-TMA tiles (mbarrier)
constexpr long long BT_WAIT_LIMIT = 4000000000LL;   // ~2 s at 2 GHz
constexpr long long BT_TEST_WAIT_LIMIT = 2000000LL; // ~1 ms (MSBM_FLAG_TEST_TIMEOUT)

enum BStageType { BS_COPY = 0, BS_PYR, BS_COARSE, BS_FULL, BS_STATS, BS_RESTR };

struct BLevel {
    int W, H, Dk, pitch;
    uint8_t *L, *R;          // image origins in the apron buffers
    int16_t *d;              // maps of levels >= 1
    float *c;
    int2 *rstat;             // right-window statistics plane (levels below the coarsest)
    int rspitch;
    int sx, zblock;          // full-range tiling (coarsest level only)
};

struct BStage {
    int type;                // BStageType
    int arg;                 // BS_PYR: fused group; BS_COARSE / BS_FULL / BS_RESTR: level
    int tiles_x, ntiles;     // tiles across (per image for BS_PYR) and in total
};

struct BPair {
    int W, H, D, K, nh, r, nst;
    BStage st[BT_MAXS];
    PyrFuseArgs pf[BT_MAXG];           // fused pyramid groups (group 0 reads the caller's images)
    int pf_nby[BT_MAXG];               // tile rows of each group's coarsest level
    int sfirst[BT_MAXK + 1], stx[BT_MAXK];   // statistics stage: first tile and tiles across per level
    BLevel lv[BT_MAXK];
};

struct BMaps {               // TMA descriptors of one (pair, level), 64-byte aligned
    CUtensorMap mRL, mR128, mR256, mF256, mFL, mS128, mS256;
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
    int *done;               // [pair * BT_MAXS + stage] finished tiles
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

// The non-TMA tiles are called out of line so that each keeps its own register allocation
// inside the persistent kernel's 128-register budget.
template <int F>
__device__ __noinline__ void pyr_item(const PyrFuseArgs &pf, const uint8_t *src, size_t spitch, int bx, int by,
                                      int img, int nbx, int nby, uint8_t *sm) {
    pyr_fused_tile<F, BT_THREADS>(pf, src, spitch, bx, by, img, nbx, nby, sm);
}

template <int NH>
__device__ __noinline__ void stats_item(const BLevel &l, int bx, int by, uint8_t *sm) {
    stats_tile<NH, BT_THREADS>(l.R, l.pitch, l.W, l.H, l.rstat, l.rspitch, bx, by, sm);
}

template <int NH>
__device__ __noinline__ void coarse_item(const BLevel &l, int16_t *d_out, float *c_out, unsigned long long *evals,
                                         int bx, int by, uint8_t *sm) {
    coarse_tile<NH, BT_CO_TY, BT_THREADS>(l.L, l.R, l.pitch, l.W, l.H, l.Dk, d_out, c_out, evals, bx, by, sm);
}

template <int NH, bool FULL>
__device__ bool run_item(const BatchArgs &a, const BPair &P, const BMaps *mp, const BIO &io, const BStage &S,
                         int tile, uint8_t *smem, uint32_t &parity) {
    const int K = P.K;
    if (S.type == BS_PYR) {
        const PyrFuseArgs &pf = P.pf[S.arg];
        const int per = S.ntiles / 2, img = tile / per, t = tile - img * per;
        const int by = t / S.tiles_x, bx = t - by * S.tiles_x;
        const uint8_t *src = S.arg == 0 ? (img ? io.R : io.L) : pf.src[img];
        const size_t spitch = S.arg == 0 ? io.pitch : pf.spitch;
        switch (pf.F) {
            case 1: pyr_item<1>(pf, src, spitch, bx, by, img, S.tiles_x, P.pf_nby[S.arg], smem + BT_AUX); break;
            case 2: pyr_item<2>(pf, src, spitch, bx, by, img, S.tiles_x, P.pf_nby[S.arg], smem + BT_AUX); break;
            default: pyr_item<3>(pf, src, spitch, bx, by, img, S.tiles_x, P.pf_nby[S.arg], smem + BT_AUX); break;
        }
        return true;
    }
    if (S.type == BS_STATS) {
        int k = 0;
        while (k + 1 < K - 1 && tile >= P.sfirst[k + 1]) ++k;
        const int t = tile - P.sfirst[k], by = t / P.stx[k], bx = t - by * P.stx[k];
        stats_item<NH>(P.lv[k], bx, by, smem + BT_AUX);
        return true;
    }
    const int k = S.arg;
    const BLevel &l = P.lv[k];
    int16_t *d_out = k == 0 ? io.d : l.d;
    float *c_out = k == 0 ? io.c : l.c;
    const int by = tile / S.tiles_x, bx = tile - by * S.tiles_x;
    if (S.type == BS_COARSE) {
        coarse_item<NH>(l, d_out, c_out, a.evals, bx, by, smem + BT_AUX);
        return true;
    }
    if constexpr (FULL) {
      if (S.type == BS_FULL) {
        FullTileArgs t = {};
        t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.zblock = l.zblock;
        t.d_out = d_out; t.c_out = c_out;
        t.evals = a.evals; t.err = a.err; t.force_timeout = 0;
        if (l.sx == 1) return full_tile<NH, 1, BT_ZC>(t, &mp[k].mFL, &mp[k].mF256, bx, by, smem, parity);
        return full_tile<NH, 2, BT_ZC>(t, &mp[k].mFL, &mp[k].mF256, bx, by, smem, parity);
      }
    }
    RestrTileArgs t = {};
    t.Limg = l.L; t.Rimg = l.R; t.pitch = l.pitch;
    t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.r = P.r;
    t.prior = P.lv[k + 1].d; t.Wp = P.lv[k + 1].W; t.Hp = P.lv[k + 1].H;
    t.d_out = d_out; t.c_out = c_out;
    t.evals = a.evals; t.err = a.err; t.force_timeout = 0;
    const BMaps &m = mp[k];
    switch (P.r) {
        case 0: return restr_tile<NH, 1, 32, BT_NCOL, true, BT_RTY>(t, &m.mRL, &m.mR128, &m.mR256, &m.mS128, &m.mS256, bx, by, smem, parity);
        case 1: return restr_tile<NH, 3, 32, BT_NCOL, true, BT_RTY>(t, &m.mRL, &m.mR128, &m.mR256, &m.mS128, &m.mS256, bx, by, smem, parity);
        case 2: return restr_tile<NH, 5, 32, BT_NCOL, true, BT_RTY>(t, &m.mRL, &m.mR128, &m.mR256, &m.mS128, &m.mS256, bx, by, smem, parity);
        default: return restr_tile<NH, 7, 32, BT_NCOL, true, BT_RTY>(t, &m.mRL, &m.mR128, &m.mR256, &m.mS128, &m.mS256, bx, by, smem, parity);
    }
}

template <bool FULL>
__global__ void __launch_bounds__(BT_THREADS, FULL ? BT_CTAS_FULL : BT_CTAS_LEAN)
    batch_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ long long item_s;
    __shared__ int seg_s;
    __shared__ int ok_s;
    const int tid = threadIdx.x;
    // thread 0 reserves the CTA's next item while the current one runs (the atomic's latency
    // hides behind the work); items are still taken in increasing order, and the smallest
    // unfinished item is always one a CTA is working on, so reservations cannot deadlock
    long long next = 0;
    int last_seg = -1;       // thread 0: segment of the previous item (its dependency already met)
    if (tid == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
        seg_s = 0;
        next = atomicAdd(a.head, 1);
    }
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();   // the previous item is finished with shared memory
        if (tid == 0) {
            const long long it = next;
            item_s = it;
            if (it < a.total) next = atomicAdd(a.head, 1);
            // segment of this item: the last segment whose start is <= it.  Items are handed
            // out in increasing order, so this CTA's segment only moves forward.
            int sgi = seg_s;
            while (sgi + 1 < a.nseg && a.segs[sgi + 1].start <= it) ++sgi;
            seg_s = sgi;
        }
        __syncthreads();
        const long long it = item_s;
        if (it >= a.total) break;
        const BSeg sg = a.segs[seg_s];
        const int tile = static_cast<int>(it - sg.start);
        if (tid == 0) {
            int ok = 1;
            // a new segment: stop if another CTA recorded an error, else wait for the pair's
            // previous stage (later items of the same segment find it complete)
            if (seg_s != last_seg) {
                last_seg = seg_s;
                if (*reinterpret_cast<volatile int *>(a.err) != 0) ok = 0;
            } else {
                ok = 2;
            }
            if (ok == 1 && sg.stage > 0) {
                const int *cnt = a.done + sg.pair * BT_MAXS + sg.stage - 1;
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
        __syncthreads();   // orders thread 0's acquire before every thread's reads
        if (!ok_s) break;
        const BPair &P = a.pairs[sg.pair];
        const BIO io = a.io[sg.pair];
        const BStage S = P.st[sg.stage];
        bool ok = true;
        if (S.type == BS_COPY) {
            // level-0 copy (K = 1): BT_BAND apron rows
            const BLevel &d = P.lv[0];
            const int quads = (d.W + 2 * APX + 3) / 4;
            const int y0 = tile * BT_BAND - APY;
            const int nrow = min(BT_BAND, d.H + APY - y0);
            for (int i = tid; i < 2 * nrow * quads; i += BT_THREADS) {
                const int img = i / (nrow * quads), j = i - img * nrow * quads;
                const int Y = y0 + j / quads, X0 = (j % quads) * 4 - APX;
                copy_quad(img ? io.R : io.L, io.pitch, d.W, d.H, img ? d.R : d.L, d.pitch, X0, Y);
            }
        } else {
            const BMaps *mp = a.maps + sg.pair * BT_MAXK;
            switch (P.nh) {
                case 1: ok = run_item<1, FULL>(a, P, mp, io, S, tile, smem, parity); break;
                case 2: ok = run_item<2, FULL>(a, P, mp, io, S, tile, smem, parity); break;
                case 3: ok = run_item<3, FULL>(a, P, mp, io, S, tile, smem, parity); break;
                default: ok = run_item<4, FULL>(a, P, mp, io, S, tile, smem, parity); break;
            }
        }
        (void)ok;   // a failed wait has set the error word; the loop head then stops
        __syncthreads();   // every thread's stores of this item are issued
        if (tid == 0) {
            __threadfence();
            if (!(a.withhold && sg.stage == 0)) atomicAdd(a.done + sg.pair * BT_MAXS + sg.stage, 1);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Grouped launches (MSBM_FLAG_BATCH_GROUPED).  The same per-pair stage tables, run as one
// ordinary launch per group of stages that share a tile function and its template
// parameters (kind, window, tile variant) and a place in the pass order (pyramid groups,
// coarsest search, statistics planes, then restricted level k from the coarsest down).  A
// group's CTAs cover the tiles of all its (pair, stage) segments; a CTA finds its segment
// by binary search over the segments' first blocks.  Stream order between the launches of
// the captured graph replaces the persistent kernel's completion counters, so there are
// no device waits besides each tile's own TMA wait, and each tile function keeps the
// register allocation of a kernel of its own.

struct BGSeg {
    int start;               // first block of the segment in its launch
    int pair, stage;
};

struct BGArgs {
    const BPair *pairs;
    const BMaps *maps;       // [pair * BT_MAXK + level]
    const BIO *io;
    const BGSeg *segs;       // this launch's segments
    int nseg;
    unsigned long long *evals;
    int *err;
    int force_timeout;
};

__device__ __forceinline__ int bg_find(const BGArgs &a, int b) {
    int lo = 0, hi = a.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].start <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int F>
__global__ void __launch_bounds__(BT_THREADS) bg_pyr_kernel(const __grid_constant__ BGArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BStage &S = P.st[sg.stage];
    const PyrFuseArgs &pf = P.pf[S.arg];
    const int tile = blockIdx.x - sg.start, per = S.ntiles / 2, img = tile / per, t = tile - img * per;
    const int by = t / S.tiles_x, bx = t - by * S.tiles_x;
    const uint8_t *src = S.arg == 0 ? (img ? io.R : io.L) : pf.src[img];
    const size_t spitch = S.arg == 0 ? io.pitch : pf.spitch;
    pyr_fused_tile<F, BT_THREADS>(pf, src, spitch, bx, by, img, S.tiles_x, P.pf_nby[S.arg], smem);
}

__global__ void __launch_bounds__(BT_THREADS) bg_copy_kernel(const __grid_constant__ BGArgs a) {
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BLevel &d = P.lv[0];
    const int tile = blockIdx.x - sg.start;
    const int quads = (d.W + 2 * APX + 3) / 4;
    const int y0 = tile * BT_BAND - APY;
    const int nrow = min(BT_BAND, d.H + APY - y0);
    for (int i = threadIdx.x; i < 2 * nrow * quads; i += BT_THREADS) {
        const int img = i / (nrow * quads), j = i - img * nrow * quads;
        const int Y = y0 + j / quads, X0 = (j % quads) * 4 - APX;
        copy_quad(img ? io.R : io.L, io.pitch, d.W, d.H, img ? d.R : d.L, d.pitch, X0, Y);
    }
}

template <int NH>
__global__ void __launch_bounds__(BT_THREADS) bg_stats_kernel(const __grid_constant__ BGArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const int tile = blockIdx.x - sg.start, K = P.K;
    int k = 0;
    while (k + 1 < K - 1 && tile >= P.sfirst[k + 1]) ++k;
    const int t = tile - P.sfirst[k], by = t / P.stx[k], bx = t - by * P.stx[k];
    const BLevel &l = P.lv[k];
    stats_tile<NH, BT_THREADS>(l.R, l.pitch, l.W, l.H, l.rstat, l.rspitch, bx, by, smem);
}

template <int NH>
__global__ void __launch_bounds__(BT_THREADS) bg_coarse_kernel(const __grid_constant__ BGArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BStage &S = P.st[sg.stage];
    const int k = S.arg, tile = blockIdx.x - sg.start;
    const BLevel &l = P.lv[k];
    const int by = tile / S.tiles_x, bx = tile - by * S.tiles_x;
    coarse_tile<NH, BT_CO_TY, BT_THREADS>(l.L, l.R, l.pitch, l.W, l.H, l.Dk, k == 0 ? io.d : l.d,
                                          k == 0 ? io.c : l.c, a.evals, bx, by, smem);
}

template <int NH, int SX>
__global__ void __launch_bounds__(BT_THREADS, 3) bg_full_kernel(const __grid_constant__ BGArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BStage &S = P.st[sg.stage];
    const int k = S.arg, tile = blockIdx.x - sg.start;
    const BLevel &l = P.lv[k];
    FullTileArgs t = {};
    t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.zblock = l.zblock;
    t.d_out = k == 0 ? io.d : l.d;
    t.c_out = k == 0 ? io.c : l.c;
    t.evals = a.evals; t.err = a.err; t.force_timeout = a.force_timeout;
    const BMaps &m = a.maps[sg.pair * BT_MAXK + k];
    uint32_t parity = 0;
    full_tile<NH, SX, BT_ZC>(t, &m.mFL, &m.mF256, tile % S.tiles_x, tile / S.tiles_x, smem, parity);
}

template <int NH, int G>
__global__ void __launch_bounds__(BT_THREADS, 8) bg_restr_kernel(const __grid_constant__ BGArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BStage &S = P.st[sg.stage];
    const int k = S.arg, tile = blockIdx.x - sg.start;
    const BLevel &l = P.lv[k];
    RestrTileArgs t = {};
    t.Limg = l.L; t.Rimg = l.R; t.pitch = l.pitch;
    t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.r = P.r;
    t.prior = P.lv[k + 1].d; t.Wp = P.lv[k + 1].W; t.Hp = P.lv[k + 1].H;
    t.d_out = k == 0 ? io.d : l.d;
    t.c_out = k == 0 ? io.c : l.c;
    t.evals = a.evals; t.err = a.err; t.force_timeout = a.force_timeout;
    const BMaps &m = a.maps[sg.pair * BT_MAXK + k];
    uint32_t parity = 0;
    restr_tile<NH, G, 32, BT_NCOL, true, BT_RTY>(t, &m.mRL, &m.mR128, &m.mR256, &m.mS128, &m.mS256,
                                                 tile % S.tiles_x, tile / S.tiles_x, smem, parity);
}

// Restricted level, grouped mode: the cell kernel over the segment's 32 x 8 pixel tiles
template <int NH, int G>
__global__ void __launch_bounds__((BT_RTX / 2) * (BT_RTY / 2), 8) bg_cell_kernel(const __grid_constant__ BGArgs a) {
    constexpr int CX = BT_RTX / 2, CY = BT_RTY / 2;   // cells of a tile
    __shared__ unsigned long long evsum;
    if (threadIdx.x == 0) evsum = 0ull;
    __syncthreads();
    const BGSeg sg = a.segs[bg_find(a, blockIdx.x)];
    const BPair &P = a.pairs[sg.pair];
    const BIO &io = a.io[sg.pair];
    const BStage &S = P.st[sg.stage];
    const int k = S.arg, tile = blockIdx.x - sg.start;
    const BLevel &l = P.lv[k];
    RestrTileArgs t = {};
    t.Limg = l.L; t.Rimg = l.R; t.pitch = l.pitch;
    t.W = l.W; t.H = l.H; t.Dk = l.Dk; t.r = P.r;
    t.prior = P.lv[k + 1].d; t.Wp = P.lv[k + 1].W; t.Hp = P.lv[k + 1].H;
    t.d_out = k == 0 ? io.d : l.d;
    t.c_out = k == 0 ? io.c : l.c;
    t.rstat = l.rstat; t.rspitch = l.rspitch;
    const int cx = (tile % S.tiles_x) * CX + static_cast<int>(threadIdx.x) % CX;
    const int cy = (tile / S.tiles_x) * CY + static_cast<int>(threadIdx.x) / CX;
    unsigned cnt = 0;
    if (2 * cx < t.W && 2 * cy < t.H) cnt = cell_search<NH, G>(t, cx, cy);
    const unsigned wc = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((threadIdx.x & 31) == 0 && wc) atomicAdd(&evsum, static_cast<unsigned long long>(wc));
    __syncthreads();
    if (threadIdx.x == 0 && a.evals && evsum) atomicAdd(a.evals, evsum);
}

size_t batch_smem_bytes(bool full) {
    size_t m = BT_AUX + (size_t)PF_SMEM;
    for (size_t b : {RCfg<1, 32, BT_NCOL, true, BT_RTY>::BYTES, RCfg<2, 32, BT_NCOL, true, BT_RTY>::BYTES,
                     RCfg<3, 32, BT_NCOL, true, BT_RTY>::BYTES, RCfg<BT_MAX_NH, 32, BT_NCOL, true, BT_RTY>::BYTES,
                     BT_AUX + StatsCfg<1>::BYTES, BT_AUX + StatsCfg<2>::BYTES, BT_AUX + StatsCfg<3>::BYTES,
                     BT_AUX + StatsCfg<BT_MAX_NH>::BYTES, BT_AUX + CoarseCfg<1, BT_CO_TY>::BYTES,
                     BT_AUX + CoarseCfg<2, BT_CO_TY>::BYTES, BT_AUX + CoarseCfg<3, BT_CO_TY>::BYTES,
                     BT_AUX + CoarseCfg<BT_MAX_NH, BT_CO_TY>::BYTES})
        m = std::max(m, b);
    if (full)
        for (size_t b : {FullCfg<1, 2, BT_ZC>::BYTES, FullCfg<2, 2, BT_ZC>::BYTES, FullCfg<3, 2, BT_ZC>::BYTES,
                         FullCfg<BT_MAX_NH, 2, BT_ZC>::BYTES, FullCfg<BT_MAX_NH, 1, BT_ZC>::BYTES})
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

// 2-D map over a plane of 8-byte entries: `rows` rows of `pitch` entries.
bool encode_b64(CUtensorMap *m, void *base, int pitch, int rows, int bw, int bh) {
    EncodeFn fn = encode_fn_b();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 8};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline msbm_status cst(cudaError_t e) {
    return e == cudaSuccess ? MSBM_OK : (e == cudaErrorMemoryAllocation ? MSBM_ERR_OOM : MSBM_ERR_CUDA);
}

}  // namespace
}  // namespace msbm

using namespace msbm;

namespace msbm {
namespace {

// One grouped launch: a tile function with its template parameters and its segments.
// Restricted launches of grouped mode run the cell kernel (zncc_cell_tile.cuh): var = G +
// BG_CELL, BG_CELL_THREADS threads per 32 x 8 pixel tile (16 x 4 prior cells).  Under
// MSBM_FLAG_TEST_TIMEOUT they keep the staged tile, whose bounded wait that flag exercises.
constexpr int BG_CELL = 100;
constexpr int BG_CELL_THREADS = (BT_RTX / 2) * (BT_RTY / 2);

struct BGLaunch {
    int type;                // BStageType
    int nh, var;             // window half-width; F (pyramid), sx (full), G (restricted)
    int order;               // place in the pass: pyramid groups, coarsest, statistics, levels
    int nblocks;
    int seg0, nseg;          // the launch's segments in the batch's segment array
    size_t smem;
};

size_t bg_smem(int type, int nh, int var) {
    auto pick = [](int h, size_t a1, size_t a2, size_t a3, size_t a4) {
        return h == 1 ? a1 : (h == 2 ? a2 : (h == 3 ? a3 : a4));
    };
    switch (type) {
        case BS_PYR: return PF_SMEM;
        case BS_STATS: return pick(nh, StatsCfg<1>::BYTES, StatsCfg<2>::BYTES, StatsCfg<3>::BYTES, StatsCfg<4>::BYTES);
        case BS_COARSE:
            return pick(nh, CoarseCfg<1, BT_CO_TY>::BYTES, CoarseCfg<2, BT_CO_TY>::BYTES, CoarseCfg<3, BT_CO_TY>::BYTES,
                        CoarseCfg<4, BT_CO_TY>::BYTES);
        case BS_FULL:
            return var == 1 ? pick(nh, FullCfg<1, 1, BT_ZC>::BYTES, FullCfg<2, 1, BT_ZC>::BYTES, FullCfg<3, 1, BT_ZC>::BYTES,
                                   FullCfg<4, 1, BT_ZC>::BYTES)
                            : pick(nh, FullCfg<1, 2, BT_ZC>::BYTES, FullCfg<2, 2, BT_ZC>::BYTES, FullCfg<3, 2, BT_ZC>::BYTES,
                                   FullCfg<4, 2, BT_ZC>::BYTES);
        case BS_RESTR:
            if (var >= BG_CELL) return 0;
            return pick(nh, RCfg<1, 32, BT_NCOL, true, BT_RTY>::BYTES, RCfg<2, 32, BT_NCOL, true, BT_RTY>::BYTES,
                        RCfg<3, 32, BT_NCOL, true, BT_RTY>::BYTES, RCfg<4, 32, BT_NCOL, true, BT_RTY>::BYTES);
        default: return 0;
    }
}

// The kernel of a grouped launch (host-side function pointer), or nullptr.
template <int NH>
const void *bg_kernel_nh(int type, int var) {
    switch (type) {
        case BS_STATS: return reinterpret_cast<const void *>(bg_stats_kernel<NH>);
        case BS_COARSE: return reinterpret_cast<const void *>(bg_coarse_kernel<NH>);
        case BS_FULL:
            return var == 1 ? reinterpret_cast<const void *>(bg_full_kernel<NH, 1>)
                            : reinterpret_cast<const void *>(bg_full_kernel<NH, 2>);
        case BS_RESTR:
            switch (var) {
                case BG_CELL + 1: return reinterpret_cast<const void *>(bg_cell_kernel<NH, 1>);
                case BG_CELL + 3: return reinterpret_cast<const void *>(bg_cell_kernel<NH, 3>);
                case BG_CELL + 5: return reinterpret_cast<const void *>(bg_cell_kernel<NH, 5>);
                case BG_CELL + 7: return reinterpret_cast<const void *>(bg_cell_kernel<NH, 7>);
                case 1: return reinterpret_cast<const void *>(bg_restr_kernel<NH, 1>);
                case 3: return reinterpret_cast<const void *>(bg_restr_kernel<NH, 3>);
                case 5: return reinterpret_cast<const void *>(bg_restr_kernel<NH, 5>);
                default: return reinterpret_cast<const void *>(bg_restr_kernel<NH, 7>);
            }
        default: return nullptr;
    }
}

const void *bg_kernel(int type, int nh, int var) {
    if (type == BS_COPY) return reinterpret_cast<const void *>(bg_copy_kernel);
    if (type == BS_PYR)
        return var == 1 ? reinterpret_cast<const void *>(bg_pyr_kernel<1>)
                        : (var == 2 ? reinterpret_cast<const void *>(bg_pyr_kernel<2>)
                                    : reinterpret_cast<const void *>(bg_pyr_kernel<3>));
    switch (nh) {
        case 1: return bg_kernel_nh<1>(type, var);
        case 2: return bg_kernel_nh<2>(type, var);
        case 3: return bg_kernel_nh<3>(type, var);
        default: return bg_kernel_nh<4>(type, var);
    }
}

}  // namespace
}  // namespace msbm

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
    bool full = false;           // some pair's coarsest level uses the full-range tile
    bool io_uploaded = false;
    cudaGraphExec_t exec = nullptr;
    // grouped launches (MSBM_FLAG_BATCH_GROUPED)
    bool grouped = false;
    std::vector<BGLaunch> launches;
    BGSeg *d_gsegs = nullptr;
    int force_timeout = 0;
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
        if (p.flags & ~(MSBM_FLAG_NO_GRAPH | MSBM_FLAG_TEST_TIMEOUT | MSBM_FLAG_BATCH_GROUPED))
            return MSBM_ERR_INVALID_ARG;
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
    b->grouped = (pairs[0].flags & MSBM_FLAG_BATCH_GROUPED) != 0;
    b->withhold = !b->grouped && (pairs[0].flags & MSBM_FLAG_TEST_TIMEOUT) != 0;
    b->force_timeout = b->grouped && (pairs[0].flags & MSBM_FLAG_TEST_TIMEOUT) != 0 ? 1 : 0;
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
        const int rowsF = 8 + 2 * P.nh, rowsR = BT_RTY + 2 * P.nh;
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
            l.rspitch = (W + 15) / 16 * 16;
            if (k < P.K - 1) dalloc(reinterpret_cast<void **>(&l.rstat), (size_t)l.rspitch * H * sizeof(int2));
            l.sx = full_sx ? full_sx[i] : (W >= 512 ? 2 : 1);
            l.zblock = full_zblock ? full_zblock[i] : 0;
            BMaps &m = maps[(size_t)i * BT_MAXK + k];
            enc_ok = enc_ok && encode_b(&m.mRL, buf, l.pitch, rows, BT_RTX + 32, rowsR) &&
                     encode_b(&m.mR128, buf + bytes, l.pitch, rows, 128, rowsR) &&
                     encode_b(&m.mR256, buf + bytes, l.pitch, rows, 256, rowsR) &&
                     encode_b(&m.mF256, buf + bytes, l.pitch, rows, 256, rowsF) &&
                     encode_b(&m.mFL, buf, l.pitch, rows, 32 * l.sx + 32, rowsF);
            if (l.rstat)
                enc_ok = enc_ok && encode_b64(&m.mS128, l.rstat, l.rspitch, H, 128, BT_RTY) &&
                         encode_b64(&m.mS256, l.rstat, l.rspitch, H, 256, BT_RTY);
            W = (W + 1) / 2;
            H = (H + 1) / 2;
        }
        if (e != cudaSuccess) break;
        // the pair's stage table
        auto add = [&](int type, int arg, int tx, int nt) {
            BStage &S = P.st[P.nst++];
            S.type = type; S.arg = arg; S.tiles_x = tx; S.ntiles = nt;
        };
        const int K = P.K;
        if (K == 1) {
            add(BS_COPY, 0, 1, (P.lv[0].H + 2 * APY + BT_BAND - 1) / BT_BAND);
        } else {
            for (int s0 = 0, g = 0; s0 < K - 1; s0 += PF_MAXF, ++g) {
                PyrFuseArgs &f = P.pf[g];
                f.F = std::min(PF_MAXF, K - 1 - s0);
                f.write_src = s0 == 0;
                f.src[0] = P.lv[s0].L;
                f.src[1] = P.lv[s0].R;
                f.spitch = (size_t)P.lv[s0].pitch;
                for (int j = 0; j <= f.F; ++j) {
                    const BLevel &l = P.lv[s0 + j];
                    f.W[j] = l.W; f.H[j] = l.H;
                    f.dst[j][0] = l.L; f.dst[j][1] = l.R;
                    f.dpitch[j] = l.pitch;
                }
                const int tx = (f.W[f.F] + PF_TX - 1) / PF_TX, ty = (f.H[f.F] + PF_TY - 1) / PF_TY;
                P.pf_nby[g] = ty;
                add(BS_PYR, g, tx, 2 * tx * ty);
            }
        }
        {
            const BLevel &l = P.lv[K - 1];
            if (l.Dk <= BT_COARSE_DK) {
                const int tx = (l.W + CO_TX - 1) / CO_TX;
                add(BS_COARSE, K - 1, tx, tx * ((l.H + BT_CO_TY - 1) / BT_CO_TY));
            } else {
                const int tx = (l.W + 32 * l.sx - 1) / (32 * l.sx);
                add(BS_FULL, K - 1, tx, tx * ((l.H + 7) / 8));
            }
        }
        if (K >= 2) {
            P.sfirst[0] = 0;
            for (int k = 0; k < K - 1; ++k) {
                P.stx[k] = (P.lv[k].W + ST_TX - 1) / ST_TX;
                P.sfirst[k + 1] = P.sfirst[k] + P.stx[k] * ((P.lv[k].H + ST_TY - 1) / ST_TY);
            }
            add(BS_STATS, 0, 1, P.sfirst[K - 1]);
        }
        for (int k = K - 2; k >= 0; --k) {
            const int tx = (P.lv[k].W + BT_RTX - 1) / BT_RTX;
            add(BS_RESTR, k, tx, tx * ((P.lv[k].H + BT_RTY - 1) / BT_RTY));
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
    for (auto &P : b->pairs) max_stages = std::max(max_stages, P.nst);
    long long pos = 0;
    for (int s = 0; s < max_stages; ++s) {
        std::vector<int> idx;
        for (int i = 0; i < n_pairs; ++i)
            if (s < b->pairs[i].nst) idx.push_back(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            return b->pairs[x].st[s].ntiles > b->pairs[y].st[s].ntiles;
        });
        for (int i : idx) {
            BSeg g;
            g.start = pos;
            g.pair = i;
            g.stage = s;
            g.ntiles = b->pairs[i].st[s].ntiles;
            g.need = s > 0 ? b->pairs[i].st[s - 1].ntiles : 0;
            pos += g.ntiles;
            segs.push_back(g);
        }
    }
    b->nseg = (int)segs.size();
    b->total = pos;
    // grouped launches: (order, type, window, variant) -> segments of that launch
    std::vector<BGSeg> gsegs;
    if (b->grouped) {
        struct Key {
            int order, type, nh, var;
            bool operator<(const Key &o) const {
                if (order != o.order) return order < o.order;
                if (type != o.type) return type < o.type;
                if (nh != o.nh) return nh < o.nh;
                return var < o.var;
            }
        };
        std::vector<std::pair<Key, std::pair<int, int>>> items;   // key -> (pair, stage)
        for (int i = 0; i < n_pairs; ++i) {
            const BPair &P = b->pairs[i];
            for (int st = 0; st < P.nst; ++st) {
                const BStage &S = P.st[st];
                Key k{0, S.type, 0, 0};
                switch (S.type) {
                    case BS_COPY: k.order = 0; break;
                    case BS_PYR: k.order = S.arg; k.var = P.pf[S.arg].F; break;
                    case BS_COARSE: k.order = 100; k.nh = P.nh; break;
                    case BS_FULL: k.order = 100; k.nh = P.nh; k.var = P.lv[S.arg].sx; break;
                    case BS_STATS: k.order = 200; k.nh = P.nh; break;
                    default:
                        k.order = 300 + (BT_MAXK - S.arg); k.nh = P.nh; k.var = std::min(2 * P.r + 1, 7);
                        if (!b->force_timeout) k.var += BG_CELL;   // the cell kernel (no device waits)
                        break;
                }
                items.push_back({k, {i, st}});
            }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const auto &x, const auto &y) { return x.first < y.first; });
        for (size_t a0 = 0; a0 < items.size();) {
            size_t a1 = a0;
            BGLaunch L;
            L.type = items[a0].first.type; L.nh = items[a0].first.nh; L.var = items[a0].first.var;
            L.order = items[a0].first.order;
            L.seg0 = (int)gsegs.size();
            int blocks = 0;
            while (a1 < items.size() && !(items[a0].first < items[a1].first) && !(items[a1].first < items[a0].first)) {
                BGSeg g;
                g.start = blocks;
                g.pair = items[a1].second.first;
                g.stage = items[a1].second.second;
                blocks += b->pairs[g.pair].st[g.stage].ntiles;
                gsegs.push_back(g);
                ++a1;
            }
            L.nseg = (int)gsegs.size() - L.seg0;
            L.nblocks = blocks;
            L.smem = bg_smem(L.type, L.nh, L.var);
            if (L.nblocks > 0) b->launches.push_back(L);
            a0 = a1;
        }
        for (const BGLaunch &L : b->launches) {
            if (e == cudaSuccess && L.smem > 48 * 1024)
                e = cudaFuncSetAttribute(bg_kernel(L.type, L.nh, L.var), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.smem);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(bg_kernel(L.type, L.nh, L.var), cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
        }
        if (!gsegs.empty()) dalloc(reinterpret_cast<void **>(&b->d_gsegs), sizeof(BGSeg) * gsegs.size());
        if (e == cudaSuccess && !gsegs.empty())
            e = cudaMemcpy(b->d_gsegs, gsegs.data(), sizeof(BGSeg) * gsegs.size(), cudaMemcpyHostToDevice);
    }
    dalloc(reinterpret_cast<void **>(&b->d_pairs), sizeof(BPair) * n_pairs);
    dalloc(reinterpret_cast<void **>(&b->d_maps), sizeof(BMaps) * maps.size());
    dalloc(reinterpret_cast<void **>(&b->d_io), sizeof(BIO) * n_pairs);
    dalloc(reinterpret_cast<void **>(&b->d_segs), sizeof(BSeg) * segs.size());
    dalloc(reinterpret_cast<void **>(&b->d_head), sizeof(int));
    dalloc(reinterpret_cast<void **>(&b->d_done), sizeof(int) * n_pairs * BT_MAXS);
    dalloc(reinterpret_cast<void **>(&b->d_err), sizeof(int));
    dalloc(reinterpret_cast<void **>(&b->d_evals), sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pairs, b->pairs.data(), sizeof(BPair) * n_pairs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_maps, maps.data(), sizeof(BMaps) * maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_segs, segs.data(), sizeof(BSeg) * segs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_evals, 0, sizeof(unsigned long long));
    b->full = false;
    for (auto &P : b->pairs)
        for (int s = 0; s < P.nst; ++s) b->full = b->full || P.st[s].type == BS_FULL;
    b->smem = batch_smem_bytes(b->full);
    const void *kern = b->full ? reinterpret_cast<const void *>(batch_kernel<true>)
                               : reinterpret_cast<const void *>(batch_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BT_THREADS, b->smem);
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

static msbm_status batch_enqueue_grouped(msbm_batch *b, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (const BGLaunch &L : b->launches) {
        BGArgs a;
        memset(&a, 0, sizeof(a));
        a.pairs = b->d_pairs; a.maps = b->d_maps; a.io = b->d_io;
        a.segs = b->d_gsegs + L.seg0; a.nseg = L.nseg;
        a.evals = b->d_evals; a.err = b->d_err; a.force_timeout = b->force_timeout;
        void *args[] = {&a};
        const int threads = (L.type == BS_RESTR && L.var >= BG_CELL) ? BG_CELL_THREADS : BT_THREADS;
        e = cudaLaunchKernel(bg_kernel(L.type, L.nh, L.var), dim3(L.nblocks), dim3(threads), args, L.smem, st);
        if (e != cudaSuccess) break;
    }
    return cst(e);
}

static msbm_status batch_enqueue(msbm_batch *b, cudaStream_t st) {
    if (b->grouped) return batch_enqueue_grouped(b, st);
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.pairs = b->d_pairs; a.maps = b->d_maps; a.io = b->d_io; a.segs = b->d_segs;
    a.nseg = b->nseg; a.total = b->total; a.head = b->d_head; a.done = b->d_done;
    a.evals = b->d_evals; a.err = b->d_err;
    a.withhold = b->withhold ? 1 : 0;
    a.wait_limit = b->withhold ? BT_TEST_WAIT_LIMIT : BT_WAIT_LIMIT;
    cudaError_t e = cudaMemsetAsync(b->d_head, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * b->n * BT_MAXS, st);
    if (e == cudaSuccess) {
        if (b->full)
            batch_kernel<true><<<b->grid, BT_THREADS, b->smem, st>>>(a);
        else
            batch_kernel<false><<<b->grid, BT_THREADS, b->smem, st>>>(a);
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
    int err = 0;
    if (cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return MSBM_ERR_CUDA;
    if (err) {
        // cleared in the batch stream's order (see msbm_sync)
        if (cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream) != cudaSuccess) return MSBM_ERR_CUDA;
        return static_cast<msbm_status>(err);
    }
    return MSBM_OK;
}

msbm_status msbm_batch_eval_count(msbm_batch *b, int64_t *count, int32_t reset) {
    if (!b || !count) return MSBM_ERR_INVALID_ARG;
    unsigned long long v = 0;
    if (cudaMemcpyAsync(&v, b->d_evals, sizeof(v), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return MSBM_ERR_CUDA;
    *count = static_cast<int64_t>(v);
    if (reset && cudaMemsetAsync(b->d_evals, 0, sizeof(v), b->stream) != cudaSuccess) return MSBM_ERR_CUDA;
    return MSBM_OK;
}

msbm_status msbm_batch_level_result(msbm_batch *b, int32_t pair, int32_t level, int16_t *d_out,
                                    float *cost_out) {
    if (!b || pair < 0 || pair >= b->n || !d_out) return MSBM_ERR_INVALID_ARG;
    const BPair &P = b->pairs[pair];
    if (level < 1 || level >= P.K) return MSBM_ERR_INVALID_ARG;
    const BLevel &l = P.lv[level];
    const size_t n = (size_t)l.W * l.H;
    cudaError_t e = cudaMemcpyAsync(d_out, l.d, n * sizeof(int16_t), cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess && cost_out)
        e = cudaMemcpyAsync(cost_out, l.c, n * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
    return cst(e);
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
