// msbm_api.cu -- the C ABI declared in include/msbm.h: argument validation, the context
// (pyramid apron buffers, per-level maps, TMA descriptors, error and evaluation counters),
// launch orchestration of the hierarchical pass (Sec. III, Fig. 1) and its CUDA-graph
// replay.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>
#include <stdio.h>

#include "msbm.h"
#include "msbm_internal.h"

using namespace msbm;

namespace {
// NVTX range for profilers (nsys, ncu's range filters): one per pass, level and host frame.
// Header-only NVTX v3: without a profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    NvtxRange(const char *what, int k) {
        char buf[48];
        snprintf(buf, sizeof(buf), "%s %d", what, k);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Pass pipelines (and staging sets) of msbm_disparity_host_frames.  The hierarchical pass is
// a chain of small, latency-bound launches, so passes of consecutive frames on several
// pipelines overlap: 1400 x 1000 pair, 128 frames from page-locked buffers, disparity maps
// back: 20 900 frames/s with two pipelines, 24 990 with three, 27 970 with four, 29 120 with
// six, 28 720 with eight (with the cost maps too, about 17 200 for all: the host link).
constexpr int HOST_PIPES = 6;

struct msbm_ctx {
    msbm_params p{};
    int nh = 0;
    int device = 0;
    int num_sms = 0;
    // matching kernels of the level chain launch as programmatic dependents of their stream
    // predecessor, so that each is scheduled while the previous level drains
    bool pdl = true;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // second stream of the pass: the statistics planes, beside the coarsest level's search
    // and the coarser restricted levels; ev_stat[k]: level k's plane is written
    cudaStream_t side_stream = nullptr;
    // third stream of the pass: level 0's planes (the largest), from the fork on
    cudaStream_t side_stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_stat[12] = {};
    std::vector<LevelBuf> lv;
    int *d_err = nullptr;
    unsigned long long *d_evals = nullptr;
    // graph replay of msbm_disparity: one instantiated pass graph per set of caller
    // pointers, for the two most recent sets (the pipelined host path alternates two
    // staging sets)
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const void *key[4] = {nullptr, nullptr, nullptr, nullptr};
        size_t pitch = 0;
        unsigned long long used = 0;
    };
    GraphSlot graphs[2];
    unsigned long long graph_clock = 0;
    int graph_kernels = 0;       // kernel nodes of the captured pass graph
    int *h_err = nullptr;        // page-locked copy of d_err read by msbm_sync
    // level-0 cost when the caller passes none but a gated step needs one
    float *c0 = nullptr;
    // pipelined host path (msbm_disparity_host_frames): two device staging sets, an upload
    // and a download stream, and per set the events that order its reuse
    uint8_t *sL[HOST_PIPES] = {}, *sR[HOST_PIPES] = {};
    int16_t *sd[HOST_PIPES] = {};
    float *sc[HOST_PIPES] = {};
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    // second pass pipeline of the host frames path: a context of the same parameters (its own
    // level buffers) on its own stream, taking every other frame, so that one frame's coarse,
    // latency-bound levels run beside the previous frame's finest level
    // further pass pipelines of msbm_disparity_host_frames (contexts with the same
    // parameters on their own streams); pipeline 0 is this context
    msbm_ctx *twin[HOST_PIPES] = {};
    cudaStream_t twin_stream[HOST_PIPES] = {};
    cudaEvent_t ev_up[HOST_PIPES] = {}, ev_pass[HOST_PIPES] = {}, ev_down[HOST_PIPES] = {};
};

namespace {

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool encode_u8(CUtensorMap *m, uint8_t *base, int pitch, int rows, int box_w, int box_h) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D map over a plane of 8-byte entries: `rows` rows of `pitch` entries.
bool encode_u64(CUtensorMap *m, void *base, int pitch, int rows, int box_w, int box_h) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 8};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

msbm_status validate(const msbm_params *p) {
    if (!p) return MSBM_ERR_INVALID_ARG;
    if (p->width < 1 || p->width > 16384 || p->height < 1 || p->height > 16384)
        return MSBM_ERR_INVALID_ARG;
    if (p->max_disp < 1 || p->max_disp > 4096) return MSBM_ERR_INVALID_ARG;
    if (p->levels < 1 || p->levels > 12) return MSBM_ERR_INVALID_ARG;
    if (p->window < 3 || p->window > 13 || (p->window & 1) == 0) return MSBM_ERR_INVALID_ARG;
    if (p->radius < 0 || p->radius > 16) return MSBM_ERR_INVALID_ARG;
    if (p->flags & ~(MSBM_FLAG_NO_GRAPH | MSBM_FLAG_TEST_TIMEOUT | MSBM_FLAGS_FULL_METHOD | MSBM_FLAG_WINDOW_HALVING))
        return MSBM_ERR_INVALID_ARG;
    if ((p->flags & (MSBM_FLAG_ALPHA_REFINE | MSBM_FLAG_SELECTIVE_MEDIAN)) && !(p->alpha > -2.f && p->alpha < 2.f))
        return MSBM_ERR_INVALID_ARG;
    if ((p->flags & MSBM_FLAG_BETA_FALLBACK) && !(p->beta > -2.f && p->beta < 2.f)) return MSBM_ERR_INVALID_ARG;
    return MSBM_OK;
}

int choose_sx(int W, int H, int sms) {
    for (int sx = 4; sx > 1; sx /= 2) {
        long ctas = (long)((W + 32 * sx - 1) / (32 * sx)) * ((H + 7) / 8);
        if (ctas >= 2L * sms) return sx;
    }
    return 1;
}

void free_ctx(msbm_ctx *c) {
    if (!c) return;
    for (int q = 1; q < HOST_PIPES; ++q) {
        if (c->twin[q]) {
            cudaStreamSynchronize(c->twin_stream[q]);
            free_ctx(c->twin[q]);
        }
        if (c->twin_stream[q]) cudaStreamDestroy(c->twin_stream[q]);
    }
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto &l : c->lv) {
        cudaFree(l.base[0]);
        cudaFree(l.d);
        cudaFree(l.c);
        cudaFree(l.dtmp);
        cudaFree(l.mask);
        cudaFree(l.cells);
        cudaFree(l.rstat);
    }
    cudaFree(c->c0);
    cudaFree(c->d_err);
    cudaFreeHost(c->h_err);
    cudaFree(c->d_evals);
    for (int b = 0; b < HOST_PIPES; ++b) {
        cudaFree(c->sL[b]);
        cudaFree(c->sR[b]);
        cudaFree(c->sd[b]);
        cudaFree(c->sc[b]);
        if (c->ev_up[b]) cudaEventDestroy(c->ev_up[b]);
        if (c->ev_pass[b]) cudaEventDestroy(c->ev_pass[b]);
        if (c->ev_down[b]) cudaEventDestroy(c->ev_down[b]);
    }
    if (c->up_stream) cudaStreamDestroy(c->up_stream);
    if (c->down_stream) cudaStreamDestroy(c->down_stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    if (c->side_stream2) cudaStreamDestroy(c->side_stream2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    for (cudaEvent_t ev : c->ev_stat)
        if (ev) cudaEventDestroy(ev);
    delete c;
}

inline msbm_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MSBM_OK;
    if (e == cudaErrorMemoryAllocation) return MSBM_ERR_OOM;
    return MSBM_ERR_CUDA;
}

// The pyramid: a plain copy for one level, else fused launches of up to PF_MAXF reductions
// each (the first also writing level 0).
msbm_status enqueue_pyramid(msbm_ctx *c, const uint8_t *L, const uint8_t *R, size_t pitch,
                            cudaStream_t st) {
    const int K = c->p.levels;
    if (K == 1) return cuda_status(launch_apron_copy(L, R, pitch, c->lv[0], st));
    cudaError_t e = cudaSuccess;
    for (int s = 0; e == cudaSuccess && s < K - 1; s += PF_MAXF) {
        PyrFuseArgs a;
        memset(&a, 0, sizeof(a));
        a.F = std::min(PF_MAXF, K - 1 - s);
        a.write_src = s == 0;
        a.src[0] = s == 0 ? L : c->lv[s].img(0);
        a.src[1] = s == 0 ? R : c->lv[s].img(1);
        a.spitch = s == 0 ? pitch : (size_t)c->lv[s].pitch;
        for (int j = 0; j <= a.F; ++j) {
            const LevelBuf &l = c->lv[s + j];
            a.W[j] = l.W;
            a.H[j] = l.H;
            a.dst[j][0] = l.img(0);
            a.dst[j][1] = l.img(1);
            a.dpitch[j] = l.pitch;
        }
        e = launch_pyr_fused(a, st);
    }
    return cuda_status(e);
}

// Statistics planes of levels 0 .. n-1: one launch per run of levels with the same window.
cudaError_t launch_stats_levels(msbm_ctx *c, int n, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int k0 = 0; e == cudaSuccess && k0 < n;) {
        int k1 = k0 + 1;
        while (k1 < n && c->lv[k1].nh == c->lv[k0].nh) ++k1;
        e = launch_level_stats(c->lv.data() + k0, k1 - k0, c->lv[k0].nh, st);
        k0 = k1;
    }
    return e;
}

// stats_ready: the level's right-window statistics plane is already computed in stream order.
msbm_status enqueue_level(msbm_ctx *c, int k, const int16_t *prior, int16_t *d, float *cost,
                          cudaStream_t st, const uint8_t *skip = nullptr, bool stats_ready = false) {
    const LevelBuf &l = c->lv[k];
    const int force = (c->p.flags & MSBM_FLAG_TEST_TIMEOUT) ? 1 : 0;
    cudaError_t e;
    if (!prior && l.coarse) {
        e = launch_zncc_coarse(l, l.nh, d, cost, c->d_evals, st, c->pdl);
    } else if (!prior) {
        FullArgs a;
        memset(&a, 0, sizeof(a));
        a.tmL = l.tmFL;
        a.tmR = l.tmR256;
        a.t.W = l.W; a.t.H = l.H; a.t.Dk = l.Dk; a.t.zblock = l.full_zblock;
        a.t.d_out = d; a.t.c_out = cost;
        a.t.evals = c->d_evals; a.t.err = c->d_err; a.t.force_timeout = force;
        e = launch_zncc_full(a, l.nh, l.full_sx, st, c->pdl);
    } else {
        RestrArgs a;
        memset(&a, 0, sizeof(a));
        a.tmL = l.tmRL;
        a.tmR128 = l.tmRR128;
        a.tmR256 = l.tmRR256;
        a.tmS = l.tmS128;
        a.tmS256 = l.tmS256;
        a.t.skip = skip;
        a.t.Limg = l.img(0); a.t.Rimg = l.img(1); a.t.pitch = l.pitch;
        a.t.W = l.W; a.t.H = l.H; a.t.Dk = l.Dk; a.t.r = c->p.radius;
        a.t.prior = prior; a.t.Wp = (l.W + 1) / 2; a.t.Hp = (l.H + 1) / 2;
        a.t.d_out = d; a.t.c_out = cost;
        a.t.evals = c->d_evals; a.t.err = c->d_err; a.t.force_timeout = force;
        a.t.rstat = l.rstat; a.t.rspitch = l.rspitch;
        e = stats_ready ? cudaSuccess : launch_level_stats(&l, 1, l.nh, st);
        if (e == cudaSuccess) e = launch_zncc_restricted(a, l.nh, st, c->pdl);
    }
    return cuda_status(e);
}

// Eq. 8-9 with both branches at level k: gate from the coarser cost, restricted search for
// every pixel (fallback pixels are not counted), then the full search of the fallback
// pixels only (zncc_sparse.cu), overwriting them.
msbm_status enqueue_level_beta(msbm_ctx *c, int k, const int16_t *prior, const float *cprior, int16_t *d,
                               float *cost, cudaStream_t st, bool stats_ready = false) {
    LevelBuf &l = c->lv[k];
    const LevelBuf &lp = c->lv[k + 1];
    cudaError_t e = launch_beta_gate(cprior, lp.W, lp.H, l.W, l.H, c->p.beta, l.mask, l.cells, st);
    if (e != cudaSuccess) return cuda_status(e);
    msbm_status s = enqueue_level(c, k, prior, d, cost, st, l.mask, stats_ready);
    if (s != MSBM_OK) return s;
    // the restricted search above left the level's statistics plane in stream order
    return cuda_status(launch_zncc_sparse(l, l.nh, d, cost, c->d_evals, st));
}

// Level k of the pass with the gated steps the context's flags select: the full-range
// search (+ alpha refinement) at the coarsest level, the restricted search (+ beta fallback,
// + selective median) below it.  Writes the level's final map to d / cost at level 0.
// stats_ready: the restricted levels' statistics planes are already computed in stream order.
msbm_status enqueue_match(msbm_ctx *c, int k, int16_t *d, float *cost, cudaStream_t st,
                          bool stats_ready = false) {
    const int K = c->p.levels;
    const uint32_t f = c->p.flags;
    LevelBuf &l = c->lv[k];
    int16_t *dk = k == 0 ? d : l.d;                        // final map of this level
    float *ck = k == 0 ? (cost ? cost : c->c0) : l.c;      // its cost
    msbm_status s;
    if (k == K - 1) {
        s = enqueue_level(c, k, nullptr, dk, ck, st);
        if (s == MSBM_OK && (f & MSBM_FLAG_ALPHA_REFINE))
            s = cuda_status(launch_alpha_refine(l, l.nh, c->p.alpha, dk, ck, c->d_evals, st));
        return s;
    }
    const int16_t *prior = c->lv[k + 1].d;
    const bool med = (f & MSBM_FLAG_SELECTIVE_MEDIAN) != 0;
    int16_t *dm = med ? l.dtmp : dk;                      // matching output
    if (f & MSBM_FLAG_BETA_FALLBACK)
        s = enqueue_level_beta(c, k, prior, c->lv[k + 1].c, dm, ck, st, stats_ready);
    else
        s = enqueue_level(c, k, prior, dm, ck, st, nullptr, stats_ready);
    if (s == MSBM_OK && med) s = cuda_status(launch_selective_median(dm, ck, l.W, l.H, c->p.alpha, dk, st));
    return s;
}

msbm_status enqueue_all(msbm_ctx *c, const uint8_t *L, const uint8_t *R, size_t pitch, int16_t *d,
                        float *cost, cudaStream_t st) {
    msbm_status s = enqueue_pyramid(c, L, R, pitch, st);
    const int K = c->p.levels;
    // fork: the statistics planes of levels K-2 .. 1, coarsest first, on one side stream
    // and level 0's on another, beside the coarsest level's full-range search and the
    // coarser restricted levels; each restricted level joins on its own plane only
    if (s == MSBM_OK && K >= 2) {
        cudaError_t e = cudaEventRecord(c->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side_stream, c->ev_fork, 0);
        if (e == cudaSuccess && K >= 3) e = cudaStreamWaitEvent(c->side_stream2, c->ev_fork, 0);
        for (int k = K - 2; e == cudaSuccess && k >= 0; --k) {
            cudaStream_t ss = (k == 0 && K >= 3) ? c->side_stream2 : c->side_stream;
            e = launch_level_stats(&c->lv[k], 1, c->lv[k].nh, ss);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_stat[k], ss);
        }
        s = cuda_status(e);
    }
    for (int k = K - 1; s == MSBM_OK && k >= 0; --k) {
        NvtxRange range("msbm level", k);
        if (k <= K - 2) s = cuda_status(cudaStreamWaitEvent(st, c->ev_stat[k], 0));
        if (s == MSBM_OK) s = enqueue_match(c, k, d, cost, st, true);
    }
    return s;
}

}  // namespace

extern "C" {

int msbm_version(void) { return 10000; }

const char *msbm_status_string(msbm_status s) {
    switch (s) {
        case MSBM_OK: return "ok";
        case MSBM_ERR_INVALID_ARG: return "invalid argument";
        case MSBM_ERR_ALIGNMENT: return "misaligned buffer";
        case MSBM_ERR_OOM: return "out of memory";
        case MSBM_ERR_CUDA: return "CUDA error";
        case MSBM_ERR_TIMEOUT: return "device wait timed out";
        case MSBM_ERR_UNSUPPORTED: return "unsupported device or size";
    }
    return "unknown status";
}

msbm_status msbm_create(const msbm_params *params, void *cuda_stream, msbm_ctx **out) {
    if (!out) return MSBM_ERR_INVALID_ARG;
    *out = nullptr;
    msbm_status s = validate(params);
    if (s != MSBM_OK) return s;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return MSBM_ERR_UNSUPPORTED;
    if (!(prop.major == 10 && prop.minor == 3)) return MSBM_ERR_UNSUPPORTED;
    if (!encode_fn()) return MSBM_ERR_UNSUPPORTED;

    msbm_ctx *c = new (std::nothrow) msbm_ctx();
    if (!c) return MSBM_ERR_OOM;
    c->p = *params;
    c->nh = params->window / 2;
    c->device = dev;
    c->num_sms = prop.multiProcessorCount;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side_stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int k = 0; e == cudaSuccess && k < params->levels; ++k)
        e = cudaEventCreateWithFlags(&c->ev_stat[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_evals, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_evals, 0, sizeof(unsigned long long));
    int W = params->width, H = params->height;
    for (int k = 0; e == cudaSuccess && k < params->levels; ++k) {
        LevelBuf l;
        l.W = W; l.H = H;
        l.Dk = (int)(((long)params->max_disp + (1L << k) - 1) >> k);
        l.nh = (params->flags & MSBM_FLAG_WINDOW_HALVING) ? std::max(1, c->nh >> k) : c->nh;
        const int rowsT = 8 + 2 * l.nh;    // staged rows of the full-range tile
        l.pitch = (W + 2 * APX + 127) / 128 * 128;
        l.rows = H + 2 * APY;
        size_t bytes = (size_t)l.pitch * l.rows;
        uint8_t *buf = nullptr;
        e = cudaMalloc(&buf, 2 * bytes);
        if (e != cudaSuccess) break;
        l.base[0] = buf;
        l.base[1] = buf + bytes;
        e = cudaMemset(buf, 0, 2 * bytes);
        if (e == cudaSuccess && k > 0) e = cudaMalloc(&l.d, (size_t)W * H * sizeof(int16_t));
        if (e == cudaSuccess && k > 0) e = cudaMalloc(&l.c, (size_t)W * H * sizeof(float));
        l.rspitch = (W + 15) / 16 * 16;
        if (e == cudaSuccess) e = cudaMalloc(&l.rstat, (size_t)l.rspitch * H * sizeof(int2));
        const bool finer = k < params->levels - 1;
        if (e == cudaSuccess && finer && (params->flags & MSBM_FLAG_SELECTIVE_MEDIAN))
            e = cudaMalloc(&l.dtmp, (size_t)W * H * sizeof(int16_t));
        if (e == cudaSuccess && finer && (params->flags & MSBM_FLAG_BETA_FALLBACK))
            e = cudaMalloc(&l.mask, (size_t)W * H);
        if (e == cudaSuccess && finer && (params->flags & MSBM_FLAG_BETA_FALLBACK))
            e = cudaMalloc(&l.cells, (2 + (size_t)((W + 1) / 2) * ((H + 1) / 2)) * sizeof(unsigned));
        l.full_sx = choose_sx(W, H, c->num_sms);
        l.coarse = zncc_coarse_fits(W, H, c->num_sms);
        if (e == cudaSuccess) {
            const int rowsR = l.rty + 2 * l.nh;
            bool ok = encode_u8(&l.tmFL, l.base[0], l.pitch, l.rows, 32 * l.full_sx + 32, rowsT) &&
                      encode_u8(&l.tmR256, l.base[1], l.pitch, l.rows, 256, rowsT) &&
                      encode_u8(&l.tmRL, l.base[0], l.pitch, l.rows, 64, rowsR) &&
                      encode_u8(&l.tmRR128, l.base[1], l.pitch, l.rows, 128, rowsR) &&
                      encode_u8(&l.tmRR256, l.base[1], l.pitch, l.rows, 256, rowsR) &&
                      encode_u64(&l.tmS128, l.rstat, l.rspitch, H, 128, l.rty) &&
                      encode_u64(&l.tmS256, l.rstat, l.rspitch, H, 256, l.rty);
            if (!ok) { c->lv.push_back(l); free_ctx(c); return MSBM_ERR_UNSUPPORTED; }
        }
        if (e == cudaSuccess) e = zncc_full_prepare(l.nh, l.full_sx);
        if (e == cudaSuccess) e = zncc_restricted_prepare(l.nh);
        c->lv.push_back(l);
        W = (W + 1) / 2;
        H = (H + 1) / 2;
    }
    if (e == cudaSuccess && (params->flags & MSBM_FLAGS_FULL_METHOD))
        e = cudaMalloc(&c->c0, (size_t)params->width * params->height * sizeof(float));
    if (e != cudaSuccess) {
        msbm_status st = cuda_status(e);
        free_ctx(c);
        return st;
    }
    *out = c;
    return MSBM_OK;
}

msbm_status msbm_destroy(msbm_ctx *ctx) {
    if (!ctx) return MSBM_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return MSBM_OK;
}

msbm_status msbm_set_stream(msbm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return MSBM_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return MSBM_OK;
}

msbm_status msbm_level_shape(const msbm_ctx *ctx, int32_t level, int32_t *w, int32_t *h,
                             int32_t *d_k) {
    if (!ctx || level < 0 || level >= ctx->p.levels) return MSBM_ERR_INVALID_ARG;
    const LevelBuf &l = ctx->lv[level];
    if (w) *w = l.W;
    if (h) *h = l.H;
    if (d_k) *d_k = l.Dk;
    return MSBM_OK;
}

msbm_status msbm_set_level_tuning(msbm_ctx *ctx, int32_t level, int32_t sx, int32_t zblock) {
    if (!ctx || level < 0 || level >= ctx->p.levels) return MSBM_ERR_INVALID_ARG;
    if ((sx != 1 && sx != 2 && sx != 4) || zblock < 0 || zblock % 32 != 0) return MSBM_ERR_INVALID_ARG;
    LevelBuf &l = ctx->lv[level];
    const int rowsT = 8 + 2 * l.nh;
    if (!encode_u8(&l.tmFL, l.base[0], l.pitch, l.rows, 32 * sx + 32, rowsT)) return MSBM_ERR_UNSUPPORTED;
    cudaError_t e = zncc_full_prepare(l.nh, sx);
    if (e != cudaSuccess) return cuda_status(e);
    l.full_sx = sx;
    l.full_zblock = zblock;
    l.coarse = false;            // explicit tuning selects the full-range tile kernel
    for (auto &g : ctx->graphs) {   // the captured graphs hold the old launch configuration
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = msbm_ctx::GraphSlot();
    }
    return MSBM_OK;
}

msbm_status msbm_pyramid(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                         size_t pitch_bytes) {
    if (!ctx || !d_left || !d_right || pitch_bytes < (size_t)ctx->p.width) return MSBM_ERR_INVALID_ARG;
    return enqueue_pyramid(ctx, d_left, d_right, pitch_bytes, ctx->stream);
}

msbm_status msbm_level_image(msbm_ctx *ctx, int32_t level, int32_t which, uint8_t *d_out) {
    if (!ctx || level < 0 || level >= ctx->p.levels || (which != 0 && which != 1) || !d_out)
        return MSBM_ERR_INVALID_ARG;
    return cuda_status(launch_level_extract(ctx->lv[level], which, d_out, ctx->stream));
}

msbm_status msbm_match_level(msbm_ctx *ctx, int32_t level, const int16_t *d_prior, int16_t *d_out,
                             float *cost_out) {
    if (!ctx || level < 0 || level >= ctx->p.levels || !d_out) return MSBM_ERR_INVALID_ARG;
    return enqueue_level(ctx, level, d_prior, d_out, cost_out, ctx->stream);
}

msbm_status msbm_alpha_refine(msbm_ctx *ctx, int32_t level, int16_t *d, float *cost) {
    if (!ctx || level < 0 || level >= ctx->p.levels || !d || !cost) return MSBM_ERR_INVALID_ARG;
    return cuda_status(launch_alpha_refine(ctx->lv[level], ctx->lv[level].nh, ctx->p.alpha, d, cost, ctx->d_evals, ctx->stream));
}

msbm_status msbm_selective_median(msbm_ctx *ctx, int32_t level, const int16_t *d_in, const float *cost,
                                  int16_t *d_out) {
    if (!ctx || level < 0 || level >= ctx->p.levels || !d_in || !cost || !d_out || d_in == d_out)
        return MSBM_ERR_INVALID_ARG;
    const LevelBuf &l = ctx->lv[level];
    return cuda_status(launch_selective_median(d_in, cost, l.W, l.H, ctx->p.alpha, d_out, ctx->stream));
}

msbm_status msbm_match_level_beta(msbm_ctx *ctx, int32_t level, const int16_t *d_prior, const float *cost_prior,
                                  int16_t *d_out, float *cost_out, uint8_t *fallback_out) {
    if (!ctx || level < 0 || level >= ctx->p.levels - 1 || !d_prior || !cost_prior || !d_out || !cost_out)
        return MSBM_ERR_INVALID_ARG;
    if (!(ctx->p.flags & MSBM_FLAG_BETA_FALLBACK)) return MSBM_ERR_INVALID_ARG;   // buffers not allocated
    msbm_status s = enqueue_level_beta(ctx, level, d_prior, cost_prior, d_out, cost_out, ctx->stream);
    if (s == MSBM_OK && fallback_out) {
        const LevelBuf &l = ctx->lv[level];
        s = cuda_status(cudaMemcpyAsync(fallback_out, l.mask, (size_t)l.W * l.H, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return s;
}

msbm_status msbm_disparity(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                           size_t pitch_bytes, int16_t *d_out, float *cost_out) {
    if (!ctx || !d_left || !d_right || !d_out || pitch_bytes < (size_t)ctx->p.width)
        return MSBM_ERR_INVALID_ARG;
    NvtxRange range("msbm_disparity");
    if (ctx->p.flags & MSBM_FLAG_NO_GRAPH)
        return enqueue_all(ctx, d_left, d_right, pitch_bytes, d_out, cost_out, ctx->stream);
    const void *key[4] = {d_left, d_right, d_out, cost_out};
    msbm_ctx::GraphSlot *slot = nullptr;
    for (auto &g : ctx->graphs)
        if (g.exec && g.pitch == pitch_bytes && memcmp(key, g.key, sizeof(key)) == 0) slot = &g;
    if (!slot) {
        // capture the pass for these pointers into the least recently used slot (updating
        // its executable graph in place when the topology allows)
        slot = &ctx->graphs[0];
        for (auto &g : ctx->graphs)
            if (g.used < slot->used) slot = &g;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return MSBM_ERR_CUDA;
        msbm_status s = enqueue_all(ctx, d_left, d_right, pitch_bytes, d_out, cost_out, ctx->cap_stream);
        e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (s != MSBM_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return s != MSBM_OK ? s : MSBM_ERR_CUDA;
        }
        if (slot->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(slot->exec, g, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(slot->exec);
                slot->exec = nullptr;
            }
        }
        if (!slot->exec) e = cudaGraphInstantiate(&slot->exec, g, 0);
        ctx->graph_kernels = count_kernel_nodes(g);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            slot->exec = nullptr;
            return cuda_status(e);
        }
        memcpy(slot->key, key, sizeof(key));
        slot->pitch = pitch_bytes;
    }
    slot->used = ++ctx->graph_clock;
    return cuda_status(cudaGraphLaunch(slot->exec, ctx->stream));
}

msbm_status msbm_disparity_host_frames(msbm_ctx *ctx, int32_t n_frames, const uint8_t *const *h_lefts,
                                       const uint8_t *const *h_rights, size_t pitch_bytes, int16_t *const *h_ds,
                                       float *const *h_costs) {
    if (!ctx || n_frames < 1 || !h_lefts || !h_rights || !h_ds || pitch_bytes < (size_t)ctx->p.width)
        return MSBM_ERR_INVALID_ARG;
    for (int i = 0; i < n_frames; ++i)
        if (!h_lefts[i] || !h_rights[i] || !h_ds[i]) return MSBM_ERR_INVALID_ARG;
    const size_t W = ctx->p.width, H = ctx->p.height;
    cudaError_t e = cudaSuccess;
    if (!ctx->up_stream) {
        // staging images are dense (pitch W); images at another pitch are copied row by row
        for (int b = 0; e == cudaSuccess && b < HOST_PIPES; ++b) {
            e = cudaMalloc(&ctx->sL[b], W * H);
            if (e == cudaSuccess) e = cudaMalloc(&ctx->sR[b], W * H);
            if (e == cudaSuccess) e = cudaMalloc(&ctx->sd[b], W * H * sizeof(int16_t));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->sc[b], W * H * sizeof(float));
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_up[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_pass[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_down[b], cudaEventDisableTiming);
        }
        cudaStream_t up = nullptr, down = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (up) cudaStreamDestroy(up);
            if (down) cudaStreamDestroy(down);
            return cuda_status(e);
        }
        ctx->up_stream = up;
        ctx->down_stream = down;
    }
    const int np = std::min(n_frames, HOST_PIPES);     // pass pipelines this call uses
    for (int q = 1; q < np; ++q) {
        if (ctx->twin[q]) continue;
        cudaStream_t ts = nullptr;
        e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
        msbm_ctx *tw = nullptr;
        msbm_status s = msbm_create(&ctx->p, ts, &tw);
        if (s != MSBM_OK) {
            cudaStreamDestroy(ts);
            return s;
        }
        ctx->twin[q] = tw;
        ctx->twin_stream[q] = ts;
    }
    cudaStream_t up = ctx->up_stream, down = ctx->down_stream;
    // Frame i uses staging set b = i % np: its upload waits for the pass of frame i-np
    // (which read set b's images), its pass for its upload and for the download of frame
    // i-np (which read set b's maps), its download for its pass.  So the next frames'
    // uploads and the previous frames' downloads run beside frame i's pass.  Frames rotate
    // over the pass pipelines as they do over the staging sets: frame i runs on pipeline b
    // (the context itself for b = 0, its twin b otherwise), so consecutive passes overlap.
    for (int i = 0; i < n_frames && e == cudaSuccess; ++i) {
        NvtxRange range("msbm host frame", i);
        const int b = i % np;
        msbm_ctx *pc = b > 0 ? ctx->twin[b] : ctx;
        cudaStream_t st = pc->stream;
        const bool want_cost = h_costs && h_costs[i];
        if (i >= np) e = cudaStreamWaitEvent(up, ctx->ev_pass[b], 0);
        if (e == cudaSuccess) {
            if (pitch_bytes == W) {
                e = cudaMemcpyAsync(ctx->sL[b], h_lefts[i], W * H, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->sR[b], h_rights[i], W * H, cudaMemcpyHostToDevice, up);
            } else {
                e = cudaMemcpy2DAsync(ctx->sL[b], W, h_lefts[i], pitch_bytes, W, H, cudaMemcpyHostToDevice, up);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(ctx->sR[b], W, h_rights[i], pitch_bytes, W, H, cudaMemcpyHostToDevice, up);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_up[b], up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->ev_up[b], 0);
        if (e == cudaSuccess && i >= np) e = cudaStreamWaitEvent(st, ctx->ev_down[b], 0);
        if (e != cudaSuccess) break;
        msbm_status s = msbm_disparity(pc, ctx->sL[b], ctx->sR[b], W, ctx->sd[b], want_cost ? ctx->sc[b] : nullptr);
        if (s != MSBM_OK) {
            cudaStreamSynchronize(up);
            cudaStreamSynchronize(down);
            return s;
        }
        e = cudaEventRecord(ctx->ev_pass[b], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, ctx->ev_pass[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_ds[i], ctx->sd[b], W * H * sizeof(int16_t), cudaMemcpyDeviceToHost, down);
        if (e == cudaSuccess && want_cost)
            e = cudaMemcpyAsync(h_costs[i], ctx->sc[b], W * H * sizeof(float), cudaMemcpyDeviceToHost, down);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_down[b], down);
    }
    cudaError_t e2 = cudaStreamSynchronize(up);
    cudaError_t e3 = cudaStreamSynchronize(down);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
    if (e != cudaSuccess) return cuda_status(e);
    msbm_status s = MSBM_OK;
    for (int q = 1; q < HOST_PIPES; ++q) {
        if (!ctx->twin[q]) continue;
        const msbm_status sq = msbm_sync(ctx->twin[q]);
        if (s == MSBM_OK) s = sq;
    }
    msbm_status s0 = msbm_sync(ctx);
    return s0 != MSBM_OK ? s0 : s;
}

msbm_status msbm_disparity_host(msbm_ctx *ctx, const uint8_t *h_left, const uint8_t *h_right,
                                size_t pitch_bytes, int16_t *h_d, float *h_cost) {
    // one frame of the pipelined host path: the images are copied into device staging
    // buffers, the pass runs on them and the maps are copied back.  On page-locked buffers
    // these linear DMA copies beat letting the kernels read and write host memory across the
    // link themselves (measured 7100 vs 6650 frames/s for the 1400 x 1000 pair, maps written
    // by the kernels 6340).
    if (!h_left || !h_right || !h_d) return MSBM_ERR_INVALID_ARG;
    return msbm_disparity_host_frames(ctx, 1, &h_left, &h_right, pitch_bytes, &h_d, h_cost ? &h_cost : nullptr);
}

msbm_status msbm_level_result(msbm_ctx *ctx, int32_t level, int16_t *d_out, float *cost_out) {
    if (!ctx || level < 1 || level >= ctx->p.levels || !d_out) return MSBM_ERR_INVALID_ARG;
    const LevelBuf &l = ctx->lv[level];
    const size_t n = (size_t)l.W * l.H;
    cudaError_t e = cudaMemcpyAsync(d_out, l.d, n * sizeof(int16_t), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && cost_out)
        e = cudaMemcpyAsync(cost_out, l.c, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
    return cuda_status(e);
}

msbm_status msbm_profile_disparity(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                                   size_t pitch_bytes, int16_t *d_out, float *cost_out,
                                   float *stage_ms, int32_t n_stages) {
    if (!ctx || !d_left || !d_right || !d_out || !stage_ms || pitch_bytes < (size_t)ctx->p.width)
        return MSBM_ERR_INVALID_ARG;
    const int K = ctx->p.levels;
    if (n_stages != K + 2) return MSBM_ERR_INVALID_ARG;
    std::vector<cudaEvent_t> ev(K + 3, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    cudaStream_t st = ctx->stream;
    msbm_status s = cuda_status(e);
    int i = 0;
    if (s == MSBM_OK) s = cuda_status(cudaEventRecord(ev[i++], st));
    {
        NvtxRange range("msbm pyramid");
        if (s == MSBM_OK) s = enqueue_pyramid(ctx, d_left, d_right, pitch_bytes, st);
    }
    if (s == MSBM_OK) s = cuda_status(cudaEventRecord(ev[i++], st));
    {
        NvtxRange range("msbm statistics planes");
        if (s == MSBM_OK && K >= 2) s = cuda_status(launch_stats_levels(ctx, K - 1, st));
    }
    if (s == MSBM_OK) s = cuda_status(cudaEventRecord(ev[i++], st));
    for (int k = K - 1; s == MSBM_OK && k >= 0; --k) {
        NvtxRange range("msbm level", k);
        s = enqueue_match(ctx, k, d_out, cost_out, st, true);
        if (s == MSBM_OK) s = cuda_status(cudaEventRecord(ev[i++], st));
    }
    if (s == MSBM_OK) s = cuda_status(cudaStreamSynchronize(st));
    for (int j = 0; s == MSBM_OK && j < K + 2; ++j)
        s = cuda_status(cudaEventElapsedTime(&stage_ms[j], ev[j], ev[j + 1]));
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    return s;
}

msbm_status msbm_pass_kernel_count(const msbm_ctx *ctx, int32_t *count) {
    if (!ctx || !count) return MSBM_ERR_INVALID_ARG;
    *count = ctx->graph_clock ? ctx->graph_kernels : 0;
    return MSBM_OK;
}

msbm_status msbm_sync(msbm_ctx *ctx) {
    if (!ctx) return MSBM_ERR_INVALID_ARG;
    // the error word rides the stream to page-locked host memory: one wait, no extra round trip
    cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return MSBM_ERR_CUDA;
    const int err = *ctx->h_err;
    if (err != 0) {
        // cleared in the context stream's order, so it cannot wipe a status that work
        // enqueued on that stream after this call records
        if (cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream) != cudaSuccess) return MSBM_ERR_CUDA;
        return static_cast<msbm_status>(err);
    }
    return MSBM_OK;
}

msbm_status msbm_eval_count(msbm_ctx *ctx, int64_t *count, int32_t reset) {
    if (!ctx || !count) return MSBM_ERR_INVALID_ARG;
    unsigned long long v = 0;
    if (cudaMemcpyAsync(&v, ctx->d_evals, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return MSBM_ERR_CUDA;
    *count = static_cast<int64_t>(v);
    if (reset && cudaMemsetAsync(ctx->d_evals, 0, sizeof(v), ctx->stream) != cudaSuccess) return MSBM_ERR_CUDA;
    return MSBM_OK;
}

}  // extern "C"
