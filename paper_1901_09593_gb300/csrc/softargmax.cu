// softargmax.cu -- differentiable ZNCC level: soft-argmax disparity readout over a level's
// cost volume and its backward with respect to both images.  The paper's ZNCC (Eq. 2) on
// float images, with an epsilon-regularised denominator,
//     rho(p, z) = sum ac*bc / sqrt((sum ac^2 + eps)(sum bc^2 + eps)),   ac = a - mean(a)
// over candidates 0 <= z <= min(ndisp - 1, x); p_z = softmax_z(rho / T);
// d_soft = sum_z z p_z.  This stands beside the hard winner-take-all of the method
// (Sec. III-A, Eq. 3) as a differentiable readout; the cost volume is never stored.
//
// Forward (one thread per pixel, 32 x 8 pixels per CTA): both images' tiles are staged in
// shared memory (clamp-to-edge); right-window means and rsqrt(sum bc^2 + eps) are computed
// per CTA two-pass; the left window is centred in registers (two-pass); per candidate the
// right window slides one column (a (2n+1) x (2n+1) register window used cyclically, so one
// new column is loaded per candidate); the softmax is accumulated online in base 2.  Saved:
// d_soft and the softmax max m and sum l per pixel.
//
// Backward.  With g = dLoss/dd_soft, g_rho = g p_z (z - d_soft) / T and s = the denominator,
// the derivative of rho through the centred windows (the mean terms cancel because centred
// entries sum to zero) gives, for every image position q of the clamp-extended images,
//   gL(q)  = sum_z R(q - z) A_z(q) - box(zeta)(q) - L(q) box(beta)(q) + box(beta*ma)(q)
//   gR(q') = sum_z L(q' + z) A_z(q' + z) - box(er)(q') - R(q') box(delta)(q') + box(delta*mb)(q')
// where A_z = box filter over the window of alpha(p, z) = g_rho / s, and per pixel / right
// centre r:  beta(p) = sum_z g_rho rho / (Saa + eps),  zeta(p) = sum_z alpha mb(p - z),
// delta(r) = sum_z g_rho rho / (Sbb + eps) and er(r) = sum_z alpha ma at p = r + z.
// Positions outside the image are folded into the clamped edge pixel.  Two kernels: the
// coefficients (writes the alpha volume and the per-pixel / per-centre sums) and the
// gradients (box filter of alpha per tile and candidate, both gathers; the box-filtered
// volume is never stored).  Everything is FP32.
//
// Saved or recomputed.  msbm_zncc_softargmax_fwd_saved also keeps, in caller-owned memory,
// rho for every (image, z, pixel) it evaluated and the left and right window statistics
// {mean, rsqrt(sum c^2 + eps)}; the matching backward's coefficient kernel then reads them
// (one coalesced load per (pixel, z)) instead of staging both images and recomputing the
// (2n+1)^2-term products.  The values are those the recomputation gives, bit for bit (the
// same code computes them), so both backwards agree.  msbm_zncc_softargmax_fwd / _bwd keep
// nothing and recompute.
#include <math.h>

#include "msbm.h"
#include "msbm_device.cuh"
#include "msbm_internal.h"

namespace msbm {

namespace {

constexpr int SA_TX = 32, SA_TY = 8;
constexpr float LOG2E = 1.4426950408889634f;

struct SaArgs {
    const float *L, *R;
    int B, H, W, ndisp;
    float invT2;    // log2(e) / T
    float invT;     // 1 / T
    float eps;
    // forward outputs / backward inputs
    float *dsoft, *m2, *l;
    // backward
    const float *g;
    float *alpha;   // [B][Z][H][W]
    float *zeta, *beta, *ma, *mb, *delta, *er;   // [B][H][W]
    // saved by the forward (nullptr: not kept / recompute): rho [B][Z][H][W] (admissible z
    // only), left statistics {ma, rsa} and right statistics {mb, rsb} per pixel [B][H][W]
    float *rho;
    float2 *lst, *rst;
    // the gradients' box terms per clamp-extended position [B][H+2n][W+2n] (sa_box_kernel)
    float4 *box;
};

template <int NH>
struct SaCfg {
    static constexpr int WIN = 2 * NH + 1;
    static constexpr int N = WIN * WIN;
    static constexpr int ROWS = SA_TY + 2 * NH;
    static constexpr int LTP = SA_TX + 2 * NH;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Stage the left tile, the right span and the right-window statistics of one CTA.
// Layout: Lt[ROWS][LTP], Rt[ROWS][RTP], st[TY][RSW] (float2 {mean, rsqrt(Sbb + eps)}).  RTP
// and RSW are the widths of the right span and of its statistics; RS, when not 0, is a
// compile-time row stride of Rt (>= RTP; st's is RS - 2n) so that the scan's loads of a
// column take constant offsets.
template <int NH, int RS = 0>
__device__ void sa_stage(const SaArgs &a, const float *L, const float *R, int x0, int y0, float *Lt, float *Rt,
                         float2 *st, int RTP, int RSW) {
    using C = SaCfg<NH>;
    const int RTPS = RS ? RS : RTP, RSWS = RS ? RS - 2 * NH : RSW;   // row strides
    const int tid = threadIdx.y * SA_TX + threadIdx.x, nthr = SA_TX * SA_TY;
    const int W = a.W, H = a.H;
    for (int i = tid; i < C::ROWS * C::LTP; i += nthr) {
        int t = i / C::LTP, u = i - t * C::LTP;
        int yy = clampi(y0 - NH + t, 0, H - 1), xx = clampi(x0 - NH + u, 0, W - 1);
        Lt[i] = L[(size_t)yy * W + xx];
    }
    const int rx0 = x0 - (a.ndisp - 1) - NH;   // image column of Rt column 0
    for (int i = tid; i < C::ROWS * RTP; i += nthr) {
        int t = i / RTP, u = i - t * RTP;
        int yy = clampi(y0 - NH + t, 0, H - 1), xx = clampi(rx0 + u, 0, W - 1);
        Rt[t * RTPS + u] = R[(size_t)yy * W + xx];
    }
    __syncthreads();
    // right centre v <-> image column x0 - (ndisp-1) + v; its window is Rt cols v .. v+2n
    for (int i = tid; i < SA_TY * RSW; i += nthr) {
        int ry = i / RSW, v = i - ry * RSW;
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < C::WIN; ++t)
#pragma unroll
            for (int j = 0; j < C::WIN; ++j) s += Rt[(ry + t) * RTPS + v + j];
        const float mean = s * (1.0f / C::N);
        float q = 0.f;
#pragma unroll
        for (int t = 0; t < C::WIN; ++t)
#pragma unroll
            for (int j = 0; j < C::WIN; ++j) {
                float d = Rt[(ry + t) * RTPS + v + j] - mean;
                q = fmaf(d, d, q);
            }
        st[ry * RSWS + v] = make_float2(mean, rsqrtf(q + a.eps));
    }
    __syncthreads();
}

// Per-pixel ZNCC over all admissible candidates, calling visit(z, rho, v2, mb, rsb) for each.
template <int NH, int RS = 0, typename F>
__device__ __forceinline__ void sa_scan(const SaArgs &a, const float *Lt, const float *Rt, const float2 *st,
                                        int RTPw, int RSWw, int tx, int ty, int x, float &ma_out, float &rsa_out,
                                        F &&visit) {
    const int RTP = RS ? RS : RTPw, RSW = RS ? RS - 2 * NH : RSWw;   // row strides (see sa_stage)
    using C = SaCfg<NH>;
    constexpr int WIN = C::WIN;
    float ac[WIN][WIN];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < WIN; ++i)
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
            ac[i][j] = Lt[(ty + i) * C::LTP + tx + j];
            s += ac[i][j];
        }
    const float ma = s * (1.0f / C::N);
    float saa = 0.f, sac = 0.f;
#pragma unroll
    for (int i = 0; i < WIN; ++i)
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
            ac[i][j] -= ma;
            saa = fmaf(ac[i][j], ac[i][j], saa);
            sac += ac[i][j];
        }
    const float rsa = rsqrtf(saa + a.eps);
    ma_out = ma;
    rsa_out = rsa;
    const int zmax = min(a.ndisp - 1, x);
    // Rt column of image column (x - n - z) is tx + ndisp - 1 - z
    const int cb = tx + a.ndisp - 1;
    float rw[WIN][WIN];
#pragma unroll
    for (int i = 0; i < WIN; ++i)
#pragma unroll
        for (int j = 0; j < WIN; ++j) rw[i][j] = Rt[(ty + i) * RTP + cb + j];
    for (int z0 = 0; z0 <= zmax; z0 += WIN) {
#pragma unroll
        for (int zz = 0; zz < WIN; ++zz) {
            const int z = z0 + zz;
            if (z > zmax) break;
            if (z > 0) {
                // new logical column 0 (image column x - z - n) goes into the slot of the
                // column that just left the window; logical column j lives in slot
                // (j - zz) mod WIN, so the indices below are compile-time constants
#pragma unroll
                for (int i = 0; i < WIN; ++i) rw[i][(WIN - zz) % WIN] = Rt[(ty + i) * RTP + cb - z];
            }
            float sab = 0.f;
#pragma unroll
            for (int i = 0; i < WIN; ++i)
#pragma unroll
                for (int j = 0; j < WIN; ++j) sab = fmaf(ac[i][j], rw[i][(j - zz + WIN) % WIN], sab);
            const float2 q = st[ty * RSW + cb - z];   // statistics of the right centre x - z
            // sum ac*(b - mb) = sum ac*b - mb * sum ac (sum ac is the centring residual)
            const float rho = (sab - q.x * sac) * rsa * q.y;
            visit(z, rho, rho * a.invT2, q.x, q.y);
        }
    }
}

// ZP: ndisp rounded up to 64, 128 or 256; the staged rows take the compile-time stride of ZP
// candidates
template <int NH, int ZP>
__global__ void __launch_bounds__(256) sa_fwd_kernel(const SaArgs a) {
    using C = SaCfg<NH>;
    constexpr int RS = SA_TX + ZP - 1 + 2 * NH, RSWS = RS - 2 * NH;
    extern __shared__ float sm[];
    const int RTP = SA_TX + a.ndisp - 1 + 2 * NH, RSW = SA_TX + a.ndisp - 1;   // widths
    float *Lt = sm;
    float *Rt = Lt + C::ROWS * C::LTP;
    float2 *st = reinterpret_cast<float2 *>(Rt + ((C::ROWS * RS + 1) & ~1));
    const int b = blockIdx.z, x0 = blockIdx.x * SA_TX, y0 = blockIdx.y * SA_TY;
    const size_t plane = (size_t)a.H * a.W;
    sa_stage<NH, RS>(a, a.L + b * plane, a.R + b * plane, x0, y0, Lt, Rt, st, RTP, RSW);
    const int tx = threadIdx.x, ty = threadIdx.y, x = x0 + tx, y = y0 + ty;
    if (x >= a.W || y >= a.H) return;
    float m2 = -INFINITY, l = 0.f, s = 0.f, ma, rsa;
    float *rho_p = a.rho ? a.rho + (size_t)b * a.ndisp * plane + (size_t)y * a.W + x : nullptr;
    sa_scan<NH, RS>(a, Lt, Rt, st, RTP, RSW, tx, ty, x, ma, rsa, [&](int z, float rho, float v2, float, float) {
        if (rho_p) rho_p[(size_t)z * plane] = rho;
        if (v2 > m2) {
            const float sc = exp2f(m2 - v2);
            l = fmaf(l, sc, 1.f);
            s = fmaf(s, sc, static_cast<float>(z));
            m2 = v2;
        } else {
            const float e = exp2f(v2 - m2);
            l += e;
            s = fmaf(static_cast<float>(z), e, s);
        }
    });
    const size_t p = b * plane + (size_t)y * a.W + x;
    a.dsoft[p] = s / l;
    a.m2[p] = m2;
    a.l[p] = l;
    if (a.lst) {
        a.lst[p] = make_float2(ma, rsa);
        a.rst[p] = st[ty * RSWS + tx + a.ndisp - 1];   // right centre x
    }
}

// Two CTAs per SM: at 7 x 7 the unconstrained build took 148 registers (one CTA per SM);
// at 128 registers a few hundred bytes spill and forward + backward of the 8 x 640 x 480,
// 64-candidate workload went 2.58 -> 2.29 ms.
template <int NH>
__global__ void __launch_bounds__(256, 2) sa_bwd_coef_kernel(const SaArgs a) {
    using C = SaCfg<NH>;
    extern __shared__ float sm[];
    const int RTP = SA_TX + a.ndisp - 1 + 2 * NH, RSW = SA_TX + a.ndisp - 1;
    float *Lt = sm;
    float *Rt = Lt + C::ROWS * C::LTP;
    float2 *st = reinterpret_cast<float2 *>(Rt + ((C::ROWS * RTP + 1) & ~1));
    float *accD = reinterpret_cast<float *>(st + SA_TY * RSW);
    float *accE = accD + SA_TY * RSW;
    const int b = blockIdx.z, x0 = blockIdx.x * SA_TX, y0 = blockIdx.y * SA_TY;
    const size_t plane = (size_t)a.H * a.W;
    const int tid = threadIdx.y * SA_TX + threadIdx.x;
    for (int i = tid; i < 2 * SA_TY * RSW; i += SA_TX * SA_TY) accD[i] = 0.f;
    sa_stage<NH>(a, a.L + b * plane, a.R + b * plane, x0, y0, Lt, Rt, st, RTP, RSW);
    const int tx = threadIdx.x, ty = threadIdx.y, x = x0 + tx, y = y0 + ty;
    // a warp is one tile row; when all its in-image lanes walk the same candidates, lane l at
    // z and lane l+1 at z+1 are the only writers of a right centre, so ordered plain updates
    // (one __syncwarp per candidate) replace the shared atomics
    const bool inside = x < a.W && y < a.H;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, inside);
    const bool lockstep = __ballot_sync(0xFFFFFFFFu, inside && min(a.ndisp - 1, x) == a.ndisp - 1) == am;
    if (inside) {
        const size_t p = b * plane + (size_t)y * a.W + x;
        const float d = a.dsoft[p], m2 = a.m2[p];
        const float gs = a.g[p] * a.invT / a.l[p];             // g p_z (z - d) / T = gs 2^(..) (z - d)
        float beta = 0.f, zeta = 0.f, ma = 0.f, rsa = 0.f;
        float *alpha = a.alpha + (size_t)b * a.ndisp * plane + (size_t)y * a.W + x;
        float *accDrow = accD + ty * RSW + tx + a.ndisp - 1;   // right centre x - z at [-z]
        float *accErow = accE + ty * RSW + tx + a.ndisp - 1;
        int zmax = -1;   // ma and rsa are set by sa_scan before its first callback
        // the same arithmetic as sa_bwd_coef_saved_kernel, so both backwards give the same
        // coefficients
        sa_scan<NH>(a, Lt, Rt, st, RTP, RSW, tx, ty, x, ma, rsa, [&](int z, float rho, float, float mb, float rsb) {
            const float grho = gs * exp2f(fmaf(rho, a.invT2, -m2)) * (static_cast<float>(z) - d);
            const float al = grho * rsa * rsb;
            const float gr = grho * rho;
            beta = fmaf(gr, rsa * rsa, beta);
            zeta = fmaf(al, mb, zeta);
            if (lockstep) {
                accDrow[-z] = fmaf(gr, rsb * rsb, accDrow[-z]);
                accErow[-z] = fmaf(al, ma, accErow[-z]);
                __syncwarp(am);
            } else {
                atomicAdd(accDrow - z, gr * rsb * rsb);
                atomicAdd(accErow - z, al * ma);
            }
            alpha[(size_t)z * plane] = al;
            zmax = z;
        });
        for (int z = zmax + 1; z < a.ndisp; ++z) alpha[(size_t)z * plane] = 0.f;
        a.beta[p] = beta;
        a.zeta[p] = zeta;
        a.ma[p] = ma;
        a.mb[p] = st[ty * RSW + tx + a.ndisp - 1].x;   // right centre x (z = 0)
    }
    __syncthreads();
    // flush the right-centre accumulators: centre v <-> image column x0 - (ndisp-1) + v
    float *delta = a.delta + b * plane, *er = a.er + b * plane;
    for (int i = tid; i < SA_TY * RSW; i += SA_TX * SA_TY) {
        int ry = i / RSW, v = i - ry * RSW;
        int yy = y0 + ry, xx = x0 - (a.ndisp - 1) + v;
        if (yy >= a.H || xx < 0 || xx >= a.W) continue;
        if (accD[i] != 0.f) atomicAdd(delta + (size_t)yy * a.W + xx, accD[i]);
        if (accE[i] != 0.f) atomicAdd(er + (size_t)yy * a.W + xx, accE[i]);
    }
}

// The coefficient kernel on the forward's saved rho and window statistics: the same
// per-(pixel, z) coefficients and sums as sa_bwd_coef_kernel, with rho, {ma, rsa} and
// {mb, rsb} loaded instead of recomputed (no image staging, no window products).
__global__ void __launch_bounds__(256) sa_bwd_coef_saved_kernel(const SaArgs a) {
    extern __shared__ float sm[];
    const int RSW = SA_TX + a.ndisp - 1;
    float *accD = sm;
    float *accE = accD + SA_TY * RSW;
    const int b = blockIdx.z, x0 = blockIdx.x * SA_TX, y0 = blockIdx.y * SA_TY;
    const size_t plane = (size_t)a.H * a.W;
    const int tid = threadIdx.y * SA_TX + threadIdx.x;
    for (int i = tid; i < 2 * SA_TY * RSW; i += SA_TX * SA_TY) accD[i] = 0.f;
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, x = x0 + tx, y = y0 + ty;
    // lockstep as in sa_bwd_coef_kernel: ordered plain updates when a warp's in-image lanes
    // all walk every candidate
    const bool inside = x < a.W && y < a.H;
    const unsigned am = __ballot_sync(0xFFFFFFFFu, inside);
    const bool lockstep = __ballot_sync(0xFFFFFFFFu, inside && min(a.ndisp - 1, x) == a.ndisp - 1) == am;
    if (inside) {
        const size_t p = b * plane + (size_t)y * a.W + x;
        const float d = a.dsoft[p], m2 = a.m2[p];
        const float gs = a.g[p] * a.invT / a.l[p];             // g p_z (z - d) / T = gs 2^(..) (z - d)
        const float2 ls = a.lst[p];
        const float ma = ls.x, rsa = ls.y, rsa2 = rsa * rsa;
        float beta = 0.f, zeta = 0.f;
        float *alpha = a.alpha + (size_t)b * a.ndisp * plane + (size_t)y * a.W + x;
        const float *rho_p = a.rho + (size_t)b * a.ndisp * plane + (size_t)y * a.W + x;
        const uint32_t pl = static_cast<uint32_t>(plane);       // H * W < 2^32
        const float2 *rs = a.rst + p;                            // right centre x - z at [-z]
        float *accDrow = accD + ty * RSW + tx + a.ndisp - 1;
        float *accErow = accE + ty * RSW + tx + a.ndisp - 1;
        const int zmax = min(a.ndisp - 1, x);
        // the loads of SB_AHEAD candidates are issued together: the volume comes from DRAM,
        // and one candidate's latency per iteration would bound the loop (measured backward:
        // 1.20 ms one at a time, 0.96 ms four, 1.08 / 1.14 ms eight / sixteen)
        constexpr int SB_AHEAD = 4;
        for (int z0 = 0; z0 <= zmax; z0 += SB_AHEAD) {
            float rv[SB_AHEAD];
            float2 qv[SB_AHEAD];
#pragma unroll
            for (int u = 0; u < SB_AHEAD; ++u) {
                const int z = z0 + u;
                rv[u] = z <= zmax ? __ldg(rho_p + static_cast<uint64_t>(static_cast<uint32_t>(z)) * pl) : 0.f;
                qv[u] = z <= zmax ? __ldg(rs - z) : make_float2(0.f, 0.f);
            }
            float zd = static_cast<float>(z0) - d;
#pragma unroll
            for (int u = 0; u < SB_AHEAD; ++u, zd += 1.f) {
                const int z = z0 + u;
                if (z > zmax) break;
                const float rho = rv[u], mb = qv[u].x, rsb = qv[u].y;
                const float grho = gs * exp2f(fmaf(rho, a.invT2, -m2)) * zd;
                const float al = grho * rsa * rsb;
                const float gr = grho * rho;
                beta = fmaf(gr, rsa2, beta);
                zeta = fmaf(al, mb, zeta);
                if (lockstep) {
                    accDrow[-z] = fmaf(gr, rsb * rsb, accDrow[-z]);
                    accErow[-z] = fmaf(al, ma, accErow[-z]);
                    __syncwarp(am);
                } else {
                    atomicAdd(accDrow - z, gr * rsb * rsb);
                    atomicAdd(accErow - z, al * ma);
                }
                alpha[static_cast<uint64_t>(static_cast<uint32_t>(z)) * pl] = al;
            }
        }
        for (int z = zmax + 1; z < a.ndisp; ++z) alpha[(size_t)z * plane] = 0.f;
        a.beta[p] = beta;
        a.zeta[p] = zeta;
        a.ma[p] = ma;
        a.mb[p] = rs[0].x;
    }
    __syncthreads();
    float *delta = a.delta + b * plane, *er = a.er + b * plane;
    for (int i = tid; i < SA_TY * RSW; i += SA_TX * SA_TY) {
        int ry = i / RSW, v = i - ry * RSW;
        int yy = y0 + ry, xx = x0 - (a.ndisp - 1) + v;
        if (yy >= a.H || xx < 0 || xx >= a.W) continue;
        if (accD[i] != 0.f) atomicAdd(delta + (size_t)yy * a.W + xx, accD[i]);
        if (accE[i] != 0.f) atomicAdd(er + (size_t)yy * a.W + xx, accE[i]);
    }
}

constexpr int SG_BOX = 32;                        // box-term tile side

// The gradients' box terms (the last three of gL and gR in the file header) per position of
// the clamp-extended domain (Y in [0, H+2n), X in [0, W+2n); image position q = (Y-n, X-n)),
// summed over the image pixels of q's window:
//   x = sum(beta ma) - sum(zeta),  y = sum(beta),  z = sum(delta mb) - sum(er),  w = sum(delta)
// so that gL(q) gets x - L(q) y and gR(q) gets z - R(q) w.  Per 32 x 32 tile of positions the
// four summands' (32 + 2n)^2 image region (zero outside the image) is staged in shared
// memory, then summed horizontally and vertically.
template <int NH>
__global__ void __launch_bounds__(256) sa_box_kernel(const SaArgs a) {
    constexpr int WIN = 2 * NH + 1, TR = SG_BOX + 2 * NH, TCP = TR + 1;
    __shared__ float sv[4][TR][TCP];
    __shared__ float hv[4][TR][SG_BOX + 1];
    const int b = blockIdx.z, X0 = blockIdx.x * SG_BOX, Y0 = blockIdx.y * SG_BOX;
    const int tid = threadIdx.y * SA_TX + threadIdx.x;
    const size_t plane = (size_t)a.H * a.W;
    const float *zeta = a.zeta + b * plane, *beta = a.beta + b * plane, *ma = a.ma + b * plane;
    const float *er = a.er + b * plane, *delta = a.delta + b * plane, *mb = a.mb + b * plane;
    for (int i = tid; i < TR * TR; i += SA_TX * 8) {
        const int t = i / TR, u = i - t * TR;
        const int yy = Y0 - 2 * NH + t, xx = X0 - 2 * NH + u;
        float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
            const size_t o = (size_t)yy * a.W + xx;
            v1 = beta[o];
            v0 = fmaf(v1, ma[o], -zeta[o]);
            v3 = delta[o];
            v2 = fmaf(v3, mb[o], -er[o]);
        }
        sv[0][t][u] = v0;
        sv[1][t][u] = v1;
        sv[2][t][u] = v2;
        sv[3][t][u] = v3;
    }
    __syncthreads();
    for (int i = tid; i < 4 * TR * SG_BOX; i += SA_TX * 8) {
        const int m = i / (TR * SG_BOX), r = i - m * TR * SG_BOX, t = r / SG_BOX, u = r - t * SG_BOX;
        float h = 0.f;
#pragma unroll
        for (int j = 0; j < WIN; ++j) h += sv[m][t][u + j];
        hv[m][t][u] = h;
    }
    __syncthreads();
    const int Wp = a.W + 2 * NH, Hp = a.H + 2 * NH;
    float4 *out = a.box + (size_t)b * Hp * Wp;
    for (int i = tid; i < SG_BOX * SG_BOX; i += SA_TX * 8) {
        const int t = i / SG_BOX, u = i - t * SG_BOX;
        const int Y = Y0 + t, X = X0 + u;
        if (Y >= Hp || X >= Wp) continue;
        float r[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < WIN; ++k) v += hv[m][t + k][u];
            r[m] = v;
        }
        out[(size_t)Y * Wp + X] = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// Both image gradients over the clamp-extended domain (Y in [0, H+2n), X in [0, W+2n); image
// position q = (Y-n, X-n), folded into the clamped edge pixel by atomicAdd).  Per 32 x 32
// tile (each thread a column of 4 positions) and candidate z the CTA box-filters alpha(b, z)
// in shared memory:
//   A_z(Y, X) = sum of alpha(b, z) over the (2n+1)^2 image pixels around (Y-n, X-n)
// (zero outside the image; horizontal sums, then a vertical sliding sum), then
//   gL(Y, X)     += R(q - z) A_z(Y, X)                      (z <= X; A_z is 0 beyond)
//   gR(Y, X - z) += L(q)     A_z(Y, X)                      (X - z >= 0)
// with R(q - z) read from the tile's right rows staged once, and gR accumulated in a shared
// row buffer spanning the tile and the ndisp - 1 columns to its left, flushed once per tile.
// The box terms of both gradients (zeta, beta, ma / er, delta, mb) are added for the tile's
// own positions.  The A volume is never stored.
constexpr int SG_TY = 32, SG_PER = SG_TY / 8;     // tile rows, rows per thread

template <int NH>
struct SgCfg {
    static constexpr int TR = SG_TY + 2 * NH, TC = SA_TX + 2 * NH;
    static constexpr int TCP = TC + 1, HSP = SA_TX + 1;
    static size_t bytes(int ndisp) {
        const size_t aw = SA_TX + ndisp - 1;
        return sizeof(float) * ((size_t)TR * TCP + (size_t)TR * HSP + 2 * (size_t)SG_TY * aw);
    }
};

template <int NH>
__global__ void __launch_bounds__(256) sa_grad_kernel(const SaArgs a, float *gL, float *gR) {
    using C = SgCfg<NH>;
    constexpr int WIN = 2 * NH + 1, TR = C::TR, TC = C::TC, TCP = C::TCP, HSP = C::HSP;
    extern __shared__ float sm[];
    float *tile = sm;                                 // [TR][TCP]
    float *hs = tile + TR * TCP;                      // [TR][HSP]
    const int AW = SA_TX + a.ndisp - 1;               // column c <-> extended X0 - (ndisp-1) + c
    float *Rs = hs + TR * HSP;                        // [SG_TY][AW]: R at row q_y, column X - n - z
    float *accR = Rs + SG_TY * AW;                    // [SG_TY][AW]
    const int b = blockIdx.z;
    const int Wp = a.W + 2 * NH, Hp = a.H + 2 * NH;
    const int X0 = blockIdx.x * SA_TX, Y0 = blockIdx.y * SG_TY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * SA_TX + tx;
    const size_t plane = (size_t)a.H * a.W;
    const float *Lb = a.L + b * plane, *Rb = a.R + b * plane;
    for (int r = ty; r < SG_TY; r += 8)
        for (int c = tx; c < AW; c += SA_TX) {
            const int cy = clampi(Y0 + r - NH, 0, a.H - 1);
            const int xx = clampi(X0 - (a.ndisp - 1) + c - NH, 0, a.W - 1);
            Rs[r * AW + c] = Rb[(size_t)cy * a.W + xx];
            accR[r * AW + c] = 0.f;
        }
    const int X = X0 + tx, qx = X - NH;
    const int r0 = SG_PER * ty;                       // this thread's first tile row
    float Lq[SG_PER], gl[SG_PER], racc[SG_PER];
#pragma unroll
    for (int k = 0; k < SG_PER; ++k) {
        racc[k] = 0.f;
        const int cy = clampi(Y0 + r0 + k - NH, 0, a.H - 1);
        Lq[k] = Lb[(size_t)cy * a.W + clampi(qx, 0, a.W - 1)];
        gl[k] = 0.f;
    }
    const bool colin = X < Wp;
    // the tile's elements e = tid + 256 k, (t, u) = (e / TC, e % TC) <-> image
    // (Y0 - 2n + t, X0 - 2n + u); the next candidate's are loaded into registers while the
    // current one is processed
    constexpr int NE = (TR * TC + SA_TX * 8 - 1) / (SA_TX * 8);
    int off[NE];                                      // element offset in an alpha plane, or -1
    int soff[NE];                                     // its place in the shared tile, or -1
#pragma unroll
    for (int k = 0; k < NE; ++k) {
        const int e = tid + SA_TX * 8 * k, t = e / TC, u = e - t * TC;
        const int yy = Y0 - 2 * NH + t, xx = X0 - 2 * NH + u;
        soff[k] = e < TR * TC ? t * TCP + u : -1;
        off[k] = (e < TR * TC && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) ? yy * a.W + xx : -1;
    }
    float nxt[NE];
    const float *al0 = a.alpha + (size_t)b * a.ndisp * plane;
#pragma unroll
    for (int k = 0; k < NE; ++k) nxt[k] = off[k] >= 0 ? __ldg(al0 + off[k]) : 0.f;
    for (int z = 0; z < a.ndisp; ++z) {
        __syncthreads();   // the previous candidate's tile and sums are consumed
#pragma unroll
        for (int k = 0; k < NE; ++k)
            if (soff[k] >= 0) tile[soff[k]] = nxt[k];
        if (z + 1 < a.ndisp) {
            const float *al = al0 + (size_t)(z + 1) * plane;
#pragma unroll
            for (int k = 0; k < NE; ++k) nxt[k] = off[k] >= 0 ? __ldg(al + off[k]) : 0.f;
        }
        __syncthreads();
        // horizontal window sums: each of TR x 4 items slides over 8 columns of one row
        for (int i = tid; i < TR * 4; i += SA_TX * 8) {
            const int t = i >> 2, c0 = (i & 3) * 8;
            const float *row = tile + t * TCP + c0;
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < WIN; ++j) s += row[j];
            float *h = hs + t * HSP + c0;
            h[0] = s;
#pragma unroll
            for (int u = 1; u < 8; ++u) {
                s += row[u + WIN - 1] - row[u - 1];
                h[u] = s;
            }
        }
        __syncthreads();
        const int c = tx + a.ndisp - 1 - z;           // column of extended X - z
        float v[SG_PER];
#pragma unroll
        for (int k = 0; k < SG_PER; ++k) v[k] = 0.f;
        if (colin && z <= X) {
            float A = 0.f;
#pragma unroll
            for (int i = 0; i < WIN; ++i) A += hs[(r0 + i) * HSP + tx];
#pragma unroll
            for (int k = 0; k < SG_PER; ++k) {
                if (k > 0) A += hs[(r0 + k + WIN - 1) * HSP + tx] - hs[(r0 + k - 1) * HSP + tx];
                gl[k] = fmaf(Rs[(r0 + k) * AW + c], A, gl[k]);
                v[k] = Lq[k] * A;
            }
        }
        // gR(Y, X - z) += L(q) A_z: the partial of column c moves one lane up per candidate
        // (lane tx + 1 reaches the same column at z + 1); lane 31's leaves the warp complete
#pragma unroll
        for (int k = 0; k < SG_PER; ++k) {
            racc[k] += v[k];
            if (tx == SA_TX - 1) accR[(r0 + k) * AW + c] += racc[k];
            racc[k] = __shfl_up_sync(0xFFFFFFFFu, racc[k], 1);
            if (tx == 0) racc[k] = 0.f;
        }
    }
    // the partials still in flight: lane tx holds column tx - 1 (that lane tx - 1 had at the
    // last candidate), then the box terms below update the tile's own columns
#pragma unroll
    for (int k = 0; k < SG_PER; ++k)
        if (tx > 0) accR[(r0 + k) * AW + tx - 1] += racc[k];
    __syncwarp();
    __syncthreads();
    const float4 *box = a.box + (size_t)b * Hp * Wp;
#pragma unroll
    for (int k = 0; k < SG_PER; ++k) {
        const int Y = Y0 + r0 + k, qy = Y - NH;
        if (!colin || Y >= Hp) continue;
        const float4 t = box[(size_t)Y * Wp + X];           // the box terms (sa_box_kernel)
        const size_t o = (size_t)clampi(qy, 0, a.H - 1) * a.W + clampi(qx, 0, a.W - 1);
        atomicAdd(gL + b * plane + o, gl[k] + t.x - Lq[k] * t.y);
        accR[(r0 + k) * AW + tx + a.ndisp - 1] += t.z - Rb[o] * t.w;
    }
    __syncthreads();
    float *gRb = gR + b * plane;
    for (int i = tid; i < SG_TY * AW; i += SA_TX * 8) {
        const int r = i / AW, c = i - r * AW;
        const int Xe = X0 - (a.ndisp - 1) + c, Ye = Y0 + r;
        if (Xe < 0 || Xe >= Wp || Ye >= Hp || accR[i] == 0.f) continue;
        atomicAdd(gRb + (size_t)clampi(Ye - NH, 0, a.H - 1) * a.W + clampi(Xe - NH, 0, a.W - 1), accR[i]);
    }
}

size_t sa_fwd_smem(int nh, int ndisp, bool bwd) {
    const int rows = SA_TY + 2 * nh, ltp = SA_TX + 2 * nh;
    const int rtp = SA_TX + ndisp - 1 + 2 * nh, rsw = SA_TX + ndisp - 1;
    size_t f = (size_t)rows * ltp + (((size_t)rows * rtp + 1) & ~(size_t)1) + 2 * (size_t)SA_TY * rsw;
    if (bwd) f += 2 * (size_t)SA_TY * rsw;
    return f * sizeof(float);
}

template <int NH>
cudaError_t sa_run(const SaArgs &a, bool bwd, float *gL, float *gR, cudaStream_t st) {
    dim3 blk(SA_TX, SA_TY);
    dim3 grd((a.W + SA_TX - 1) / SA_TX, (a.H + SA_TY - 1) / SA_TY, a.B);
    size_t smem = sa_fwd_smem(NH, a.ndisp, bwd);
    cudaError_t e;
    if (!bwd) {
        const int zp = a.ndisp <= 64 ? 64 : (a.ndisp <= 128 ? 128 : 256);
        const size_t fsm = sa_fwd_smem(NH, zp, false);
        auto kern = zp == 64 ? sa_fwd_kernel<NH, 64> : (zp == 128 ? sa_fwd_kernel<NH, 128> : sa_fwd_kernel<NH, 256>);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        if (e != cudaSuccess) return e;
        kern<<<grd, blk, fsm, st>>>(a);
        return cudaGetLastError();
    }
    if (a.rho) {
        const size_t csm = 2 * (size_t)SA_TY * (SA_TX + a.ndisp - 1) * sizeof(float);
        sa_bwd_coef_saved_kernel<<<grd, blk, csm, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(sa_bwd_coef_kernel<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        sa_bwd_coef_kernel<NH><<<grd, blk, smem, st>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int Wp = a.W + 2 * NH, Hp = a.H + 2 * NH;
    dim3 gbox((Wp + SG_BOX - 1) / SG_BOX, (Hp + SG_BOX - 1) / SG_BOX, a.B);
    sa_box_kernel<NH><<<gbox, blk, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 gext((Wp + SA_TX - 1) / SA_TX, (Hp + SG_TY - 1) / SG_TY, a.B);
    const size_t gsm = SgCfg<NH>::bytes(a.ndisp);
    e = cudaFuncSetAttribute(sa_grad_kernel<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    if (e != cudaSuccess) return e;
    sa_grad_kernel<NH><<<gext, blk, gsm, st>>>(a, gL, gR);
    return cudaGetLastError();
}

cudaError_t sa_dispatch(int nh, const SaArgs &a, bool bwd, float *gL, float *gR, cudaStream_t st) {
    switch (nh) {
        case 1: return sa_run<1>(a, bwd, gL, gR, st);
        case 2: return sa_run<2>(a, bwd, gL, gR, st);
        case 3: return sa_run<3>(a, bwd, gL, gR, st);
        case 4: return sa_run<4>(a, bwd, gL, gR, st);
        default: return cudaErrorInvalidValue;
    }
}

bool sa_sizes_ok(int B, int H, int W, int window, int ndisp) {
    if (B < 1 || B > 65535 || H < 1 || H > 16384 || W < 1 || W > 16384) return false;
    if (window < 3 || window > 9 || (window & 1) == 0) return false;
    return ndisp >= 1 && ndisp <= 256;
}

msbm_status sa_validate(const float *L, const float *R, int B, int H, int W, int window, int ndisp, float T,
                        float eps) {
    if (!L || !R) return MSBM_ERR_INVALID_ARG;
    if (!sa_sizes_ok(B, H, W, window, ndisp)) return MSBM_ERR_INVALID_ARG;
    if (!(T > 0.f) || !(eps >= 0.f) || !isfinite(T) || !isfinite(eps)) return MSBM_ERR_INVALID_ARG;
    return MSBM_OK;
}

struct SaWorkspace {
    size_t alpha, arrays, box, total;
};

// Saved-forward memory: rho [B][Z][H][W], then {ma, rsa} and {mb, rsb} per pixel, each
// part 256-byte aligned.
struct SaSaved {
    size_t rho, stats, total;
};

SaSaved sa_saved(int B, int H, int W, int ndisp) {
    SaSaved v;
    auto al = [](size_t n) { return (n + 255) / 256 * 256; };
    v.rho = al((size_t)B * ndisp * H * W * sizeof(float));
    v.stats = al((size_t)B * H * W * sizeof(float2));
    v.total = v.rho + 2 * v.stats;
    return v;
}

void sa_bind_saved(SaArgs &a, void *saved, const SaSaved &v) {
    uint8_t *m = static_cast<uint8_t *>(saved);
    a.rho = reinterpret_cast<float *>(m);
    a.lst = reinterpret_cast<float2 *>(m + v.rho);
    a.rst = reinterpret_cast<float2 *>(m + v.rho + v.stats);
}

SaWorkspace sa_workspace(int B, int H, int W, int window, int ndisp) {
    SaWorkspace w;
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const int nh = window / 2;
    w.alpha = al((size_t)B * ndisp * H * W * sizeof(float));
    w.arrays = al((size_t)B * H * W * sizeof(float));
    w.box = al((size_t)B * (H + 2 * nh) * (W + 2 * nh) * sizeof(float4));
    w.total = w.alpha + 6 * w.arrays + w.box;
    return w;
}

}  // namespace

}  // namespace msbm

using namespace msbm;

extern "C" {

msbm_status msbm_zncc_softargmax_fwd(const float *d_left, const float *d_right, int32_t batch, int32_t height,
                                     int32_t width, int32_t window, int32_t ndisp, float temperature, float eps,
                                     float *d_soft, float *m_out, float *l_out, void *cuda_stream) {
    msbm_status s = sa_validate(d_left, d_right, batch, height, width, window, ndisp, temperature, eps);
    if (s != MSBM_OK) return s;
    if (!d_soft || !m_out || !l_out) return MSBM_ERR_INVALID_ARG;
    SaArgs a = {};
    a.L = d_left; a.R = d_right;
    a.B = batch; a.H = height; a.W = width; a.ndisp = ndisp;
    a.invT2 = LOG2E / temperature; a.invT = 1.f / temperature; a.eps = eps;
    a.dsoft = d_soft; a.m2 = m_out; a.l = l_out;
    cudaError_t e = sa_dispatch(window / 2, a, false, nullptr, nullptr, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? MSBM_OK : MSBM_ERR_CUDA;
}

size_t msbm_zncc_softargmax_workspace_bytes(int32_t batch, int32_t height, int32_t width, int32_t window,
                                            int32_t ndisp) {
    if (!sa_sizes_ok(batch, height, width, window, ndisp)) return 0;
    return sa_workspace(batch, height, width, window, ndisp).total;
}

msbm_status msbm_zncc_softargmax_bwd(const float *d_left, const float *d_right, int32_t batch, int32_t height,
                                     int32_t width, int32_t window, int32_t ndisp, float temperature, float eps,
                                     const float *d_soft, const float *m_in, const float *l_in, const float *g_d,
                                     float *g_left, float *g_right, void *workspace, size_t workspace_bytes,
                                     void *cuda_stream) {
    msbm_status s = sa_validate(d_left, d_right, batch, height, width, window, ndisp, temperature, eps);
    if (s != MSBM_OK) return s;
    if (!d_soft || !m_in || !l_in || !g_d || !g_left || !g_right || !workspace) return MSBM_ERR_INVALID_ARG;
    SaWorkspace w = sa_workspace(batch, height, width, window, ndisp);
    if (workspace_bytes < w.total) return MSBM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return MSBM_ERR_ALIGNMENT;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    SaArgs a = {};
    a.L = d_left; a.R = d_right;
    a.B = batch; a.H = height; a.W = width; a.ndisp = ndisp;
    a.invT2 = LOG2E / temperature; a.invT = 1.f / temperature; a.eps = eps;
    a.dsoft = const_cast<float *>(d_soft); a.m2 = const_cast<float *>(m_in); a.l = const_cast<float *>(l_in);
    a.g = g_d;
    a.alpha = reinterpret_cast<float *>(ws);
    float *arr = reinterpret_cast<float *>(ws + w.alpha);
    const size_t na = w.arrays / sizeof(float);
    a.zeta = arr; a.beta = arr + na; a.ma = arr + 2 * na; a.mb = arr + 3 * na; a.delta = arr + 4 * na;
    a.er = arr + 5 * na;
    a.box = reinterpret_cast<float4 *>(ws + w.alpha + 6 * w.arrays);
    const size_t plane_bytes = (size_t)batch * height * width * sizeof(float);
    cudaError_t e = cudaMemsetAsync(a.delta, 0, 2 * w.arrays, st);   // delta and er accumulate
    if (e == cudaSuccess) e = cudaMemsetAsync(g_left, 0, plane_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_right, 0, plane_bytes, st);
    if (e == cudaSuccess) e = sa_dispatch(window / 2, a, true, g_left, g_right, st);
    return e == cudaSuccess ? MSBM_OK : MSBM_ERR_CUDA;
}

size_t msbm_zncc_softargmax_saved_bytes(int32_t batch, int32_t height, int32_t width, int32_t window,
                                        int32_t ndisp) {
    if (!sa_sizes_ok(batch, height, width, window, ndisp)) return 0;
    return sa_saved(batch, height, width, ndisp).total;
}

msbm_status msbm_zncc_softargmax_fwd_saved(const float *d_left, const float *d_right, int32_t batch,
                                           int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                           float temperature, float eps, float *d_soft, float *m_out, float *l_out,
                                           void *saved, size_t saved_bytes, void *cuda_stream) {
    msbm_status s = sa_validate(d_left, d_right, batch, height, width, window, ndisp, temperature, eps);
    if (s != MSBM_OK) return s;
    if (!d_soft || !m_out || !l_out || !saved) return MSBM_ERR_INVALID_ARG;
    const SaSaved v = sa_saved(batch, height, width, ndisp);
    if (saved_bytes < v.total) return MSBM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(saved) % 256 != 0) return MSBM_ERR_ALIGNMENT;
    SaArgs a = {};
    a.L = d_left; a.R = d_right;
    a.B = batch; a.H = height; a.W = width; a.ndisp = ndisp;
    a.invT2 = LOG2E / temperature; a.invT = 1.f / temperature; a.eps = eps;
    a.dsoft = d_soft; a.m2 = m_out; a.l = l_out;
    sa_bind_saved(a, saved, v);
    cudaError_t e = sa_dispatch(window / 2, a, false, nullptr, nullptr, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? MSBM_OK : MSBM_ERR_CUDA;
}

msbm_status msbm_zncc_softargmax_bwd_saved(const float *d_left, const float *d_right, int32_t batch,
                                           int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                           float temperature, float eps, const float *d_soft, const float *m_in,
                                           const float *l_in, const float *g_d, const void *saved,
                                           size_t saved_bytes, float *g_left, float *g_right, void *workspace,
                                           size_t workspace_bytes, void *cuda_stream) {
    msbm_status s = sa_validate(d_left, d_right, batch, height, width, window, ndisp, temperature, eps);
    if (s != MSBM_OK) return s;
    if (!d_soft || !m_in || !l_in || !g_d || !g_left || !g_right || !workspace || !saved)
        return MSBM_ERR_INVALID_ARG;
    const SaSaved v = sa_saved(batch, height, width, ndisp);
    SaWorkspace w = sa_workspace(batch, height, width, window, ndisp);
    if (saved_bytes < v.total || workspace_bytes < w.total) return MSBM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0 || reinterpret_cast<uintptr_t>(saved) % 256 != 0)
        return MSBM_ERR_ALIGNMENT;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    SaArgs a = {};
    a.L = d_left; a.R = d_right;
    a.B = batch; a.H = height; a.W = width; a.ndisp = ndisp;
    a.invT2 = LOG2E / temperature; a.invT = 1.f / temperature; a.eps = eps;
    a.dsoft = const_cast<float *>(d_soft); a.m2 = const_cast<float *>(m_in); a.l = const_cast<float *>(l_in);
    a.g = g_d;
    sa_bind_saved(a, const_cast<void *>(saved), v);
    a.alpha = reinterpret_cast<float *>(ws);
    float *arr = reinterpret_cast<float *>(ws + w.alpha);
    const size_t na = w.arrays / sizeof(float);
    a.zeta = arr; a.beta = arr + na; a.ma = arr + 2 * na; a.mb = arr + 3 * na; a.delta = arr + 4 * na;
    a.er = arr + 5 * na;
    a.box = reinterpret_cast<float4 *>(ws + w.alpha + 6 * w.arrays);
    const size_t plane_bytes = (size_t)batch * height * width * sizeof(float);
    cudaError_t e = cudaMemsetAsync(a.delta, 0, 2 * w.arrays, st);   // delta and er accumulate
    if (e == cudaSuccess) e = cudaMemsetAsync(g_left, 0, plane_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_right, 0, plane_bytes, st);
    if (e == cudaSuccess) e = sa_dispatch(window / 2, a, true, g_left, g_right, st);
    return e == cudaSuccess ? MSBM_OK : MSBM_ERR_CUDA;
}

}  // extern "C"
