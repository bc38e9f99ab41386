/*
 * msbm_oracle.c -- plain, slow FP64 CPU oracle for multi-scale hierarchical ZNCC block
 * matching (Kaushik & Lall, "Fast Hierarchical depth map computation from stereo").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark call this code.  It shares nothing with the CUDA library: no header, no
 * helper, no table.  Every function follows the paper's steps in its own order and
 * notation, with no blocking, fusion or reordering, so it can be read against the paper.
 *
 * Conventions (readings of the paper; each is listed with its reason in the design notes):
 *   - images are row-major, (y, x) = (row, column), the LEFT image is the reference and
 *     candidate disparity z pairs left column x with right column x - z (Eq. 1);
 *   - window half-width n, side w = 2n+1, N = w*w window pixels; pixels outside the image
 *     are read clamp-to-edge;
 *   - D candidates 0..D-1 at level 0, D_k = ceil(D / 2^k) at level k (Sec. III);
 *   - a candidate is admissible only if z <= x (its right centre lies in the image).
 *
 * Parity status: pyramid, ZNCC, WTA, the hierarchical driver and the soft-argmax level are
 * pinned by the tests in tests/test_oracle_*.py (brute force, invariants, planted scenes,
 * finite differences).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------------
 * Gaussian pyramid (Sec. III, Fig. 1).  The paper names a Gaussian pyramid without the
 * kernel.  Reading: the 5-tap binomial 1,4,6,4,1 on each axis (weights /16 each, /256 in
 * 2-D), clamp-to-edge, output ceil(W/2) x ceil(H/2), integer result rounded to nearest
 * ((sum + 128) >> 8).  Written as the direct 2-D weighted sum.
 * ---------------------------------------------------------------------------------- */
void oracle_reduce(const uint8_t *src, int W, int H, uint8_t *dst) {
    static const int c[5] = {1, 4, 6, 4, 1};
    int W2 = (W + 1) / 2, H2 = (H + 1) / 2;
    for (int y = 0; y < H2; ++y)
        for (int x = 0; x < W2; ++x) {
            long s = 0;
            for (int a = -2; a <= 2; ++a)
                for (int b = -2; b <= 2; ++b) {
                    int yy = clampi(2 * y + a, 0, H - 1);
                    int xx = clampi(2 * x + b, 0, W - 1);
                    s += (long)c[a + 2] * c[b + 2] * src[(long)yy * W + xx];
                }
            dst[(long)y * W2 + x] = (uint8_t)((s + 128) >> 8);
        }
}

/* Level sizes: level 0 is W x H, level k is ceil(W_{k-1}/2) x ceil(H_{k-1}/2). */
void oracle_level_size(int W, int H, int k, int *Wk, int *Hk) {
    for (int i = 0; i < k; ++i) { W = (W + 1) / 2; H = (H + 1) / 2; }
    *Wk = W; *Hk = H;
}

/* Candidate count at level k: D_k = ceil(D / 2^k) (Sec. III, d^k_max = D_max / 2^k). */
int oracle_level_disp(int D, int k) { return (int)((D + (1L << k) - 1) >> k); }

/* All K levels of one image, concatenated level 0 first. */
void oracle_pyramid(const uint8_t *img, int W, int H, int K, uint8_t *out) {
    memcpy(out, img, (size_t)W * H);
    const uint8_t *prev = out;
    int w = W, h = H;
    uint8_t *cur = out + (size_t)W * H;
    for (int k = 1; k < K; ++k) {
        oracle_reduce(prev, w, h, cur);
        prev = cur;
        cur += (size_t)((w + 1) / 2) * ((h + 1) / 2);
        w = (w + 1) / 2; h = (h + 1) / 2;
    }
}

/* ------------------------------------------------------------------------------------
 * ZNCC matching cost (Eq. 2) between the left window centred at (y, x) and the right
 * window centred at (y, x - z) (Eq. 1).  The paper's printed normalisation is garbled;
 * read as the standard zero-mean normalised cross-correlation in [-1, 1]:
 *     rho = sum (a - mean a)(b - mean b) / sqrt(sum (a - mean a)^2 * sum (b - mean b)^2)
 * evaluated from exact integer sums as
 *     c = N*Sab - Sa*Sb,  Va = N*Saa - Sa^2,  Vb = N*Sbb - Sb^2,  rho = c / sqrt(Va*Vb)
 * (the N factors cancel).  A flat window (Va == 0 or Vb == 0) has rho = 0; the result is
 * clamped to [-1, 1] against rounding.
 * ---------------------------------------------------------------------------------- */
double oracle_zncc(const uint8_t *A, const uint8_t *B, int W, int H, int n, int y, int x, int z) {
    long long Sa = 0, Sb = 0, Saa = 0, Sbb = 0, Sab = 0;
    long long N = (long long)(2 * n + 1) * (2 * n + 1);
    for (int i = -n; i <= n; ++i) {
        int yy = clampi(y + i, 0, H - 1);
        for (int j = -n; j <= n; ++j) {
            long long a = A[(long)yy * W + clampi(x + j, 0, W - 1)];
            long long b = B[(long)yy * W + clampi(x - z + j, 0, W - 1)];
            Sa += a; Sb += b; Saa += a * a; Sbb += b * b; Sab += a * b;
        }
    }
    long long Va = N * Saa - Sa * Sa;
    long long Vb = N * Sbb - Sb * Sb;
    if (Va == 0 || Vb == 0) return 0.0;
    double c = (double)(N * Sab - Sa * Sb);
    double rho = c / sqrt((double)Va * (double)Vb);
    if (rho > 1.0) rho = 1.0;
    if (rho < -1.0) rho = -1.0;
    return rho;
}

/* ------------------------------------------------------------------------------------
 * One level of winner-take-all matching.
 *   prior == NULL: the coarsest-level search of Sec. III-A (Eq. 3-4) over every
 *                  admissible candidate 0 <= z <= min(D_k - 1, x).
 *   prior != NULL: the refinement branch of Sec. III-C (Eq. 8-9, first case) at a finer
 *                  level.  The prior is the coarser level's disparity map (Wp x Hp); its
 *                  nearest-neighbour upsample scaled to this level's units is
 *                  dhat = 2 * prior(y/2, x/2)  (the paper writes NN(d^{k+1}) and omits the
 *                  factor 2 that the doubled resolution implies).  The candidates are the
 *                  closed span dhat - r .. dhat + r (the paper's open interval around dhat
 *                  with r = 1 gives its "3 comparisons") clipped to the admissible range.
 *                  dhat is first clamped to 0 .. min(D_k - 1, x); for any prior produced by
 *                  the coarser level this clamp changes nothing.
 * Outputs: d (argmax; ties to the smallest z), C (max, Eq. 4/9), C2 (second-best value,
 * -INFINITY when only one candidate exists).  Returns the number of (pixel, z) ZNCC
 * evaluations.
 * ---------------------------------------------------------------------------------- */
long long oracle_match_level(const uint8_t *A, const uint8_t *B, int W, int H, int n, int Dk,
                             int r, const int16_t *prior, int Wp, int Hp, int16_t *d,
                             double *C, double *C2) {
    long long evals = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : evals)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int zmax = Dk - 1 < x ? Dk - 1 : x;
            int lo = 0, hi = zmax;
            if (prior) {
                int py = clampi(y / 2, 0, Hp - 1), px = clampi(x / 2, 0, Wp - 1);
                int dh = clampi(2 * (int)prior[(long)py * Wp + px], 0, zmax);
                lo = dh - r < 0 ? 0 : dh - r;
                hi = dh + r > zmax ? zmax : dh + r;
            }
            double best = -INFINITY, second = -INFINITY;
            int bz = lo;
            for (int z = lo; z <= hi; ++z) {
                double rho = oracle_zncc(A, B, W, H, n, y, x, z);
                if (rho > best) { second = best; best = rho; bz = z; }
                else if (rho > second) second = rho;
            }
            evals += hi - lo + 1;
            d[(long)y * W + x] = (int16_t)bz;
            C[(long)y * W + x] = best;
            C2[(long)y * W + x] = second;
        }
    }
    return evals;
}

/* ------------------------------------------------------------------------------------
 * The whole hierarchical pass (Sec. III, Fig. 1) in its plain form: pyramid of both
 * images, full search at the coarsest level K-1, then for k = K-2 .. 0 the restricted
 * search around the upsampled coarser disparity.  (The alpha refinement of Sec. III-B, the
 * beta fallback of Eq. 8-9 and the selective median of Sec. III-D are separate functions
 * below.)  K = 1 is flat block matching.
 * Outputs are all levels concatenated, level 0 first: d_all, C_all, C2_all sized
 * sum_k W_k*H_k.  Returns the total evaluation count, or -1 on bad arguments.
 * ---------------------------------------------------------------------------------- */
long long oracle_disparity(const uint8_t *L, const uint8_t *R, int W, int H, int D, int K,
                           int w, int r, int16_t *d_all, double *C_all, double *C2_all) {
    if (W < 1 || H < 1 || D < 1 || K < 1 || w < 1 || (w & 1) == 0 || r < 0) return -1;
    int n = w / 2;
    size_t total = 0;
    for (int k = 0; k < K; ++k) { int a, b; oracle_level_size(W, H, k, &a, &b); total += (size_t)a * b; }
    uint8_t *pl = (uint8_t *)malloc(total), *pr = (uint8_t *)malloc(total);
    size_t *off = (size_t *)malloc(sizeof(size_t) * K);
    if (!pl || !pr || !off) { free(pl); free(pr); free(off); return -1; }
    oracle_pyramid(L, W, H, K, pl);
    oracle_pyramid(R, W, H, K, pr);
    size_t o = 0;
    for (int k = 0; k < K; ++k) { int a, b; oracle_level_size(W, H, k, &a, &b); off[k] = o; o += (size_t)a * b; }
    long long evals = 0;
    for (int k = K - 1; k >= 0; --k) {
        int Wk, Hk, Wp = 0, Hp = 0;
        oracle_level_size(W, H, k, &Wk, &Hk);
        const int16_t *prior = NULL;
        if (k < K - 1) { oracle_level_size(W, H, k + 1, &Wp, &Hp); prior = d_all + off[k + 1]; }
        evals += oracle_match_level(pl + off[k], pr + off[k], Wk, Hk, n, oracle_level_disp(D, k),
                                    r, prior, Wp, Hp, d_all + off[k], C_all + off[k],
                                    C2_all + off[k]);
    }
    free(pl); free(pr); free(off);
    return evals;
}

/* ------------------------------------------------------------------------------------
 * Differentiable level (float images).  ZNCC with two-pass window means and an
 * epsilon-regularised denominator,
 *     rho_eps = sum ac*bc / sqrt((sum ac^2 + eps) (sum bc^2 + eps)),  ac = a - mean a,
 * over candidates 0 <= z <= min(ndisp - 1, x); p = softmax(rho / T) over the admissible
 * candidates; d_soft = sum z p_z.  Images are B x H x W, row-major per image.
 * rho_out (optional, may be NULL) receives rho for every (b, y, x, z), -INFINITY where z
 * is not admissible.
 * ---------------------------------------------------------------------------------- */
static double zncc_eps_window(const double *A, const double *Bm, int W, int H, int n, int y,
                              int x, int z, double eps, double *ac, double *bc, double *Saa_o,
                              double *Sbb_o) {
    int w = 2 * n + 1, N = w * w, t = 0;
    double ma = 0.0, mb = 0.0;
    for (int i = -n; i <= n; ++i)
        for (int j = -n; j <= n; ++j, ++t) {
            int yy = clampi(y + i, 0, H - 1);
            ac[t] = A[(long)yy * W + clampi(x + j, 0, W - 1)];
            bc[t] = Bm[(long)yy * W + clampi(x - z + j, 0, W - 1)];
            ma += ac[t]; mb += bc[t];
        }
    ma /= N; mb /= N;
    double Saa = 0.0, Sbb = 0.0, Sab = 0.0;
    for (t = 0; t < N; ++t) {
        ac[t] -= ma; bc[t] -= mb;
        Saa += ac[t] * ac[t]; Sbb += bc[t] * bc[t]; Sab += ac[t] * bc[t];
    }
    *Saa_o = Saa; *Sbb_o = Sbb;
    return Sab / sqrt((Saa + eps) * (Sbb + eps));
}

void oracle_softargmax_fwd(const double *L, const double *R, int Bn, int H, int W, int n,
                           int ndisp, double T, double eps, double *dsoft, double *rho_out) {
    int N = (2 * n + 1) * (2 * n + 1);
#pragma omp parallel
    {
        double *ac = (double *)malloc(sizeof(double) * N), *bc = (double *)malloc(sizeof(double) * N);
        double *rho = (double *)malloc(sizeof(double) * (ndisp > 0 ? ndisp : 1));
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (int b = 0; b < Bn; ++b)
            for (int y = 0; y < H; ++y) {
                const double *A = L + (long)b * H * W, *Bm = R + (long)b * H * W;
                for (int x = 0; x < W; ++x) {
                    int zmax = ndisp - 1 < x ? ndisp - 1 : x;
                    double Saa, Sbb, m = -INFINITY;
                    for (int z = 0; z <= zmax; ++z) {
                        rho[z] = zncc_eps_window(A, Bm, W, H, n, y, x, z, eps, ac, bc, &Saa, &Sbb);
                        if (rho[z] / T > m) m = rho[z] / T;
                    }
                    double s = 0.0, sz = 0.0;
                    for (int z = 0; z <= zmax; ++z) {
                        double e = exp(rho[z] / T - m);
                        s += e; sz += z * e;
                    }
                    long pix = ((long)b * H + y) * W + x;
                    dsoft[pix] = sz / s;
                    if (rho_out)
                        for (int z = 0; z < ndisp; ++z) rho_out[pix * ndisp + z] = z <= zmax ? rho[z] : -INFINITY;
                }
            }
        free(ac); free(bc); free(rho);
    }
}

/* Backward of the soft-argmax readout with respect to both images.  With
 * p_z = softmax(rho_z / T) and d = sum z p_z:  dd/drho_z = p_z (z - d) / T.  For the
 * centred window entries,  drho/dac_i = bc_i / s - rho * ac_i / (Saa + eps)  and
 * drho/dbc_i = ac_i / s - rho * bc_i / (Sbb + eps)  with s = sqrt((Saa+eps)(Sbb+eps)); the
 * derivative through the mean vanishes because the centred entries sum to zero.  Each
 * window entry's gradient goes to the image pixel it was read from (clamped positions
 * accumulate at the edge pixel).  g_d is dLoss/dd_soft; gL, gR are overwritten. */
void oracle_softargmax_bwd(const double *L, const double *R, int Bn, int H, int W, int n,
                           int ndisp, double T, double eps, const double *g_d, double *gL,
                           double *gR) {
    int w = 2 * n + 1, N = w * w;
    memset(gL, 0, sizeof(double) * Bn * H * W);
    memset(gR, 0, sizeof(double) * Bn * H * W);
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < Bn; ++b) {
        double *ac = (double *)malloc(sizeof(double) * N), *bc = (double *)malloc(sizeof(double) * N);
        double *rho = (double *)malloc(sizeof(double) * (ndisp > 0 ? ndisp : 1));
        const double *A = L + (long)b * H * W, *Bm = R + (long)b * H * W;
        double *gA = gL + (long)b * H * W, *gB = gR + (long)b * H * W;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int zmax = ndisp - 1 < x ? ndisp - 1 : x;
                double Saa, Sbb, m = -INFINITY;
                for (int z = 0; z <= zmax; ++z) {
                    rho[z] = zncc_eps_window(A, Bm, W, H, n, y, x, z, eps, ac, bc, &Saa, &Sbb);
                    if (rho[z] / T > m) m = rho[z] / T;
                }
                double s = 0.0, sz = 0.0;
                for (int z = 0; z <= zmax; ++z) { double e = exp(rho[z] / T - m); s += e; sz += z * e; }
                double dsoft = sz / s;
                double g = g_d[((long)b * H + y) * W + x];
                if (g == 0.0) continue;
                for (int z = 0; z <= zmax; ++z) {
                    double p = exp(rho[z] / T - m) / s;
                    double grho = g * p * (z - dsoft) / T;
                    double r_ = zncc_eps_window(A, Bm, W, H, n, y, x, z, eps, ac, bc, &Saa, &Sbb);
                    double sq = sqrt((Saa + eps) * (Sbb + eps));
                    int t = 0;
                    for (int i = -n; i <= n; ++i)
                        for (int j = -n; j <= n; ++j, ++t) {
                            int yy = clampi(y + i, 0, H - 1);
                            double da = bc[t] / sq - r_ * ac[t] / (Saa + eps);
                            double db = ac[t] / sq - r_ * bc[t] / (Sbb + eps);
                            gA[(long)yy * W + clampi(x + j, 0, W - 1)] += grho * da;
                            gB[(long)yy * W + clampi(x - z + j, 0, W - 1)] += grho * db;
                        }
                }
            }
        free(ac); free(bc); free(rho);
    }
}

/* ====================================================================================
 * The gated steps of the full method (Sec. III-B, III-C second branch, III-D).
 * ==================================================================================== */

/* Keys cubic convolution kernel with a = -1/2 (Catmull-Rom). */
static double cubic_w(double t) {
    t = fabs(t);
    if (t < 1.0) return (1.5 * t - 2.5) * t * t + 1.0;
    if (t < 2.0) return ((-0.5 * t + 2.5) * t - 4.0) * t + 2.0;
    return 0.0;
}

/* Sec. III-C: the cost prior C_hat^k = BI(C^{k+1}), bicubic upsampling.  Reading: the fine
 * pixel (y, x) sits at coarse coordinates (y/2, x/2) (coarse pixel i is the reduce of fine
 * pixel 2i), samples outside the coarse map are clamped to its edge.  Written as the plain
 * 4 x 4 weighted sum. */
double oracle_bicubic_at(const double *Cc, int Wc, int Hc, double cy, double cx) {
    int iy = (int)floor(cy), ix = (int)floor(cx);
    double fy = cy - iy, fx = cx - ix, s = 0.0;
    for (int a = -1; a <= 2; ++a) {
        double wy = cubic_w(a - fy);
        int yy = clampi(iy + a, 0, Hc - 1);
        for (int b = -1; b <= 2; ++b) {
            double wx = cubic_w(b - fx);
            int xx = clampi(ix + b, 0, Wc - 1);
            s += wy * wx * Cc[(long)yy * Wc + xx];
        }
    }
    return s;
}

void oracle_upsample_cost(const double *Cc, int Wc, int Hc, int W, int H, double *out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) out[(long)y * W + x] = oracle_bicubic_at(Cc, Wc, Hc, 0.5 * y, 0.5 * x);
}

/* Eq. 8-9, both branches: where the upsampled cost C_hat exceeds beta the restricted
 * search around dhat (first branch, as oracle_match_level), otherwise the full search over
 * 0 .. min(D_k - 1, x) (second branch).  Cprior is the coarser level's cost map (Wp x Hp).
 * fallback (optional) receives 1 where the second branch was taken; chat (optional)
 * receives C_hat.  Returns the evaluation count. */
long long oracle_match_level_beta(const uint8_t *A, const uint8_t *B, int W, int H, int n, int Dk,
                                  int r, const int16_t *prior, const double *Cprior, int Wp, int Hp,
                                  double beta, int16_t *d, double *C, double *C2, uint8_t *fallback,
                                  double *chat) {
    long long evals = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : evals)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int zmax = Dk - 1 < x ? Dk - 1 : x;
            double ch = oracle_bicubic_at(Cprior, Wp, Hp, 0.5 * y, 0.5 * x);
            int full = !(ch > beta);
            int lo = 0, hi = zmax;
            if (!full) {
                int py = clampi(y / 2, 0, Hp - 1), px = clampi(x / 2, 0, Wp - 1);
                int dh = clampi(2 * (int)prior[(long)py * Wp + px], 0, zmax);
                lo = dh - r < 0 ? 0 : dh - r;
                hi = dh + r > zmax ? zmax : dh + r;
            }
            double best = -INFINITY, second = -INFINITY;
            int bz = lo;
            for (int z = lo; z <= hi; ++z) {
                double rho = oracle_zncc(A, B, W, H, n, y, x, z);
                if (rho > best) { second = best; best = rho; bz = z; }
                else if (rho > second) second = rho;
            }
            evals += hi - lo + 1;
            long o = (long)y * W + x;
            d[o] = (int16_t)bz; C[o] = best; C2[o] = second;
            if (fallback) fallback[o] = (uint8_t)full;
            if (chat) chat[o] = ch;
        }
    }
    return evals;
}

/* Sec. III-B, Eq. 5-7: for every pixel whose matched cost C' is not above alpha, average
 * the DSI over its 3 x 3 neighbourhood N(i, j) (neighbours inside the image; the paper
 * leaves the size unstated and writes a sum, which has the same argmax; the average keeps
 * C on the ZNCC scale) and take the argmax over the pixel's own admissible candidates
 * 0 .. min(D_k - 1, x).  Each neighbour's E(z) is the ZNCC of its window at disparity z
 * (clamp-to-edge windows).  d, C are updated in place from copies of the inputs; C2
 * receives the second-best averaged value for refined pixels (untouched otherwise);
 * refined (optional) marks the refined pixels. */
void oracle_alpha_refine(const uint8_t *A, const uint8_t *B, int W, int H, int n, int Dk,
                         double alpha, int16_t *d, double *C, double *C2, uint8_t *refined) {
    double *Cin = (double *)malloc(sizeof(double) * (size_t)W * H);
    memcpy(Cin, C, sizeof(double) * (size_t)W * H);
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            long o = (long)y * W + x;
            if (refined) refined[o] = 0;
            if (Cin[o] > alpha) continue;
            int zmax = Dk - 1 < x ? Dk - 1 : x;
            double best = -INFINITY, second = -INFINITY;
            int bz = 0;
            for (int z = 0; z <= zmax; ++z) {
                double s = 0.0;
                int cnt = 0;
                for (int m = y - 1; m <= y + 1; ++m)
                    for (int q = x - 1; q <= x + 1; ++q) {
                        if (m < 0 || m >= H || q < 0 || q >= W) continue;
                        s += oracle_zncc(A, B, W, H, n, m, q, z);
                        ++cnt;
                    }
                double e = s / cnt;
                if (e > best) { second = best; best = e; bz = z; }
                else if (e > second) second = e;
            }
            d[o] = (int16_t)bz;
            C[o] = best;
            C2[o] = second;
            if (refined) refined[o] = 1;
        }
    }
    free(Cin);
}

/* Sec. III-D, Eq. 10: for every pixel whose cost is not above alpha, the median of the
 * disparities of the 5 x 5 neighbours (inside the image) whose cost is above alpha; the
 * lower median for an even count; unchanged when no neighbour qualifies.  Reads d_in, C;
 * writes d_out (may not alias d_in). */
void oracle_selective_median(const int16_t *d_in, const double *C, int W, int H, double alpha,
                             int16_t *d_out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long o = (long)y * W + x;
            d_out[o] = d_in[o];
            if (C[o] > alpha) continue;
            int v[25], cnt = 0;
            for (int m = y - 2; m <= y + 2; ++m)
                for (int q = x - 2; q <= x + 2; ++q) {
                    if (m < 0 || m >= H || q < 0 || q >= W) continue;
                    long p = (long)m * W + q;
                    if (C[p] > alpha) v[cnt++] = d_in[p];
                }
            if (cnt == 0) continue;
            for (int i = 1; i < cnt; ++i) {            /* insertion sort */
                int t = v[i], j = i - 1;
                while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
                v[j + 1] = t;
            }
            d_out[o] = (int16_t)v[(cnt - 1) / 2];
        }
}

/* Window half-width at level k when the block size halves per level (Sec. III: the
 * matching block size decreases by a factor of 2 at every pyramid level; Sec. IV gives the
 * block of the full-resolution level): n_k = max(1, n_0 >> k), i.e. windows 2 n_k + 1. */
int oracle_level_half_width(int n0, int k) {
    int n = n0 >> k;
    return n < 1 ? 1 : n;
}

/* The full method of Sec. III (Fig. 1): coarsest WTA, then (flags & 1) alpha refinement;
 * at each finer level the beta-gated search (flags & 2; else the restricted branch only),
 * then (flags & 4) the selective median.  flags & 8: level k matches with half-width
 * oracle_level_half_width(w / 2, k) instead of w / 2 at every level.  Outputs as
 * oracle_disparity: all levels, level 0 first; d_all holds each level's final
 * (post-median) map, C_all its cost (the median changes d only), C2_all the second-best
 * cost.  Returns the evaluation count (alpha refinement counts its 3x3 x candidates
 * evaluations), or -1 on bad arguments. */
long long oracle_disparity_full(const uint8_t *L, const uint8_t *R, int W, int H, int D, int K,
                                int w, int r, double alpha, double beta, int flags, int16_t *d_all,
                                double *C_all, double *C2_all) {
    if (W < 1 || H < 1 || D < 1 || K < 1 || w < 1 || (w & 1) == 0 || r < 0) return -1;
    int n = w / 2;
    size_t total = 0;
    for (int k = 0; k < K; ++k) { int a, b; oracle_level_size(W, H, k, &a, &b); total += (size_t)a * b; }
    uint8_t *pl = (uint8_t *)malloc(total), *pr = (uint8_t *)malloc(total);
    size_t *off = (size_t *)malloc(sizeof(size_t) * K);
    int16_t *tmp = (int16_t *)malloc(sizeof(int16_t) * (size_t)W * H);
    if (!pl || !pr || !off || !tmp) { free(pl); free(pr); free(off); free(tmp); return -1; }
    oracle_pyramid(L, W, H, K, pl);
    oracle_pyramid(R, W, H, K, pr);
    size_t o = 0;
    for (int k = 0; k < K; ++k) { int a, b; oracle_level_size(W, H, k, &a, &b); off[k] = o; o += (size_t)a * b; }
    long long evals = 0;
    const int n0 = n;
    for (int k = K - 1; k >= 0; --k) {
        int Wk, Hk, Wp = 0, Hp = 0;
        oracle_level_size(W, H, k, &Wk, &Hk);
        int Dk = oracle_level_disp(D, k);
        n = (flags & 8) ? oracle_level_half_width(n0, k) : n0;
        int16_t *dk = d_all + off[k];
        double *ck = C_all + off[k], *c2k = C2_all + off[k];
        if (k == K - 1) {
            evals += oracle_match_level(pl + off[k], pr + off[k], Wk, Hk, n, Dk, 0, NULL, 0, 0, dk, ck, c2k);
            if (flags & 1) {
                for (long i = 0; i < (long)Wk * Hk; ++i)
                    if (ck[i] <= alpha) {
                        int x = (int)(i % Wk), y = (int)(i / Wk);
                        int cnt = (y > 0) + 1 + (y < Hk - 1);
                        cnt *= (x > 0) + 1 + (x < Wk - 1);
                        evals += (long long)cnt * ((Dk - 1 < x ? Dk - 1 : x) + 1);
                    }
                oracle_alpha_refine(pl + off[k], pr + off[k], Wk, Hk, n, Dk, alpha, dk, ck, c2k, NULL);
            }
            continue;
        }
        oracle_level_size(W, H, k + 1, &Wp, &Hp);
        const int16_t *prior = d_all + off[k + 1];
        if (flags & 2)
            evals += oracle_match_level_beta(pl + off[k], pr + off[k], Wk, Hk, n, Dk, r, prior,
                                             C_all + off[k + 1], Wp, Hp, beta, dk, ck, c2k, NULL, NULL);
        else
            evals += oracle_match_level(pl + off[k], pr + off[k], Wk, Hk, n, Dk, r, prior, Wp, Hp, dk, ck, c2k);
        if (flags & 4) {
            oracle_selective_median(dk, ck, Wk, Hk, alpha, tmp);
            memcpy(dk, tmp, sizeof(int16_t) * (size_t)Wk * Hk);
        }
    }
    free(pl); free(pr); free(off); free(tmp);
    return evals;
}
